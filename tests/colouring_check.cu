// Host-side check of the conflict-free assembly rules the cell kernels use
// (fe_cell_kernel.cuh): along one direction of a structured mesh, for every
// global node exactly one of the (cell, local node) pairs that hold it is the
// first writer, and that cell has the strictly lowest colour among them; cells
// of one colour share no node; Dirichlet boundary nodes are exactly the two
// ends.  The 3-D colour is the lexicographic combination of the per-direction
// colours (z slowest), so the per-direction properties give the 3-D ones.
// Runs on the CPU (no device code is called); prints "ok" or the first failure.
#include <cstdio>
#include <vector>

#include "fe_cell_kernel.cuh"

using namespace fe;

static int fail(const char* what, int n, int P, int periodic, int g) {
  std::printf("FAIL %s: n=%d P=%d periodic=%d node=%d\n", what, n, P, periodic, g);
  return 1;
}

int main() {
  for (int periodic = 0; periodic <= 1; ++periodic)
    for (int n = periodic ? 2 : 1; n <= 13; ++n)
      for (int P = 1; P <= 8; ++P) {
        // three colours along a periodic direction with an odd cell count
        const int last_odd = periodic && (n & 1) && n > 1;
        const int N = periodic ? n * P : n * P + 1;
        std::vector<std::vector<int>> holders(N);   // cells holding each node
        for (int c = 0; c < n; ++c)
          for (int i = 0; i <= P; ++i) {
            const int g = node_coord(c, i, P, N, periodic);
            if (g < 0 || g >= N) return fail("node coordinate out of range", n, P, periodic, g);
            holders[g].push_back(c * (P + 1) + i);
          }
        for (int g = 0; g < N; ++g) {
          int firsts = 0, first_colour = -1, min_colour = 99, at_min = 0;
          for (int h : holders[g]) {
            const int c = h / (P + 1), i = h % (P + 1);
            const int k = dir_color(c, n, last_odd);
            if (first_along(c, n, i, P, periodic, last_odd)) { ++firsts; first_colour = k; }
            if (k < min_colour) { min_colour = k; at_min = 1; } else if (k == min_colour) ++at_min;
          }
          if (holders[g].empty()) return fail("node held by no cell", n, P, periodic, g);
          if (firsts != 1) return fail("not exactly one first writer", n, P, periodic, g);
          if (first_colour != min_colour || at_min != 1) return fail("first writer not the unique lowest colour", n, P, periodic, g);
          // cells of one colour share no node
          for (size_t a = 0; a < holders[g].size(); ++a)
            for (size_t b = a + 1; b < holders[g].size(); ++b) {
              const int ca = holders[g][a] / (P + 1), cb = holders[g][b] / (P + 1);
              if (ca != cb && dir_color(ca, n, last_odd) == dir_color(cb, n, last_odd))
                return fail("two cells of one colour share a node", n, P, periodic, g);
            }
          const bool end = !periodic && (g == 0 || g == N - 1);
          if (on_boundary(g, N, periodic) != end) return fail("boundary flag", n, P, periodic, g);
        }
        // colour count: 1 for one cell, 3 for odd periodic counts, else 2
        int kmax = 0;
        for (int c = 0; c < n; ++c) kmax = dir_color(c, n, last_odd) > kmax ? dir_color(c, n, last_odd) : kmax;
        const int want = n == 1 ? 1 : (last_odd ? 3 : 2);
        if (kmax + 1 != want) return fail("colour count", n, P, periodic, -1);
      }
  std::printf("ok\n");
  return 0;
}
