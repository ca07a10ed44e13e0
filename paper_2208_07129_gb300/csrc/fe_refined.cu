// Host setup of a one-level adaptively refined mesh with hanging nodes
// (Sec. 3.2.2: constraints u_S = W u_M; the adaptive meshes of the paper's
// Sec. 4 benchmarks).
//
// A Dirichlet box of nx x ny x nz coarse cells of size H; the coarse cells in
// [refine_lo, refine_hi) are split into 2 x 2 x 2 children.  Cells are listed
// coarse cell by coarse cell (x fastest), a refined cell replaced by its 8
// children (x fastest).  Node positions along one direction (units of H/4):
//   vertex m of the half-size grid:        2m          key (V, m)
//   interior GLL node i of coarse cell c:  4c + 2(1 + g_i)   key (C, c, i)
//     (the middle node of an even degree is the vertex 2c + 1)
//   interior GLL node j of fine cell f:    2f + (1 + g_j)    key (F, f, j)
// Two nodes are one DoF when their three keys agree; DoFs are numbered by
// position, z slowest, x fastest.  A fine-cell node on the closure of an
// unrefined coarse cell C that is not one of C's nodes is a slave: its value
// is C's interpolant there (masters on the boundary carry 0 and are dropped).
#include <algorithm>
#include <array>
#include <cmath>
#include <map>
#include <new>
#include <unordered_map>
#include <vector>

#include "fe_internal.h"

using namespace fe;

namespace {

fe_status from_cuda(cudaError_t e) {
  return fe::cuda_status(e);
}

constexpr long long kV = 0, kC = 1, kF = 2;

struct Comp {
  long long key;   // kind << 40 | a << 8 | i
  double pos;      // units of H/4
};

Comp comp(int level, int c, int i, int p, const double* g) {
  auto K = [](long long kind, long long a, long long idx) { return (kind << 40) | (a << 8) | idx; };
  if (level == 0) {
    if (i == 0) return {K(kV, 2LL * c, 0), 4.0 * c};
    if (i == p) return {K(kV, 2LL * c + 2, 0), 4.0 * c + 4.0};
    if (p % 2 == 0 && i == p / 2) return {K(kV, 2LL * c + 1, 0), 4.0 * c + 2.0};
    return {K(kC, c, i), 4.0 * c + 2.0 * (1.0 + g[i])};
  }
  if (i == 0) return {K(kV, c, 0), 2.0 * c};
  if (i == p) return {K(kV, (long long)c + 1, 0), 2.0 * c + 2.0};
  return {K(kF, c, i), 2.0 * c + (1.0 + g[i])};
}

using Key3 = std::array<long long, 3>;
struct Key3Hash {
  size_t operator()(const Key3& k) const {
    size_t h = 1469598103934665603ull;
    for (long long v : k) h = (h ^ (size_t)v) * 1099511628211ull;
    return h;
  }
};

}  // namespace

namespace fe {
void free_refined(fe_ctx* c) {
  for (int* p : {c->d_map, c->d_row_slave, c->d_sl_ptr, c->d_sl_idx, c->d_slaves, c->d_ma_rows, c->d_ma_ptr,
                 c->d_ma_idx})
    cudaFree(p);
  cudaFree(c->d_sl_w);
  cudaFree(c->d_sl_w32);
  cudaFree(c->d_ma_w);
  cudaFree(c->d_ma_w32);
  cudaFree(c->d_xc);
}
}  // namespace fe

extern "C" fe_status fe_setup_refined(const fe_refined_desc* md, int p, const fe_quad_desc* quad, double mu,
                                      fe_ctx** out) {
  if (!out) return FE_EINVAL;
  *out = nullptr;
  if (!md || !quad || !std::isfinite(mu)) return FE_EINVAL;
  const int n[3] = {md->nx, md->ny, md->nz};
  for (int d = 0; d < 3; ++d) {
    if (n[d] < 1 || !(md->hi[d] > md->lo[d])) return FE_EINVAL;
    if (md->refine_lo[d] < 0 || md->refine_hi[d] > n[d] || md->refine_lo[d] > md->refine_hi[d]) return FE_EINVAL;
  }
  if (quad->kind != FE_QUAD_GAUSS && quad->kind != FE_QUAD_GLL) return FE_EINVAL;
  if (p < 1 || p > kMaxP || quad->n_q < p + 1 || quad->n_q > p + 3) return FE_EUNSUPPORTED;
  const long long ncoarse = (long long)n[0] * n[1] * n[2];
  if (ncoarse > (1LL << 24)) return FE_EINVAL;

  fe_ctx* c = new (std::nothrow) fe_ctx();
  if (!c) return FE_ENOMEM;
  c->refined = 1;
  c->nx = n[0]; c->ny = n[1]; c->nz = n[2];
  c->periodic = 0;
  c->p = p; c->np = p + 1; c->nq = quad->n_q; c->quad_kind = quad->kind; c->mu = mu;
  c->general = 0;
  if (quad->n_q >= 9) { c->vb64 = 4; c->nty64 = 32; c->vb32 = 4; c->nty32 = 64; c->vbdf = 4; c->ntydf = 64; }
  c->fp32_variant = 3;
  build_tables(c);
  const int np = c->np, nq = c->nq, NP3 = np * np * np;
  const double* g = c->gll.data();
  double H[3];
  for (int d = 0; d < 3; ++d) H[d] = (md->hi[d] - md->lo[d]) / n[d];
  auto refined = [&](int cx, int cy, int cz) {
    return cx >= md->refine_lo[0] && cx < md->refine_hi[0] && cy >= md->refine_lo[1] && cy < md->refine_hi[1] &&
           cz >= md->refine_lo[2] && cz < md->refine_hi[2];
  };

  // ---- cells ----
  struct Cell { int level, idx[3]; };
  std::vector<Cell> cells;
  for (int cz = 0; cz < n[2]; ++cz)
    for (int cy = 0; cy < n[1]; ++cy)
      for (int cx = 0; cx < n[0]; ++cx) {
        if (refined(cx, cy, cz)) {
          for (int k = 0; k < 8; ++k)
            cells.push_back({1, {2 * cx + (k & 1), 2 * cy + ((k >> 1) & 1), 2 * cz + ((k >> 2) & 1)}});
        } else {
          cells.push_back({0, {cx, cy, cz}});
        }
      }
  const size_t E = cells.size();

  // ---- nodes: keys, positions, numbering ----
  std::unordered_map<Key3, int, Key3Hash> id;
  std::vector<std::array<double, 3>> pos;
  std::vector<Key3> keys;
  std::vector<int> local(E * NP3);
  std::vector<char> on_fine;
  for (size_t e = 0; e < E; ++e) {
    const Cell& C = cells[e];
    Comp cp[3][kMaxP + 1];
    for (int d = 0; d < 3; ++d)
      for (int i = 0; i < np; ++i) cp[d][i] = comp(C.level, C.idx[d], i, p, g);
    for (int i3 = 0; i3 < np; ++i3)
      for (int i2 = 0; i2 < np; ++i2)
        for (int i1 = 0; i1 < np; ++i1) {
          const Key3 k{cp[0][i1].key, cp[1][i2].key, cp[2][i3].key};
          auto it = id.find(k);
          int v;
          if (it == id.end()) {
            v = (int)keys.size();
            id.emplace(k, v);
            keys.push_back(k);
            pos.push_back({cp[0][i1].pos, cp[1][i2].pos, cp[2][i3].pos});
            on_fine.push_back(0);
          } else {
            v = it->second;
          }
          if (C.level == 1) on_fine[v] = 1;
          local[e * NP3 + (i3 * np + i2) * np + i1] = v;
        }
  }
  const size_t N = keys.size();
  if (N >= (size_t)kMapIndex) { fe_destroy(c); return FE_EINVAL; }
  std::vector<int> order(N);
  for (size_t i = 0; i < N; ++i) order[i] = (int)i;
  std::sort(order.begin(), order.end(), [&](int a, int b) {
    if (pos[a][2] != pos[b][2]) return pos[a][2] < pos[b][2];
    if (pos[a][1] != pos[b][1]) return pos[a][1] < pos[b][1];
    return pos[a][0] < pos[b][0];
  });
  std::vector<int> dof(N);
  for (size_t r = 0; r < N; ++r) dof[order[r]] = (int)r;
  c->n_dofs = N;
  c->n_cells = E;
  std::vector<char> boundary(N), fine(N);
  for (size_t v = 0; v < N; ++v) {
    bool b = false;
    for (int d = 0; d < 3; ++d) {
      const long long k = keys[v][d];
      if ((k >> 40) == kV) {
        const long long m = (k >> 8) & 0xffffffffLL;
        if (m == 0 || m == 2LL * n[d]) b = true;
      }
    }
    boundary[dof[v]] = b;
    fine[dof[v]] = on_fine[v];
  }

  // ---- hanging nodes ----
  // slave DoF -> (master DoF, weight) list
  std::map<int, std::vector<std::pair<int, double>>> slaves;
  for (size_t v = 0; v < N; ++v) {
    const int dv = dof[v];
    if (boundary[dv] || !fine[dv]) continue;
    int cand[3][2], nc[3];
    for (int d = 0; d < 3; ++d) {
      const int a = (int)std::floor(pos[v][d] / 4.0), b = (int)std::ceil(pos[v][d] / 4.0) - 1;
      nc[d] = 0;
      for (int x : {b, a})
        if (x >= 0 && x < n[d] && (nc[d] == 0 || cand[d][0] != x)) cand[d][nc[d]++] = x;
    }
    int owner[3] = {-1, -1, -1};
    bool shared = false, any = false;
    for (int z = 0; z < nc[2]; ++z)
      for (int y = 0; y < nc[1]; ++y)
        for (int x = 0; x < nc[0]; ++x) {
          const int C3[3] = {cand[0][x], cand[1][y], cand[2][z]};
          if (refined(C3[0], C3[1], C3[2])) continue;
          bool own = true;
          for (int d = 0; d < 3 && own; ++d) {
            bool hit = false;
            for (int i = 0; i < np; ++i) hit = hit || comp(0, C3[d], i, p, g).key == keys[v][d];
            own = hit;
          }
          if (own) shared = true;
          if (!any) { any = true; owner[0] = C3[0]; owner[1] = C3[1]; owner[2] = C3[2]; }
        }
    if (!any || shared) continue;
    double ph[3][kMaxP + 1];
    for (int d = 0; d < 3; ++d) {
      const double xi = (pos[v][d] - 4.0 * owner[d]) / 2.0 - 1.0;
      for (int i = 0; i < np; ++i) ph[d][i] = lagrange_1d(g, np, i, xi);
    }
    std::vector<std::pair<int, double>> ms;
    for (int i3 = 0; i3 < np; ++i3)
      for (int i2 = 0; i2 < np; ++i2)
        for (int i1 = 0; i1 < np; ++i1) {
          const double w = ph[0][i1] * ph[1][i2] * ph[2][i3];
          if (std::fabs(w) <= 1e-14) continue;
          const Key3 mk{comp(0, owner[0], i1, p, g).key, comp(0, owner[1], i2, p, g).key,
                        comp(0, owner[2], i3, p, g).key};
          auto it = id.find(mk);
          if (it == id.end()) { fe_destroy(c); return FE_EINVAL; }   // a coarse node of C must exist
          const int dm = dof[it->second];
          if (!boundary[dm]) ms.emplace_back(dm, w);
        }
    slaves[dv] = ms;
  }

  // ---- colours: coarse cells by parity (0..7), fine cells by parity (8..15) ----
  std::vector<int> col(E);
  int count[16] = {0};
  for (size_t e = 0; e < E; ++e) {
    const Cell& C = cells[e];
    col[e] = (C.level ? 8 : 0) + (C.idx[0] & 1) + 2 * (C.idx[1] & 1) + 4 * (C.idx[2] & 1);
    count[col[e]]++;
  }
  c->colors.n_colors = 16;
  c->colors.offset.assign(17, 0);
  for (int k = 0; k < 16; ++k) c->colors.offset[k + 1] = c->colors.offset[k] + count[k];
  c->cells_by_color.resize(E);
  std::vector<int> fill(c->colors.offset.begin(), c->colors.offset.end() - 1);
  for (size_t e = 0; e < E; ++e) c->cells_by_color[fill[col[e]]++] = (int)e;
  // first writer of every node in colour order
  std::vector<int> map(E * NP3);
  std::vector<char> written(N, 0);
  for (int k = 0; k < 16; ++k)
    for (int t = c->colors.offset[k]; t < c->colors.offset[k + 1]; ++t) {
      const int e = c->cells_by_color[t];
      for (int j = 0; j < NP3; ++j) {
        const int dv = dof[local[(size_t)e * NP3 + j]];
        int code = dv;
        if (boundary[dv]) code |= kMapConstrained;
        if (!written[dv]) { code |= kMapFirst; written[dv] = 1; }
        map[(size_t)e * NP3 + j] = code;
      }
    }

  // ---- geometry: axis-aligned boxes ----
  const size_t nq3 = (size_t)nq * nq * nq;
  c->cell_lo.resize(3 * E);
  c->cell_h.resize(3 * E);
  c->cellG.resize(E * 6);
  c->detJ.resize(E * nq3);
  for (size_t e = 0; e < E; ++e) {
    const Cell& C = cells[e];
    double h[3];
    for (int d = 0; d < 3; ++d) {
      h[d] = C.level ? H[d] / 2.0 : H[d];
      c->cell_h[3 * e + d] = h[d];
      c->cell_lo[3 * e + d] = md->lo[d] + C.idx[d] * h[d];
    }
    const double det = h[0] * h[1] * h[2] / 8.0;
    // mu det J J^-1 J^-T with J = diag(h / 2)
    const double G[6] = {mu * det * 4.0 / (h[0] * h[0]), 0.0, 0.0, mu * det * 4.0 / (h[1] * h[1]), 0.0,
                         mu * det * 4.0 / (h[2] * h[2])};
    for (int k = 0; k < 6; ++k) c->cellG[e * 6 + k] = G[k];
    for (size_t Q = 0; Q < nq3; ++Q) c->detJ[e * nq3 + Q] = det;
  }
  c->mdev = MeshDev{1, 1, 1, 1, 1, 1, 0, 1, 1, 0, 0, 0};

  // ---- constraints as CSR (slave rows and master rows) ----
  std::vector<int> row_slave(N, -1), sl_ptr(1, 0), sl_idx, slave_dof;
  std::vector<double> sl_w;
  std::map<int, std::vector<std::pair<int, double>>> by_master;
  for (const auto& kv : slaves) {
    row_slave[kv.first] = (int)slave_dof.size();
    slave_dof.push_back(kv.first);
    for (const auto& mw : kv.second) {
      sl_idx.push_back(mw.first);
      sl_w.push_back(mw.second);
      by_master[mw.first].emplace_back(kv.first, mw.second);
    }
    sl_ptr.push_back((int)sl_idx.size());
  }
  std::vector<int> ma_rows, ma_ptr(1, 0), ma_idx;
  std::vector<double> ma_w;
  for (const auto& kv : by_master) {
    ma_rows.push_back(kv.first);
    for (const auto& sw : kv.second) {
      ma_idx.push_back(sw.first);
      ma_w.push_back(sw.second);
    }
    ma_ptr.push_back((int)ma_idx.size());
  }
  c->n_slaves = (int)slave_dof.size();
  c->n_masters = (int)ma_rows.size();
  c->node_xyz.resize(3 * N);
  for (size_t v = 0; v < N; ++v)
    for (int d = 0; d < 3; ++d) c->node_xyz[3 * (size_t)dof[v] + d] = md->lo[d] + pos[v][d] * H[d] / 4.0;

  // ---- uploads ----
  cudaError_t err = upload_ints(&c->d_cells, c->cells_by_color);
  if (err == cudaSuccess) err = upload_ints(&c->d_map, map);
  if (err == cudaSuccess) err = upload_doubles(&c->d_cellG64, c->cellG);
  if (err == cudaSuccess) err = upload_floats(&c->d_cellG32, c->cellG);
  if (err == cudaSuccess) err = upload_ffs(&c->d_cellGff, c->cellG);
  if (err == cudaSuccess) err = upload_ints(&c->d_row_slave, row_slave);
  if (err == cudaSuccess && c->n_slaves > 0) {
    err = upload_ints(&c->d_sl_ptr, sl_ptr);
    if (err == cudaSuccess) err = upload_ints(&c->d_slaves, slave_dof);
    if (err == cudaSuccess && !sl_idx.empty()) err = upload_ints(&c->d_sl_idx, sl_idx);
    if (err == cudaSuccess && !sl_w.empty()) err = upload_doubles(&c->d_sl_w, sl_w);
    if (err == cudaSuccess && !sl_w.empty()) err = upload_floats(&c->d_sl_w32, sl_w);
  }
  if (err == cudaSuccess && c->n_masters > 0) {
    err = upload_ints(&c->d_ma_rows, ma_rows);
    if (err == cudaSuccess) err = upload_ints(&c->d_ma_ptr, ma_ptr);
    if (err == cudaSuccess) err = upload_ints(&c->d_ma_idx, ma_idx);
    if (err == cudaSuccess) err = upload_doubles(&c->d_ma_w, ma_w);
    if (err == cudaSuccess) err = upload_floats(&c->d_ma_w32, ma_w);
  }
  if (err == cudaSuccess) err = cudaMalloc(&c->d_status, sizeof(int));
  if (err == cudaSuccess) err = cudaMemset(c->d_status, 0, sizeof(int));
  if (err == cudaSuccess) err = upload_point_coeff(c, std::vector<double>(E * nq3, 0.0));
  if (err != cudaSuccess) { fe_destroy(c); return from_cuda(err); }
  *out = c;
  return FE_OK;
}

extern "C" int fe_num_slaves(const fe_ctx* c) { return c ? c->n_slaves : 0; }

extern "C" fe_status fe_node_coords(const fe_ctx* c, double* xyz) {
  if (!c || !xyz) return FE_EINVAL;
  if (c->refined) {
    std::copy(c->node_xyz.begin(), c->node_xyz.end(), xyz);
    return FE_OK;
  }
  // structured numbering: node (gx, gy, gz) at the GLL node of its cell
  const int P = c->p, Nx = c->mdev.Nx, Ny = c->mdev.Ny, Nz = c->mdev.Nz;
  for (int gz = 0; gz < Nz; ++gz)
    for (int gy = 0; gy < Ny; ++gy)
      for (int gx = 0; gx < Nx; ++gx) {
        const int g3[3] = {gx, gy, gz};
        double x[3];
        if (c->general) {
          // trilinear cells: evaluate the map of the cell that owns the node
          double X8[8][3];
          int cidx[3], li[3];
          const int nc[3] = {c->nx, c->ny, c->nz};
          for (int d = 0; d < 3; ++d) {
            cidx[d] = std::min(g3[d] / P, nc[d] - 1);
            li[d] = g3[d] - cidx[d] * P;
          }
          for (int k = 0; k < 8; ++k) {
            const size_t vi = (size_t)(cidx[0] + (k & 1)) +
                              (size_t)(c->nx + 1) * ((cidx[1] + ((k >> 1) & 1)) + (size_t)(c->ny + 1) * (cidx[2] + ((k >> 2) & 1)));
            for (int d = 0; d < 3; ++d) X8[k][d] = c->vertices[3 * vi + d];
          }
          double xi[3];
          for (int d = 0; d < 3; ++d) xi[d] = c->gll[li[d]];
          for (int d = 0; d < 3; ++d) x[d] = 0.0;
          for (int k = 0; k < 8; ++k) {
            const double w = 0.125 * (1 + ((k & 1) ? 1 : -1) * xi[0]) * (1 + (((k >> 1) & 1) ? 1 : -1) * xi[1]) *
                             (1 + (((k >> 2) & 1) ? 1 : -1) * xi[2]);
            for (int d = 0; d < 3; ++d) x[d] += w * X8[k][d];
          }
        } else {
          for (int d = 0; d < 3; ++d) {
            const int cd = g3[d] / P, ld = g3[d] - cd * P;
            x[d] = c->box_lo[d] + c->box_h[d] * (cd + 0.5 * (1.0 + c->gll[ld]));
          }
        }
        for (int d = 0; d < 3; ++d) xyz[3 * (gx + (size_t)Nx * (gy + (size_t)Ny * gz)) + d] = x[d];
      }
  return FE_OK;
}
