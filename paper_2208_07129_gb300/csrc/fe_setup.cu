// Host-side setup of libfe (FP64): 1D quadrature and basis tables, geometry
// at the quadrature points, cell colouring, and the C ABI calls that build
// and query a context.
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>

#include "fe_internal.h"

namespace fe {
namespace {

// Legendre P_n and P_n' at x by the three-term recurrence and the
// derivative identity (1 - x^2) P_n' = n (P_{n-1} - x P_n).
void legendre_pd(int n, double x, double* P, double* dP) {
  double p0 = 1.0, p1 = x;
  if (n == 0) { *P = 1.0; *dP = 0.0; return; }
  for (int k = 2; k <= n; ++k) {
    const double p2 = ((2 * k - 1) * x * p1 - (k - 1) * p0) / k;
    p0 = p1;
    p1 = p2;
  }
  *P = p1;
  *dP = n * (p0 - x * p1) / (1.0 - x * x);
}

// Gauss-Legendre: Newton on P_n from the asymptotic guesses cos(pi (i+3/4)/(n+1/2)).
void gauss_rule(int n, double* x, double* w) {
  for (int i = 0; i < n; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
    for (int it = 0; it < 100; ++it) {
      double P, dP;
      legendre_pd(n, z, &P, &dP);
      const double dz = P / dP;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    double P, dP;
    legendre_pd(n, z, &P, &dP);
    x[n - 1 - i] = z;
    w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dP * dP);
  }
}

// Gauss-Lobatto-Legendre: the end points and the zeros of P'_{n-1}, found by
// Newton with P'' from Legendre's equation, started at the Chebyshev-Lobatto
// points; weights 2 / (n (n-1) P_{n-1}^2).
void gll_rule(int n, double* x, double* w) {
  const int m = n - 1;
  for (int j = 0; j < n; ++j) {
    double z = -std::cos(M_PI * j / m);
    if (j > 0 && j < m) {
      for (int it = 0; it < 100; ++it) {
        double P, dP;
        legendre_pd(m, z, &P, &dP);
        const double d2P = (2.0 * z * dP - m * (m + 1.0) * P) / (1.0 - z * z);
        const double dz = dP / d2P;
        z -= dz;
        if (std::fabs(dz) < 1e-16) break;
      }
    }
    double P, dP;
    legendre_pd(m, z, &P, &dP);
    x[j] = z;
    w[j] = 2.0 / (n * (n - 1.0) * P * P);
  }
}

// Lagrange polynomial l_k on nodes xs[0..n-1] and its derivative at t:
//   l_k(t)  = prod_{j != k} (t - x_j) / (x_k - x_j)
//   l_k'(t) = sum_{m != k} 1/(x_k - x_m) prod_{j != k, m} (t - x_j) / (x_k - x_j)
double lagrange_value(const double* xs, int n, int k, double t) {
  double v = 1.0;
  for (int j = 0; j < n; ++j)
    if (j != k) v *= (t - xs[j]) / (xs[k] - xs[j]);
  return v;
}

double lagrange_deriv(const double* xs, int n, int k, double t) {
  double s = 0.0;
  for (int m = 0; m < n; ++m) {
    if (m == k) continue;
    double term = 1.0 / (xs[k] - xs[m]);
    for (int j = 0; j < n; ++j)
      if (j != k && j != m) term *= (t - xs[j]) / (xs[k] - xs[j]);
    s += term;
  }
  return s;
}

// Corner k = a + 2b + 4c of cell (cx, cy, cz).
void corner(const fe_ctx* c, int cx, int cy, int cz, int k, const fe_mesh_desc* md, double out[3]) {
  const int a = k & 1, b = (k >> 1) & 1, cc = (k >> 2) & 1;
  if (!c->vertices.empty()) {
    const size_t vi = (size_t)(cx + a) + (size_t)(c->nx + 1) * ((cy + b) + (size_t)(c->ny + 1) * (cz + cc));
    for (int d = 0; d < 3; ++d) out[d] = c->vertices[3 * vi + d];
  } else {
    const int idx[3] = {cx + a, cy + b, cz + cc};
    const int n[3] = {c->nx, c->ny, c->nz};
    for (int d = 0; d < 3; ++d) out[d] = md->lo[d] + (md->hi[d] - md->lo[d]) * idx[d] / n[d];
  }
}

// Position and Jacobian dx/dxi of the trilinear map at xi, written as the
// corner sum with hat functions (1 -+ xi)/2.
void trilinear_map(const double X[8][3], const double xi[3], double x[3], double J[3][3]) {
  for (int i = 0; i < 3; ++i) {
    x[i] = 0;
    J[i][0] = J[i][1] = J[i][2] = 0;
  }
  for (int k = 0; k < 8; ++k) {
    const double s0 = (k & 1) ? 1.0 : -1.0, s1 = ((k >> 1) & 1) ? 1.0 : -1.0, s2 = ((k >> 2) & 1) ? 1.0 : -1.0;
    const double h0 = 0.5 * (1 + s0 * xi[0]), h1 = 0.5 * (1 + s1 * xi[1]), h2 = 0.5 * (1 + s2 * xi[2]);
    for (int i = 0; i < 3; ++i) {
      x[i] += X[k][i] * h0 * h1 * h2;
      J[i][0] += X[k][i] * 0.5 * s0 * h1 * h2;
      J[i][1] += X[k][i] * h0 * 0.5 * s1 * h2;
      J[i][2] += X[k][i] * h0 * h1 * 0.5 * s2;
    }
  }
}

// mu det J J^-1 J^-T = mu adj(J) adj(J)^T / det J, adj the adjugate.
double metric(const double J[3][3], double mu, double G[6]) {
  double adj[3][3];
  adj[0][0] = J[1][1] * J[2][2] - J[1][2] * J[2][1];
  adj[0][1] = J[0][2] * J[2][1] - J[0][1] * J[2][2];
  adj[0][2] = J[0][1] * J[1][2] - J[0][2] * J[1][1];
  adj[1][0] = J[1][2] * J[2][0] - J[1][0] * J[2][2];
  adj[1][1] = J[0][0] * J[2][2] - J[0][2] * J[2][0];
  adj[1][2] = J[0][2] * J[1][0] - J[0][0] * J[1][2];
  adj[2][0] = J[1][0] * J[2][1] - J[1][1] * J[2][0];
  adj[2][1] = J[0][1] * J[2][0] - J[0][0] * J[2][1];
  adj[2][2] = J[0][0] * J[1][1] - J[0][1] * J[1][0];
  const double det = J[0][0] * adj[0][0] + J[0][1] * adj[1][0] + J[0][2] * adj[2][0];
  const int ij[6][2] = {{0, 0}, {0, 1}, {0, 2}, {1, 1}, {1, 2}, {2, 2}};
  for (int k = 0; k < 6; ++k) {
    const int s = ij[k][0], d = ij[k][1];
    G[k] = mu * (adj[s][0] * adj[d][0] + adj[s][1] * adj[d][1] + adj[s][2] * adj[d][2]) / det;
  }
  return det;
}

int dir_colors(int n, int periodic) { return (periodic && (n & 1) && n > 1) ? 3 : (n > 1 ? 2 : 1); }
int host_dir_color(int c, int n, int last_odd) { return (last_odd && c == n - 1) ? 2 : (c & 1); }

template <typename T>
cudaError_t upload(T** dst, const T* src, size_t n) {
  if (n == 0) { *dst = nullptr; return cudaSuccess; }
  cudaError_t e = cudaMalloc(dst, n * sizeof(T));
  if (e != cudaSuccess) return e;
  return cudaMemcpy(*dst, src, n * sizeof(T), cudaMemcpyHostToDevice);
}

template <typename T>
cudaError_t upload_as_float(float** dst, const std::vector<T>& src) {
  std::vector<float> f(src.begin(), src.end());
  return upload(dst, f.data(), f.size());
}

cudaError_t upload_as_ff(ff** dst, const std::vector<double>& src) {
  std::vector<ff> tmp(src.size());
  for (size_t i = 0; i < src.size(); ++i) tmp[i] = ff(src[i]);
  return upload(dst, tmp.data(), tmp.size());
}

}  // namespace

// GLL nodes and weights (n_p points), the quadrature rule, and the 1D
// tables: N (values at the points) and D~ (collocation derivative), plain
// and with sqrt(w) folded in (Sec. 3.2.4).  Needs c->np, c->nq, c->quad_kind.
void build_tables(fe_ctx* c) {
  const int np = c->np, nq = c->nq;
  c->gll.resize(np); c->wgll.resize(np); c->qx.resize(nq); c->qw.resize(nq);
  gll_rule(np, c->gll.data(), c->wgll.data());
  if (c->quad_kind == FE_QUAD_GAUSS) gauss_rule(nq, c->qx.data(), c->qw.data());
  else gll_rule(nq, c->qx.data(), c->qw.data());
  c->N1.resize(nq * np); c->D1.resize(nq * nq); c->Nf.resize(nq * np); c->Df.resize(nq * nq);
  for (int q = 0; q < nq; ++q) {
    for (int i = 0; i < np; ++i) {
      c->N1[q * np + i] = lagrange_value(c->gll.data(), np, i, c->qx[q]);
      c->Nf[q * np + i] = c->N1[q * np + i] * std::sqrt(c->qw[q]);
    }
    for (int k = 0; k < nq; ++k) {
      c->D1[q * nq + k] = lagrange_deriv(c->qx.data(), nq, k, c->qx[q]);
      c->Df[q * nq + k] = c->D1[q * nq + k] * std::sqrt(c->qw[q] / c->qw[k]);
    }
  }
}

double lagrange_1d(const double* xs, int n, int k, double t) { return lagrange_value(xs, n, k, t); }

cudaError_t upload_ints(int** dst, const std::vector<int>& src) { return upload(dst, src.data(), src.size()); }
cudaError_t upload_doubles(double** dst, const std::vector<double>& src) { return upload(dst, src.data(), src.size()); }
cudaError_t upload_floats(float** dst, const std::vector<double>& src) { return upload_as_float(dst, src); }
cudaError_t upload_ffs(ff** dst, const std::vector<double>& src) { return upload_as_ff(dst, src); }

// Geometry and per-point value coefficient uploads (FP64, FP32 and double-float copies).
cudaError_t upload_point_coeff(fe_ctx* c, const std::vector<double>& ptC) {
  cudaFree(c->d_ptC64);
  cudaFree(c->d_ptC32);
  cudaFree(c->d_ptCff);
  c->d_ptC64 = nullptr;
  c->d_ptC32 = nullptr;
  c->d_ptCff = nullptr;
  cudaError_t e = upload(&c->d_ptC64, ptC.data(), ptC.size());
  if (e == cudaSuccess) e = upload_as_float(&c->d_ptC32, ptC);
  if (e == cudaSuccess) e = upload_as_ff(&c->d_ptCff, ptC);
  // tcgen05 kernel, n_q = 8: per cell, plane q3 at a pitch of 72 floats and
  // its rows q2 >= 4 shifted by 4, so that the kernel's one bulk copy per
  // cell lands in a layout whose reads meet no bank conflict
  cudaFree(c->d_ptCtc);
  c->d_ptCtc = nullptr;
  if (e == cudaSuccess && !c->refined && c->nq == 8) {
    std::vector<double> skew(c->n_cells * (size_t)kTcCvWords, 0.0);
    for (size_t k = 0; k < c->n_cells; ++k)
      for (int q3 = 0; q3 < 8; ++q3)
        for (int q2 = 0; q2 < 8; ++q2)
          for (int q1 = 0; q1 < 8; ++q1)
            skew[k * kTcCvWords + 72 * q3 + 8 * q2 + (q2 >= 4 ? 4 : 0) + q1] = ptC[k * 512 + 64 * q3 + 8 * q2 + q1];
    e = upload_as_float(&c->d_ptCtc, skew);
  }
  return e;
}

// Diagonal mass by the (p+1)-point GLL rule on the element nodes (Sec. 4.3):
// node (i1, i2, i3) of cell e contributes w_i1 w_i2 w_i3 det J_e(node).
void build_gll_mass(fe_ctx* c) {
  if (!c->mass.empty()) return;
  const int P = c->p, np = c->np;
  const int Nx = c->mdev.Nx, Ny = c->mdev.Ny, Nz = c->mdev.Nz;
  fe_mesh_desc md{};
  c->mass.assign(c->n_dofs, 0.0);
  for (int cz = 0; cz < c->nz; ++cz)
    for (int cy = 0; cy < c->ny; ++cy)
      for (int cx = 0; cx < c->nx; ++cx) {
        double X[8][3];
        for (int k = 0; k < 8; ++k) {
          if (c->general) {
            corner(c, cx, cy, cz, k, &md, X[k]);
          } else {
            const int idx[3] = {cx + (k & 1), cy + ((k >> 1) & 1), cz + ((k >> 2) & 1)};
            for (int d = 0; d < 3; ++d) X[k][d] = c->box_lo[d] + c->box_h[d] * idx[d];
          }
        }
        for (int i3 = 0; i3 < np; ++i3)
          for (int i2 = 0; i2 < np; ++i2)
            for (int i1 = 0; i1 < np; ++i1) {
              const double xi[3] = {c->gll[i1], c->gll[i2], c->gll[i3]};
              double x[3], J[3][3];
              trilinear_map(X, xi, x, J);
              const double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                                 J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                                 J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
              int g[3] = {cx * P + i1, cy * P + i2, cz * P + i3};
              if (c->periodic) { g[0] %= Nx; g[1] %= Ny; g[2] %= Nz; }
              c->mass[g[0] + (size_t)Nx * (g[1] + (size_t)Ny * g[2])] +=
                  c->wgll[i1] * c->wgll[i2] * c->wgll[i3] * det;
            }
      }
  if (!c->periodic)
    for (int gz = 0; gz < Nz; ++gz)
      for (int gy = 0; gy < Ny; ++gy)
        for (int gx = 0; gx < Nx; ++gx)
          if (gx == 0 || gy == 0 || gz == 0 || gx == Nx - 1 || gy == Ny - 1 || gz == Nz - 1)
            c->mass[gx + (size_t)Nx * (gy + (size_t)Ny * gz)] = 1.0;
}

}  // namespace fe

using namespace fe;

static fe_status from_cuda(cudaError_t e) { return fe::cuda_status(e); }

extern "C" fe_status fe_setup(const fe_mesh_desc* mesh, int p, const fe_quad_desc* quad, double mu, fe_ctx** out) {
  if (!out) return FE_EINVAL;
  *out = nullptr;
  if (!mesh || !quad) return FE_EINVAL;
  if (mesh->nx < 1 || mesh->ny < 1 || mesh->nz < 1) return FE_EINVAL;
  if (mesh->bc != FE_BC_DIRICHLET0 && mesh->bc != FE_BC_PERIODIC) return FE_EINVAL;
  if (mesh->bc == FE_BC_PERIODIC && (mesh->nx < 2 || mesh->ny < 2 || mesh->nz < 2)) return FE_EINVAL;
  if (quad->kind != FE_QUAD_GAUSS && quad->kind != FE_QUAD_GLL) return FE_EINVAL;
  if (!std::isfinite(mu)) return FE_EINVAL;
  if (!mesh->vertex_xyz)
    for (int d = 0; d < 3; ++d)
      if (!(mesh->hi[d] > mesh->lo[d])) return FE_EINVAL;
  if (p < 1 || p > kMaxP || quad->n_q < p + 1 || quad->n_q > p + 3) return FE_EUNSUPPORTED;
  if (quad->kind == FE_QUAD_GLL && quad->n_q < 2) return FE_EINVAL;
  const long long ncell = (long long)mesh->nx * mesh->ny * mesh->nz;
  if (ncell > (1LL << 30)) return FE_EINVAL;

  fe_ctx* c = new (std::nothrow) fe_ctx();
  if (!c) return FE_ENOMEM;
  c->nx = mesh->nx; c->ny = mesh->ny; c->nz = mesh->nz;
  c->periodic = mesh->bc == FE_BC_PERIODIC;
  c->p = p; c->np = p + 1; c->nq = quad->n_q; c->quad_kind = quad->kind; c->mu = mu;
  c->general = mesh->vertex_xyz != nullptr;
  // FP64 tile measured on GB300: 8 vectors x 16 lines up to n_q = 8, 4 x 32 above;
  // FP32: even-odd line kernel, 8 x 32 up to n_q = 8, 4 x 64 above (two more
  // CTAs per SM in the 48 KB of shared memory that 4 vectors of n_q = 10 take)
  // double-float: 8 x 32 up to n_q = 8, 4 x 64 above
  c->fp32_variant = 3;
  if (quad->n_q >= 9) { c->vb64 = 4; c->nty64 = 32; c->vb32 = 4; c->nty32 = 64; c->vbdf = 4; c->ntydf = 64; }
  const int np = c->np, nq = c->nq;
  const int add = c->periodic ? 0 : 1;
  c->mdev.nx = c->nx; c->mdev.ny = c->ny; c->mdev.nz = c->nz;
  c->mdev.Nx = c->nx * p + add; c->mdev.Ny = c->ny * p + add; c->mdev.Nz = c->nz * p + add;
  c->mdev.periodic = c->periodic;
  c->n_dofs = (size_t)c->mdev.Nx * c->mdev.Ny * c->mdev.Nz;
  c->n_cells = (size_t)ncell;
  for (int d = 0; d < 3; ++d) {
    c->box_lo[d] = mesh->lo[d];
    c->box_h[d] = (mesh->hi[d] - mesh->lo[d]) / (d == 0 ? c->nx : (d == 1 ? c->ny : c->nz));
  }
  if (c->general) {
    const size_t nv = (size_t)(c->nx + 1) * (c->ny + 1) * (c->nz + 1) * 3;
    c->vertices.assign(mesh->vertex_xyz, mesh->vertex_xyz + nv);
  }

  // ---- 1D tables ----
  build_tables(c);

  // ---- geometry (FP64) ----
  const size_t E = c->n_cells, nq3 = (size_t)nq * nq * nq;
  c->detJ.resize(E * nq3);
  if (c->general) c->ptG.resize(E * 6 * nq3);
  else c->cellG.resize(E * 6);
  bool bad = false;
  for (int cz = 0; cz < c->nz && !bad; ++cz)
    for (int cy = 0; cy < c->ny && !bad; ++cy)
      for (int cx = 0; cx < c->nx && !bad; ++cx) {
        const size_t e = cx + (size_t)c->nx * (cy + (size_t)c->ny * cz);
        double X[8][3];
        for (int k = 0; k < 8; ++k) corner(c, cx, cy, cz, k, mesh, X[k]);
        if (!c->general) {
          double J[3][3] = {{(X[1][0] - X[0][0]) / 2, 0, 0}, {0, (X[2][1] - X[0][1]) / 2, 0},
                            {0, 0, (X[4][2] - X[0][2]) / 2}};
          double G[6];
          const double det = metric(J, mu, G);
          // an axis-aligned box: the metric is diagonal, which the cell
          // kernels without per-point geometry rely on
          if (G[1] != 0.0 || G[2] != 0.0 || G[4] != 0.0) bad = true;
          for (int k = 0; k < 6; ++k) c->cellG[e * 6 + k] = G[k];
          for (size_t Q = 0; Q < nq3; ++Q) c->detJ[e * nq3 + Q] = det;
        } else {
          for (int q3 = 0; q3 < nq; ++q3)
            for (int q2 = 0; q2 < nq; ++q2)
              for (int q1 = 0; q1 < nq; ++q1) {
                const size_t Q = q1 + (size_t)nq * (q2 + (size_t)nq * q3);
                const double xi[3] = {c->qx[q1], c->qx[q2], c->qx[q3]};
                double x[3], J[3][3], G[6];
                trilinear_map(X, xi, x, J);
                const double det = metric(J, mu, G);
                if (!(det > 0.0) || !std::isfinite(det)) bad = true;
                c->detJ[e * nq3 + Q] = det;
                for (int k = 0; k < 6; ++k) c->ptG[(e * 6 + k) * nq3 + Q] = G[k];
              }
        }
      }
  if (bad) { fe_destroy(c); return FE_EINVAL; }

  // ---- colours (conflict-free assembly) ----
  const int Cx = dir_colors(c->nx, c->periodic), Cy = dir_colors(c->ny, c->periodic),
            Cz = dir_colors(c->nz, c->periodic);
  c->mdev.cx_col = Cx; c->mdev.cy_col = Cy;
  c->mdev.last_odd_x = Cx == 3; c->mdev.last_odd_y = Cy == 3; c->mdev.last_odd_z = Cz == 3;
  c->colors.n_colors = Cx * Cy * Cz;
  std::vector<int> count(c->colors.n_colors, 0), col(E);
  for (int cz = 0; cz < c->nz; ++cz)
    for (int cy = 0; cy < c->ny; ++cy)
      for (int cx = 0; cx < c->nx; ++cx) {
        const size_t e = cx + (size_t)c->nx * (cy + (size_t)c->ny * cz);
        const int k = host_dir_color(cx, c->nx, Cx == 3) +
                      Cx * (host_dir_color(cy, c->ny, Cy == 3) + Cy * host_dir_color(cz, c->nz, Cz == 3));
        col[e] = k;
        count[k]++;
      }
  c->colors.offset.assign(c->colors.n_colors + 1, 0);
  for (int k = 0; k < c->colors.n_colors; ++k) c->colors.offset[k + 1] = c->colors.offset[k] + count[k];
  c->cells_by_color.resize(E);
  std::vector<int> fill(c->colors.offset.begin(), c->colors.offset.end() - 1);
  for (size_t e = 0; e < E; ++e) c->cells_by_color[fill[col[e]]++] = (int)e;

  // ---- uploads ----
  cudaError_t err = upload(&c->d_cells, c->cells_by_color.data(), E);
  if (err == cudaSuccess && !c->general) err = upload(&c->d_cellG64, c->cellG.data(), c->cellG.size());
  if (err == cudaSuccess && !c->general) err = upload_as_float(&c->d_cellG32, c->cellG);
  if (err == cudaSuccess && c->general) err = upload(&c->d_ptG64, c->ptG.data(), c->ptG.size());
  if (err == cudaSuccess && c->general) err = upload_as_float(&c->d_ptG32, c->ptG);
  if (err == cudaSuccess && !c->general) err = upload_as_ff(&c->d_cellGff, c->cellG);
  if (err == cudaSuccess && c->general) err = upload_as_ff(&c->d_ptGff, c->ptG);
  if (err == cudaSuccess) err = cudaMalloc(&c->d_status, sizeof(int));
  if (err == cudaSuccess) err = cudaMemset(c->d_status, 0, sizeof(int));
  if (err == cudaSuccess) {
    std::vector<double> zero(E * nq3, 0.0);
    err = upload_point_coeff(c, zero);
  }
  if (err == cudaSuccess) err = build_tc_images(c);
  if (err == cudaSuccess && E * (size_t)c->np * c->np * c->np <= kSmallSlots) {
    c->small_bytes = E * (size_t)c->np * c->np * c->np * 64 * sizeof(double);
    err = cudaMalloc(&c->d_small, c->small_bytes);
  }
  if (err != cudaSuccess) { fe_destroy(c); return from_cuda(err); }
  *out = c;
  return FE_OK;
}

extern "C" void fe_destroy(fe_ctx* c) {
  if (!c) return;
  cudaFree(c->d_cells); cudaFree(c->d_cellG64); cudaFree(c->d_ptG64); cudaFree(c->d_ptC64);
  cudaFree(c->d_cellG32); cudaFree(c->d_ptG32); cudaFree(c->d_ptC32); cudaFree(c->d_ptCtc); cudaFree(c->d_detJ);
  cudaFree(c->d_cellGff); cudaFree(c->d_ptGff); cudaFree(c->d_ptCff);
  cudaFree(c->d_status); cudaFree(c->d_stage);
  cudaFree(c->d_tcimg[0]); cudaFree(c->d_tcimg[1]); cudaFree(c->d_tcmask); cudaFree(c->d_tcq); cudaFree(c->d_small);
  if (c->copy_in) cudaStreamDestroy(c->copy_in);
  if (c->copy_out) cudaStreamDestroy(c->copy_out);
  for (cudaEvent_t ev : {c->ev_start, c->ev_in[0], c->ev_in[1], c->ev_comp[0], c->ev_comp[1], c->ev_out[0], c->ev_out[1]})
    if (ev) cudaEventDestroy(ev);
  free_solver_workspace(c);
  free_learned(c);
  free_eig(c);
  free_refined(c);
  delete c;
}

extern "C" size_t fe_num_dofs(const fe_ctx* c) { return c ? c->n_dofs : 0; }
extern "C" size_t fe_num_cells(const fe_ctx* c) { return c ? c->n_cells : 0; }
extern "C" int fe_num_quad_points_1d(const fe_ctx* c) { return c ? c->nq : 0; }

extern "C" fe_status fe_quadrature_points(const fe_ctx* c, double* xyz) {
  if (!c || !xyz) return FE_EINVAL;
  const int nq = c->nq;
  const size_t nq3 = (size_t)nq * nq * nq;
  if (c->refined) {   // axis-aligned boxes of the refined mesh, in cell order
    for (size_t e = 0; e < c->n_cells; ++e)
      for (int q3 = 0; q3 < nq; ++q3)
        for (int q2 = 0; q2 < nq; ++q2)
          for (int q1 = 0; q1 < nq; ++q1) {
            const size_t Q = q1 + (size_t)nq * (q2 + (size_t)nq * q3);
            const int qq[3] = {q1, q2, q3};
            for (int d = 0; d < 3; ++d)
              xyz[(e * nq3 + Q) * 3 + d] = c->cell_lo[3 * e + d] + 0.5 * (1.0 + c->qx[qq[d]]) * c->cell_h[3 * e + d];
          }
    return FE_OK;
  }
  fe_mesh_desc md{};
  md.nx = c->nx; md.ny = c->ny; md.nz = c->nz;
  for (int cz = 0; cz < c->nz; ++cz)
    for (int cy = 0; cy < c->ny; ++cy)
      for (int cx = 0; cx < c->nx; ++cx) {
        const size_t e = cx + (size_t)c->nx * (cy + (size_t)c->ny * cz);
        double X[8][3];
        for (int k = 0; k < 8; ++k) {
          if (c->general) {
            corner(c, cx, cy, cz, k, &md, X[k]);
          } else {
            const int idx[3] = {cx + (k & 1), cy + ((k >> 1) & 1), cz + ((k >> 2) & 1)};
            for (int d = 0; d < 3; ++d) X[k][d] = c->box_lo[d] + c->box_h[d] * idx[d];
          }
        }
        for (int q3 = 0; q3 < nq; ++q3)
          for (int q2 = 0; q2 < nq; ++q2)
            for (int q1 = 0; q1 < nq; ++q1) {
              const size_t Q = q1 + (size_t)nq * (q2 + (size_t)nq * q3);
              const double xi[3] = {c->qx[q1], c->qx[q2], c->qx[q3]};
              double x[3], J[3][3];
              trilinear_map(X, xi, x, J);
              for (int d = 0; d < 3; ++d) xyz[(e * nq3 + Q) * 3 + d] = x[d];
            }
      }
  return FE_OK;
}

extern "C" fe_status fe_set_potential(fe_ctx* c, const double* Vq) {
  if (!c) return FE_EINVAL;
  const size_t n = c->n_cells * (size_t)c->nq * c->nq * c->nq;
  std::vector<double> ptC(n, 0.0);
  if (Vq)
    for (size_t i = 0; i < n; ++i) {
      if (!std::isfinite(Vq[i])) return FE_EINVAL;
      ptC[i] = c->detJ[i] * Vq[i];
    }
  return from_cuda(upload_point_coeff(c, ptC));
}

extern "C" fe_status fe_set_mode(fe_ctx* c, fe_mode m) {
  if (!c) return FE_EINVAL;
  if (m != FE_FP64 && m != FE_FP32 && m != FE_TF32 && m != FE_BF16 && m != FE_TF32X3 && m != FE_DF64 &&
      m != FE_BF16S)
    return FE_EINVAL;
  c->mode = m;
  return FE_OK;
}

extern "C" fe_mode fe_get_mode(const fe_ctx* c) { return c ? c->mode : FE_FP64; }

extern "C" fe_status fe_set_tile(fe_ctx* c, fe_mode mode, int vectors_per_cta, int lines, int variant) {
  if (!c || vectors_per_cta < 1 || vectors_per_cta > 32 || (vectors_per_cta & (vectors_per_cta - 1)) != 0 ||
      lines < 1 || lines > 256 || variant < 0 || variant > 3)
    return FE_EINVAL;
  if (mode == FE_FP64) {
    if (variant >= 2) return FE_EINVAL;
    c->vb64 = vectors_per_cta;
    c->nty64 = lines;
    c->fp64_variant = variant;
  } else if (mode == FE_DF64) {
    if (variant != 0) return FE_EINVAL;
    c->vbdf = vectors_per_cta;
    c->ntydf = lines;
  } else if (mode == FE_FP32) {
    if (variant == 2 && c->nq > 8) return FE_EUNSUPPORTED;
    c->vb32 = vectors_per_cta;
    c->nty32 = lines;
    c->fp32_variant = variant;
  } else if (mode == FE_TF32 || mode == FE_BF16) {
    if (variant > 2) return FE_EINVAL;   // tensor-core tiles are fixed: only the kernel is chosen
    c->tc_variant = variant;
  } else if (mode == FE_BF16S) {
    if (variant != 0 && variant != 2) return FE_EINVAL;   // tcgen05 only
    c->tc_variant = variant;
  } else {
    return FE_EUNSUPPORTED;
  }
  return FE_OK;
}
