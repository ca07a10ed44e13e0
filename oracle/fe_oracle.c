/*
 * fe_oracle.c -- plain FP64 CPU oracle for the finite-element operator
 *
 *     A = K + M^V,   K_IJ = int mu grad N_I . grad N_J,   M^V_IJ = int V N_I N_J
 *
 * discretised with degree-p Lagrange elements on Gauss-Lobatto-Legendre (GLL)
 * nodes over a structured hexahedral mesh (Sec. 2.1, the stiffness / mass
 * integrals; Sec. 2.2, the cell stiffness by quadrature and the weighted mass
 * N^T G N).  A is DEFINED with the tensor n_q-point quadrature rule, exactly as
 * the paper evaluates its cell integrals.
 *
 * THIS FILE IS TEST INFRASTRUCTURE.  Only the tests, the smoke check and the
 * CPU-baseline leg of the benchmark may load it.  It shares no code, header,
 * table or constant with the CUDA library: it computes its own quadrature
 * (root bracketing + bisection of Legendre polynomials), its own Lagrange
 * basis (barycentric form), its own trilinear geometry, forms dense cell
 * matrices by direct quadrature loops, and assembles A row by row into CSR.
 * There is deliberately no sum factorisation, no weight folding and no
 * blocking here: every formula is the textbook definition written out.
 *
 * Conventions (the oracle's own):
 *   reference cell [-1,1]^3, local node I = i1 + n_p*(i2 + n_p*i3),
 *   quadrature point Q = q1 + n_q*(q2 + n_q*q3), cell e = cx + nx*(cy + ny*cz),
 *   global node (gx,gy,gz) -> gx + Nx*(gy + Ny*gz), with Nx = nx*p + 1 for a
 *   Dirichlet box and Nx = nx*p (wrap-around) for a periodic box.
 *   Dirichlet: the constrained operator is P A P, P zeroing boundary nodes
 *   (Sec. 3.2.2: Dirichlet constraints have no master nodes, so the constrained
 *   values are simply set, here to zero).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_OK 0
#define OR_EINVAL 1
#define OR_ENOMEM 2
#define OR_EGEOM 3

typedef struct {
  int nx, ny, nz;
  int periodic;              /* 0: Dirichlet box, 1: periodic box */
  double lo[3], hi[3];
  const double* vertex_xyz;  /* NULL (uniform) or (nx+1)(ny+1)(nz+1)*3, x fastest */
} oracle_mesh;

/* ------------------------------------------------------------------------- */
/* 1D: Legendre polynomials and quadrature rules (Sec. 2.2, tensor quadrature) */
/* ------------------------------------------------------------------------- */

/* P_n(x) by the three-term recurrence (k+1) P_{k+1} = (2k+1) x P_k - k P_{k-1}. */
static double legendre(int n, double x) {
  if (n == 0) return 1.0;
  double pm = 1.0, pk = x;
  for (int k = 1; k < n; ++k) {
    double pn = ((2.0 * k + 1.0) * x * pk - k * pm) / (k + 1.0);
    pm = pk;
    pk = pn;
  }
  return pk;
}

/* P_n'(x) from the identity (x^2 - 1) P_n' = n (x P_n - P_{n-1}), |x| < 1. */
static double legendre_deriv(int n, double x) {
  if (n == 0) return 0.0;
  return n * (x * legendre(n, x) - legendre(n - 1, x)) / (x * x - 1.0);
}

typedef double (*scalar_fn)(int, double);

/* All roots of f(n, .) in (-1, 1): bracket sign changes on a fine grid, then
 * bisect each bracket down to adjacent doubles.  Returns the number found. */
static int roots_in_open_interval(scalar_fn f, int n, double* out, int max_out) {
  const int samples = 4000 * (n + 1);
  int count = 0;
  double a = -1.0 + 1e-13;
  double fa = f(n, a);
  for (int s = 1; s <= samples; ++s) {
    double b = (s == samples) ? 1.0 - 1e-13 : -1.0 + 2.0 * s / samples;
    double fb = f(n, b);
    if (fa == 0.0) {
      if (count < max_out) out[count] = a;
      ++count;
    } else if (fa * fb < 0.0) {
      double l = a, r = b, fl = fa;
      for (int it = 0; it < 200; ++it) {
        double m = 0.5 * (l + r);
        if (m == l || m == r) break;
        double fm = f(n, m);
        if (fm == 0.0) { l = r = m; break; }
        if (fl * fm < 0.0) { r = m; } else { l = m; fl = fm; }
      }
      if (count < max_out) out[count] = 0.5 * (l + r);
      ++count;
    }
    a = b;
    fa = fb;
  }
  return count;
}

/* Gauss-Legendre rule with n points: nodes are the roots of P_n, weights
 * w = 2 / ((1 - x^2) P_n'(x)^2).  Returns 0 on success. */
int oracle_gauss(int n, double* x, double* w) {
  if (n < 1 || n > 40) return OR_EINVAL;
  if (n == 1) { x[0] = 0.0; w[0] = 2.0; return OR_OK; }
  int c = roots_in_open_interval(legendre, n, x, n);
  if (c != n) return OR_EINVAL;
  for (int i = 0; i < n; ++i) {
    double d = legendre_deriv(n, x[i]);
    w[i] = 2.0 / ((1.0 - x[i] * x[i]) * d * d);
  }
  return OR_OK;
}

/* Gauss-Lobatto-Legendre rule with n >= 2 points: -1, +1 and the roots of
 * P_{n-1}'; weights w = 2 / (n (n-1) P_{n-1}(x)^2). */
int oracle_gll(int n, double* x, double* w) {
  if (n < 2 || n > 40) return OR_EINVAL;
  x[0] = -1.0;
  x[n - 1] = 1.0;
  if (n > 2) {
    int c = roots_in_open_interval(legendre_deriv, n - 1, x + 1, n - 2);
    if (c != n - 2) return OR_EINVAL;
  }
  for (int i = 0; i < n; ++i) {
    double pl = legendre(n - 1, x[i]);
    w[i] = 2.0 / (n * (n - 1.0) * pl * pl);
  }
  return OR_OK;
}

/* Barycentric Lagrange basis on nodes xn[0..n-1] at t: phi[j], dphi[j].
 * lambda_j = 1 / prod_{k!=j} (x_j - x_k).  Off the nodes:
 *   phi_j = l(t) lambda_j / (t - x_j),  l(t) = prod_k (t - x_k),
 *   phi_j' = phi_j * sum_{k != j} 1 / (t - x_k).
 * At a node x_i: phi_j = delta_ij, phi_j' = (lambda_j / lambda_i) / (x_i - x_j)
 * for j != i and phi_i' = sum_{k != i} 1 / (x_i - x_k). */
void oracle_lagrange(int n, const double* xn, double t, double* phi, double* dphi) {
  double lam[64];
  for (int j = 0; j < n; ++j) {
    double prod = 1.0;
    for (int k = 0; k < n; ++k)
      if (k != j) prod *= (xn[j] - xn[k]);
    lam[j] = 1.0 / prod;
  }
  int at = -1;
  for (int j = 0; j < n; ++j)
    if (t == xn[j]) at = j;
  if (at >= 0) {
    for (int j = 0; j < n; ++j) {
      phi[j] = (j == at) ? 1.0 : 0.0;
      if (j == at) {
        double s = 0.0;
        for (int k = 0; k < n; ++k)
          if (k != at) s += 1.0 / (xn[at] - xn[k]);
        dphi[j] = s;
      } else {
        dphi[j] = (lam[j] / lam[at]) / (xn[at] - xn[j]);
      }
    }
    return;
  }
  double l = 1.0;
  for (int k = 0; k < n; ++k) l *= (t - xn[k]);
  for (int j = 0; j < n; ++j) {
    phi[j] = l * lam[j] / (t - xn[j]);
    double s = 0.0;
    for (int k = 0; k < n; ++k)
      if (k != j) s += 1.0 / (t - xn[k]);
    dphi[j] = phi[j] * s;
  }
}

/* ------------------------------------------------------------------------- */
/* Mesh, DoF numbering, geometry                                              */
/* ------------------------------------------------------------------------- */

static int mesh_ok(const oracle_mesh* m, int p) {
  if (!m || p < 1 || p > 16) return 0;
  if (m->nx < 1 || m->ny < 1 || m->nz < 1) return 0;
  for (int d = 0; d < 3; ++d)
    if (!(m->hi[d] > m->lo[d])) return 0;
  return 1;
}

static long nodes_dir(const oracle_mesh* m, int p, int d) {
  int n = d == 0 ? m->nx : (d == 1 ? m->ny : m->nz);
  return (long)n * p + (m->periodic ? 0 : 1);
}

long oracle_num_dofs(const oracle_mesh* m, int p) {
  if (!mesh_ok(m, p)) return -1;
  return nodes_dir(m, p, 0) * nodes_dir(m, p, 1) * nodes_dir(m, p, 2);
}

long oracle_num_cells(const oracle_mesh* m) {
  return (long)m->nx * m->ny * m->nz;
}

/* Global index of local node (i1,i2,i3) of cell e: the Boolean map Q^(e)
 * (Sec. 2.2, Eq. for V = A U with the cell-to-subdomain map). */
static long cell_dof(const oracle_mesh* m, int p, long e, int i1, int i2, int i3) {
  long cx = e % m->nx, cy = (e / m->nx) % m->ny, cz = e / ((long)m->nx * m->ny);
  long Nx = nodes_dir(m, p, 0), Ny = nodes_dir(m, p, 1), Nz = nodes_dir(m, p, 2);
  long gx = cx * p + i1, gy = cy * p + i2, gz = cz * p + i3;
  if (m->periodic) { gx %= Nx; gy %= Ny; gz %= Nz; }
  return gx + Nx * (gy + Ny * gz);
}

int oracle_cell_dofs(const oracle_mesh* m, int p, long e, long* dofs) {
  if (!mesh_ok(m, p) || e < 0 || e >= oracle_num_cells(m)) return OR_EINVAL;
  int np = p + 1;
  for (int i3 = 0; i3 < np; ++i3)
    for (int i2 = 0; i2 < np; ++i2)
      for (int i1 = 0; i1 < np; ++i1)
        dofs[i1 + np * (i2 + np * i3)] = cell_dof(m, p, e, i1, i2, i3);
  return OR_OK;
}

/* 1 if the global node lies on the Dirichlet boundary. */
int oracle_is_constrained(const oracle_mesh* m, int p, long dof) {
  if (m->periodic) return 0;
  long Nx = nodes_dir(m, p, 0), Ny = nodes_dir(m, p, 1), Nz = nodes_dir(m, p, 2);
  long gx = dof % Nx, gy = (dof / Nx) % Ny, gz = dof / (Nx * Ny);
  return gx == 0 || gy == 0 || gz == 0 || gx == Nx - 1 || gy == Ny - 1 || gz == Nz - 1;
}

/* The 8 corner coordinates of cell e, corner index a + 2b + 4c. */
static void cell_corners(const oracle_mesh* m, long e, double X[8][3]) {
  long cx = e % m->nx, cy = (e / m->nx) % m->ny, cz = e / ((long)m->nx * m->ny);
  for (int c = 0; c < 2; ++c)
    for (int b = 0; b < 2; ++b)
      for (int a = 0; a < 2; ++a) {
        long vx = cx + a, vy = cy + b, vz = cz + c;
        int k = a + 2 * b + 4 * c;
        if (m->vertex_xyz) {
          long vi = vx + (m->nx + 1) * (vy + (long)(m->ny + 1) * vz);
          for (int d = 0; d < 3; ++d) X[k][d] = m->vertex_xyz[3 * vi + d];
        } else {
          long v[3] = {vx, vy, vz};
          int n[3] = {m->nx, m->ny, m->nz};
          for (int d = 0; d < 3; ++d)
            X[k][d] = m->lo[d] + (m->hi[d] - m->lo[d]) * (double)v[d] / (double)n[d];
        }
      }
}

/* Trilinear map x(xi) = sum_corners X_abc l_a(xi1) l_b(xi2) l_c(xi3), with
 * l_0 = (1 - t)/2, l_1 = (1 + t)/2, and its Jacobian J_ij = dx_i / dxi_j. */
static void trilinear(const double X[8][3], const double xi[3], double x[3], double J[3][3]) {
  for (int i = 0; i < 3; ++i) {
    x[i] = 0.0;
    for (int j = 0; j < 3; ++j) J[i][j] = 0.0;
  }
  for (int c = 0; c < 2; ++c)
    for (int b = 0; b < 2; ++b)
      for (int a = 0; a < 2; ++a) {
        double l1 = a ? 0.5 * (1 + xi[0]) : 0.5 * (1 - xi[0]);
        double l2 = b ? 0.5 * (1 + xi[1]) : 0.5 * (1 - xi[1]);
        double l3 = c ? 0.5 * (1 + xi[2]) : 0.5 * (1 - xi[2]);
        double d1 = a ? 0.5 : -0.5, d2 = b ? 0.5 : -0.5, d3 = c ? 0.5 : -0.5;
        const double* P = X[a + 2 * b + 4 * c];
        for (int i = 0; i < 3; ++i) {
          x[i] += P[i] * l1 * l2 * l3;
          J[i][0] += P[i] * d1 * l2 * l3;
          J[i][1] += P[i] * l1 * d2 * l3;
          J[i][2] += P[i] * l1 * l2 * d3;
        }
      }
}

/* det and inverse of a 3x3 matrix by cofactors. */
static double inv3(const double J[3][3], double Ji[3][3]) {
  double c00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
  double c01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
  double c02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
  double det = J[0][0] * c00 + J[0][1] * c01 + J[0][2] * c02;
  Ji[0][0] = c00 / det;
  Ji[1][0] = c01 / det;
  Ji[2][0] = c02 / det;
  Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
  Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
  Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
  Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
  Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
  Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
  return det;
}

/* ------------------------------------------------------------------------- */
/* Reference element tables                                                   */
/* ------------------------------------------------------------------------- */

typedef struct {
  int np, nq;
  double node[32];          /* GLL nodes (n_p) */
  double qx[32], qw[32];    /* quadrature points / weights (n_q) */
  double phi[32][32];       /* phi[q][i]  = l_i(xi_q)  */
  double dphi[32][32];      /* dphi[q][i] = l_i'(xi_q) */
} ref1d;

static int make_ref1d(int p, int nq, int quad_kind, ref1d* r) {
  if (p < 1 || p > 16 || nq < 1 || nq > 30) return OR_EINVAL;
  r->np = p + 1;
  r->nq = nq;
  double wn[32];
  if (oracle_gll(r->np, r->node, wn) != OR_OK) return OR_EINVAL;
  int st = quad_kind == 1 ? oracle_gll(nq, r->qx, r->qw) : oracle_gauss(nq, r->qx, r->qw);
  if (st != OR_OK) return OR_EINVAL;
  for (int q = 0; q < nq; ++q) oracle_lagrange(r->np, r->node, r->qx[q], r->phi[q], r->dphi[q]);
  return OR_OK;
}

/* Physical quadrature point coordinates, xyz[(e*nq^3 + Q)*3 + d]. */
int oracle_quad_points(const oracle_mesh* m, int p, int nq, int quad_kind, double* xyz) {
  if (!mesh_ok(m, p)) return OR_EINVAL;
  ref1d r;
  if (make_ref1d(p, nq, quad_kind, &r) != OR_OK) return OR_EINVAL;
  long E = oracle_num_cells(m);
  long nq3 = (long)nq * nq * nq;
#pragma omp parallel for schedule(static)
  for (long e = 0; e < E; ++e) {
    double X[8][3];
    cell_corners(m, e, X);
    for (int q3 = 0; q3 < nq; ++q3)
      for (int q2 = 0; q2 < nq; ++q2)
        for (int q1 = 0; q1 < nq; ++q1) {
          double xi[3] = {r.qx[q1], r.qx[q2], r.qx[q3]}, x[3], J[3][3];
          trilinear(X, xi, x, J);
          long Q = q1 + nq * (q2 + (long)nq * q3);
          for (int d = 0; d < 3; ++d) xyz[(e * nq3 + Q) * 3 + d] = x[d];
        }
  }
  return OR_OK;
}

/* ------------------------------------------------------------------------- */
/* Cell matrix by direct quadrature (Sec. 2.2: K^(e) by the n_q-point rule,   */
/* M^{kappa,(e)} = N^T G N with G_QQ = kappa det J w_Q)                        */
/* ------------------------------------------------------------------------- */

/* Per-point data of one cell, as the two factors of A^(e) = B^T W B:
 *   B[I][4Q + d] = (J^{-T} grad_xi N_I)_d (d = 0,1,2) and B[I][4Q + 3] = N_I,
 *   W[4Q + d]   = mu w_Q det J  (d < 3)  and W[4Q + 3] = V_Q w_Q det J,
 * all at the quadrature point xi_Q.  Then
 *   A_IJ = sum_Q w_Q det J [ mu (J^{-T} grad N_I).(J^{-T} grad N_J) + V_Q N_I N_J ]
 *        = sum_k B[I][k] W[k] B[J][k]. */
typedef struct {
  double* B;   /* n_p^3 x 4 n_q^3 */
  double* W;   /* 4 n_q^3 */
} cell_points;

static int cell_point_data(const oracle_mesh* m, const ref1d* r, long e, double mu,
                           const double* Vq_cell, cell_points* cp) {
  int np = r->np, nq = r->nq;
  long nq3 = (long)nq * nq * nq;
  double X[8][3];
  cell_corners(m, e, X);
  for (int q3 = 0; q3 < nq; ++q3)
    for (int q2 = 0; q2 < nq; ++q2)
      for (int q1 = 0; q1 < nq; ++q1) {
        long Q = q1 + nq * (q2 + (long)nq * q3);
        double xi[3] = {r->qx[q1], r->qx[q2], r->qx[q3]}, x[3], J[3][3], Ji[3][3];
        trilinear(X, xi, x, J);
        double det = inv3(J, Ji);
        if (!(det > 0.0)) return OR_EGEOM;
        double wdet = r->qw[q1] * r->qw[q2] * r->qw[q3] * det;
        for (int d = 0; d < 3; ++d) cp->W[4 * Q + d] = mu * wdet;
        cp->W[4 * Q + 3] = (Vq_cell ? Vq_cell[Q] : 0.0) * wdet;
        for (int i3 = 0; i3 < np; ++i3)
          for (int i2 = 0; i2 < np; ++i2)
            for (int i1 = 0; i1 < np; ++i1) {
              long I = i1 + np * (i2 + (long)np * i3);
              double g[3];
              g[0] = r->dphi[q1][i1] * r->phi[q2][i2] * r->phi[q3][i3];
              g[1] = r->phi[q1][i1] * r->dphi[q2][i2] * r->phi[q3][i3];
              g[2] = r->phi[q1][i1] * r->phi[q2][i2] * r->dphi[q3][i3];
              double* b = cp->B + I * 4 * nq3 + 4 * Q;
              /* (J^{-T} g)_d = sum_k (J^{-1})_{kd} g_k */
              for (int d = 0; d < 3; ++d) b[d] = Ji[0][d] * g[0] + Ji[1][d] * g[1] + Ji[2][d] * g[2];
              b[3] = r->phi[q1][i1] * r->phi[q2][i2] * r->phi[q3][i3];
            }
      }
  return OR_OK;
}

/* Rows [i0, i1) of the cell matrix A^(e) = K^(e) + M^{V,(e)} (B^T W B). */
static void cell_matrix_rows(const ref1d* r, const cell_points* cp, long i0, long i1,
                             double* out /* (i1-i0) x np3 */) {
  long np3 = (long)r->np * r->np * r->np, nk = 4L * r->nq * r->nq * r->nq;
  for (long I = i0; I < i1; ++I) {
    const double* bI = cp->B + I * nk;
    for (long J = 0; J < np3; ++J) {
      const double* bJ = cp->B + J * nk;
      double s = 0.0;
      for (long k = 0; k < nk; ++k) s += bI[k] * cp->W[k] * bJ[k];
      out[(I - i0) * np3 + J] = s;
    }
  }
}

static int alloc_points(const ref1d* r, cell_points* cp) {
  long np3 = (long)r->np * r->np * r->np, nk = 4L * r->nq * r->nq * r->nq;
  cp->B = (double*)malloc(sizeof(double) * np3 * nk);
  cp->W = (double*)malloc(sizeof(double) * nk);
  if (!cp->B || !cp->W) {
    free(cp->B); free(cp->W);
    return OR_ENOMEM;
  }
  return OR_OK;
}

static void free_points(cell_points* cp) {
  free(cp->B); free(cp->W);
}

/* Dense cell matrix A^(e) (n_p^3 x n_p^3, row-major), unconstrained. */
int oracle_cell_matrix(const oracle_mesh* m, int p, int nq, int quad_kind, double mu,
                       const double* Vq, long e, double* Ae) {
  if (!mesh_ok(m, p) || e < 0 || e >= oracle_num_cells(m)) return OR_EINVAL;
  ref1d r;
  if (make_ref1d(p, nq, quad_kind, &r) != OR_OK) return OR_EINVAL;
  cell_points cp;
  if (alloc_points(&r, &cp) != OR_OK) return OR_ENOMEM;
  long np3 = (long)r.np * r.np * r.np, nq3 = (long)nq * nq * nq;
  int st = cell_point_data(m, &r, e, mu, Vq ? Vq + e * nq3 : NULL, &cp);
  if (st == OR_OK) cell_matrix_rows(&r, &cp, 0, np3, Ae);
  free_points(&cp);
  return st;
}

/* ------------------------------------------------------------------------- */
/* Global assembly into CSR, row by row (Sec. 2.2, A = sum_e Q^T A^(e) Q,     */
/* constrained by C: Dirichlet rows and columns removed when `constrain`)     */
/* ------------------------------------------------------------------------- */

/* Cells incident to a global node and the node's local index in each. */
static int incident_cells(const oracle_mesh* m, int p, long dof, long* cells, int* locals) {
  long N[3] = {nodes_dir(m, p, 0), nodes_dir(m, p, 1), nodes_dir(m, p, 2)};
  int nc[3] = {m->nx, m->ny, m->nz};
  long g[3] = {dof % N[0], (dof / N[0]) % N[1], dof / (N[0] * N[1])};
  long cand_c[3][2];
  int cand_l[3][2], cnt[3];
  for (int d = 0; d < 3; ++d) {
    cnt[d] = 0;
    /* cell c holds node g iff c*p <= g' <= c*p + p for some g' equal to g (mod N if periodic) */
    for (long c = 0; c < nc[d]; ++c)
      for (int l = 0; l <= p; ++l) {
        long gg = c * p + l;
        if (m->periodic) gg %= N[d];
        if (gg == g[d]) {
          cand_c[d][cnt[d]] = c;
          cand_l[d][cnt[d]] = l;
          cnt[d]++;
        }
      }
  }
  int k = 0;
  int np = p + 1;
  for (int a = 0; a < cnt[0]; ++a)
    for (int b = 0; b < cnt[1]; ++b)
      for (int c = 0; c < cnt[2]; ++c) {
        cells[k] = cand_c[0][a] + m->nx * (cand_c[1][b] + (long)m->ny * cand_c[2][c]);
        locals[k] = cand_l[0][a] + np * (cand_l[1][b] + np * cand_l[2][c]);
        ++k;
      }
  return k;
}

/* Merge a cell-matrix row into a row accumulator.  pos[] (one slot per global
 * DoF, -1 when unused) maps a column to its slot in cols/vals. */
static long merge_row(const oracle_mesh* m, int p, int constrain, const long* gdofs, long np3,
                      const double* arow, long n, long* cols, double* vals, long* pos) {
  for (long J = 0; J < np3; ++J) {
    long c = gdofs[J];
    if (constrain && oracle_is_constrained(m, p, c)) continue;
    if (pos[c] < 0) { pos[c] = n; cols[n] = c; vals[n] = arow[J]; ++n; }
    else vals[pos[c]] += arow[J];
  }
  return n;
}

static void sort_row(long n, long* cols, double* vals) {
  for (long i = 1; i < n; ++i) {
    long c = cols[i];
    double v = vals[i];
    long j = i - 1;
    while (j >= 0 && cols[j] > c) { cols[j + 1] = cols[j]; vals[j + 1] = vals[j]; --j; }
    cols[j + 1] = c;
    vals[j + 1] = v;
  }
}

/* Assemble the global CSR matrix.  Two calls: first with col == NULL to get
 * rowptr (n_dofs + 1 entries, rowptr[n_dofs] = nnz), then with col/val sized
 * nnz.  All cell matrices are formed first (E * n_p^6 doubles held), then each
 * row sums the matching rows of the cell matrices of its incident cells. */
int oracle_assemble_csr(const oracle_mesh* m, int p, int nq, int quad_kind, double mu, const double* Vq,
                        int constrain, long* rowptr, long* col, double* val) {
  if (!mesh_ok(m, p)) return OR_EINVAL;
  ref1d r;
  if (make_ref1d(p, nq, quad_kind, &r) != OR_OK) return OR_EINVAL;
  long n = oracle_num_dofs(m, p), E = oracle_num_cells(m);
  long np3 = (long)r.np * r.np * r.np, nq3 = (long)nq * nq * nq;
  double* Ae = (double*)malloc(sizeof(double) * E * np3 * np3);
  long* gd = (long*)malloc(sizeof(long) * E * np3);
  if (!Ae || !gd) { free(Ae); free(gd); return OR_ENOMEM; }
  int status = OR_OK;
#pragma omp parallel
  {
    cell_points cp;
    if (alloc_points(&r, &cp) != OR_OK) {
#pragma omp critical
      status = OR_ENOMEM;
    } else {
#pragma omp for schedule(dynamic, 1)
      for (long e = 0; e < E; ++e) {
        oracle_cell_dofs(m, p, e, gd + e * np3);
        if (cell_point_data(m, &r, e, mu, Vq ? Vq + e * nq3 : NULL, &cp) != OR_OK) {
#pragma omp critical
          status = OR_EGEOM;
          continue;
        }
        cell_matrix_rows(&r, &cp, 0, np3, Ae + e * np3 * np3);
      }
      free_points(&cp);
    }
  }
  if (status == OR_OK) {
#pragma omp parallel
    {
      long* cols = (long*)malloc(sizeof(long) * 8 * np3);
      double* vals = (double*)malloc(sizeof(double) * 8 * np3);
      long* pos = (long*)malloc(sizeof(long) * n);
      for (long I = 0; I < n; ++I) pos[I] = -1;
      long cells[8];
      int locals[8];
#pragma omp for schedule(dynamic, 64)
      for (long I = 0; I < n; ++I) {
        long cnt = 0;
        if (!(constrain && oracle_is_constrained(m, p, I))) {
          int nc = incident_cells(m, p, I, cells, locals);
          for (int k = 0; k < nc; ++k)
            cnt = merge_row(m, p, constrain, gd + cells[k] * np3, np3,
                            Ae + cells[k] * np3 * np3 + locals[k] * np3, cnt, cols, vals, pos);
          for (long t = 0; t < cnt; ++t) pos[cols[t]] = -1;
          sort_row(cnt, cols, vals);
        }
        if (col == NULL) {
          rowptr[I + 1] = cnt;
        } else {
          for (long t = 0; t < cnt; ++t) {
            col[rowptr[I] + t] = cols[t];
            val[rowptr[I] + t] = vals[t];
          }
        }
      }
      free(cols);
      free(vals);
      free(pos);
    }
    if (col == NULL) {
      rowptr[0] = 0;
      for (long I = 0; I < n; ++I) rowptr[I + 1] += rowptr[I];
    }
  }
  free(Ae);
  free(gd);
  return status;
}

/* Rows rows[0..n_rows) of the global CSR matrix, assembled without forming
 * whole cell matrices: each row sums, over its incident cells, the one
 * matching row of the cell matrix (the same quadrature sums and the same
 * merge as oracle_assemble_csr, restricted to the requested rows).  Two calls
 * as for oracle_assemble_csr: first with col == NULL for rowptr (n_rows + 1
 * entries), then with col/val sized rowptr[n_rows].  Used to time the CSR x
 * block product on a bounded row block of a mesh too large to assemble. */
int oracle_assemble_rows_csr(const oracle_mesh* m, int p, int nq, int quad_kind, double mu, const double* Vq,
                             int constrain, const long* rows, long n_rows, long* rowptr, long* col, double* val) {
  if (!mesh_ok(m, p)) return OR_EINVAL;
  ref1d r;
  if (make_ref1d(p, nq, quad_kind, &r) != OR_OK) return OR_EINVAL;
  long n = oracle_num_dofs(m, p);
  long np3 = (long)r.np * r.np * r.np, nq3 = (long)nq * nq * nq;
  int status = OR_OK;
#pragma omp parallel
  {
    cell_points cp;
    int ok = alloc_points(&r, &cp) == OR_OK;
    double* rowbuf = (double*)malloc(sizeof(double) * np3);
    long* gdofs = (long*)malloc(sizeof(long) * np3);
    long* cols = (long*)malloc(sizeof(long) * 8 * np3);
    double* vals = (double*)malloc(sizeof(double) * 8 * np3);
    long* pos = (long*)malloc(sizeof(long) * n);
    long cells[8];
    int locals[8];
    if (!ok || !rowbuf || !gdofs || !cols || !vals || !pos) {
#pragma omp critical
      status = OR_ENOMEM;
    } else {
      for (long I = 0; I < n; ++I) pos[I] = -1;
#pragma omp for schedule(dynamic, 1)
      for (long k = 0; k < n_rows; ++k) {
        long I = rows[k], cnt = 0;
        if (I < 0 || I >= n) {
#pragma omp critical
          status = OR_EINVAL;
          continue;
        }
        if (!(constrain && oracle_is_constrained(m, p, I))) {
          int nc = incident_cells(m, p, I, cells, locals);
          for (int c = 0; c < nc; ++c) {
            if (cell_point_data(m, &r, cells[c], mu, Vq ? Vq + cells[c] * nq3 : NULL, &cp) != OR_OK) {
#pragma omp critical
              status = OR_EGEOM;
              break;
            }
            cell_matrix_rows(&r, &cp, locals[c], locals[c] + 1, rowbuf);
            oracle_cell_dofs(m, p, cells[c], gdofs);
            cnt = merge_row(m, p, constrain, gdofs, np3, rowbuf, cnt, cols, vals, pos);
          }
          for (long t = 0; t < cnt; ++t) pos[cols[t]] = -1;
          sort_row(cnt, cols, vals);
        }
        if (col == NULL) {
          rowptr[k + 1] = cnt;
        } else {
          for (long t = 0; t < cnt; ++t) {
            col[rowptr[k] + t] = cols[t];
            val[rowptr[k] + t] = vals[t];
          }
        }
      }
    }
    if (ok) free_points(&cp);
    free(rowbuf); free(gdofs); free(cols); free(vals); free(pos);
  }
  if (status == OR_OK && col == NULL) {
    rowptr[0] = 0;
    for (long k = 0; k < n_rows; ++k) rowptr[k + 1] += rowptr[k];
  }
  return status;
}

/* Y = A X for a CSR matrix and a DoF-major block X[dof * n_vec + v]. */
int oracle_csr_spmm(long n_rows, const long* rowptr, const long* col, const double* val,
                    const double* X, int n_vec, double* Y) {
#pragma omp parallel for schedule(dynamic, 64)
  for (long I = 0; I < n_rows; ++I) {
    double* y = Y + I * n_vec;
    for (int v = 0; v < n_vec; ++v) y[v] = 0.0;
    for (long t = rowptr[I]; t < rowptr[I + 1]; ++t) {
      double a = val[t];
      const double* x = X + col[t] * n_vec;
      for (int v = 0; v < n_vec; ++v) y[v] += a * x[v];
    }
  }
  return OR_OK;
}

/* Selected rows of Y = A X without storing A: row I of the (optionally
 * constrained) global matrix is sum_e Q^(e)T A^(e) Q^(e), so
 *   Y[I, :] = sum over cells e containing I, local index i of I in e, of
 *             sum_J A^(e)[i, J] X[dof(e, J), :]      (constrained J dropped).
 * Output Y_rows[k * n_vec + v] for rows[k]. */
int oracle_apply_rows(const oracle_mesh* m, int p, int nq, int quad_kind, double mu, const double* Vq,
                      int constrain, const double* X, int n_vec, const long* rows, long n_rows,
                      double* Y_rows) {
  if (!mesh_ok(m, p)) return OR_EINVAL;
  ref1d r;
  if (make_ref1d(p, nq, quad_kind, &r) != OR_OK) return OR_EINVAL;
  long np3 = (long)r.np * r.np * r.np, nq3 = (long)nq * nq * nq;
  long n = oracle_num_dofs(m, p);
  int status = OR_OK;
#pragma omp parallel
  {
    cell_points cp;
    int ok = alloc_points(&r, &cp) == OR_OK;
    double* rowbuf = (double*)malloc(sizeof(double) * np3);
    long* gdofs = (long*)malloc(sizeof(long) * np3);
    long cells[8];
    int locals[8];
    if (!ok || !rowbuf || !gdofs) {
#pragma omp critical
      status = OR_ENOMEM;
    } else {
#pragma omp for schedule(dynamic, 1)
      for (long k = 0; k < n_rows; ++k) {
        long I = rows[k];
        double* y = Y_rows + k * n_vec;
        for (int v = 0; v < n_vec; ++v) y[v] = 0.0;
        if (I < 0 || I >= n) {
#pragma omp critical
          status = OR_EINVAL;
          continue;
        }
        if (constrain && oracle_is_constrained(m, p, I)) continue;
        int nc = incident_cells(m, p, I, cells, locals);
        for (int c = 0; c < nc; ++c) {
          if (cell_point_data(m, &r, cells[c], mu, Vq ? Vq + cells[c] * nq3 : NULL, &cp) != OR_OK) {
#pragma omp critical
            status = OR_EGEOM;
            break;
          }
          cell_matrix_rows(&r, &cp, locals[c], locals[c] + 1, rowbuf);
          oracle_cell_dofs(m, p, cells[c], gdofs);
          for (long J = 0; J < np3; ++J) {
            if (constrain && oracle_is_constrained(m, p, gdofs[J])) continue;
            const double* x = X + gdofs[J] * n_vec;
            for (int v = 0; v < n_vec; ++v) y[v] += rowbuf[J] * x[v];
          }
        }
      }
    }
    if (ok) free_points(&cp);
    free(rowbuf); free(gdofs);
  }
  return status;
}

int oracle_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
