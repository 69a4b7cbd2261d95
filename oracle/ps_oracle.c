/*
 * ps_oracle.c -- plain FP64 CPU oracle of the parareal + splitting method of
 * Arraras, Gaspar, Jimenez-Ciga, Portero, "Space-time parallel iterative
 * solvers for the integration of parabolic problems" (arXiv 2502.08370).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * reference that the CUDA path is compared against.  Only the tests, the
 * smoke check and the CPU-baseline leg of the benchmark may load it.  It
 * shares no code, header, table or helper with the CUDA library.
 *
 * What it computes, in the paper's order and notation:
 *   - model problem u_t = div(D grad u) - c u + f, u = 0 on the boundary
 *     (Sec. 2.1, eq. cont_problem), D = a(x) I with a nodal scalar a, or in 2-D
 *     the full tensor D = [[a, d12], [d12, a]] of Sec. 5.2 (domain-decomposition
 *     splitting only: the mixed derivatives give a 9-point stencil);
 *   - f(x, t) = src(x) src_t(t) + src2(x) src2_t(t) (two separable terms, enough
 *     for the manufactured solutions of Sec. 5);
 *   - method of lines with second-order finite differences on a uniform
 *     grid of interior nodes (Sec. 2.2, eq. semidisc_prob; Sec. 5);
 *   - dimensional splitting L_j u = (a u_{x_j})_{x_j} - c u / M (Sec. 2.1);
 *   - domain-decomposition splitting L_j u = div(rho_j a grad u) - rho_j c u
 *     with a partition of unity rho_j over overlapping boxes (Sec. 2.1,
 *     eq. partition_unity_M2 and the suboperator definition after it);
 *   - the fractional implicit Euler step (Sec. 2.2, eq. FIE_method);
 *   - the parareal iteration with G = FIE at step DeltaT and F = s FIE steps
 *     of step delta t (Sec. 3, the parareal recursion);
 *   - the Douglas-Rachford step (Sec. 2.2, eq. DR_method) and the pairing
 *     G = FIE, F = s DR steps (Parareal/FIE-DR, Sec. 4.2);
 *   - the discrete adjoint of the sequential fine solution (no counterpart in
 *     the paper; the transpose of the FIE steps above).
 *
 * Readings where the paper is silent (each one is also listed in the design
 * notes of the repository):
 *   - edge coefficient a_{i+1/2} = (a_i + a_{i+1}) / 2 from the nodal a;
 *   - full tensor: A_j is assembled from one quadratic form per grid cell, with D
 *     (the mean of its four nodal values) and rho_j taken at the cell centre, the
 *     x-differences of the cell's bottom and top edges, the y-differences of its
 *     left and right edges, and cell-averaged gradients in the d12 term.  Each
 *     cell's form is positive semidefinite when D is SPD, so every A_j is
 *     symmetric negative semidefinite, sum_j A_j = A, and the stencil has 9
 *     points (5 when d12 = 0);
 *   - DD weights rho_j evaluated at edge midpoints, so sum_j A_j = A;
 *   - the overlap ramp is cos^2 over an overlap of width beta centred on
 *     each core boundary (C^1, where the paper asks for C^infinity);
 *   - substep order x, y, z; DD colours (bx%2, by%2) = (0,0),(1,0),(0,1),(1,1);
 *   - the source is evaluated at the end time of each (sub)step;
 *   - correction evaluated as F + (G_new - G_old); stop at the first k >= 1
 *     with max_n ||U_n^k - U_n^{k-1}||_inf < tol, or at k = N.
 *
 * Arrays are dense, x fastest: U[(k*ny + j)*nx + i] over interior nodes,
 * a[(k*(ny+2) + j)*(nx+2) + i] over the grid including the boundary.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
  int dim;             /* 2 or 3 */
  int nx, ny, nz;      /* interior nodes per direction (nz = 1 in 2-D) */
  const double* a;     /* nodal diffusion incl. boundary; NULL means a = 1 */
  double c;            /* reaction coefficient (c >= 0) */
  const double* src;   /* spatial source on interior nodes; NULL means f = 0 */
  const double* src_t; /* time factor at fine times t_j = j*dt; NULL means 1 */
  int src_t_len;
  int split;           /* 0 = dimensional, 1 = domain decomposition (2-D) */
  int boxes_x, boxes_y;/* DD: boxes per direction */
  double overlap;      /* DD: overlap width beta (absolute, in [0,1] units) */
  const double* d12;   /* 2-D nodal off-diagonal diffusion incl. boundary; NULL means 0 */
  const double* src2;  /* second separable source term src2(x) src2_t(t); NULL means 0 */
  const double* src2_t;
  int src2_t_len;
} or_problem;

/* ------------------------------------------------------------------ */
/* grid helpers                                                        */
/* ------------------------------------------------------------------ */
static int nn(const or_problem* p, int d) { return d == 0 ? p->nx : d == 1 ? p->ny : p->nz; }
static double hh(const or_problem* p, int d) { return 1.0 / (nn(p, d) + 1); }
static long n_total(const or_problem* p) { return (long)p->nx * p->ny * (p->dim == 3 ? p->nz : 1); }
int or_num_substeps(const or_problem* p) {
  if (p->split == 0) return p->dim;
  return (p->boxes_x > 1 ? 2 : 1) * (p->boxes_y > 1 ? 2 : 1);
}

/* nodal coefficient at grid indices (i,j,k) in 0..n+1 (boundary included) */
static double a_node(const or_problem* p, int i, int j, int k) {
  if (!p->a) return 1.0;
  long nx2 = p->nx + 2, ny2 = p->ny + 2;
  if (p->dim == 2) k = 0;
  return p->a[((long)k * ny2 + j) * nx2 + i];
}

/* nodal off-diagonal coefficient at (i,j) in 0..n+1 (2-D) */
static double d12_node(const or_problem* p, int i, int j) {
  return p->d12 ? p->d12[(long)j * (p->nx + 2) + i] : 0.0;
}

/* ------------------------------------------------------------------ */
/* partition of unity (DD splitting, Sec. 2.1)                         */
/* ------------------------------------------------------------------ */
/* ramp across an overlap of width w centred at cb: 1 left, 0 right, cos^2 in between */
static double ramp_down(double x, double cb, double w) {
  double lo = cb - 0.5 * w, hi = cb + 0.5 * w;
  if (x <= lo) return 1.0;
  if (x >= hi) return 0.0;
  double s = cos(0.5 * M_PI * (x - lo) / w);
  return s * s;
}
/* 1-D partition function of box b out of B on [0,1]: cores [b/B, (b+1)/B] */
double or_phi1d(int b, int B, double w, double x) {
  if (B <= 1) return 1.0;
  double left = (b == 0) ? 1.0 : 1.0 - ramp_down(x, (double)b / B, w);
  double right = (b == B - 1) ? 1.0 : ramp_down(x, (double)(b + 1) / B, w);
  return left * right;
}
static int colour_of(const or_problem* p, int bx, int by) {
  int ncx = p->boxes_x > 1 ? 2 : 1;
  return (bx % 2) + ncx * (by % 2);
}
/* rho_colour(x, y) = sum of its boxes' products phi_bx(x) * phi_by(y) */
double or_rho(const or_problem* p, int colour, double x, double y) {
  double s = 0.0;
  for (int by = 0; by < p->boxes_y; ++by)
    for (int bx = 0; bx < p->boxes_x; ++bx)
      if (colour_of(p, bx, by) == colour)
        s += or_phi1d(bx, p->boxes_x, p->overlap, x) * or_phi1d(by, p->boxes_y, p->overlap, y);
  return s;
}
/* node range [lo, hi] (1-based interior) of 1-D box b: nodes touching a point
   (node or adjacent edge midpoint) where phi_b > 0.  The adjacent midpoints are
   also the centres of the cells around the node, which the full-tensor operator
   weights, so the range serves both operators. */
int or_box_range(const or_problem* p, int d, int b, int* lo, int* hi) {
  int n = nn(p, d), B = d == 0 ? p->boxes_x : p->boxes_y;
  double h = hh(p, d);
  *lo = n + 1; *hi = 0;
  for (int i = 1; i <= n; ++i) {
    double f = or_phi1d(b, B, p->overlap, i * h);
    double fl = or_phi1d(b, B, p->overlap, (i - 0.5) * h);
    double fr = or_phi1d(b, B, p->overlap, (i + 0.5) * h);
    if (f > 0.0 || fl > 0.0 || fr > 0.0) {
      if (i < *lo) *lo = i;
      if (i > *hi) *hi = i;
    }
  }
  return *hi >= *lo;
}

/* ------------------------------------------------------------------ */
/* operators A_j (method of lines, Sec. 2.2)                           */
/* ------------------------------------------------------------------ */
/* value of U at interior index (i,j,k) 1-based, zero on the boundary */
static double uval(const or_problem* p, const double* u, int i, int j, int k) {
  if (i < 1 || i > p->nx || j < 1 || j > p->ny) return 0.0;
  if (p->dim == 3 && (k < 1 || k > p->nz)) return 0.0;
  if (p->dim == 2) k = 1;
  return u[((long)(k - 1) * p->ny + (j - 1)) * p->nx + (i - 1)];
}
/* weight of edge between node (i,j,k) and its +e_d neighbour for substep m */
static double edge_weight(const or_problem* p, int m, int d, int i, int j, int k) {
  (void)k;
  if (p->split == 0) return d == m ? 1.0 : 0.0;
  double x = i * hh(p, 0), y = j * hh(p, 1);
  if (d == 0) x += 0.5 * hh(p, 0); else y += 0.5 * hh(p, 1);
  return or_rho(p, m, x, y);
}
static double node_reaction_weight(const or_problem* p, int m, int i, int j) {
  if (p->split == 0) return 1.0 / p->dim;
  return or_rho(p, m, i * hh(p, 0), j * hh(p, 1));
}
/* Full tensor D = [[a, d12], [d12, a]] (2-D): the quadratic form of cell (ci, cj), the
   cell with lower-left node (ci, cj), ci in 0..nx, cj in 0..ny, weighted by rho_m at its
   centre.  Corners 0 = (ci, cj), 1 = (ci+1, cj), 2 = (ci, cj+1), 3 = (ci+1, cj+1).  With
   the edge differences Dx_b = u1 - u0, Dx_t = u3 - u2, Dy_l = u2 - u0, Dy_r = u3 - u1 and
   the cell gradient (gx, gy) = ((Dx_b + Dx_t)/(2hx), (Dy_l + Dy_r)/(2hy)):
     Q(u, v) = d11 (Dx_b(u) Dx_b(v) + Dx_t(u) Dx_t(v)) / (2 hx^2)
             + d22 (Dy_l(u) Dy_l(v) + Dy_r(u) Dy_r(v)) / (2 hy^2)
             + d12 (gx(u) gy(v) + gx(v) gy(u)),
   the one-cell approximation of the integral of grad v . D grad u divided by the cell
   area.  K[p][q] = rho Q(e_q, e_p); (A_m u)_P = -sum over the cells at P of K[p][q] u_q. */
static void cell_form(const or_problem* p, int m, int ci, int cj, double K[4][4]) {
  double hx = hh(p, 0), hy = hh(p, 1);
  double rho = p->split == 0 ? 1.0 : or_rho(p, m, (ci + 0.5) * hx, (cj + 0.5) * hy);
  double d = 0.25 * (a_node(p, ci, cj, 0) + a_node(p, ci + 1, cj, 0) + a_node(p, ci, cj + 1, 0) +
                     a_node(p, ci + 1, cj + 1, 0));
  double b = 0.25 * (d12_node(p, ci, cj) + d12_node(p, ci + 1, cj) + d12_node(p, ci, cj + 1) +
                     d12_node(p, ci + 1, cj + 1));
  static const double ex_b[4] = {-1, 1, 0, 0}, ex_t[4] = {0, 0, -1, 1};
  static const double ey_l[4] = {-1, 0, 1, 0}, ey_r[4] = {0, -1, 0, 1};
  static const double gx[4] = {-0.5, 0.5, -0.5, 0.5}, gy[4] = {-0.5, -0.5, 0.5, 0.5};
  for (int r = 0; r < 4; ++r)
    for (int q = 0; q < 4; ++q) {
      double v = d * (ex_b[r] * ex_b[q] + ex_t[r] * ex_t[q]) / (2.0 * hx * hx) +
                 d * (ey_l[r] * ey_l[q] + ey_r[r] * ey_r[q]) / (2.0 * hy * hy) +
                 b * (gx[q] * gy[r] + gx[r] * gy[q]) / (hx * hy);
      K[r][q] = rho * v;
    }
}
/* (A_m u)_P without the reaction, full-tensor form, P = (i, j) interior */
static double tensor_apply(const or_problem* p, int m, const double* u, int i, int j) {
  double s = 0.0, K[4][4];
  for (int cj = j - 1; cj <= j; ++cj)
    for (int ci = i - 1; ci <= i; ++ci) {
      cell_form(p, m, ci, cj, K);
      int pl = (i - ci) + 2 * (j - cj);
      for (int q = 0; q < 4; ++q) s -= K[pl][q] * uval(p, u, ci + q % 2, cj + q / 2, 1);
    }
  return s;
}

/* out = A_m u (full grid) */
void or_apply_A(const or_problem* p, int m, const double* u, double* out) {
  int nz = p->dim == 3 ? p->nz : 1;
#pragma omp parallel for collapse(2) schedule(static)
  for (int k = 1; k <= nz; ++k)
    for (int j = 1; j <= p->ny; ++j)
      for (int i = 1; i <= p->nx; ++i) {
        int id[3] = {i, j, k};
        double uc = uval(p, u, i, j, k), s = 0.0;
        if (p->d12) {
          s = tensor_apply(p, m, u, i, j) - p->c * node_reaction_weight(p, m, i, j) * uc;
          out[(long)(j - 1) * p->nx + (i - 1)] = s;
          continue;
        }
        for (int d = 0; d < p->dim; ++d) {
          double h2 = hh(p, d) * hh(p, d);
          int ip[3] = {id[0], id[1], id[2]}, im[3] = {id[0], id[1], id[2]};
          ip[d] += 1; im[d] -= 1;
          double wp = edge_weight(p, m, d, i, j, k);
          double wm = edge_weight(p, m, d, im[0], im[1], im[2]);
          double ap = 0.5 * (a_node(p, i, j, k) + a_node(p, ip[0], ip[1], ip[2]));
          double am = 0.5 * (a_node(p, i, j, k) + a_node(p, im[0], im[1], im[2]));
          double up = uval(p, u, ip[0], ip[1], ip[2]), um = uval(p, u, im[0], im[1], im[2]);
          s += (wp * ap * (up - uc) - wm * am * (uc - um)) / h2;
        }
        s -= p->c * node_reaction_weight(p, m, i, j) * uc;
        out[((long)(k - 1) * p->ny + (j - 1)) * p->nx + (i - 1)] = s;
      }
}

/* ------------------------------------------------------------------ */
/* substep solves (I - tau A_m) x = b                                  */
/* ------------------------------------------------------------------ */
/* textbook Thomas algorithm: sub a[1..n-1], diag b[0..n-1], super c[0..n-2] */
static void thomas(int n, const double* lo, const double* di, const double* up, double* x,
                   double* cp, double* dp) {
  cp[0] = n > 1 ? up[0] / di[0] : 0.0;
  dp[0] = x[0] / di[0];
  for (int i = 1; i < n; ++i) {
    double den = di[i] - lo[i] * cp[i - 1];
    cp[i] = i < n - 1 ? up[i] / den : 0.0;
    dp[i] = (x[i] - lo[i] * dp[i - 1]) / den;
  }
  x[n - 1] = dp[n - 1];
  for (int i = n - 2; i >= 0; --i) x[i] = dp[i] - cp[i] * x[i + 1];
}

/* dimensional substep along direction m: one tridiagonal system per line.
   A line is the set of interior nodes that differ only in coordinate m; it is
   identified by its first node (coordinate m equal to 1). */
static void solve_dim(const or_problem* p, int m, double tau, double* u) {
  int n = nn(p, m);
  double h2 = hh(p, m) * hh(p, m);
  int nz = p->dim == 3 ? p->nz : 1;
  long stride = m == 0 ? 1 : m == 1 ? p->nx : (long)p->nx * p->ny;
#pragma omp parallel
  {
    double* lo = malloc(sizeof(double) * n);
    double* di = malloc(sizeof(double) * n);
    double* up = malloc(sizeof(double) * n);
    double* x = malloc(sizeof(double) * n);
    double* cp = malloc(sizeof(double) * n);
    double* dp = malloc(sizeof(double) * n);
#pragma omp for collapse(3) schedule(static)
    for (int k = 1; k <= nz; ++k)
      for (int j = 1; j <= p->ny; ++j)
        for (int i = 1; i <= p->nx; ++i) {
          int id[3] = {i, j, k};
          if (id[m] != 1) continue;
          long base = ((long)(k - 1) * p->ny + (j - 1)) * p->nx + (i - 1);
          for (int t = 0; t < n; ++t) {
            int c0[3] = {i, j, k}, cm[3], cq[3];
            c0[m] = t + 1;
            memcpy(cm, c0, sizeof cm); cm[m] -= 1;
            memcpy(cq, c0, sizeof cq); cq[m] += 1;
            double a0 = a_node(p, c0[0], c0[1], c0[2]);
            double am = 0.5 * (a0 + a_node(p, cm[0], cm[1], cm[2]));
            double ap = 0.5 * (a0 + a_node(p, cq[0], cq[1], cq[2]));
            di[t] = 1.0 + tau * (am + ap) / h2 + tau * p->c / p->dim;
            lo[t] = -tau * am / h2;
            up[t] = -tau * ap / h2;
            x[t] = u[base + t * stride];
          }
          thomas(n, lo, di, up, x, cp, dp);
          for (int t = 0; t < n; ++t) u[base + t * stride] = x[t];
        }
    free(lo); free(di); free(up); free(x); free(cp); free(dp);
  }
}

/* textbook banded Cholesky of an SPD matrix with half-bandwidth w.
   Band storage: B[i*(w+1) + (i-j)] holds entry (i, j) for i-w <= j <= i. */
static int band_cholesky(long n, int w, double* B) {
  for (long i = 0; i < n; ++i) {
    long j0 = i - w < 0 ? 0 : i - w;
    for (long j = j0; j <= i; ++j) {
      double s = B[i * (w + 1) + (i - j)];
      long k0 = (i - w > j - w ? i - w : j - w);
      if (k0 < 0) k0 = 0;
      for (long k = k0; k < j; ++k) s -= B[i * (w + 1) + (i - k)] * B[j * (w + 1) + (j - k)];
      if (j == i) {
        if (s <= 0.0) return -1;
        B[i * (w + 1)] = sqrt(s);
      } else {
        B[i * (w + 1) + (i - j)] = s / B[j * (w + 1)];
      }
    }
  }
  return 0;
}
static void band_cholesky_solve(long n, int w, const double* L, double* x) {
  for (long i = 0; i < n; ++i) {  /* L y = b */
    double s = x[i];
    long k0 = i - w < 0 ? 0 : i - w;
    for (long k = k0; k < i; ++k) s -= L[i * (w + 1) + (i - k)] * x[k];
    x[i] = s / L[i * (w + 1)];
  }
  for (long i = n - 1; i >= 0; --i) {  /* L^T x = y */
    double s = x[i];
    long k1 = i + w > n - 1 ? n - 1 : i + w;
    for (long k = i + 1; k <= k1; ++k) s -= L[k * (w + 1) + (k - i)] * x[k];
    x[i] = s / L[i * (w + 1)];
  }
}

/* DD substep for colour m: block-diagonal system, one block per box of the
   colour, identity rows elsewhere.  Each block is assembled from the edge
   weights and solved by banded Cholesky in the box's x-fastest ordering
   (half-bandwidth w, the box width; w + 1 for the full tensor, whose corner
   couplings (i-1, j-1) and (i+1, j-1) sit at offsets w + 1 and w - 1). */
static int solve_dd(const or_problem* p, int m, double tau, double* u) {
  double hx2 = hh(p, 0) * hh(p, 0), hy2 = hh(p, 1) * hh(p, 1);
  int nb = p->boxes_x * p->boxes_y;
  int err = 0;
#pragma omp parallel for schedule(dynamic) reduction(| : err)
  for (int b = 0; b < nb; ++b) {
    int bx = b % p->boxes_x, by = b / p->boxes_x;
    if (colour_of(p, bx, by) != m) continue;
    int x0, x1, y0, y1;
    if (!or_box_range(p, 0, bx, &x0, &x1) || !or_box_range(p, 1, by, &y0, &y1)) continue;
    int w = x1 - x0 + 1, hgt = y1 - y0 + 1;
    int bw = p->d12 ? w + 1 : w;
    long nloc = (long)w * hgt;
    double* B = calloc((size_t)nloc * (bw + 1), sizeof(double));
    double* x = malloc(sizeof(double) * nloc);
    for (int j = y0; j <= y1; ++j)
      for (int i = x0; i <= x1; ++i) {
        long r = (long)(j - y0) * w + (i - x0);
        x[r] = u[(long)(j - 1) * p->nx + (i - 1)];
        if (p->d12) {
          /* full tensor: row P = (i, j) of (I - tau A_m) from the forms of the four cells at P */
          B[r * (bw + 1)] = 1.0 + tau * p->c * node_reaction_weight(p, m, i, j);
          double K[4][4];
          for (int cj = j - 1; cj <= j; ++cj)
            for (int ci = i - 1; ci <= i; ++ci) {
              cell_form(p, m, ci, cj, K);
              int pl = (i - ci) + 2 * (j - cj);
              for (int q = 0; q < 4; ++q) {
                int qi = ci + q % 2, qj = cj + q / 2;
                if (qi < 1 || qi > p->nx || qj < 1 || qj > p->ny) continue; /* boundary: u = 0 */
                if (qi < x0 || qi > x1 || qj < y0 || qj > y1) {  /* couplings that leave the box */
                  if (K[pl][q] != 0.0) err |= 1;
                  continue;
                }
                long c = (long)(qj - y0) * w + (qi - x0);
                if (c <= r) B[r * (bw + 1) + (r - c)] += tau * K[pl][q];
              }
            }
          continue;
        }
        double a0 = a_node(p, i, j, 0);
        /* four edges: +x, -x, +y, -y */
        double wxp = edge_weight(p, m, 0, i, j, 0) * 0.5 * (a0 + a_node(p, i + 1, j, 0)) / hx2;
        double wxm = edge_weight(p, m, 0, i - 1, j, 0) * 0.5 * (a0 + a_node(p, i - 1, j, 0)) / hx2;
        double wyp = edge_weight(p, m, 1, i, j, 0) * 0.5 * (a0 + a_node(p, i, j + 1, 0)) / hy2;
        double wym = edge_weight(p, m, 1, i, j - 1, 0) * 0.5 * (a0 + a_node(p, i, j - 1, 0)) / hy2;
        B[r * (bw + 1)] = 1.0 + tau * (wxp + wxm + wyp + wym) + tau * p->c * node_reaction_weight(p, m, i, j);
        if (i > x0) B[r * (bw + 1) + 1] = -tau * wxm;
        if (j > y0) B[r * (bw + 1) + w] = -tau * wym;
        /* couplings that leave the box must vanish (or point at the boundary) */
        if (i == x0 && i > 1 && wxm != 0.0) err |= 1;
        if (i == x1 && i < p->nx && wxp != 0.0) err |= 1;
        if (j == y0 && j > 1 && wym != 0.0) err |= 1;
        if (j == y1 && j < p->ny && wyp != 0.0) err |= 1;
      }
    if (band_cholesky(nloc, bw, B) != 0) err |= 2;
    else {
      band_cholesky_solve(nloc, bw, B, x);
      for (int j = y0; j <= y1; ++j)
        for (int i = x0; i <= x1; ++i) u[(long)(j - 1) * p->nx + (i - 1)] = x[(long)(j - y0) * w + (i - x0)];
    }
    free(B); free(x);
  }
  return err ? -1 : 0;
}

int or_substep_solve(const or_problem* p, int m, double tau, double* u) {
  if (p->d12 && (p->split == 0 || p->dim != 2)) return -3; /* mixed terms: 2-D DD only */
  if (p->split == 0) { solve_dim(p, m, tau, u); return 0; }
  if (p->dim != 2) return -2;
  return solve_dd(p, m, tau, u);
}

/* ------------------------------------------------------------------ */
/* FIE step (eq. FIE_method) and propagators                           */
/* ------------------------------------------------------------------ */
static double time_factor_of(const double* tf, int len, int t_index) {
  if (!tf) return 1.0;
  if (t_index < 0 || t_index >= len) return NAN;
  return tf[t_index];
}
static double time_factor(const or_problem* p, int t_index) {
  return time_factor_of(p->src_t, p->src_t_len, t_index);
}
/* u += tau f(t_end), f = src src_t + src2 src2_t */
static void add_source(const or_problem* p, double tau, int t_end, double* u) {
  long nt = n_total(p);
  if (p->src) {
    double ft = time_factor(p, t_end);
    for (long i = 0; i < nt; ++i) u[i] += tau * p->src[i] * ft;
  }
  if (p->src2) {
    double ft = time_factor_of(p->src2_t, p->src2_t_len, t_end);
    for (long i = 0; i < nt; ++i) u[i] += tau * p->src2[i] * ft;
  }
}
/* u <- U_{n+1} of eq. FIE_method from U_n = u; source at fine time index t_end.
   reversed != 0 applies the substeps in the order M..1 (the transpose of a
   step, used by the adjoint). */
int or_fie_step(const or_problem* p, double tau, int t_end, int reversed, double* u) {
  add_source(p, tau, t_end, u);
  int M = or_num_substeps(p);
  for (int q = 0; q < M; ++q) {
    int m = reversed ? M - 1 - q : q;
    int rc = or_substep_solve(p, m, tau, u);
    if (rc) return rc;
  }
  return 0;
}
/* nsteps FIE steps of size tau; step q ends at fine time index t0 + (q+1)*tstride */
int or_propagate(const or_problem* p, double tau, int nsteps, int t0, int tstride, double* u) {
  for (int q = 0; q < nsteps; ++q) {
    int rc = or_fie_step(p, tau, t0 + (q + 1) * tstride, 0, u);
    if (rc) return rc;
  }
  return 0;
}

/* coarse propagator G over slice n: g FIE steps of DeltaT/g */
static int prop_G(const or_problem* p, double T, int N, int g, int s, int n, double* u) {
  return or_propagate(p, T / N / g, g, n * s, s / g, u);
}
/* fine propagator F^s over slice n: s FIE steps of dt = DeltaT/s */
static int prop_F(const or_problem* p, double T, int N, int s, int n, double* u) {
  return or_propagate(p, T / N / s, s, n * s, 1, u);
}

/* sequential fine solution at the coarse times: U[n] for n = 0..N */
int or_fine_sequential(const or_problem* p, double T, int N, int s, const double* u0, double* U) {
  long nt = n_total(p);
  memcpy(U, u0, sizeof(double) * nt);
  for (int n = 0; n < N; ++n) {
    memcpy(U + (n + 1) * nt, U + n * nt, sizeof(double) * nt);
    int rc = prop_F(p, T, N, s, n, U + (n + 1) * nt);
    if (rc) return rc;
  }
  return 0;
}
/* coarse-only sequential solution U[n] = G^n(u0) */
int or_coarse_sequential(const or_problem* p, double T, int N, int g, int s, const double* u0, double* U) {
  long nt = n_total(p);
  memcpy(U, u0, sizeof(double) * nt);
  for (int n = 0; n < N; ++n) {
    memcpy(U + (n + 1) * nt, U + n * nt, sizeof(double) * nt);
    int rc = prop_G(p, T, N, g, s, n, U + (n + 1) * nt);
    if (rc) return rc;
  }
  return 0;
}

/* Parareal (Sec. 3).  U holds (N+1)*nt values: on return U_n^k for the last k.
   hist[k-1] = max_{n} ||U_n^k - U_n^{k-1}||_inf.  Iterates k = 1, 2, ... and
   stops at the first k with hist < tol, or k = N, or k = max_iter.
   pG and pF are the problems whose splittings the coarse and fine propagators
   use (the same problem, or two DD decompositions of it as in Sec. 5.1's
   scalability experiment).  Returns 0 and *iters = k, or a negative code. */
/* fine propagator of slice n with method `fine`: 0 = FIE (eq. FIE_method), 1 = DR (eq. DR_method) */
int or_propagate_dr(const or_problem* p, double tau, int nsteps, int t0, int tstride, double* u);
static int prop_F_method(const or_problem* p, int fine, double T, int N, int s, int n, double* u) {
  if (fine == 1) return or_propagate_dr(p, T / N / s, s, n * s, 1, u);
  return prop_F(p, T, N, s, n, u);
}
int or_parareal_fine(const or_problem* pG, const or_problem* pF, int fine, double T, int N, int g, int s,
                     const double* u0, double tol, int max_iter, double* U, double* hist, int* iters);
int or_parareal2(const or_problem* pG, const or_problem* pF, double T, int N, int g, int s,
                 const double* u0, double tol, int max_iter, double* U, double* hist, int* iters) {
  return or_parareal_fine(pG, pF, 0, T, N, g, s, u0, tol, max_iter, U, hist, iters);
}
/* Parareal with G = FIE on pG and F = `fine` (0 FIE, 1 DR) on pF. */
int or_parareal_fine(const or_problem* pG, const or_problem* pF, int fine, double T, int N, int g, int s,
                     const double* u0, double tol, int max_iter, double* U, double* hist, int* iters) {
  if (fine != 0 && fine != 1) return -3;
  long nt = n_total(pF);
  if (g < 1 || s < 1 || N < 1 || s % g || n_total(pG) != nt) return -3;
  double* Fv = malloc(sizeof(double) * nt * N);
  double* Gold = malloc(sizeof(double) * nt * N);
  double* Unew = malloc(sizeof(double) * nt * (N + 1));
  double* gtmp = malloc(sizeof(double) * nt);
  int rc = or_coarse_sequential(pG, T, N, g, s, u0, U);   /* U^0 */
  int k = 0;
  if (max_iter > N) max_iter = N;
  while (!rc && k < max_iter) {
    ++k;
    for (int n = 0; n < N && !rc; ++n) {          /* F(U_n^{k-1}) and G(U_n^{k-1}) */
      memcpy(Fv + n * nt, U + n * nt, sizeof(double) * nt);
      rc |= prop_F_method(pF, fine, T, N, s, n, Fv + n * nt);
      memcpy(Gold + n * nt, U + n * nt, sizeof(double) * nt);
      rc |= prop_G(pG, T, N, g, s, n, Gold + n * nt);
    }
    memcpy(Unew, u0, sizeof(double) * nt);        /* U_0^k = P u0 */
    for (int n = 0; n < N && !rc; ++n) {          /* sequential correction */
      memcpy(gtmp, Unew + n * nt, sizeof(double) * nt);
      rc |= prop_G(pG, T, N, g, s, n, gtmp);
      for (long i = 0; i < nt; ++i)
        Unew[(n + 1) * nt + i] = Fv[n * nt + i] + (gtmp[i] - Gold[n * nt + i]);
    }
    double inc = 0.0;
    for (long i = nt; i < nt * (N + 1); ++i) {
      double d = fabs(Unew[i] - U[i]);
      if (d > inc || d != d) inc = d;
    }
    memcpy(U, Unew, sizeof(double) * nt * (N + 1));
    hist[k - 1] = inc;
    if (inc < tol) break;
  }
  *iters = k;
  free(Fv); free(Gold); free(Unew); free(gtmp);
  return rc;
}
int or_parareal(const or_problem* p, double T, int N, int g, int s, const double* u0, double tol,
                int max_iter, double* U, double* hist, int* iters) {
  return or_parareal2(p, p, T, N, g, s, u0, tol, max_iter, U, hist, iters);
}

/* ------------------------------------------------------------------ */
/* Douglas-Rachford step (eq. DR_method) and Parareal/FIE-DR (Sec. 4.2) */
/* ------------------------------------------------------------------ */
/* u <- U_{n+1} of eq. DR_method from U_n = u, source at fine time index t_end:
     U_{n,0} = (I + tau A) U_n + tau F_{n+1},   A = A_1 + ... + A_M,
     (I - tau A_j) U_{n,j} = U_{n,j-1} - tau A_j U_n,   j = 1..M,
     U_{n+1} = U_{n,M}. */
int or_dr_step(const or_problem* p, double tau, int t_end, double* u) {
  long nt = n_total(p);
  int M = or_num_substeps(p);
  double* AU = malloc(sizeof(double) * nt * M); /* A_j U_n, j = 1..M */
  double* v = malloc(sizeof(double) * nt);
  if (!AU || !v) { free(AU); free(v); return -4; }
  for (int j = 0; j < M; ++j) or_apply_A(p, j, u, AU + j * nt);
  for (long i = 0; i < nt; ++i) {
    double s = u[i];
    for (int j = 0; j < M; ++j) s += tau * AU[j * nt + i];
    v[i] = s;
  }
  add_source(p, tau, t_end, v);
  int rc = 0;
  for (int j = 0; j < M && !rc; ++j) {
    for (long i = 0; i < nt; ++i) v[i] -= tau * AU[j * nt + i];
    rc = or_substep_solve(p, j, tau, v);
  }
  if (!rc) memcpy(u, v, sizeof(double) * nt);
  free(AU); free(v);
  return rc;
}
/* nsteps DR steps of size tau; step q ends at fine time index t0 + (q+1)*tstride */
int or_propagate_dr(const or_problem* p, double tau, int nsteps, int t0, int tstride, double* u) {
  for (int q = 0; q < nsteps; ++q) {
    int rc = or_dr_step(p, tau, t0 + (q + 1) * tstride, u);
    if (rc) return rc;
  }
  return 0;
}
/* sequential fine solution with s DR steps per slice, at the coarse times */
int or_fine_sequential_dr(const or_problem* p, double T, int N, int s, const double* u0, double* U) {
  long nt = n_total(p);
  memcpy(U, u0, sizeof(double) * nt);
  for (int n = 0; n < N; ++n) {
    memcpy(U + (n + 1) * nt, U + n * nt, sizeof(double) * nt);
    int rc = or_propagate_dr(p, T / N / s, s, n * s, 1, U + (n + 1) * nt);
    if (rc) return rc;
  }
  return 0;
}

/* ------------------------------------------------------------------ */
/* discrete adjoint of the sequential fine solution                    */
/* ------------------------------------------------------------------ */
/* J = 1/2 sum_i (U_N[i] - target[i])^2 with U_N the sequential fine solution
   of N*s FIE steps of dt = T/(N s).  Returns J, dJ/du0 (interior) and dJ/da
   (nodal, boundary included).  Dimensional splitting only.  Every state is
   kept (memory N*s*M*nt doubles): for small grids only. */
int or_adjoint(const or_problem* p, double T, int N, int s, const double* u0, const double* target,
               double* J, double* grad_u0, double* grad_a) {
  if (p->split != 0) return -2;
  long nt = n_total(p);
  int M = or_num_substeps(p);
  long nsteps = (long)N * s;
  double dt = T / N / s;
  /* W[q][j] = state after substep j of step q, j = 0 is the input plus source */
  double* W = malloc(sizeof(double) * nt * (M + 1) * nsteps);
  if (!W) return -4;
  double* cur = malloc(sizeof(double) * nt);
  memcpy(cur, u0, sizeof(double) * nt);
  for (long q = 0; q < nsteps; ++q) {
    double* w0 = W + (q * (M + 1)) * nt;
    memcpy(w0, cur, sizeof(double) * nt);
    add_source(p, dt, (int)(q + 1), w0);
    for (int j = 1; j <= M; ++j) {
      double* wj = W + (q * (M + 1) + j) * nt;
      memcpy(wj, wj - nt, sizeof(double) * nt);
      solve_dim(p, j - 1, dt, wj);
    }
    memcpy(cur, W + (q * (M + 1) + M) * nt, sizeof(double) * nt);
  }
  double jj = 0.0;
  double* lam = malloc(sizeof(double) * nt);
  for (long i = 0; i < nt; ++i) { lam[i] = cur[i] - target[i]; jj += 0.5 * lam[i] * lam[i]; }
  *J = jj;
  long na = (long)(p->nx + 2) * (p->ny + 2) * (p->dim == 3 ? p->nz + 2 : 1);
  memset(grad_a, 0, sizeof(double) * na);
  long nx2 = p->nx + 2, ny2 = p->ny + 2;
  for (long q = nsteps - 1; q >= 0; --q) {
    for (int j = M; j >= 1; --j) {
      /* w_j = T_j^{-1} w_{j-1}; adjoint nu = T_j^{-T} lam = T_j^{-1} lam (T_j symmetric) */
      solve_dim(p, j - 1, dt, lam);
      const double* wj = W + (q * (M + 1) + j) * nt;
      int d = j - 1;
      double h2 = hh(p, d) * hh(p, d);
      int nz = p->dim == 3 ? p->nz : 1;
      /* dJ/da_e += dt * nu^T (dA_j/da_e) w_j = -dt (nu_q - nu_p)(w_q - w_p)/h^2,
         over every edge p -> q = p + e_d, boundary edges included */
      int lim[3] = {p->nx, p->ny, nz};
      for (int k = (p->dim == 3 ? 0 : 1); k <= (p->dim == 3 ? nz : 1); ++k)
        for (int jy = 0; jy <= p->ny; ++jy)
          for (int ix = 0; ix <= p->nx; ++ix) {
            int P[3] = {ix, jy, k}, Q[3] = {ix, jy, k};
            Q[d] += 1;
            /* the edge must lie along lines of interior nodes in the other directions */
            int ok = 1;
            for (int e = 0; e < p->dim; ++e) {
              if (e == d) { if (P[e] < 0 || Q[e] > lim[e] + 1) ok = 0; }
              else if (P[e] < 1 || P[e] > lim[e]) ok = 0;
            }
            if (!ok) continue;
            double np_ = uval(p, lam, P[0], P[1], P[2]), nq = uval(p, lam, Q[0], Q[1], Q[2]);
            double wp = uval(p, wj, P[0], P[1], P[2]), wq = uval(p, wj, Q[0], Q[1], Q[2]);
            double ge = -dt * (nq - np_) * (wq - wp) / h2;
            int kp = p->dim == 3 ? P[2] : 0, kq = p->dim == 3 ? Q[2] : 0;
            grad_a[((long)kp * ny2 + P[1]) * nx2 + P[0]] += 0.5 * ge;
            grad_a[((long)kq * ny2 + Q[1]) * nx2 + Q[0]] += 0.5 * ge;
          }
    }
  }
  memcpy(grad_u0, lam, sizeof(double) * nt);
  free(W); free(cur); free(lam);
  return 0;
}

int or_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
void or_set_num_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}
