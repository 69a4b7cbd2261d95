// ps_dd.cu -- domain-decomposition splitting (Sec. 2.1): partition of unity over
// overlapping boxes, blocked subdomain factorisation and batched subdomain solves.
//
// Colour j's suboperator is L_j u = div(rho_j a grad u) - rho_j c u (Sec. 2.1).  With
// rho_j evaluated at edge midpoints, (I - tau A_j) is the identity outside the boxes of
// colour j and block diagonal over its boxes (Sec. 2.2: one independent subsystem per
// connected component).  Ordered line by line (the box's shorter extent w fastest, m lines),
// a box block is SPD block tridiagonal: tridiagonal w x w blocks T_k on the diagonal and
// diagonal couplings C_k = diag(c_k) between lines k-1 and k.  It is solved by block
// elimination with explicit inverses of the Schur complements,
//     S_0 = T_0,  S_k = T_k - C_k S_{k-1}^{-1} C_k,
//     y_k = S_k^{-1} (b_k - C_k y_{k-1}),   x_k = y_k - S_k^{-1} C_{k+1} x_{k+1},
// which is the same LU factorisation as the banded Cholesky of the oracle, grouped by lines:
// the dependent chain of a solve is m block steps instead of m*w scalar ones, and each step
// is a dense (w x w)(w x slices) product spread over a CTA.
//
// Factors per box and line k, contiguous: S_k^{-1} (w x w, column-major; symmetric),
// F_k = S_k^{-1} C_{k+1}^T (w x w, column-major), then the couplings of line k to line k-1:
// c_k (w), and for the full tensor also its neighbours c^-_k, c^+_k (C_k tridiagonal); each
// padded to 16 bytes.
//
// Full diffusion tensor D = [[a, d12], [d12, a]] (Sec. 5.2): the mixed derivatives couple
// every node to its eight neighbours ("nonadiagonal" systems).  The operator is assembled
// from one quadratic form per grid cell, with D the mean of the cell's four nodal values and
// rho_j taken at the cell centre: with the cell's edge differences and its mean gradient,
//     Q(u, v) = a/(2hx^2) (dx_b u dx_b v + dx_t u dx_t v) + a/(2hy^2) (dy_l u dy_l v + dy_r u dy_r v)
//             + d12 (g_x u g_y v + g_x v g_y u),
// (I - tau A_j) = I + tau sum over cells of rho_j Q (plus tau rho_j c on the diagonal).  Each
// cell's form is positive semidefinite when D is SPD, so every block stays SPD.  In the
// line-by-line order C_k becomes tridiagonal; S_k and F_k keep their dense form.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "ps_async.h"
#include "ps_dd.h"

namespace ps {
namespace {

// 1-D partition function of box b of B over [0,1]: cores [b/B, (b+1)/B], cos^2 ramps of
// width w centred on every interior core boundary (1 on the left of the ramp, 0 right).
__host__ __device__ inline double ramp_down(double x, double cb, double w) {
  const double lo = cb - 0.5 * w, hi = cb + 0.5 * w;
  if (x <= lo) return 1.0;
  if (x >= hi) return 0.0;
  const double s = cos(0.5 * M_PI * (x - lo) / w);
  return s * s;
}
__host__ __device__ inline double phi1d(int b, int B, double w, double x) {
  if (B <= 1) return 1.0;
  const double left = (b == 0) ? 1.0 : 1.0 - ramp_down(x, (double)b / B, w);
  const double right = (b == B - 1) ? 1.0 : ramp_down(x, (double)(b + 1) / B, w);
  return left * right;
}

// Assembled row r of (I - tau A_j) restricted to the box: the diagonal, the coupling to the
// previous position on the same line (lead), and the couplings to the previous line at the
// same position (other) and, for the full tensor, at the positions before and after it
// (other_m, other_p).  Couplings that leave the box are dropped (their weights vanish).
struct RowEntries {
  double diag, lead, other, other_m, other_p;
};
__device__ RowEntries assemble_row_5pt(const DDBox& bx, const DDGeomArgs& ga, int r) {
  int slow = r / bx.lead, fast = r - slow * bx.lead;
  int i, j;  // 1-based interior node
  if (bx.xfast) {
    i = bx.x0 + fast;
    j = bx.y0 + slow;
  } else {
    i = bx.x0 + slow;
    j = bx.y0 + fast;
  }
  const double hx = 1.0 / (ga.nx + 1), hy = 1.0 / (ga.ny + 1);
  const int nx2 = ga.nx + 2;
  auto A = [&](int ii, int jj) { return ga.a ? ga.a[(long long)jj * nx2 + ii] : 1.0; };
  auto chi = [&](double x, double y) {
    return phi1d(bx.bx, ga.Bx, ga.overlap, x) * phi1d(bx.by, ga.By, ga.overlap, y);
  };
  const double a0 = A(i, j);
  const double wxp = chi((i + 0.5) * hx, j * hy) * 0.5 * (a0 + A(i + 1, j)) / (hx * hx);
  const double wxm = chi((i - 0.5) * hx, j * hy) * 0.5 * (a0 + A(i - 1, j)) / (hx * hx);
  const double wyp = chi(i * hx, (j + 0.5) * hy) * 0.5 * (a0 + A(i, j + 1)) / (hy * hy);
  const double wym = chi(i * hx, (j - 0.5) * hy) * 0.5 * (a0 + A(i, j - 1)) / (hy * hy);
  RowEntries e;
  e.diag = 1.0 + ga.tau * (wxp + wxm + wyp + wym) + ga.tau * ga.c * chi(i * hx, j * hy);
  if (bx.xfast) {
    e.lead = fast > 0 ? -ga.tau * wxm : 0.0;
    e.other = slow > 0 ? -ga.tau * wym : 0.0;
  } else {
    e.lead = fast > 0 ? -ga.tau * wym : 0.0;
    e.other = slow > 0 ? -ga.tau * wxm : 0.0;
  }
  e.other_m = e.other_p = 0.0;
  return e;
}

// Weights of cell (ci, cj) (lower-left node; 0..nx, 0..ny, boundary nodes included) in the
// full-tensor form: rho a / (2 hx^2), rho a / (2 hy^2), rho d12 / (hx hy), with a and d12 the
// means of the cell's four nodal values and rho the box weight at the cell centre.
struct CellW {
  double ax, ay, g;
};
__device__ CellW cell_weights(const DDBox& bx, const DDGeomArgs& ga, int ci, int cj, double hx, double hy) {
  const int nx2 = ga.nx + 2;
  auto mean4 = [&](const double* f) {
    if (!f) return 1.0;
    const long long i0 = (long long)cj * nx2 + ci;
    return 0.25 * (f[i0] + f[i0 + 1] + f[i0 + nx2] + f[i0 + nx2 + 1]);
  };
  const double rho = phi1d(bx.bx, ga.Bx, ga.overlap, (ci + 0.5) * hx) * phi1d(bx.by, ga.By, ga.overlap, (cj + 0.5) * hy);
  const double a = mean4(ga.a);
  const double b = ga.d12 ? mean4(ga.d12) : 0.0;
  CellW w;
  w.ax = rho * a / (2.0 * hx * hx);
  w.ay = rho * a / (2.0 * hy * hy);
  w.g = rho * b / (hx * hy);
  return w;
}

// Full-tensor row of node P = (i, j): the four cells around P (SW, SE, NW, NE) each add their
// form's entries.  With (ax, ay, g) of a cell and P at its corner, the diagonal takes
// ax + ay + g/2 from SW and NE and ax + ay - g/2 from SE and NW; the edge neighbours take
// -ax (W: from SW and NW) or -ay (S: from SW and SE); the corner neighbours take -g/2 (SW)
// and +g/2 (SE from cell SE, NW from cell NW).  Rows of (I - tau A_j) carry these times tau.
__device__ RowEntries assemble_row_full(const DDBox& bx, const DDGeomArgs& ga, int r) {
  const int slow = r / bx.lead, fast = r - slow * bx.lead;
  int i, j;
  if (bx.xfast) {
    i = bx.x0 + fast;
    j = bx.y0 + slow;
  } else {
    i = bx.x0 + slow;
    j = bx.y0 + fast;
  }
  const double hx = 1.0 / (ga.nx + 1), hy = 1.0 / (ga.ny + 1);
  const CellW sw = cell_weights(bx, ga, i - 1, j - 1, hx, hy), se = cell_weights(bx, ga, i, j - 1, hx, hy);
  const CellW nw = cell_weights(bx, ga, i - 1, j, hx, hy), ne = cell_weights(bx, ga, i, j, hx, hy);
  const double t = ga.tau;
  const double rho0 = phi1d(bx.bx, ga.Bx, ga.overlap, i * hx) * phi1d(bx.by, ga.By, ga.overlap, j * hy);
  RowEntries e;
  e.diag = 1.0 + t * ((sw.ax + sw.ay + 0.5 * sw.g) + (se.ax + se.ay - 0.5 * se.g) + (nw.ax + nw.ay - 0.5 * nw.g) +
                      (ne.ax + ne.ay + 0.5 * ne.g)) +
           t * ga.c * rho0;
  const double W = -t * (sw.ax + nw.ax), Sv = -t * (sw.ay + se.ay);
  const double cSW = -t * 0.5 * sw.g, cSE = t * 0.5 * se.g, cNW = t * 0.5 * nw.g;
  const bool first_pos = fast == 0, last_pos = fast == bx.lead - 1, first_line = slow == 0;
  if (bx.xfast) {  // positions along x, lines along y: previous line = (., j - 1)
    e.lead = first_pos ? 0.0 : W;
    e.other = first_line ? 0.0 : Sv;
    e.other_m = (first_line || first_pos) ? 0.0 : cSW;
    e.other_p = (first_line || last_pos) ? 0.0 : cSE;
  } else {  // positions along y, lines along x: previous line = (i - 1, .)
    e.lead = first_pos ? 0.0 : Sv;
    e.other = first_line ? 0.0 : W;
    e.other_m = (first_line || first_pos) ? 0.0 : cSW;
    e.other_p = (first_line || last_pos) ? 0.0 : cNW;
  }
  return e;
}

__device__ __forceinline__ RowEntries assemble_row(const DDBox& bx, const DDGeomArgs& ga, int r) {
  return ga.full ? assemble_row_full(bx, ga, r) : assemble_row_5pt(bx, ga, r);
}

// Entries of the box block: line k, position i (0-based, w positions per line).
__device__ __forceinline__ int box_row(const DDBox& bx, int k, int i) { return k * bx.lead + i; }

// Node (0-based index into a slice) of line k, position i.
__device__ __forceinline__ long long line_node(const DDBox& bx, int nx, int k, int i) {
  const int gx = bx.xfast ? bx.x0 + i : bx.x0 + k;
  const int gy = bx.xfast ? bx.y0 + k : bx.y0 + i;
  return (long long)(gy - 1) * nx + (gx - 1);
}

__host__ __device__ inline long long dd_sq(int w) { return ((long long)w * w + 1) & ~1LL; }
__host__ __device__ inline long long dd_vec(int w) { return (w + 1) & ~1; }
// one line's record: S_k^{-1}, F_k, then c_k (and c^-_k, c^+_k for the full tensor)
__host__ __device__ inline long long dd_line_stride(int w, int full) { return 2 * dd_sq(w) + (full ? 3 : 1) * dd_vec(w); }

// The factorisation holds one w x w Schur complement and ten w-vectors in shared memory, and
// the solve runs one thread per line position (at most 192).
constexpr int kMaxLead = 160;
constexpr int kFactorVecs = 10;

// ---------------------------------------------------------------------------------------
// a1 (DD): one CTA per box.  The Schur complement of the current line lives in shared
// memory; it is inverted in place by Gauss-Jordan elimination without pivoting (SPD), its
// inverse stored, and the next line's complement formed from it.  *status = 1 on a
// non-positive pivot (the blocks are SPD, so only on bad input).
//     S_k = T_k - C_k S_{k-1}^{-1} C_k^T,   F_k = S_k^{-1} C_{k+1}^T
// With the five-point operator C_k = diag(c_k) and the product is formed in place; for the
// full tensor C_k is tridiagonal and entry (i, j) of C_k S_{k-1}^{-1} C_k^T sums nine terms
// of S_{k-1}^{-1}, read from its stored copy (global memory, written by this CTA).
// Shared memory: A (w x w, row-major), then kFactorVecs w-vectors.
template <bool FULL>
__global__ void __launch_bounds__(512) dd_factor_kernel(const DDBox* __restrict__ boxes, DDGeomArgs ga,
                                                        double* __restrict__ fac, int* status) {
  const DDBox bx = boxes[blockIdx.x];
  const int w = bx.lead, m = bx.n / w;
  extern __shared__ double sm[];
  double* A = sm;
  double* rs = A + w * w;  // pivot row / pivot
  double* cp = rs + w;     // pivot column
  double* dg = cp + w;     // diagonal of T_k
  double* ld = dg + w;     // sub-diagonal of T_k (entry (i, i-1))
  double* k0 = ld + w;     // C_k: coupling of line k to line k-1, same position
  double* km = k0 + w;     //      ... position - 1 (full tensor)
  double* kp = km + w;     //      ... position + 1 (full tensor)
  double* n0 = kp + w;     // C_{k+1}, same layout (for F_k)
  double* nm = n0 + w;
  double* np = nm + w;
  __shared__ double s_inv;
  const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + ty * blockDim.x, nthr = blockDim.x * blockDim.y;
  double* base = fac + bx.offset;
  const long long ls = dd_line_stride(w, FULL), sq = dd_sq(w), vec = dd_vec(w);
  for (int k = 0; k < m; ++k) {
    double* Sinv = base + k * ls;
    double* Fk = Sinv + sq;
    double* ck = Sinv + 2 * sq;  // c_k, then (full tensor) c^-_k, c^+_k
    for (int e = tid; e < w; e += nthr) {
      const RowEntries re = assemble_row(bx, ga, box_row(bx, k, e));
      dg[e] = re.diag;
      ld[e] = re.lead;
      k0[e] = re.other;
      ck[e] = re.other;
      if (FULL) {
        km[e] = re.other_m;
        kp[e] = re.other_p;
        ck[vec + e] = re.other_m;
        ck[2 * vec + e] = re.other_p;
      }
    }
    __syncthreads();
    // S_k = T_k - C_k S_{k-1}^{-1} C_k^T   (A holds S_{k-1}^{-1}; full tensor: its stored copy)
    const double* Pg = base + (k - 1) * ls;  // S_{k-1}^{-1}, column-major, symmetric
    for (int i = ty; i < w; i += blockDim.y)
      for (int j = tx; j < w; j += blockDim.x) {
        double t = (i == j) ? dg[i] : (j == i - 1 ? ld[i] : (i == j - 1 ? ld[j] : 0.0));
        if (k > 0) {
          if (FULL) {
            double acc = 0.0;
            for (int da = -1; da <= 1; ++da) {
              const int a = i + da;
              if (a < 0 || a >= w) continue;
              const double cia = da < 0 ? km[i] : (da == 0 ? k0[i] : kp[i]);
              if (cia == 0.0) continue;
              double row = 0.0;
              for (int db = -1; db <= 1; ++db) {
                const int b = j + db;
                if (b < 0 || b >= w) continue;
                const double cjb = db < 0 ? km[j] : (db == 0 ? k0[j] : kp[j]);
                row = fma(Pg[(long long)b * w + a], cjb, row);
              }
              acc = fma(cia, row, acc);
            }
            t -= acc;
          } else {
            t -= k0[i] * A[i * w + j] * k0[j];
          }
        }
        A[i * w + j] = t;
      }
    __syncthreads();
    for (int p = 0; p < w; ++p) {
      for (int e = tid; e < w; e += nthr) {
        rs[e] = A[p * w + e];
        cp[e] = A[e * w + p];
      }
      __syncthreads();
      if (tid == 0) {
        const double piv = rs[p];
        if (!(piv > 0.0)) atomicExch(status, 1);
        s_inv = 1.0 / (piv > 0.0 ? piv : 1.0);
      }
      __syncthreads();
      const double inv = s_inv;
      for (int e = tid; e < w; e += nthr) rs[e] *= inv;
      __syncthreads();
      for (int i = ty; i < w; i += blockDim.y) {
        const double ci = cp[i];
        for (int j = tx; j < w; j += blockDim.x) {
          double v;
          if (i == p) v = (j == p) ? inv : rs[j];
          else if (j == p) v = -ci * inv;
          else v = fma(-ci, rs[j], A[i * w + j]);
          A[i * w + j] = v;
        }
      }
      __syncthreads();
    }
    // S_k^{-1}, column-major
    for (int i = ty; i < w; i += blockDim.y)
      for (int j = tx; j < w; j += blockDim.x) Sinv[(long long)j * w + i] = A[i * w + j];
    // C_{k+1} and F_k = S_k^{-1} C_{k+1}^T, column-major
    for (int e = tid; e < w; e += nthr) {
      if (k + 1 < m) {
        const RowEntries re = assemble_row(bx, ga, box_row(bx, k + 1, e));
        n0[e] = re.other;
        nm[e] = re.other_m;
        np[e] = re.other_p;
      } else {
        n0[e] = nm[e] = np[e] = 0.0;
      }
    }
    __syncthreads();
    for (int i = ty; i < w; i += blockDim.y)
      for (int j = tx; j < w; j += blockDim.x) {
        double f;
        if (FULL) {
          // sum over b of S_k^{-1}[i][b] C_{k+1}[j][b], b = j - 1, j, j + 1
          f = A[i * w + j] * n0[j];
          if (j > 0) f = fma(A[i * w + j - 1], nm[j], f);
          if (j + 1 < w) f = fma(A[i * w + j + 1], np[j], f);
        } else {
          f = A[i * w + j] * n0[j];
        }
        Fk[(long long)j * w + i] = f;
      }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------------------
// a3 (DD): block forward and backward substitution of one box for S slices, in place in the
// state array.  One thread per position of a line (w <= blockDim.x); each thread keeps two
// partial sums per slice (2S independent FMA chains).  The m matrices S_k^{-1} of the forward
// pass and the m - 1 matrices F_k of the backward pass stream through shared memory in
// chunks of kChunk columns: two buffers, bulk copies completing on one mbarrier each, the
// copy of chunk g + 2 issued as soon as chunk g has been consumed, so the stream runs ahead
// across block steps.  Waits are bounded: on a timeout the CTA sets *err = 1, waits (again
// bounded) for its copies in flight and returns.
constexpr int kChunk = 32;

struct DDChunk {
  const double* src;
  int j0, cols;  // first column, columns used
  uint32_t bytes;
};

// Chunk g of the stream: forward matrices k = 0..m-1, then backward ones k = m-2..0.
__device__ __forceinline__ DDChunk dd_chunk(const double* base, long long ls, long long sq, int w, int m, int nch,
                                            long long g) {
  const long long mat = g / nch;
  const int c = (int)(g - mat * nch);
  const double* M = mat < m ? base + mat * ls : base + (long long)(2 * m - 2 - mat) * ls + sq;
  DDChunk ch;
  ch.j0 = c * kChunk;
  ch.cols = min(kChunk, w - ch.j0);
  // an even column count keeps the size a multiple of 16 bytes when w is odd; the extra column
  // lies inside the line's record (padding, F_k or c_k) and is not used
  const int cols_even = (ch.cols + 1) & ~1;
  ch.src = M + (long long)ch.j0 * w;
  ch.bytes = (uint32_t)((long long)cols_even * w * sizeof(double));
  return ch;
}

template <int S, bool FULL>
__global__ void __launch_bounds__(192) dd_solve_kernel(const DDBox* __restrict__ boxes, int nx, long long nt,
                                                       const double* __restrict__ fac, double* state, int nslices,
                                                       int ld_buf, int* err) {
  const DDBox bx = boxes[blockIdx.x];
  const int w = bx.lead, m = bx.n / w;
  const int s0 = blockIdx.y * S;
  const int ns = min(S, nslices - s0);
  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw);  // two barriers, 128 bytes reserved
  double* buf0 = reinterpret_cast<double*>(smem_raw + 128);
  double* bufs[2] = {buf0, buf0 + (size_t)kChunk * ld_buf};
  double* t = buf0 + 2 * (size_t)kChunk * ld_buf;  // S x w
  double* v = t + S * w;                           // S x w
  __shared__ int s_ok;
  const int r = threadIdx.x;
  const bool act = r < w;
  const double* base = fac + bx.offset;
  const long long ls = dd_line_stride(w, FULL), sq = dd_sq(w), vec = dd_vec(w);
  const int nch = (w + kChunk - 1) / kChunk;
  const long long total = (long long)(2 * m - 1) * nch;
  if (r == 0) {
    s_ok = *reinterpret_cast<volatile int*>(err) ? 0 : 1;
    if (s_ok) {
      mbar_init(&bar[0], 1);
      mbar_init(&bar[1], 1);
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
      for (long long g = 0; g < 2 && g < total; ++g) {
        const DDChunk ch = dd_chunk(base, ls, sq, w, m, nch, g);
        mbar_expect_tx(&bar[g], ch.bytes);
        bulk_load(bufs[g], ch.src, ch.bytes, &bar[g]);
      }
    }
  }
  __syncthreads();
  if (!s_ok) return;
  double* st[S];
#pragma unroll
  for (int q = 0; q < S; ++q) st[q] = state + (long long)(s0 + (q < ns ? q : 0)) * nt;
  long long g = 0;  // next chunk of the stream
  // consumes the nch chunks of one matrix: acc += M t (sign +1) or acc -= M t (sign -1);
  // returns false (uniformly) when a copy did not arrive in time
  auto matvec = [&](const double* vec, double sign, double* a0, double* a1) -> bool {
    for (int c = 0; c < nch; ++c, ++g) {
      const int b = (int)(g & 1);
      if (r == 0) s_ok = mbar_wait(&bar[b], (uint32_t)((g >> 1) & 1)) ? 1 : 0;
      __syncthreads();
      if (!s_ok) return false;
      const double* M = bufs[b];
      const int j0 = c * kChunk, cols = min(kChunk, w - j0);
      if (act) {
        int jj = 0;
#pragma unroll 4
        for (; jj + 1 < cols; jj += 2) {
          const double d0 = sign * M[(size_t)jj * w + r], d1 = sign * M[(size_t)(jj + 1) * w + r];
#pragma unroll
          for (int q = 0; q < S; ++q) {
            a0[q] = fma(d0, vec[q * w + j0 + jj], a0[q]);
            a1[q] = fma(d1, vec[q * w + j0 + jj + 1], a1[q]);
          }
        }
        if (jj < cols) {
          const double d0 = sign * M[(size_t)jj * w + r];
#pragma unroll
          for (int q = 0; q < S; ++q) a0[q] = fma(d0, vec[q * w + j0 + jj], a0[q]);
        }
      }
      __syncthreads();  // buffer b consumed
      if (r == 0 && g + 2 < total) {
        fence_async_smem();
        const DDChunk ch = dd_chunk(base, ls, sq, w, m, nch, g + 2);
        mbar_expect_tx(&bar[b], ch.bytes);
        bulk_load(bufs[b], ch.src, ch.bytes, &bar[b]);
      }
    }
    return true;
  };
  bool ok = true;
  // forward: y_k = S_k^{-1} (b_k - C_k y_{k-1})
  for (int k = 0; k < m && ok; ++k) {
    const long long node = act ? line_node(bx, nx, k, r) : 0;
    // the full tensor's C_k reads y_{k-1} of the neighbouring positions: wait for all of v
    if (FULL && k > 0) __syncthreads();
    if (act) {
      const double c = base[k * ls + 2 * sq + r];
      const double cm = FULL ? base[k * ls + 2 * sq + vec + r] : 0.0;
      const double cpl = FULL ? base[k * ls + 2 * sq + 2 * vec + r] : 0.0;
#pragma unroll
      for (int q = 0; q < S; ++q)
        if (q < ns) {
          // explicit FMA: the same rounding in every instance of the kernel (any S), so the
          // solve of a slice does not depend on how many slices share its CTA
          const double b = st[q][node];
          double tv = k > 0 ? fma(-c, v[q * w + r], b) : b;
          if (FULL && k > 0) {
            if (r > 0) tv = fma(-cm, v[q * w + r - 1], tv);
            if (r + 1 < w) tv = fma(-cpl, v[q * w + r + 1], tv);
          }
          t[q * w + r] = tv;
        }
    }
    double a0[S], a1[S];
#pragma unroll
    for (int q = 0; q < S; ++q) a0[q] = a1[q] = 0.0;
    ok = matvec(t, 1.0, a0, a1);  // starts with a barrier: t is complete
    if (ok && act) {
      // v[., r] is read only by this thread in the next right-hand side
#pragma unroll
      for (int q = 0; q < S; ++q)
        if (q < ns) {
          const double y = a0[q] + a1[q];
          v[q * w + r] = y;
          st[q][node] = y;
        }
    }
  }
  // backward: x_{m-1} = y_{m-1} (in v and in the state); x_k = y_k - F_k x_{k+1}
  for (int k = m - 2; k >= 0 && ok; --k) {
    const long long node = act ? line_node(bx, nx, k, r) : 0;
    double a0[S], a1[S];
#pragma unroll
    for (int q = 0; q < S; ++q) {
      a0[q] = (act && q < ns) ? st[q][node] : 0.0;
      a1[q] = 0.0;
    }
    __syncthreads();  // v holds x_{k+1} of every position
    ok = matvec(v, -1.0, a0, a1);
    if (ok && act) {
#pragma unroll
      for (int q = 0; q < S; ++q)
        if (q < ns) {
          const double x = a0[q] + a1[q];
          v[q * w + r] = x;
          st[q][node] = x;
        }
    }
  }
  if (!ok && r == 0) {
    atomicExch(err, 1);
    // the copies still in flight land in this CTA's shared memory: wait for them (bounded)
    for (long long h = g; h < g + 2 && h < total; ++h) mbar_wait(&bar[h & 1], (uint32_t)((h >> 1) & 1));
  }
}

// out = in + tau (src src_t + src2 src2_t) (all nodes, nslices states); out may alias in.
__global__ void dd_rhs_kernel(const double* in, double* out, long long total, long long nt, SourceArgs sa) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    double v = in[i];
    if (sa.src) {
      const long long sl = i / nt;
      const long long ti = sa.t0 + sl * sa.tstride;
      const double ft = sa.src_t ? sa.src_t[ti] : 1.0;
      v = v + sa.tau * sa.src[i - sl * nt] * ft;
      if (sa.src2) {
        const double ft2 = sa.src2_t ? sa.src2_t[ti] : 1.0;
        v = v + sa.tau * sa.src2[i - sl * nt] * ft2;
      }
    }
    out[i] = v;
  }
}

__global__ void dd_correct_kernel(long long nt, const double* __restrict__ g, CorrArgs ca) {
  double my = 0.0, nrm = 0.0;
  bool bad = false;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nt; i += (long long)gridDim.x * blockDim.x) {
    const double gi = g[i];
    if (ca.mode == 1) {
      const double unew = ca.Fout[i] + (gi - ca.Gold[i]);
      my = fmax(my, fabs(unew - ca.U_next[i]));
      nrm = fmax(nrm, fabs(unew));
      if (!isfinite(unew)) bad = true;
      ca.Gold[i] = gi;
      ca.U_next[i] = unew;
    } else {
      if (!isfinite(gi)) bad = true;
      ca.Gold[i] = gi;
      ca.U_next[i] = gi;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    my = fmax(my, __shfl_xor_sync(0xffffffffu, my, o));
    nrm = fmax(nrm, __shfl_xor_sync(0xffffffffu, nrm, o));
  }
  if ((threadIdx.x & 31) == 0 && my > 0.0) atomicMax(ca.inc, (unsigned long long)__double_as_longlong(my));
  if ((threadIdx.x & 31) == 0 && ca.slice_stats) {
    if (my > 0.0) atomicMax(ca.slice_stats, (unsigned long long)__double_as_longlong(my));
    if (nrm > 0.0) atomicMax(ca.slice_stats + 1, (unsigned long long)__double_as_longlong(nrm));
  }
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicExch(ca.nonfinite, 1);
}

}  // namespace

// Node range [lo, hi] (1-based) of 1-D box b: nodes at which phi_b is positive at the node
// or at an adjacent edge midpoint.
static bool box_range(int n, int b, int B, double w, int* lo, int* hi) {
  const double h = 1.0 / (n + 1);
  *lo = n + 1;
  *hi = 0;
  for (int i = 1; i <= n; ++i) {
    if (phi1d(b, B, w, i * h) > 0.0 || phi1d(b, B, w, (i - 0.5) * h) > 0.0 || phi1d(b, B, w, (i + 0.5) * h) > 0.0) {
      *lo = std::min(*lo, i);
      *hi = std::max(*hi, i);
    }
  }
  return *hi >= *lo;
}

void dd_plan(const Geom& g, const ps_dd_params& dd, bool full, DDPlan& plan) {
  PS_REQUIRE(g.dim == 2, "DD splitting is 2-D");
  plan.full = full ? 1 : 0;
  const int Bx = dd.boxes[0], By = dd.boxes[1];
  const int ncx = Bx > 1 ? 2 : 1;
  plan.M = ncx * (By > 1 ? 2 : 1);
  plan.colours.assign(plan.M, {});
  std::vector<std::pair<int, int>> rx(Bx), ry(By);
  for (int b = 0; b < Bx; ++b)
    if (!box_range(g.n[0], b, Bx, dd.overlap, &rx[b].first, &rx[b].second)) rx[b] = {1, 0};
  for (int b = 0; b < By; ++b)
    if (!box_range(g.n[1], b, By, dd.overlap, &ry[b].first, &ry[b].second)) ry[b] = {1, 0};
  // boxes of one colour must not touch: the overlap must be narrower than a core
  for (int b = 2; b < Bx; ++b)
    PS_REQUIRE(rx[b].first > rx[b - 2].second + 1, "DD overlap too wide for the box count in x");
  for (int b = 2; b < By; ++b)
    PS_REQUIRE(ry[b].first > ry[b - 2].second + 1, "DD overlap too wide for the box count in y");
  long long off = 0;
  for (int by = 0; by < By; ++by)
    for (int bxi = 0; bxi < Bx; ++bxi) {
      DDBox b{};
      b.bx = bxi;
      b.by = by;
      b.x0 = rx[bxi].first;
      b.y0 = ry[by].first;
      const int wx = rx[bxi].second - rx[bxi].first + 1, wy = ry[by].second - ry[by].first + 1;
      if (wx <= 0 || wy <= 0) continue;
      b.xfast = wx <= wy ? 1 : 0;
      b.lead = b.xfast ? wx : wy;
      b.n = wx * wy;
      if (b.lead > kMaxLead)
        throw Error(PS_ERR_UNSUPPORTED, "DD box too wide: its shorter extent must be at most " +
                                            std::to_string(kMaxLead) + " nodes (use more boxes)");
      b.offset = off;
      off += (long long)(b.n / b.lead) * dd_line_stride(b.lead, plan.full);
      plan.colours[(bxi % 2) + ncx * (by % 2)].push_back(b);
    }
  plan.fac_len = off;
  plan.max_lead = 0;
  plan.nodes.assign(plan.M, 0.0);
  plan.fac_entries.assign(plan.M, 0.0);
  for (int c = 0; c < plan.M; ++c)
    for (auto& b : plan.colours[c]) {
      plan.max_lead = std::max(plan.max_lead, b.lead);
      plan.nodes[c] += b.n;
      plan.fac_entries[c] += (double)(b.n / b.lead) * (2.0 * b.lead * b.lead + (plan.full ? 3.0 : 1.0) * b.lead);
    }
}

void dd_factor(const Geom& g, const ps_dd_params& dd, const double* a_nodal, const double* d12_nodal, double c,
               double tau, DDFactors& f, cudaStream_t st) {
  dd_plan(g, dd, d12_nodal != nullptr, f.plan);
  f.tau = tau;
  f.fac.alloc((size_t)f.plan.fac_len);
  f.status.alloc(1);
  PS_CUDA(cudaMemsetAsync(f.status.p, 0, sizeof(int), st));
  f.dev_boxes.resize(f.plan.M);
  DDGeomArgs ga;
  ga.nx = g.n[0];
  ga.ny = g.n[1];
  ga.a = a_nodal;
  ga.d12 = d12_nodal;
  ga.full = d12_nodal != nullptr ? 1 : 0;
  ga.c = c;
  ga.tau = tau;
  ga.Bx = dd.boxes[0];
  ga.By = dd.boxes[1];
  ga.overlap = dd.overlap;
  const int w = f.plan.max_lead;
  const size_t smem = ((size_t)w * w + kFactorVecs * (size_t)w) * sizeof(double);
  int dev = 0, maxsm = 0;
  PS_CUDA(cudaGetDevice(&dev));
  PS_CUDA(cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  if ((int)smem + 64 > maxsm) throw Error(PS_ERR_UNSUPPORTED, "DD box too wide for the shared-memory factorisation");
  auto fkern = ga.full ? dd_factor_kernel<true> : dd_factor_kernel<false>;
  PS_CUDA(cudaFuncSetAttribute(fkern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  std::vector<DDBox> all;
  for (int c = 0; c < f.plan.M; ++c) {
    auto& boxes = f.plan.colours[c];
    f.dev_boxes[c].alloc(boxes.size());
    if (boxes.empty()) continue;
    PS_CUDA(cudaMemcpyAsync(f.dev_boxes[c].p, boxes.data(), sizeof(DDBox) * boxes.size(), cudaMemcpyHostToDevice,
                            st));
    all.insert(all.end(), boxes.begin(), boxes.end());
  }
  if (!all.empty()) {
    // every box of every colour in one launch: each CTA runs its box's m dense inversions
    f.dev_all.alloc(all.size());
    PS_CUDA(cudaMemcpyAsync(f.dev_all.p, all.data(), sizeof(DDBox) * all.size(), cudaMemcpyHostToDevice, st));
    fkern<<<(unsigned)all.size(), dim3(32, 16), smem, st>>>(f.dev_all.p, ga, f.fac.p, f.status.p);
    PS_CUDA(cudaGetLastError());
  }
  int h = 0;
  PS_CUDA(cudaMemcpyAsync(&h, f.status.p, sizeof(int), cudaMemcpyDeviceToHost, st));
  PS_CUDA(cudaStreamSynchronize(st));
  if (h) throw Error(PS_ERR_INVALID, "DD factorisation met a non-positive pivot (is a > 0?)");
}

void dd_solve(const Geom& g, int nslices, const DDFactors& f, int colour, double* state, int slices_per_block,
              int* err, cudaStream_t st) {
  const auto& boxes = f.plan.colours[colour];
  if (boxes.empty()) return;
  // slices per CTA: each streamed factor entry serves S slices; fewer CTAs as S grows
  const int S = nslices == 1 ? 1 : (slices_per_block >= 4 ? 4 : (slices_per_block == 1 ? 1 : 2));
  const int ld = f.plan.max_lead;
  const int threads = (ld + 31) / 32 * 32;
  const size_t smem = 128 + (2 * (size_t)kChunk * ld + 2 * (size_t)S * ld) * sizeof(double);
  dim3 grid((unsigned)boxes.size(), (unsigned)((nslices + S - 1) / S));
  auto launch = [&](auto kern) {
    PS_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<grid, threads, smem, st>>>(f.dev_boxes[colour].p, g.n[0], g.nt, f.fac.p, state, nslices, ld, err);
  };
  if (f.plan.full) {
    if (S == 1) launch(dd_solve_kernel<1, true>);
    else if (S == 2) launch(dd_solve_kernel<2, true>);
    else launch(dd_solve_kernel<4, true>);
  } else {
    if (S == 1) launch(dd_solve_kernel<1, false>);
    else if (S == 2) launch(dd_solve_kernel<2, false>);
    else launch(dd_solve_kernel<4, false>);
  }
  PS_CUDA(cudaGetLastError());
}

void dd_rhs(const Geom& g, int nslices, const double* in, double* out, const SourceArgs& sa, cudaStream_t st) {
  const long long total = g.nt * nslices;
  long long blocks = std::min<long long>((total + 255) / 256, 152 * 16);
  dd_rhs_kernel<<<(unsigned)blocks, 256, 0, st>>>(in, out, total, g.nt, sa);
  PS_CUDA(cudaGetLastError());
}

void dd_correct(const Geom& g, const double* gstate, const CorrArgs& ca, cudaStream_t st) {
  long long blocks = std::min<long long>((g.nt + 255) / 256, 152 * 8);
  dd_correct_kernel<<<(unsigned)blocks, 256, 0, st>>>(g.nt, gstate, ca);
  PS_CUDA(cudaGetLastError());
}

}  // namespace ps
