// ps_coarse.cu -- the coarse propagator's line sweeps on one slice: the FP64 x-sweep by
// warp-private Thomas chunks (the default; also the batches' grouped x-sweep), the sweeps
// staged whole through shared memory (an autotuner candidate), and the FP32 PCR x-sweep.
//
// The coarse chain of parareal (Sec. 3) advances one slice at a time, U_{n+1} = G(U_n) +
// correction, so its sweeps see only the lines of one slice (n^{d-1} lines per direction) and
// each line is a dependent recurrence of n steps.  Streamed from global memory, every step of
// that recurrence waits on a load.  Here a CTA first copies its lines -- right-hand side and,
// for variable coefficients, both factor vectors of every node -- into shared memory with
// asynchronous copies (cp.async; all of them in flight at once), then one thread per line runs
// the two recurrences of the L D L^T solve from shared memory,
//     forward   y_i = b_i - l_i y_{i-1}            (+ tau f_i on the way in, x-lines)
//     backward  x_i = r_i y_i - l_{i+1} x_{i+1},
// and all threads write the lines back, coalesced, with the parareal correction (eq. of the
// parareal recursion, written as F + (G_new - G_old)) or the initial-sweep epilogue fused in.
// Two such CTAs share an SM, so one's copies overlap the other's recurrences.
//
// x-lines are contiguous rows: a CTA takes R whole rows, staged row-major with an odd pitch
// (thread t's row at t * pitch, so the R threads' shared-memory accesses fall in distinct banks).
// y- and z-lines are strided: a CTA takes XB consecutive x positions of one plane, staged
// node-major [i][x] (thread t at column t), so every copy and store of a warp covers whole
// 8-/16-element row segments of the grid.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "ps_internal.h"

namespace ps {
namespace {

constexpr int kThreads = 256;
constexpr size_t kSmemBudget = 100 * 1024;  // per CTA, so that two CTAs share an SM

__device__ __forceinline__ uint32_t sh_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
// one asynchronous 4- or 8-byte copy global -> shared (cp.async, cache at all levels)
template <typename T>
__device__ __forceinline__ void cp_async(T* dst, const T* src) {
  static_assert(sizeof(T) == 4 || sizeof(T) == 8, "4- or 8-byte elements");
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(sh_addr(dst)), "l"(src), "n"(sizeof(T)) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

// The two recurrences on one line in shared memory: element i of the right-hand side at
// x[i * xs], factors l_i, r_i at L[i * fs], Rf[i * fs] (l_0 = 0), source f_i at s[i * xs]
// added as b_i + c f_i when SRC.  Loads run one chunk of four nodes ahead of the arithmetic,
// in registers (shared-memory latency is paid once per chunk, not per node); the arithmetic
// is the same in every order: y = b - l y and x = r y - l' x as one FMA each after the product.
template <typename T, bool SRC>
__device__ __forceinline__ void thomas_staged(T* x, int xs, const T* L, const T* Rf, int fs, const T* s, T c,
                                              int n) {
  const int nq = n / 4;
  T y = T(0);
  T bn[4], ln[4], sn[4];
  if (nq > 0) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      bn[u] = x[u * xs];
      ln[u] = L[u * fs];
      sn[u] = SRC ? s[u * xs] : T(0);
    }
  }
  for (int q = 0; q < nq; ++q) {
    T b[4], l[4], f[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      b[u] = bn[u];
      l[u] = ln[u];
      f[u] = sn[u];
    }
    if (q + 1 < nq) {
      const int i1 = 4 * (q + 1);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        bn[u] = x[(i1 + u) * xs];
        ln[u] = L[(i1 + u) * fs];
        sn[u] = SRC ? s[(i1 + u) * xs] : T(0);
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      T bb = b[u];
      if (SRC) bb = fma(c, f[u], bb);
      y = fma(-l[u], y, bb);
      x[(4 * q + u) * xs] = y;
    }
  }
  for (int i = 4 * nq; i < n; ++i) {
    T bb = x[i * xs];
    if (SRC) bb = fma(c, s[i * xs], bb);
    y = fma(-L[i * fs], y, bb);
    x[i * xs] = y;
  }
  // backward, from the end of the line; l_{i+1} of the last node is 0
  T xn = T(0), lnext = T(0);
  const int tail = n - 4 * nq;
  for (int i = n - 1; i >= n - tail; --i) {
    xn = fma(-lnext, xn, Rf[i * fs] * x[i * xs]);
    x[i * xs] = xn;
    lnext = L[i * fs];
  }
  T yn[4], rn[4];
  if (nq > 0) {
    const int i0 = 4 * (nq - 1);
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      yn[u] = x[(i0 + u) * xs];
      rn[u] = Rf[(i0 + u) * fs];
      ln[u] = L[(i0 + u) * fs];
    }
  }
  for (int q = nq - 1; q >= 0; --q) {
    T yy[4], r[4], l[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      yy[u] = yn[u];
      r[u] = rn[u];
      l[u] = ln[u];
    }
    if (q > 0) {
      const int i1 = 4 * (q - 1);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        yn[u] = x[(i1 + u) * xs];
        rn[u] = Rf[(i1 + u) * fs];
        ln[u] = L[(i1 + u) * fs];
      }
    }
#pragma unroll
    for (int u = 3; u >= 0; --u) {
      const T l1 = u == 3 ? lnext : l[u + 1];
      xn = fma(-l1, xn, r[u] * yy[u]);
      x[(4 * q + u) * xs] = xn;
    }
    lnext = l[0];
  }
}

// |v| as the bit pattern of a nonnegative double: maxima of such patterns are taken with
// 64-bit integer instructions (they order like the values), off the FP64 pipe.
__device__ __forceinline__ unsigned long long abs_bits(double v) {
  return (unsigned long long)__double_as_longlong(v) & 0x7fffffffffffffffull;
}
constexpr unsigned long long kInfBits = 0x7ff0000000000000ull;  // |v| bits >= this: inf or NaN

// ---------------------------------------------------------------------------------------
// x-lines (contiguous rows) of one slice, FP64.  A CTA stages R rows of the right-hand side
// (and of the source when SRC), plus their factors, at pitch `ld` (odd); threads t < R solve
// row t; the CTA writes the rows back.  VAR: factors per node in the transposed layout
// [i][row] (consecutive rows of one i are consecutive); otherwise one vector of n_x shared by
// all rows.  Shared memory: x | (source) | l | r.
template <bool VAR, bool SRC>
__global__ void __launch_bounds__(kThreads) coarse_x_staged_kernel(const double* __restrict__ in,
                                                                   double* __restrict__ out, int nx, long long rows,
                                                                   int R, int ld, const double* __restrict__ fl,
                                                                   const double* __restrict__ fr, SourceArgs sa) {
  extern __shared__ __align__(16) double xsm[];
  double* xb = xsm;
  double* sb = xb + (size_t)R * ld;
  double* lb = SRC ? sb + (size_t)R * ld : sb;
  double* rb = lb + (VAR ? (size_t)R * ld : (size_t)ld);
  const long long row0 = (long long)blockIdx.x * R;
  const int nr = (int)min((long long)R, rows - row0);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  // rows of the right-hand side and source: one warp per row, lanes along the row
  for (int rr = warp; rr < nr; rr += nw) {
    const double* g = in + (row0 + rr) * nx;
    for (int i = lane; i < nx; i += 32) cp_async(xb + rr * ld + i, g + i);
    if (SRC) {
      const double* gs = sa.src + (row0 + rr) * nx;
      for (int i = lane; i < nx; i += 32) cp_async(sb + rr * ld + i, gs + i);
    }
  }
  if (VAR) {
    // factor i of rows row0 .. row0 + nr - 1 are consecutive: half a warp per i (16 rows)
    const int half = lane >> 4, r16 = lane & 15;
    for (int i = warp * 2 + half; i < nx; i += nw * 2)
      for (int rr = r16; rr < nr; rr += 16) {
        cp_async(lb + rr * ld + i, fl + (long long)i * rows + row0 + rr);
        cp_async(rb + rr * ld + i, fr + (long long)i * rows + row0 + rr);
      }
  } else {
    for (int i = tid; i < nx; i += blockDim.x) {
      cp_async(lb + i, fl + i);
      cp_async(rb + i, fr + i);
    }
  }
  cp_async_wait_all();
  __syncthreads();
  if (tid < nr) {
    const double c = SRC ? sa.tau * (sa.src_t ? sa.src_t[sa.t0] : 1.0) : 0.0;
    const int fo = VAR ? tid * ld : 0;
    thomas_staged<double, SRC>(xb + tid * ld, 1, lb + fo, rb + fo, 1, sb + tid * ld, c, nx);
  }
  __syncthreads();
  for (int rr = warp; rr < nr; rr += nw) {
    double* g = out + (row0 + rr) * nx;
    for (int i = lane; i < nx; i += 32) g[i] = xb[rr * ld + i];
  }
}

// ---------------------------------------------------------------------------------------
// y- or z-lines of one slice: a CTA stages XB consecutive x positions of one plane, every node
// i of the line, node-major [i][x]; threads t < (valid columns) solve column t; all threads
// write back with the epilogue.  Line node i of column t sits at base + i * S + t.  VAR:
// factors per node in the state layout (same offsets as the state); otherwise one vector of
// n_m.  T is the recurrence and storage type of the right-hand side; the epilogues:
//   EPI 0  out = x (type T)
//   EPI 1  (T = double) U_{n+1} <- Fout + (g - Gold), Gold <- g, increment and norms
//   EPI 2  U_{n+1} <- g, and Gold <- g when given (initial coarse sweep)
//   EPI 3  (T = float, increment form) U_{n+1} <- Fout + g, the new FP32 increment to dnext
template <typename T, bool VAR, int EPI>
__global__ void __launch_bounds__(kThreads) coarse_strided_staged_kernel(const T* __restrict__ in, T* __restrict__ out,
                                                                         int nx, int nm, long long S, int nxb,
                                                                         long long outer_stride, int XB,
                                                                         const T* __restrict__ fl,
                                                                         const T* __restrict__ fr, CorrArgs ca) {
  extern __shared__ __align__(16) unsigned char ssm_raw[];
  T* tb = reinterpret_cast<T*>(ssm_raw);
  T* lb = tb + (size_t)nm * XB;
  T* rb = lb + (VAR ? (size_t)nm * XB : (size_t)nm);
  const int xblk = blockIdx.x % nxb;
  const long long outer = blockIdx.x / nxb;
  const int x0 = xblk * XB;
  const int nxv = min(XB, nx - x0);
  const long long base = outer * outer_stride + x0;
  const int tid = threadIdx.x;
  const int lgx = __ffs(XB) - 1;  // XB is a power of two
  const int total = nm * XB;
  for (int e = tid; e < total; e += blockDim.x) {
    const int i = e >> lgx, t = e & (XB - 1);
    if (t < nxv) {
      const long long gi = base + (long long)i * S + t;
      cp_async(tb + e, in + gi);
      if (VAR) {
        cp_async(lb + e, fl + gi);
        cp_async(rb + e, fr + gi);
      }
    }
  }
  if (!VAR)
    for (int i = tid; i < nm; i += blockDim.x) {
      cp_async(lb + i, fl + i);
      cp_async(rb + i, fr + i);
    }
  cp_async_wait_all();
  __syncthreads();
  if (tid < nxv) {
    if (VAR) thomas_staged<T, false>(tb + tid, XB, lb + tid, rb + tid, XB, nullptr, T(0), nm);
    else thomas_staged<T, false>(tb + tid, XB, lb, rb, 1, nullptr, T(0), nm);
  }
  __syncthreads();
  unsigned long long my_inc = 0, my_norm = 0;
  bool bad = false;
  for (int e = tid; e < total; e += blockDim.x) {
    const int i = e >> lgx, t = e & (XB - 1);
    if (t >= nxv) continue;
    const long long gi = base + (long long)i * S + t;
    const T xv = tb[e];
    if (EPI == 0) {
      out[gi] = xv;
    } else if (EPI == 1) {
      const double g = (double)xv;
      const double unew = ca.Fout[gi] + (g - ca.Gold[gi]);
      const unsigned long long an = abs_bits(unew);
      bad |= an >= kInfBits;
      my_inc = max(my_inc, abs_bits(unew - ca.U_next[gi]));
      my_norm = max(my_norm, an);
      ca.Gold[gi] = g;
      ca.U_next[gi] = unew;
    } else if (EPI == 2) {
      const double g = (double)xv;
      bad |= abs_bits(g) >= kInfBits;
      if (ca.Gold) ca.Gold[gi] = g;
      ca.U_next[gi] = g;
    } else {
      // G is affine, so G(U^k) - G(U^{k-1}) is its linear part applied to the increment
      const double unew = ca.Fout[gi] + (double)xv;
      const double d = unew - ca.U_next[gi];
      const unsigned long long an = abs_bits(unew);
      bad |= an >= kInfBits;
      my_inc = max(my_inc, abs_bits(d));
      my_norm = max(my_norm, an);
      ca.U_next[gi] = unew;
      ca.dnext[gi] = (float)d;
    }
  }
  if (EPI == 1 || EPI == 3) {
    for (int o = 16; o > 0; o >>= 1) {
      my_inc = max(my_inc, __shfl_xor_sync(0xffffffffu, my_inc, o));
      my_norm = max(my_norm, __shfl_xor_sync(0xffffffffu, my_norm, o));
    }
    if ((tid & 31) == 0 && my_inc > 0) atomicMax(ca.inc, my_inc);
    if ((tid & 31) == 0 && ca.slice_stats) {
      if (my_inc > 0) atomicMax(ca.slice_stats, my_inc);
      if (my_norm > 0) atomicMax(ca.slice_stats + 1, my_norm);
    }
  }
  if (EPI != 0)
    if (__any_sync(0xffffffffu, bad) && (tid & 31) == 0) atomicExch(ca.nonfinite, 1);
}

// ---------------------------------------------------------------------------------------
// x-lines of one slice, FP32, by parallel cyclic reduction: one warp per row of L <= 256 nodes,
// lane j holding equations j, j + 32, ..., j + 224 (eight per lane; past L: identity rows).
// Equation i:  e_i x_{i-1} + d_i x_i + e_{i+1} x_{i+1} = b_i  (symmetric tridiagonal,
// e_0 = e_L = 0).  Reduction step with stride s eliminates the couplings to i -+ s:
//     k1 = a_i / d_{i-s},  k2 = c_i / d_{i+s}
//     a_i <- -a_{i-s} k1,  c_i <- -c_{i+s} k2,
//     d_i <- d_i - c_{i-s} k1 - a_{i+s} k2,   b_i <- b_i - b_{i-s} k1 - b_{i+s} k2,
// for s = 1, 2, ..., 128; then x_i = b_i / d_i.  For s < 32 the partner equations live in other
// lanes (warp shuffles), for s >= 32 in the same lane (registers).  Coefficients: line-major FP32
// rows of the sub-diagonal e and the diagonal d (pitch Lp).  SRC adds tau f on the way in.
constexpr int kPcrPer = 8;  // equations per lane: L <= 256

// value of equation i - s (MINUS) or i + s of array v for lane `lane`, slot u; zero outside
template <bool MINUS>
__device__ __forceinline__ float pcr_partner(const float (&v)[kPcrPer], int u, int s, int lane) {
  const unsigned full = 0xffffffffu;
  float r;
  if (s >= 32) {
    const int du = s >> 5;
    const int uu = MINUS ? u - du : u + du;
    r = (uu >= 0 && uu < kPcrPer) ? v[uu] : 0.f;
  } else {
    // the partner is lane -+ s of the same slot, or across the slot boundary
    const int src = MINUS ? ((lane - s) & 31) : ((lane + s) & 31);
    const float same = __shfl_sync(full, v[u], src);
    const int uo = MINUS ? u - 1 : u + 1;
    const float other = __shfl_sync(full, v[(uo >= 0 && uo < kPcrPer) ? uo : u], src);
    const bool cross = MINUS ? lane < s : lane + s >= 32;
    r = cross ? ((uo >= 0 && uo < kPcrPer) ? other : 0.f) : same;
  }
  return r;
}

template <typename Tin, bool SRC>
__global__ void __launch_bounds__(256) sweep_x_pcr_kernel(const Tin* __restrict__ in, float* __restrict__ out,
                                                         long long rows, int nx, const float* __restrict__ et,
                                                         const float* __restrict__ dt, int Lp, SourceArgs sa) {
  const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const float c = SRC ? (float)(sa.tau * (sa.src_t ? sa.src_t[sa.t0] : 1.0)) : 0.f;
  for (long long row = (long long)blockIdx.x * nw + (threadIdx.x >> 5); row < rows; row += (long long)gridDim.x * nw) {
    float a[kPcrPer], d[kPcrPer], cc[kPcrPer], b[kPcrPer];
#pragma unroll
    for (int u = 0; u < kPcrPer; ++u) {
      const int i = lane + 32 * u;
      if (i < nx) {
        float bi = (float)in[row * nx + i];
        if (SRC) bi = fmaf(c, (float)sa.src[row * nx + i], bi);
        b[u] = bi;
        a[u] = et[row * Lp + i];
        d[u] = dt[row * Lp + i];
        cc[u] = i + 1 < nx ? et[row * Lp + i + 1] : 0.f;
      } else {
        a[u] = 0.f;
        d[u] = 1.f;
        cc[u] = 0.f;
        b[u] = 0.f;
      }
    }
#pragma unroll
    for (int s = 1; s < 32 * kPcrPer; s <<= 1) {  // unrolled: partner slots are compile-time constants
      float na[kPcrPer], nd[kPcrPer], nc[kPcrPer], nb[kPcrPer];
#pragma unroll
      for (int u = 0; u < kPcrPer; ++u) {
        const float am = pcr_partner<true>(a, u, s, lane), dm = pcr_partner<true>(d, u, s, lane);
        const float cm = pcr_partner<true>(cc, u, s, lane), bm = pcr_partner<true>(b, u, s, lane);
        const float ap = pcr_partner<false>(a, u, s, lane), dp = pcr_partner<false>(d, u, s, lane);
        const float cp = pcr_partner<false>(cc, u, s, lane), bp = pcr_partner<false>(b, u, s, lane);
        // partners outside the line are identity rows: d = 1, everything else 0
        const float k1 = a[u] != 0.f ? a[u] / (dm != 0.f ? dm : 1.f) : 0.f;
        const float k2 = cc[u] != 0.f ? cc[u] / (dp != 0.f ? dp : 1.f) : 0.f;
        na[u] = -am * k1;
        nc[u] = -cp * k2;
        nd[u] = d[u] - cm * k1 - ap * k2;
        nb[u] = b[u] - bm * k1 - bp * k2;
      }
#pragma unroll
      for (int u = 0; u < kPcrPer; ++u) {
        a[u] = na[u];
        d[u] = nd[u];
        cc[u] = nc[u];
        b[u] = nb[u];
      }
    }
#pragma unroll
    for (int u = 0; u < kPcrPer; ++u) {
      const int i = lane + 32 * u;
      if (i < nx) out[row * nx + i] = b[u] / d[u];
    }
  }
}

// Line-major FP32 rows [row][Lp] of the sub-diagonal e_i = -tau a_{i-1/2} / h^2 (e_0 = 0) and the
// diagonal d_i = 1 + tau (a_{i-1/2} + a_{i+1/2}) / h^2 + tau c/M of (I - tau A_x), each formed in
// FP64 from the nodal coefficient (a_{i+1/2} = (a_i + a_{i+1})/2) and rounded once.
__global__ void tridiag_x_rows_kernel(int dim, int nx, int ny, long long rows, const double* __restrict__ a,
                                      double cM, double tau, int Lp, float* __restrict__ et, float* __restrict__ dt) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= rows * Lp) return;
  const long long row = e / Lp;
  const int i = (int)(e - row * Lp);
  if (i >= nx) {
    et[e] = 0.f;
    dt[e] = 1.f;
    return;
  }
  const double h = 1.0 / (nx + 1), h2 = h * h;
  const int y = (int)(row % ny);
  const long long z = row / ny;
  const long long a0 = (dim == 3 ? (z + 1) * (ny + 2) + (y + 1) : (long long)(y + 1)) * (nx + 2) + (i + 1);
  const double ai = a ? a[a0] : 1.0;
  const double am = a ? 0.5 * (ai + a[a0 - 1]) : 1.0;
  const double ap = a ? 0.5 * (ai + a[a0 + 1]) : 1.0;
  dt[e] = (float)(1.0 + tau * (am + ap) / h2 + tau * cM);
  et[e] = i > 0 ? (float)(-tau * am / h2) : 0.f;
}


// ---------------------------------------------------------------------------------------
// FP64 x-substep, Thomas per thread, in warp-private chunks: the same operations in the same
// order as the whole-row sweep of ps_dim.cu, so the two give the same bits.  Each warp owns 32
// consecutive rows (lane = row) and works alone -- no CTA barrier couples the warps of an SM:
//   - the rows' right-hand side (and source) pass through the warp's shared memory XW_C nodes at
//     a time in two stages (cp.async; every copy instruction covers four 64-byte row segments),
//     read back by the lane of each row (row pitch XW_C + 1: distinct bank pairs);
//   - the factors l, r of the next chunk are prefetched into registers: in the transposed factor
//     layout (entry (row, i) at i * rows_per_slice + row) one node of the warp's 32 rows is one
//     coalesced 256-byte load;
//   - the forward pass writes y to `out` chunk by chunk; the backward pass copies it back one
//     chunk ahead and overwrites it with x; the last chunk's y stays in shared memory.
// On GB300 the FP64 pipe (a warp instruction per ~64 cycles per SM sub-partition, ~72 cycles of
// dependent latency) sets the pace; 9 KB of shared memory per warp leaves room for every row
// of a 255^3 slice in one wave (13-14 warps per SM), each warp never waiting on a barrier.
constexpr int XW_C = 8, XW_P = XW_C + 1, XW_WARPS = 2;
constexpr int XW_WARP_DOUBLES = 2 * 2 * 32 * XW_P;  // two stages of u and s
constexpr size_t kXwSmem = (size_t)XW_WARPS * (XW_WARP_DOUBLES + 32) * sizeof(double);

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

// Rows [row0, row0 + 32) of one x-sweep by one warp; wsm: the warp's XW_WARP_DOUBLES + 32
// doubles of shared memory.  Every copy of the warp is complete when it returns.
template <bool VAR, bool SRC>
__device__ __forceinline__ void x_thomas_warp_rows(const double* in, double* out, long long rows, int nx, int rps,
                                                   const double* __restrict__ fl, const double* __restrict__ fr,
                                                   const SourceArgs& sa, long long row0, double* wsm) {
  const int lane = threadIdx.x & 31;
  double* ub = wsm;                  // [stage][32][XW_P]: u, then y, then x
  double* sb = ub + 2 * 32 * XW_P;   // [stage][32][XW_P]: source
  long long* soff = reinterpret_cast<long long*>(sb + 2 * 32 * XW_P);  // [32]: source row offsets
  if (row0 >= rows) return;  // the whole warp: nothing below waits on another warp
  const long long myrow = row0 + lane;
  const bool active = myrow < rows;
  const int ris = active ? (int)(myrow % rps) : 0;  // row inside its slice: factor index
  double cst = 0.0;
  if (SRC) {
    soff[lane] = (long long)ris * nx;
    if (active) cst = sa.tau * (sa.src_t ? sa.src_t[sa.t0 + (myrow / rps) * sa.tstride] : 1.0);
  }
  __syncwarp();
  const int nch = (nx + XW_C - 1) / XW_C;
  // copies of a chunk: element (r, j) of the warp's 32 x XW_C block, lane -> j = lane % 8,
  // r = lane / 8 + 4 q (q = 0..7)
  const int jl = lane % XW_C, rl = lane / XW_C;
  auto stage = [&](double* dst, const double* g, bool src_rows, int k) {
    const int i = k * XW_C + jl;
#pragma unroll
    for (int q = 0; q < XW_C; ++q) {
      const int r = rl + 4 * q;
      double* d = dst + r * XW_P + jl;
      if (row0 + r < rows && i < nx) cp_async(d, g + (src_rows ? soff[r] : (row0 + r) * nx) + i);
    }
  };
  auto store = [&](const double* srcb, int k) {
    const int i = k * XW_C + jl;
#pragma unroll
    for (int q = 0; q < XW_C; ++q) {
      const int r = rl + 4 * q;
      if (row0 + r < rows && i < nx) out[(row0 + r) * nx + i] = srcb[r * XW_P + jl];
    }
  };
  // factors of nodes k * XW_C + j (+ shift) of this lane's row
  auto load_f = [&](double (&dst)[XW_C], const double* f, int k, int shift) {
#pragma unroll
    for (int j = 0; j < XW_C; ++j) {
      const int i = k * XW_C + j + shift;
      dst[j] = (active && i < nx) ? (VAR ? f[(long long)i * rps + ris] : f[i]) : 0.0;
    }
  };
  // forward  y_i = b_i - l_i y_{i-1},  b_i = u_i + c f_i (one rounding)
  double lc[XW_C], ln[XW_C];
  stage(ub, in, false, 0);
  if (SRC) stage(sb, sa.src, true, 0);
  cp_async_commit();
  load_f(lc, fl, 0, 0);
  double y = 0.0;
  for (int k = 0; k < nch; ++k) {
    const int b = k & 1;
    if (k + 1 < nch) {
      stage(ub + (b ^ 1) * 32 * XW_P, in, false, k + 1);
      if (SRC) stage(sb + (b ^ 1) * 32 * XW_P, sa.src, true, k + 1);
      load_f(ln, fl, k + 1, 0);
    }
    cp_async_commit();
    cp_async_wait1();
    __syncwarp();
    if (active) {
      double* u = ub + b * 32 * XW_P + lane * XW_P;
      const double* sv = sb + b * 32 * XW_P + lane * XW_P;
      const int len = min(XW_C, nx - k * XW_C);
#pragma unroll
      for (int j = 0; j < XW_C; ++j) {
        if (j < len) {
          const int i = k * XW_C + j;
          const double bi = SRC ? fma(cst, sv[j], u[j]) : u[j];
          y = i == 0 ? bi : fma(-lc[j], y, bi);
          u[j] = y;
        }
      }
    }
    __syncwarp();
    if (k + 1 < nch) store(ub + b * 32 * XW_P, k);
    __syncwarp();
#pragma unroll
    for (int j = 0; j < XW_C; ++j) lc[j] = ln[j];
  }
  // backward  x_i = r_i y_i - l_{i+1} x_{i+1}; its copies read back y stored above: the fence
  // orders those stores before them
  __threadfence_block();
  double rc[XW_C], rn[XW_C];
  load_f(rc, fr, nch - 1, 0);
  load_f(lc, fl, nch - 1, 1);
  double x = 0.0;
  for (int k = nch - 1; k >= 0; --k) {
    const int b = k & 1;
    if (k > 0) {
      stage(ub + (b ^ 1) * 32 * XW_P, out, false, k - 1);
      load_f(rn, fr, k - 1, 0);
      load_f(ln, fl, k - 1, 1);
    }
    cp_async_commit();
    cp_async_wait1();
    __syncwarp();
    if (active) {
      double* u = ub + b * 32 * XW_P + lane * XW_P;
      const int len = min(XW_C, nx - k * XW_C);
#pragma unroll
      for (int j = XW_C - 1; j >= 0; --j) {
        if (j < len) {
          const int i = k * XW_C + j;
          x = i == nx - 1 ? rc[j] * u[j] : fma(-lc[j], x, rc[j] * u[j]);
          u[j] = x;
        }
      }
    }
    __syncwarp();
    store(ub + b * 32 * XW_P, k);
    __syncwarp();
#pragma unroll
    for (int j = 0; j < XW_C; ++j) {
      rc[j] = rn[j];
      lc[j] = ln[j];
    }
  }
}

template <bool VAR, bool SRC>
__global__ void __launch_bounds__(32 * XW_WARPS, 8)
    sweep_x_thomas_warp_kernel(const double* in, double* out, long long rows, int nx, int rps,
                               const double* __restrict__ fl, const double* __restrict__ fr, SourceArgs sa) {
  extern __shared__ __align__(16) double xwsm[];
  const int w = threadIdx.x >> 5;
  const long long nblk = (rows + 32 * XW_WARPS - 1) / (32 * XW_WARPS);
  for (long long b = blockIdx.x; b < nblk; b += gridDim.x) {
    x_thomas_warp_rows<VAR, SRC>(in, out, rows, nx, rps, fl, fr, sa, (b * XW_WARPS + w) * 32,
                                 xwsm + w * (XW_WARP_DOUBLES + 32));
    __syncwarp();
  }
}

// Grouped coarse x-sweeps (batched 2-D problems, FP64): an item is 32 * XW_WARPS rows of one job.
template <bool VAR>
__global__ void __launch_bounds__(32 * XW_WARPS, 8)
    sweep_x_warp_grouped_kernel(const CoarseJob* __restrict__ jobs, const WorkSeg* __restrict__ segs,
                                const int* __restrict__ nseg_ptr) {
  extern __shared__ __align__(16) double xwsm[];
  const int w = threadIdx.x >> 5;
  const int nseg = *nseg_ptr;
  if (nseg <= 0) return;
  const long long total = (long long)segs[nseg - 1].prefix + segs[nseg - 1].count;
  for (long long it = blockIdx.x; it < total; it += gridDim.x) {
    int lo = 0, hi = nseg - 1;  // the last segment whose prefix is <= it
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (segs[mid].prefix <= it) lo = mid;
      else hi = mid - 1;
    }
    const WorkSeg sg = segs[lo];
    const CoarseJob& j = jobs[sg.job];
    const long long row0 = ((sg.first + (it - sg.prefix)) * XW_WARPS + w) * 32;
    if (j.sa.src)
      x_thomas_warp_rows<VAR, true>(j.xin, j.xout, j.rows, j.nx, (int)j.rows, j.lx, j.rx, j.sa, row0,
                                    xwsm + w * (XW_WARP_DOUBLES + 32));
    else
      x_thomas_warp_rows<VAR, false>(j.xin, j.xout, j.rows, j.nx, (int)j.rows, j.lx, j.rx, j.sa, row0,
                                     xwsm + w * (XW_WARP_DOUBLES + 32));
    __syncwarp();
  }
}

}  // namespace

template <typename T>
bool coarse_sweep_staged(const Geom& g, const LineFactors& f, const T* in, T* out, const SourceArgs& sa,
                         const CorrArgs& ca, cudaStream_t st) {
  const bool f64 = sizeof(T) == 8;
  const T* fl = f64 ? reinterpret_cast<const T*>(f.l64.p) : reinterpret_cast<const T*>(f.l32.p);
  const T* fr = f64 ? reinterpret_cast<const T*>(f.r64.p) : reinterpret_cast<const T*>(f.r32.p);
  if (!fl || !fr) return false;
  const bool var = f.var != 0, src = sa.src != nullptr;
  if (sa.src2) return false;
  const int m = f.m;
  if (m == 0) {
    // rows: FP64 only (the FP32 increment form's x-sweep is the warp-per-row segmented scan)
    if (!f64 || ca.mode != 0) return false;
    const int nx = g.n[0];
    const long long rows = g.nt / nx;
    const int ld = nx | 1;
    const size_t per_row = (size_t)(1 + (src ? 1 : 0) + (var ? 2 : 0)) * ld * sizeof(double);
    const size_t fixed = var ? 0 : 2 * (size_t)ld * sizeof(double);
    if (per_row + fixed > kSmemBudget) return false;
    int R = (int)std::min<size_t>(32, (kSmemBudget - fixed) / per_row);
    if (R < 2) return false;
    const size_t smem = (size_t)R * per_row + fixed;
    const unsigned blocks = (unsigned)((rows + R - 1) / R);
    auto launch = [&](auto kern) {
      PS_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      kern<<<blocks, kThreads, smem, st>>>(reinterpret_cast<const double*>(in), reinterpret_cast<double*>(out), nx,
                                           rows, R, ld, reinterpret_cast<const double*>(fl),
                                           reinterpret_cast<const double*>(fr), sa);
    };
    if (var) {
      if (src) launch(coarse_x_staged_kernel<true, true>);
      else launch(coarse_x_staged_kernel<true, false>);
    } else {
      if (src) launch(coarse_x_staged_kernel<false, true>);
      else launch(coarse_x_staged_kernel<false, false>);
    }
    PS_CUDA(cudaGetLastError());
    return true;
  }
  if (src) return false;  // the source enters with the x-substep
  if (ca.mode == 1 && !f64) return false;
  if (ca.mode == 3 && f64) return false;
  const int nx = g.n[0], nm = g.n[m];
  const long long S = g.stride(m);
  const long long nouter = m == 1 ? (g.dim == 3 ? g.n[2] : 1) : g.n[1];
  const long long outer_stride = m == 1 ? (long long)g.n[0] * g.n[1] : (long long)g.n[0];
  // columns per CTA: 128-byte row segments, fewer when the line does not fit the budget
  int XB = f64 ? 16 : 32;
  auto smem_of = [&](int xb) {
    return ((size_t)nm * xb * (var ? 3 : 1) + (var ? 0 : 2 * (size_t)nm)) * sizeof(T);
  };
  while (XB > 4 && smem_of(XB) > kSmemBudget) XB /= 2;
  if (smem_of(XB) > kSmemBudget) return false;
  while (XB > 4 && XB / 2 >= nx) XB /= 2;  // short x extent: no empty columns
  const size_t smem = smem_of(XB);
  const int nxb = (nx + XB - 1) / XB;
  const long long blocks = (long long)nxb * nouter;
  if (blocks > 0x7fffffffLL) return false;
  auto launch = [&](auto kern) {
    PS_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<(unsigned)blocks, kThreads, smem, st>>>(in, out, nx, nm, S, nxb, outer_stride, XB, fl, fr, ca);
  };
#define PS_STAGED(E)                                                  \
  do {                                                               \
    if (var) launch(coarse_strided_staged_kernel<T, true, E>);       \
    else launch(coarse_strided_staged_kernel<T, false, E>);          \
  } while (0)
  if constexpr (sizeof(T) == 8) {
    if (ca.mode == 0) PS_STAGED(0);
    else if (ca.mode == 1) PS_STAGED(1);
    else if (ca.mode == 2) PS_STAGED(2);
    else return false;
  } else {
    if (ca.mode == 0) PS_STAGED(0);
    else if (ca.mode == 2) PS_STAGED(2);
    else if (ca.mode == 3) PS_STAGED(3);
    else return false;
  }
#undef PS_STAGED
  PS_CUDA(cudaGetLastError());
  return true;
}

template bool coarse_sweep_staged<double>(const Geom&, const LineFactors&, const double*, double*, const SourceArgs&,
                                          const CorrArgs&, cudaStream_t);
template bool coarse_sweep_staged<float>(const Geom&, const LineFactors&, const float*, float*, const SourceArgs&,
                                         const CorrArgs&, cudaStream_t);

void tridiag_x_rows(const Geom& g, const double* a_nodal, double c_over_M, double tau, DevBuf<float>& et,
                    DevBuf<float>& dt, cudaStream_t st) {
  const int nx = g.n[0];
  const long long rows = g.nt / nx;
  const int Lp = (nx + 3) & ~3;
  et.alloc((size_t)rows * Lp);
  dt.alloc((size_t)rows * Lp);
  const long long total = rows * Lp;
  tridiag_x_rows_kernel<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(g.dim, nx, g.n[1], rows, a_nodal, c_over_M, tau,
                                                                          Lp, et.p, dt.p);
  PS_CUDA(cudaGetLastError());
}

template <typename Tin>
bool sweep_x_pcr(const Geom& g, const float* et, const float* dt, const Tin* in, float* out, const SourceArgs& sa,
                 cudaStream_t st) {
  const int nx = g.n[0];
  if (nx > 32 * kPcrPer || !et || !dt || sa.src2) return false;
  const long long rows = g.nt / nx;
  const int Lp = (nx + 3) & ~3;
  int dev = 0, sms = 0;
  PS_CUDA(cudaGetDevice(&dev));
  PS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const unsigned grid = (unsigned)std::min<long long>((rows + 7) / 8, (long long)sms * 8);
  if (sa.src) sweep_x_pcr_kernel<Tin, true><<<grid, 256, 0, st>>>(in, out, rows, nx, et, dt, Lp, sa);
  else sweep_x_pcr_kernel<Tin, false><<<grid, 256, 0, st>>>(in, out, rows, nx, et, dt, Lp, sa);
  PS_CUDA(cudaGetLastError());
  return true;
}
template bool sweep_x_pcr<float>(const Geom&, const float*, const float*, const float*, float*, const SourceArgs&,
                                 cudaStream_t);
template bool sweep_x_pcr<double>(const Geom&, const float*, const float*, const double*, float*, const SourceArgs&,
                                  cudaStream_t);

bool sweep_x_chunked(const Geom& g, int nslices, const LineFactors& f, const double* in, double* out,
                     const SourceArgs& sa, cudaStream_t st) {
  if (f.m != 0 || f.l64.p == nullptr) return false;
  const int nx = g.n[0];
  const long long rps = g.nt / nx;
  const long long rows = rps * nslices;
  if (rps > (1LL << 30) || nx < 2 * XW_C) return false;  // short rows: the whole-row sweep
  const bool var = f.var != 0, src = sa.src != nullptr;
  const long long warps = (rows + 31) / 32;
  long long blocks = (warps + XW_WARPS - 1) / XW_WARPS;
  if (chain_ctas_per_sm > 0) {
    int dev = 0, sms = 0;
    PS_CUDA(cudaGetDevice(&dev));
    PS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    blocks = std::min<long long>(blocks, (long long)sms * 2 * chain_ctas_per_sm);  // CTAs of two warps
  }
  auto launch = [&](auto kern) {
    kern<<<(unsigned)blocks, 32 * XW_WARPS, kXwSmem, st>>>(in, out, rows, nx, (int)rps, f.l64.p, f.r64.p, sa);
  };
  if (var) {
    if (src) launch(sweep_x_thomas_warp_kernel<true, true>);
    else launch(sweep_x_thomas_warp_kernel<true, false>);
  } else {
    if (src) launch(sweep_x_thomas_warp_kernel<false, true>);
    else launch(sweep_x_thomas_warp_kernel<false, false>);
  }
  PS_CUDA(cudaGetLastError());
  return true;
}
int coarse_x_grouped_rows() { return 32 * XW_WARPS; }

void coarse_x_grouped(bool var, const CoarseJob* jobs, const WorkSeg* segs, const int* nseg, int grid,
                      cudaStream_t st) {
  if (var) sweep_x_warp_grouped_kernel<true><<<grid, 32 * XW_WARPS, kXwSmem, st>>>(jobs, segs, nseg);
  else sweep_x_warp_grouped_kernel<false><<<grid, 32 * XW_WARPS, kXwSmem, st>>>(jobs, segs, nseg);
  PS_CUDA(cudaGetLastError());
}
}  // namespace ps
