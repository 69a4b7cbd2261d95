// ps_dim.cu -- dimensional-splitting kernels: substep factor setup, batched line solves
// with the fused right-hand side and the fused parareal correction.
//
// One substep of eq. FIE_method (Sec. 2.2) solves (I - tau A_m) x = b where, with the
// dimensional splitting of Sec. 2.1, A_m couples only nodes on a line along x_m: every
// line is an independent symmetric tridiagonal system (Sec. 2.2: "essentially
// one-dimensional uncoupled systems").  We factor each line once per step size as
// L D L^T (setup, FP64) and solve with two recurrences:
//     forward   y_i = b_i - l_i y_{i-1}
//     backward  x_i = r_i y_i - l_{i+1} x_{i+1},        r_i = 1/D_i
// All time slices are solved in one launch: the batch is (slice x line).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <type_traits>

#include "ps_internal.h"

namespace ps {
thread_local int chain_ctas_per_sm = 0;

namespace {

constexpr int kThreads = 256;

// ---------------------------------------------------------------------------------------
// a1: LDL^T factors of (I - tau A_m) along every line of direction m.
// Row i of the line: diag 1 + tau (a_{i-1/2} + a_{i+1/2}) / h^2 + tau c/M,
// off-diagonal (i, i+1) = -tau a_{i+1/2} / h^2, a_{i+1/2} = (a_i + a_{i+1}) / 2 (nodal a).
// One thread per line; lines = 1 when the coefficients are constant (var = 0).
__global__ void factor_dim_kernel(int dim, int nx, int ny, int nz, int m, const double* __restrict__ a,
                                  double cM, double tau, double* __restrict__ l, double* __restrict__ r,
                                  float* __restrict__ l32, float* __restrict__ r32, long long lines, int var) {
  long long L = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (L >= lines) return;
  const int nm = m == 0 ? nx : (m == 1 ? ny : nz);
  const long long S = m == 0 ? 1LL : (m == 1 ? (long long)nx : (long long)nx * ny);
  const long long base = (m == 0) ? L * nx : (L / S) * S * nm + (L % S);
  const int x0 = (int)(base % nx);
  const long long t = base / nx;
  const int y0 = (int)(t % ny);
  const int z0 = (int)(t / ny);
  const double h = 1.0 / (nm + 1);
  const double h2 = h * h;
  const long long as = m == 0 ? 1LL : (m == 1 ? (long long)(nx + 2) : (long long)(nx + 2) * (ny + 2));
  const long long a0 = dim == 3 ? ((long long)(z0 + 1) * (ny + 2) + (y0 + 1)) * (nx + 2) + (x0 + 1)
                                : (long long)(y0 + 1) * (nx + 2) + (x0 + 1);
  double dprev = 1.0, offprev = 0.0;
  for (int i = 0; i < nm; ++i) {
    double ai = a ? a[a0 + i * as] : 1.0;
    double am = a ? 0.5 * (ai + a[a0 + (i - 1) * as]) : 1.0;
    double ap = a ? 0.5 * (ai + a[a0 + (i + 1) * as]) : 1.0;
    double diag = 1.0 + tau * (am + ap) / h2 + tau * cM;
    double li = 0.0, di = diag;
    if (i > 0) {
      li = offprev / dprev;
      di = diag - li * offprev;
    }
    long long idx = !var ? (long long)i : (m == 0 ? (long long)i * lines + L : base + i * S);
    double ri = 1.0 / di;
    l[idx] = li;
    r[idx] = ri;
    if (l32) {
      l32[idx] = (float)li;
      r32[idx] = (float)ri;
    }
    dprev = di;
    offprev = -tau * ap / h2;
  }
}

template <typename T>
__device__ __forceinline__ T to(double v);
template <>
__device__ __forceinline__ double to<double>(double v) { return v; }
template <>
__device__ __forceinline__ float to<float>(double v) { return (float)v; }

// ---------------------------------------------------------------------------------------
// a2 + a3: x-direction substep (lines are contiguous rows).  A block stages R whole rows in
// shared memory with coalesced loads (adding tau * src * src_t on the way in when SRC), R
// threads run the two recurrences in shared memory, and the block writes the rows back
// coalesced.  ld = row pitch in shared memory, odd so that thread t's row start t*ld hits
// distinct banks.
template <typename Tin, typename Tout, typename Tc, bool VAR, bool SRC>
__device__ __forceinline__ void sweep_x_body(long long blk, Tc* sm, const Tin* in, Tout* out, long long rows, int nx,
                                             int ld, int R, long long rows_per_slice, const Tc* __restrict__ fl,
                                             const Tc* __restrict__ fr, const SourceArgs& sa) {
  const long long row0 = blk * R;
  const int nrows = (int)min((long long)R, rows - row0);
  // one warp per row, lanes along the row: coalesced, and no per-element index division
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
  for (int rr = warp; rr < nrows; rr += nwarps) {
    const long long row = row0 + rr;
    const Tin* grow = in + row * nx;
    Tc* srow = sm + rr * ld;
    if (SRC) {
      const long long sl = row / rows_per_slice;
      const double* s = sa.src + (row - sl * rows_per_slice) * nx;
      const double c = sa.tau * (sa.src_t ? sa.src_t[sa.t0 + sl * sa.tstride] : 1.0);
      if constexpr (sizeof(Tc) == 8) {
        // one rounding, as the staged coarse sweep (ps_coarse.cu) forms b + tau f
        for (int cc = lane; cc < nx; cc += 32) srow[cc] = fma(c, s[cc], (double)grow[cc]);
      } else {
        for (int cc = lane; cc < nx; cc += 32) srow[cc] = (Tc)grow[cc] + to<Tc>(c * s[cc]);
      }
    } else {
      for (int cc = lane; cc < nx; cc += 32) srow[cc] = (Tc)grow[cc];
    }
  }
  __syncthreads();
  if (threadIdx.x < nrows) {
    Tc* x = sm + threadIdx.x * ld;
    // factors: transposed layout (entry (row, i) at i * rows_per_slice + row)
    const long long ris = (row0 + threadIdx.x) % rows_per_slice;
    const Tc* L = fl + (VAR ? ris : 0);
    const Tc* Rr = fr + (VAR ? ris : 0);
    const long long fs = VAR ? rows_per_slice : 1;
    // chunks of K elements: the shared-memory and factor loads of a chunk issue together, so
    // one factor-load latency is paid per chunk (the arithmetic order does not depend on K;
    // 16-node chunks measured slower here: they cost occupancy)
    constexpr int K = 8;
    constexpr int KB = 8;
    Tc y = x[0];
    for (int i0 = 1; i0 < nx; i0 += K) {
      Tc b[K], l[K];
#pragma unroll
      for (int u = 0; u < K; ++u) {
        const int i = i0 + u;
        b[u] = i < nx ? x[i] : Tc(0);
        l[u] = i < nx ? L[i * fs] : Tc(0);
      }
#pragma unroll
      for (int u = 0; u < K; ++u) {
        if (i0 + u < nx) {
          y = fma(-l[u], y, b[u]);  // explicit: the same rounding as the staged sweeps
          x[i0 + u] = y;
        }
      }
    }
    Tc xn = y;
    for (int i0 = nx - 1; i0 >= 0; i0 -= KB) {
      Tc yy[KB], r[KB], l[KB];
#pragma unroll
      for (int u = 0; u < KB; ++u) {
        const int i = i0 - u;
        yy[u] = i >= 0 ? x[i] : Tc(0);
        r[u] = i >= 0 ? Rr[i * fs] : Tc(0);
        l[u] = (i >= 0 && i + 1 < nx) ? L[(i + 1) * fs] : Tc(0);
      }
#pragma unroll
      for (int u = 0; u < KB; ++u) {
        const int i = i0 - u;
        if (i >= 0) {
          xn = (i == nx - 1) ? r[u] * yy[u] : fma(-l[u], xn, r[u] * yy[u]);
          x[i] = xn;
        }
      }
    }
  }
  __syncthreads();
  for (int rr = warp; rr < nrows; rr += nwarps) {
    Tout* grow = out + (row0 + rr) * nx;
    const Tc* srow = sm + rr * ld;
    for (int cc = lane; cc < nx; cc += 32) grow[cc] = (Tout)srow[cc];
  }
}

template <typename Tin, typename Tout, typename Tc, bool VAR, bool SRC>
__global__ void __launch_bounds__(kThreads) sweep_x_kernel(const Tin* in, Tout* out, long long rows, int nx,
                                                          int ld, int R, long long rows_per_slice,
                                                          const Tc* __restrict__ fl, const Tc* __restrict__ fr,
                                                          SourceArgs sa) {
  extern __shared__ unsigned char smem_raw[];
  sweep_x_body<Tin, Tout, Tc, VAR, SRC>(blockIdx.x, reinterpret_cast<Tc*>(smem_raw), in, out, rows, nx, ld, R,
                                         rows_per_slice, fl, fr, sa);
}

// ---------------------------------------------------------------------------------------
// a3/a4 (coarse x-substep, FP32): one warp per row, the two recurrences of the L D L^T solve
// as segmented scans.  Both are first-order affine,  y_i = -l_i y_{i-1} + b_i  and
// x_i = -l_{i+1} x_{i+1} + r_i y_i,  so lane j composes the maps of its segment of m nodes
// (A = product of the -l, B = the segment run from a zero input), a five-step shuffle scan
// composes the segments, and each lane replays its segment from the exact incoming value.
// The dependent chain is 3m + 10 operations per recurrence instead of L.  The row and its
// factor rows are staged in shared memory with element i at i + i/m (m even), so the
// segment reads of the 32 lanes fall in distinct banks.
template <typename T>
__device__ __forceinline__ void warp_line_solve_skewed(T* xb, const T* lb, const T* rb, int L, int m,
                                                       int lane) {
  const unsigned full = 0xffffffffu;
  const int base = lane * (m + 1);
  const int cnt = max(0, min(m, L - lane * m));
  T A = T(1), B = T(0);
  for (int u = 0; u < cnt; ++u) {
    const T l = lb[base + u];
    B = xb[base + u] - l * B;
    A = -l * A;
  }
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const T Ap = __shfl_up_sync(full, A, d), Bp = __shfl_up_sync(full, B, d);
    if (lane >= d) {
      B = A * Bp + B;
      A = A * Ap;
    }
  }
  T y = __shfl_up_sync(full, B, 1);
  if (lane == 0) y = T(0);
  for (int u = 0; u < cnt; ++u) {
    y = xb[base + u] - lb[base + u] * y;
    xb[base + u] = y;
  }
  __syncwarp();
  // l_{i+1} past the segment's end: the next segment's first factor (0 past the line)
  const T lnext = (lane * m + cnt < L) ? lb[base + m + 1] : T(0);
  A = T(1);
  B = T(0);
  for (int u = cnt - 1; u >= 0; --u) {
    const T ln = (u + 1 < cnt) ? lb[base + u + 1] : lnext;
    B = rb[base + u] * xb[base + u] - ln * B;
    A = -ln * A;
  }
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const T An = __shfl_down_sync(full, A, d), Bn = __shfl_down_sync(full, B, d);
    if (lane + d < 32) {
      B = A * Bn + B;
      A = A * An;
    }
  }
  T xv = __shfl_down_sync(full, B, 1);
  if (lane == 31) xv = T(0);
  for (int u = cnt - 1; u >= 0; --u) {
    const T ln = (u + 1 < cnt) ? lb[base + u + 1] : lnext;
    xv = rb[base + u] * xb[base + u] - ln * xv;
    xb[base + u] = xv;
  }
  __syncwarp();
}

// One slice: rows of nx nodes, line-major factor rows lt/rt (pitch Lp).  SRC adds
// tau * src * src_t[t0] to the right-hand side on the way in.
// One row by one warp: stage the row (plus tau f when SRC) and its line-major factor rows in
// the warp's shared memory with the skewed pitch, solve, write back.
template <typename T, typename Tin, bool SRC>
__device__ __forceinline__ void warp_row(long long row, const Tin* __restrict__ in, T* __restrict__ out, int nx, int m,
                                         const T* __restrict__ lt, const T* __restrict__ rt, int Lp,
                                         const SourceArgs& sa, T* xb, T* lb, T* rb, int lane) {
  const double c = SRC ? sa.tau * (sa.src_t ? sa.src_t[sa.t0] : 1.0) : 0.0;
  const Tin* gin = in + row * nx;
  const T* gl = lt + row * Lp;
  const T* gr = rt + row * Lp;
  for (int i = lane; i < nx; i += 32) {
    const int k = i + i / m;
    T b = (T)gin[i];
    if constexpr (sizeof(T) == 8) {
      if (SRC) b = fma(c, sa.src[row * nx + i], (double)b);
    } else {
      if (SRC) b = b + (float)(c * sa.src[row * nx + i]);
    }
    xb[k] = b;
    lb[k] = gl[i];
    rb[k] = gr[i];
  }
  // one slot past the line: the backward step reads the next segment's first factor there
  if (lane == 0) lb[nx + nx / m] = T(0);
  __syncwarp();
  warp_line_solve_skewed(xb, lb, rb, nx, m, lane);
  for (int i = lane; i < nx; i += 32) out[row * nx + i] = xb[i + i / m];
  __syncwarp();
}

template <typename T, typename Tin, bool SRC>
__global__ void __launch_bounds__(256) sweep_x_warp_kernel(const Tin* __restrict__ in, T* __restrict__ out,
                                                           long long rows, int nx, int m, int span,
                                                           const T* __restrict__ lt, const T* __restrict__ rt,
                                                           int Lp, SourceArgs sa) {
  extern __shared__ __align__(16) unsigned char wsm_raw[];
  T* wsm = reinterpret_cast<T*>(wsm_raw);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  T* xb = wsm + (size_t)warp * 3 * span;
  T* lb = xb + span;
  T* rb = lb + span;
  for (long long row = (long long)blockIdx.x * nw + warp; row < rows; row += (long long)gridDim.x * nw)
    warp_row<T, Tin, SRC>(row, in, out, nx, m, lt, rt, Lp, sa, xb, lb, rb, lane);
}

__device__ __forceinline__ void atomic_max_nonneg(unsigned long long* addr, double v) {
  // nonnegative doubles order like their bit patterns
  atomicMax(addr, (unsigned long long)__double_as_longlong(v));
}

// |v| as the bit pattern of a nonnegative double.  Maxima of such patterns are taken with
// 64-bit integer instructions: they order like the values, and GB300's FP64 pipe, which
// the line recurrences already saturate, is left to the recurrences.
__device__ __forceinline__ unsigned long long abs_bits(double v) {
  return (unsigned long long)__double_as_longlong(v) & 0x7fffffffffffffffull;
}
constexpr unsigned long long kInfBits = 0x7ff0000000000000ull;  // |v| bits >= this: inf or NaN

// ---------------------------------------------------------------------------------------
// a3/a4: y- or z-direction substep, one thread per line; consecutive threads take
// consecutive x so every access of a warp is one coalesced row segment.  The forward
// recurrence stores y_i in `tmp` (the output, or the coarse scratch state; its type is the
// output type, which holds the recurrence type exactly), the backward one reads it back.  EPI = 1 fuses the parareal correction of Sec. 3 into the backward
// recurrence of the last sweep of a coarse step:
//     U_{n+1} <- Fout + (g - Gold),  Gold <- g,  inc <- max(inc, |U_{n+1}^new - U_{n+1}^old|)
// EPI = 2 is the initial coarse sweep: U_{n+1} <- g, Gold <- g.
template <typename Tin, typename Tout, typename Tc, bool VAR, bool SRC, int EPI, bool AHEAD>
__device__ __forceinline__ void sweep_strided_body(long long blk, const Tin* in, Tout* out, Tout* tmp, long long lines,
                                                   int nm, long long S, long long nt, const Tc* __restrict__ fl,
                                                   const Tc* __restrict__ fr, const SourceArgs& sa,
                                                   const CorrArgs& ca) {
  const long long L = blk * blockDim.x + threadIdx.x;
  unsigned long long my_inc = 0, my_norm = 0;  // bit patterns of nonnegative doubles
  bool bad = false;
  if (L < lines) {
    const long long outer = L / S;
    const long long base = outer * S * nm + (L - outer * S);
    const long long sl = base / nt;
    const long long pos = base - sl * nt;  // position inside the slice
    const Tc* Lf = fl + (VAR ? pos : 0);
    const Tc* Rf = fr + (VAR ? pos : 0);
    const long long fs = VAR ? S : 1;
    double ft = 0.0;
    if (SRC) ft = sa.tau * (sa.src_t ? sa.src_t[sa.t0 + sl * sa.tstride] : 1.0);
    // forward recurrence; the loads of each chunk of K elements are issued together (one
    // memory latency per chunk; the arithmetic order does not depend on K).  Wider chunks
    // cost registers here: every element carries its own 64-bit address.
    constexpr int K = 8;
    Tc y = (Tc)in[base];
    if (SRC) y = y + to<Tc>(ft * sa.src[pos]);
    if constexpr (AHEAD) {
      // chunk loads one chunk ahead, issued before the previous chunk's stores (the compiler
      // cannot hoist them itself: in and tmp may be the same array).  Chosen at launch for
      // short line strides (y-lines); long-stride sweeps (z-lines) keep the plain loop below,
      // which measured faster there.
      auto load_chunk = [&](int i0, Tc* b, Tc* l) {
#pragma unroll
        for (int u = 0; u < K; ++u) {
          const int i = i0 + u;
          b[u] = i < nm ? (Tc)in[base + i * S] : Tc(0);
          l[u] = i < nm ? Lf[i * fs] : Tc(0);
          if (SRC) b[u] = b[u] + (i < nm ? to<Tc>(ft * sa.src[pos + i * S]) : Tc(0));
        }
      };
      Tc bn[K], ln[K];
      load_chunk(1, bn, ln);
      tmp[base] = (Tout)y;
      for (int i0 = 1; i0 < nm; i0 += K) {
        Tc b[K], l[K];
#pragma unroll
        for (int u = 0; u < K; ++u) {
          b[u] = bn[u];
          l[u] = ln[u];
        }
        if (i0 + K < nm) load_chunk(i0 + K, bn, ln);
#pragma unroll
        for (int u = 0; u < K; ++u) {
          if (i0 + u < nm) {
            y = fma(-l[u], y, b[u]);
            tmp[base + (i0 + u) * S] = (Tout)y;
          }
        }
      }
    } else {
      tmp[base] = (Tout)y;
      for (int i0 = 1; i0 < nm; i0 += K) {
        Tc b[K], l[K];
#pragma unroll
        for (int u = 0; u < K; ++u) {
          const int i = i0 + u;
          b[u] = i < nm ? (Tc)in[base + i * S] : Tc(0);
          l[u] = i < nm ? Lf[i * fs] : Tc(0);
          if (SRC) b[u] = b[u] + (i < nm ? to<Tc>(ft * sa.src[pos + i * S]) : Tc(0));
        }
#pragma unroll
        for (int u = 0; u < K; ++u) {
          if (i0 + u < nm) {
            y = fma(-l[u], y, b[u]);
            tmp[base + (i0 + u) * S] = (Tout)y;
          }
        }
      }
    }
    // backward recurrence (chunks of KB), with the correction of Sec. 3 fused when EPI != 0
    constexpr int KB = 4;
    Tc xn = y;
    for (int i0 = nm - 1; i0 >= 0; i0 -= KB) {
      Tc yy[KB], r[KB], l[KB];
      double fo[KB], go[KB], uo[KB];
#pragma unroll
      for (int u = 0; u < KB; ++u) {
        const int i = i0 - u;
        const bool ok = i >= 0;
        yy[u] = ok ? (Tc)tmp[base + i * S] : Tc(0);
        r[u] = ok ? Rf[i * fs] : Tc(0);
        l[u] = (ok && i + 1 < nm) ? Lf[(i + 1) * fs] : Tc(0);
        if (EPI == 1 || EPI == 3) {
          const long long si = pos + (long long)(ok ? i : 0) * S;
          if (EPI == 1) go[u] = ok ? ca.Gold[si] : 0.0;
          fo[u] = ok ? ca.Fout[si] : 0.0;
          uo[u] = ok ? ca.U_next[si] : 0.0;
        }
      }
#pragma unroll
      for (int u = 0; u < KB; ++u) {
        const int i = i0 - u;
        if (i >= 0) {
          xn = (i == nm - 1) ? r[u] * yy[u] : fma(-l[u], xn, r[u] * yy[u]);
          const long long gi = base + i * S;
          if (EPI == 0) {
            out[gi] = (Tout)xn;
          } else {
            const long long si = pos + i * S;  // coarse steps run on one slice
            const double g = (double)xn;
            if (EPI == 1) {
              const double unew = fo[u] + (g - go[u]);
              const unsigned long long an = abs_bits(unew);
              bad |= an >= kInfBits;
              my_inc = max(my_inc, abs_bits(unew - uo[u]));
              my_norm = max(my_norm, an);
              ca.Gold[si] = g;
              ca.U_next[si] = unew;
            } else if (EPI == 3) {
              // G is affine, so G(U^k) - G(U^{k-1}) is its linear part applied to the increment
              const double unew = fo[u] + g;
              const double d = unew - uo[u];
              const unsigned long long an = abs_bits(unew);
              bad |= an >= kInfBits;
              my_inc = max(my_inc, abs_bits(d));
              my_norm = max(my_norm, an);
              ca.U_next[si] = unew;
              ca.dnext[si] = (float)d;
            } else {
              bad |= abs_bits(g) >= kInfBits;
              if (ca.Gold) ca.Gold[si] = g;
              ca.U_next[si] = g;
            }
          }
        }
      }
    }
  }
  if (EPI == 1 || EPI == 3) {
    for (int o = 16; o > 0; o >>= 1) {
      my_inc = max(my_inc, __shfl_xor_sync(0xffffffffu, my_inc, o));
      my_norm = max(my_norm, __shfl_xor_sync(0xffffffffu, my_norm, o));
    }
    if ((threadIdx.x & 31) == 0 && my_inc > 0) atomicMax(ca.inc, my_inc);
    if ((threadIdx.x & 31) == 0 && ca.slice_stats) {
      if (my_inc > 0) atomicMax(ca.slice_stats, my_inc);
      if (my_norm > 0) atomicMax(ca.slice_stats + 1, my_norm);
    }
  }
  if (EPI != 0) {
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicExch(ca.nonfinite, 1);
  }
}

template <typename Tin, typename Tout, typename Tc, bool VAR, bool SRC, int EPI, bool AHEAD>
__global__ void __launch_bounds__(kThreads) sweep_strided_kernel(const Tin* in, Tout* out, Tout* tmp, long long lines,
                                                                int nm, long long S, long long nt,
                                                                const Tc* __restrict__ fl, const Tc* __restrict__ fr,
                                                                SourceArgs sa, CorrArgs ca) {
  sweep_strided_body<Tin, Tout, Tc, VAR, SRC, EPI, AHEAD>(blockIdx.x, in, out, tmp, lines, nm, S, nt, fl, fr, sa, ca);
}

// ---------------------------------------------------------------------------------------
// y/z-substep without source (FP64, or FP32 for the coarse increment form), the loads pipelined
// through shared memory: the same operations in the same order as sweep_strided_body, so the
// two give the same bits.  Each
// thread copies its own line's next chunk (right-hand side or stored y, factors, and the
// correction's Gold / Fout / old U_{n+1}) with cp.async into its column of a node-major
// [array][j][t] stage while it runs the recurrences on the current chunk; no other thread
// reads that column, so the thread's own wait_group is the only synchronisation.  Every copy
// and store of a warp is one 128- or 256-byte row segment.  On GB300 the FP64 pipe, not HBM, sets the
// pace of these sweeps (6 FP64 operations per node with the correction, against 56 bytes):
// the point is to keep every line's next loads in flight so that the pipe never waits on
// memory, with one wave of 4 CTAs x 128 lines per SM.
constexpr int SC_T = 128;
constexpr int SC_NS = 3;                // stages: the copies run two chunks ahead of the recurrences
constexpr int SC_STAGE_BYTES = 16384;   // per stage and CTA
constexpr size_t kScSmem = (size_t)SC_NS * SC_STAGE_BYTES;

template <typename E>
__device__ __forceinline__ void cpa(E* dst, const E* src) {
  static_assert(sizeof(E) == 4 || sizeof(E) == 8, "4- or 8-byte elements");
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src),
               "n"(sizeof(E))
               : "memory");
}
__device__ __forceinline__ void cpa_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cpa_wait_ahead() {
  asm volatile("cp.async.wait_group %0;" ::"n"(SC_NS - 1) : "memory");
}

// Lines [blk * SC_T, blk * SC_T + SC_T) of one sweep.  T: the recurrences' type (right-hand
// side, y, x, factors); the correction's arrays (Gold, Fout, old U_{n+1}) are FP64.  csm:
// SC_NS stages of SC_STAGE_BYTES, each laid out as the sweep arrays [a][j][t] of T, then the
// correction arrays [e][j][t] of double.  Within a pass thread t touches only its own columns;
// between the passes (and between calls) the CTA synchronises.  All copies are complete when
// it returns.  Every thread of the CTA calls it.
template <typename T, bool VAR, int EPI>
__device__ __forceinline__ void strided_chunk_lines(long long blk, const T* in, T* out, T* tmp, long long lines,
                                                    int nm, long long S, long long nt, const T* __restrict__ fl,
                                                    const T* __restrict__ fr, const CorrArgs& ca,
                                                    unsigned char* csm) {
  constexpr int CF = SC_STAGE_BYTES / ((VAR ? 2 : 1) * SC_T * (int)sizeof(T));  // forward chunk: u (+ l)
  constexpr int NSB = 1 + (VAR ? 2 : 0);                                        // y (+ r, l)
  constexpr int NEB = EPI == 1 ? 3 : EPI == 3 ? 2 : 0;                          // Gold, Fout, old U
  constexpr int CBr = SC_STAGE_BYTES / (SC_T * (NSB * (int)sizeof(T) + NEB * 8));
  constexpr int CB = CBr < 24 ? CBr : 24;                                       // backward chunk
  const int tid = threadIdx.x;
  const long long L = blk * SC_T + tid;
  const bool active = L < lines;
  long long base = 0, pos = 0;
  if (active) {
    const long long outer = L / S;
    base = outer * S * nm + (L - outer * S);
    pos = base - (base / nt) * nt;
  }
  const T* Lf = fl + (VAR ? pos : 0);
  const T* Rf = fr + (VAR ? pos : 0);
  const long long fs = VAR ? S : 1;
  unsigned long long my_inc = 0, my_norm = 0;
  bool bad = false;
  // forward  y_i = b_i - l_i y_{i-1}, stored to tmp
  const int nchF = (nm + CF - 1) / CF;
  auto stage_f = [&](int k) {
    T* st = reinterpret_cast<T*>(csm + (k % SC_NS) * SC_STAGE_BYTES);
    if (active)
      for (int j = 0; j < CF; ++j) {
        const int i = k * CF + j;
        if (i < nm) {
          cpa(st + j * SC_T + tid, in + base + i * S);
          if (VAR) cpa(st + (CF + j) * SC_T + tid, Lf + i * fs);
        }
      }
    cpa_commit();
  };
  T y = T(0);
  for (int k = 0; k < SC_NS - 1; ++k) {
    if (k < nchF) stage_f(k);
    else cpa_commit();
  }
  for (int k = 0; k < nchF; ++k) {
    // chunk k + NS - 1 goes into the stage that chunk k - 1 used (its reads are done); then all
    // but the NS - 1 newest groups are complete, chunk k among them
    if (k + SC_NS - 1 < nchF) stage_f(k + SC_NS - 1);
    else cpa_commit();
    cpa_wait_ahead();
    if (active) {
      const T* st = reinterpret_cast<const T*>(csm + (k % SC_NS) * SC_STAGE_BYTES);
      const int len = min(CF, nm - k * CF);
#pragma unroll
      for (int j = 0; j < CF; ++j) {
        if (j < len) {
          const int i = k * CF + j;
          const T b = st[j * SC_T + tid];
          const T l = VAR ? st[(CF + j) * SC_T + tid] : Lf[i * fs];
          y = i == 0 ? b : fma(-l, y, b);
          tmp[base + i * S] = y;
        }
      }
    }
  }
  // The backward stages use another layout than the forward ones: with FP32 sweeps a thread's
  // FP64 correction slots overlap other threads' forward columns, so no thread may stage a
  // backward chunk while another still reads its forward chunks.  The barrier also orders this
  // thread's y stores before the copies that read them back.
  __syncthreads();
  // backward  x_i = r_i y_i - l_{i+1} x_{i+1}, nodes from the end, with the epilogue
  const int nchB = (nm + CB - 1) / CB;
  auto stage_b = [&](int k) {
    T* st = reinterpret_cast<T*>(csm + (k % SC_NS) * SC_STAGE_BYTES);
    double* se = reinterpret_cast<double*>(st + NSB * CB * SC_T);
    if (active)
      for (int j = 0; j < CB; ++j) {
        const int i = nm - 1 - (k * CB + j);
        if (i >= 0) {
          cpa(st + j * SC_T + tid, tmp + base + i * S);
          if (VAR) {
            cpa(st + (CB + j) * SC_T + tid, Rf + i * fs);
            if (i + 1 < nm) cpa(st + (2 * CB + j) * SC_T + tid, Lf + (i + 1) * fs);
          }
          const long long si = pos + (long long)i * S;
          int e = 0;
          if (EPI == 1) cpa(se + (e++ * CB + j) * SC_T + tid, ca.Gold + si);
          if (EPI == 1 || EPI == 3) {
            cpa(se + (e++ * CB + j) * SC_T + tid, ca.Fout + si);
            cpa(se + (e++ * CB + j) * SC_T + tid, ca.U_next + si);
          }
        }
      }
    cpa_commit();
  };
  // y_{nm-1} is read back like every other y: the stored value is the register's
  T xn = T(0);
  for (int k = 0; k < SC_NS - 1; ++k) {
    if (k < nchB) stage_b(k);
    else cpa_commit();
  }
  for (int k = 0; k < nchB; ++k) {
    if (k + SC_NS - 1 < nchB) stage_b(k + SC_NS - 1);
    else cpa_commit();
    cpa_wait_ahead();
    if (active) {
      const T* st = reinterpret_cast<const T*>(csm + (k % SC_NS) * SC_STAGE_BYTES);
      const double* se = reinterpret_cast<const double*>(st + NSB * CB * SC_T);
#pragma unroll
      for (int j = 0; j < CB; ++j) {
        const int i = nm - 1 - (k * CB + j);
        if (i >= 0) {
          const T yy = st[j * SC_T + tid];
          T r, l;
          if (VAR) {
            r = st[(CB + j) * SC_T + tid];
            l = i + 1 < nm ? st[(2 * CB + j) * SC_T + tid] : T(0);
          } else {
            r = Rf[i * fs];
            l = i + 1 < nm ? Lf[(i + 1) * fs] : T(0);
          }
          xn = i == nm - 1 ? r * yy : fma(-l, xn, r * yy);
          const long long si = pos + (long long)i * S;
          const double g = (double)xn;
          int e = 0;
          if (EPI == 0) {
            out[base + i * S] = xn;
          } else if (EPI == 1) {
            const double go = se[(e++ * CB + j) * SC_T + tid];
            const double fo = se[(e++ * CB + j) * SC_T + tid];
            const double uo = se[(e++ * CB + j) * SC_T + tid];
            const double unew = fo + (g - go);
            const unsigned long long an = abs_bits(unew);
            bad |= an >= kInfBits;
            my_inc = max(my_inc, abs_bits(unew - uo));
            my_norm = max(my_norm, an);
            ca.Gold[si] = g;
            ca.U_next[si] = unew;
          } else if (EPI == 3) {
            // G is affine, so G(U^k) - G(U^{k-1}) is its linear part applied to the increment
            const double fo = se[(e++ * CB + j) * SC_T + tid];
            const double uo = se[(e++ * CB + j) * SC_T + tid];
            const double unew = fo + g;
            const double d = unew - uo;
            const unsigned long long an = abs_bits(unew);
            bad |= an >= kInfBits;
            my_inc = max(my_inc, abs_bits(d));
            my_norm = max(my_norm, an);
            ca.U_next[si] = unew;
            ca.dnext[si] = (float)d;
          } else {
            bad |= abs_bits(g) >= kInfBits;
            if (ca.Gold) ca.Gold[si] = g;
            ca.U_next[si] = g;
          }
        }
      }
    }
  }
  if (EPI == 1 || EPI == 3) {
    for (int o = 16; o > 0; o >>= 1) {
      my_inc = max(my_inc, __shfl_xor_sync(0xffffffffu, my_inc, o));
      my_norm = max(my_norm, __shfl_xor_sync(0xffffffffu, my_norm, o));
    }
    if ((threadIdx.x & 31) == 0 && my_inc > 0) atomicMax(ca.inc, my_inc);
    if ((threadIdx.x & 31) == 0 && ca.slice_stats) {
      if (my_inc > 0) atomicMax(ca.slice_stats, my_inc);
      if (my_norm > 0) atomicMax(ca.slice_stats + 1, my_norm);
    }
  }
  if (EPI != 0) {
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicExch(ca.nonfinite, 1);
  }
}

template <typename T, bool VAR, int EPI>
__global__ void __launch_bounds__(SC_T, 4)
    sweep_strided_chunk_kernel(const T* in, T* out, T* tmp, long long lines, int nm, long long S, long long nt,
                               const T* __restrict__ fl, const T* __restrict__ fr, CorrArgs ca) {
  extern __shared__ __align__(16) unsigned char csm[];
  const long long nblk = (lines + SC_T - 1) / SC_T;
  for (long long blk = blockIdx.x; blk < nblk; blk += gridDim.x) {
    strided_chunk_lines<T, VAR, EPI>(blk, in, out, tmp, lines, nm, S, nt, fl, fr, ca, csm);
    __syncthreads();  // the next group of lines stages in the forward layout again
  }
}

// ---------------------------------------------------------------------------------------
// Grouped coarse steps (batched problems, 2-D, FP64, no source): one launch runs the same
// sweep of many problems' coarse step n.  jobs[j] describes problem j's sweep; the first
// *nseg segments of `segs` list (job, first block, block count, prefix) runs of blocks.
__device__ __forceinline__ int find_segment(const WorkSeg* segs, int nseg, long long it) {
  int lo = 0, hi = nseg - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (segs[mid].prefix <= it) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}


template <bool VAR, int EPI, int AX>
__global__ void __launch_bounds__(SC_T, 4) sweep_y_grouped_kernel(const CoarseJob* __restrict__ jobs,
                                                                  const WorkSeg* __restrict__ segs,
                                                                  const int* __restrict__ nseg_ptr) {
  extern __shared__ __align__(16) unsigned char csm[];
  const int nseg = *nseg_ptr;
  if (nseg <= 0) return;
  const long long total = (long long)segs[nseg - 1].prefix + segs[nseg - 1].count;
  for (long long it = blockIdx.x; it < total; it += gridDim.x) {
    const WorkSeg sg = segs[find_segment(segs, nseg, it)];
    const CoarseJob& j = jobs[sg.job];
    // AX 1: y-lines (nx * nz, stride nx); AX 2: z-lines (nx * ny, stride nx * ny)
    const long long S = AX == 1 ? (long long)j.nx : (long long)j.nx * j.ny;
    const long long lines = AX == 1 ? (long long)j.nx * j.nz : (long long)j.nx * j.ny;
    strided_chunk_lines<double, VAR, EPI>(sg.first + (it - sg.prefix), j.xout, j.xout, j.xout, lines,
                                          AX == 1 ? j.ny : j.nz, S, j.nt, AX == 1 ? j.ly : j.lz,
                                          AX == 1 ? j.ry : j.rz, j.ca, csm);
    __syncthreads();  // the next item stages in the forward layout again
  }
}

// Grouped FP32 increment-form coarse steps (batches of PS_COARSE_DELTA32 problems), the same
// per-row and per-line bodies as the single-problem launches.  x: one warp per row, eight rows
// per work item; the input is the FP64 state with the source (initial sweep) or the FP32
// increment.  y: one thread per line with the increment-form (mode 3) or initial (mode 2)
// epilogue.
__global__ void __launch_bounds__(256) sweep_x32_grouped_kernel(const XWarpJob* __restrict__ jobs,
                                                                const WorkSeg* __restrict__ segs,
                                                                const int* __restrict__ nseg_ptr, int span_max) {
  extern __shared__ __align__(16) unsigned char wsm_raw[];
  float* wsm = reinterpret_cast<float*>(wsm_raw);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  float* xb = wsm + (size_t)warp * 3 * span_max;
  float* lb = xb + span_max;
  float* rb = lb + span_max;
  const int nseg = *nseg_ptr;
  if (nseg <= 0) return;
  const long long total = (long long)segs[nseg - 1].prefix + segs[nseg - 1].count;
  for (long long it = blockIdx.x; it < total; it += gridDim.x) {
    const WorkSeg sg = segs[find_segment(segs, nseg, it)];
    const XWarpJob& j = jobs[sg.job];
    const long long row = (sg.first + (it - sg.prefix)) * nw + warp;
    if (row < j.rows) {
      if (j.in64) {
        if (j.sa.src)
          warp_row<float, double, true>(row, j.in64, j.out, j.nx, j.m, j.lt, j.rt, j.Lp, j.sa, xb, lb, rb, lane);
        else
          warp_row<float, double, false>(row, j.in64, j.out, j.nx, j.m, j.lt, j.rt, j.Lp, j.sa, xb, lb, rb, lane);
      } else {
        warp_row<float, float, false>(row, j.in32, j.out, j.nx, j.m, j.lt, j.rt, j.Lp, SourceArgs{}, xb, lb, rb,
                                      lane);
      }
    }
  }
}

template <bool VAR, int EPI, int AX>
__global__ void __launch_bounds__(SC_T) sweep_y32_grouped_kernel(const CoarseJob* __restrict__ jobs,
                                                                 const WorkSeg* __restrict__ segs,
                                                                 const int* __restrict__ nseg_ptr) {
  // FP32 lines of a batch: the streamed body (loads one chunk ahead in registers); the staged
  // chunk body measured slower here, where each problem has few lines and every line's chain
  // of dependent FP32 steps is short in time
  const int nseg = *nseg_ptr;
  if (nseg <= 0) return;
  const long long total = (long long)segs[nseg - 1].prefix + segs[nseg - 1].count;
  for (long long it = blockIdx.x; it < total; it += gridDim.x) {
    const WorkSeg sg = segs[find_segment(segs, nseg, it)];
    const CoarseJob& j = jobs[sg.job];
    const long long S = AX == 1 ? (long long)j.nx : (long long)j.nx * j.ny;
    const long long lines = AX == 1 ? (long long)j.nx * j.nz : (long long)j.nx * j.ny;
    sweep_strided_body<float, float, float, VAR, false, EPI, true>(sg.first + (it - sg.prefix), j.g32, j.g32, j.g32,
                                                                   lines, AX == 1 ? j.ny : j.nz, S, j.nt,
                                                                   AX == 1 ? j.ly32 : j.lz32,
                                                                   AX == 1 ? j.ry32 : j.rz32, SourceArgs{}, j.ca);
  }
}

__global__ void copy_inc_grouped_kernel(const CoarseJob* __restrict__ jobs, const WorkSeg* __restrict__ segs,
                                        const int* __restrict__ nseg_ptr) {
  const int nseg = *nseg_ptr;
  if (nseg <= 0) return;
  const long long total = (long long)segs[nseg - 1].prefix + segs[nseg - 1].count;
  for (long long it = blockIdx.x; it < total; it += gridDim.x) {
    const WorkSeg sg = segs[find_segment(segs, nseg, it)];
    const CoarseJob& j = jobs[sg.job];
    const long long i = (sg.first + (it - sg.prefix)) * blockDim.x + threadIdx.x;
    double my = 0.0, nrm = 0.0;
    bool bad = false;
    if (i < j.nt) {
      const double v = j.xin[i];
      const double d = v - j.xout[i];
      my = fabs(d);
      nrm = fabs(v);
      bad = !isfinite(v);
      j.xout[i] = v;
      if (j.ca.dnext) j.ca.dnext[i] = (float)d;  // the increment form's FP32 increment of slice k
    }
    for (int o = 16; o > 0; o >>= 1) {
      my = fmax(my, __shfl_xor_sync(0xffffffffu, my, o));
      nrm = fmax(nrm, __shfl_xor_sync(0xffffffffu, nrm, o));
    }
    if ((threadIdx.x & 31) == 0) {
      if (my > 0.0) atomic_max_nonneg(j.ca.inc, my);
      if (j.ca.slice_stats) {
        if (my > 0.0) atomic_max_nonneg(j.ca.slice_stats, my);
        if (nrm > 0.0) atomic_max_nonneg(j.ca.slice_stats + 1, nrm);
      }
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicExch(j.ca.nonfinite, 1);
  }
}

__global__ void copy_inc_kernel(long long n, const double* __restrict__ src, double* __restrict__ dst,
                                unsigned long long* inc, int* nonfinite, unsigned long long* slice_stats,
                                float* __restrict__ dout) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double my = 0.0, nrm = 0.0;
  bool bad = false;
  for (; i < n; i += (long long)gridDim.x * blockDim.x) {
    double v = src[i];
    const double d = v - dst[i];
    my = fmax(my, fabs(d));
    nrm = fmax(nrm, fabs(v));
    if (!isfinite(v)) bad = true;
    dst[i] = v;
    if (dout) dout[i] = (float)d;
  }
  for (int o = 16; o > 0; o >>= 1) {
    my = fmax(my, __shfl_xor_sync(0xffffffffu, my, o));
    nrm = fmax(nrm, __shfl_xor_sync(0xffffffffu, nrm, o));
  }
  if ((threadIdx.x & 31) == 0 && my > 0.0) atomic_max_nonneg(inc, my);
  if ((threadIdx.x & 31) == 0 && slice_stats) {
    if (my > 0.0) atomic_max_nonneg(slice_stats, my);
    if (nrm > 0.0) atomic_max_nonneg(slice_stats + 1, nrm);
  }
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicExch(nonfinite, 1);
}

// SMs of the current device, queried per call (the device may differ between calls)
int sm_count() {
  int dev = 0, n = 0;
  PS_CUDA(cudaGetDevice(&dev));
  PS_CUDA(cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev));
  return n;
}
int g_max_smem = 0;
int max_dyn_smem() {
  if (!g_max_smem) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  }
  return g_max_smem;
}

template <typename Tin, typename Tout, typename Tc, bool VAR, bool SRC>
void launch_x(const Geom& g, int nslices, const Tc* fl, const Tc* fr, const Tin* in, Tout* out, const SourceArgs& sa,
              cudaStream_t st) {
  const int nx = g.n[0];
  const long long rows_per_slice = g.nt / nx;
  const long long rows = rows_per_slice * nslices;
  const int ld = (nx % 2) ? nx : nx + 1;
  const int budget = 96 * 1024;
  int R = std::max(1, std::min(sizeof(Tc) == 8 ? 32 : 64, budget / (int)(ld * sizeof(Tc))));
  size_t smem = (size_t)R * ld * sizeof(Tc);
  if ((int)smem > max_dyn_smem()) throw Error(PS_ERR_UNSUPPORTED, "x-line too long for shared memory");
  auto kern = sweep_x_kernel<Tin, Tout, Tc, VAR, SRC>;
  static bool attr_set = false;
  if (!attr_set) {
    PS_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, max_dyn_smem()));
    attr_set = true;
  }
  long long blocks = (rows + R - 1) / R;
  kern<<<(unsigned)blocks, kThreads, smem, st>>>(in, out, rows, nx, ld, R, rows_per_slice, fl, fr, sa);
  PS_CUDA(cudaGetLastError());
}

template <typename Tin, typename Tout, typename Tc, bool VAR, bool SRC, int EPI>
void launch_strided(const Geom& g, int m, int nslices, const Tc* fl, const Tc* fr, const Tin* in, Tout* out, Tout* tmp,
                    const SourceArgs& sa, const CorrArgs& ca, cudaStream_t st) {
  const int nm = g.n[m];
  const long long S = g.stride(m);
  const long long lines = (g.nt / nm) * nslices;
  if constexpr (std::is_same<Tin, Tc>::value && std::is_same<Tout, Tc>::value && !SRC &&
                (sizeof(Tc) == 8 ? EPI != 3 : EPI != 1)) {
    // the loads pipelined through shared memory (same arithmetic as sweep_strided_body)
    long long cblocks = (lines + SC_T - 1) / SC_T;
    if (chain_ctas_per_sm > 0) cblocks = std::min<long long>(cblocks, (long long)sm_count() * chain_ctas_per_sm);
    sweep_strided_chunk_kernel<Tc, VAR, EPI><<<(unsigned)cblocks, SC_T, kScSmem, st>>>(
        in, out, tmp, lines, nm, S, g.nt, fl, fr, ca);
    PS_CUDA(cudaGetLastError());
    return;
  }
  long long blocks = (lines + kThreads - 1) / kThreads;
  if (S * (long long)sizeof(Tin) <= 8192)
    sweep_strided_kernel<Tin, Tout, Tc, VAR, SRC, EPI, true>
        <<<(unsigned)blocks, kThreads, 0, st>>>(in, out, tmp, lines, nm, S, g.nt, fl, fr, sa, ca);
  else
    sweep_strided_kernel<Tin, Tout, Tc, VAR, SRC, EPI, false>
        <<<(unsigned)blocks, kThreads, 0, st>>>(in, out, tmp, lines, nm, S, g.nt, fl, fr, sa, ca);
  PS_CUDA(cudaGetLastError());
}

template <typename Tin, typename Tout, typename Tc>
void dispatch(const Geom& g, int nslices, const LineFactors& f, const Tc* fl, const Tc* fr, const Tin* in, Tout* out,
              const SourceArgs& sa, const CorrArgs& ca, Tout* tmp, cudaStream_t st) {
  static_assert(sizeof(Tout) >= sizeof(Tc), "the output type must hold the recurrence type");
  const bool var = f.var != 0, src = sa.src != nullptr;
  if (f.m == 0) {
    PS_REQUIRE(ca.mode == 0, "the correction is fused into a y/z sweep only");
    if constexpr (sizeof(Tin) == 8 && sizeof(Tout) == 8 && sizeof(Tc) == 8) {
      // FP64 rows of 32 nodes or more: the chunked sweep (same arithmetic, more rows in flight)
      if (sweep_x_chunked(g, nslices, f, in, out, sa, st)) return;
    }
    if (var) {
      if (src) launch_x<Tin, Tout, Tc, true, true>(g, nslices, fl, fr, in, out, sa, st);
      else launch_x<Tin, Tout, Tc, true, false>(g, nslices, fl, fr, in, out, sa, st);
    } else {
      if (src) launch_x<Tin, Tout, Tc, false, true>(g, nslices, fl, fr, in, out, sa, st);
      else launch_x<Tin, Tout, Tc, false, false>(g, nslices, fl, fr, in, out, sa, st);
    }
    return;
  }
  Tout* t = tmp ? tmp : out;
#define PS_STRIDED(V, S_, E) launch_strided<Tin, Tout, Tc, V, S_, E>(g, f.m, nslices, fl, fr, in, out, t, sa, ca, st)
  if (ca.mode == 0) {
    if (var) { if (src) PS_STRIDED(true, true, 0); else PS_STRIDED(true, false, 0); }
    else { if (src) PS_STRIDED(false, true, 0); else PS_STRIDED(false, false, 0); }
  } else if (ca.mode == 1) {
    if constexpr (sizeof(Tc) == 8) {
      if (var) { if (src) PS_STRIDED(true, true, 1); else PS_STRIDED(true, false, 1); }
      else { if (src) PS_STRIDED(false, true, 1); else PS_STRIDED(false, false, 1); }
    } else {
      throw Error(PS_ERR_INVALID, "the standard correction runs with FP64 recurrences");
    }
  } else if (ca.mode == 3) {
    if constexpr (sizeof(Tc) == 4 && sizeof(Tout) == 4) {
      PS_REQUIRE(ca.dnext && ca.Fout && ca.U_next, "increment-form correction needs Fout, U_next and dnext");
      if (var) PS_STRIDED(true, false, 3); else PS_STRIDED(false, false, 3);
    } else {
      throw Error(PS_ERR_INVALID, "the increment-form correction runs with FP32 recurrences");
    }
  } else {
    if (var) { if (src) PS_STRIDED(true, true, 2); else PS_STRIDED(true, false, 2); }
    else { if (src) PS_STRIDED(false, true, 2); else PS_STRIDED(false, false, 2); }
  }
#undef PS_STRIDED
}

}  // namespace

void factor_dim(const Geom& g, int m, const double* a_nodal, double c_over_M, double tau, LineFactors& f,
                bool want_f32, cudaStream_t st) {
  const int nm = g.n[m];
  f.m = m;
  f.var = a_nodal ? 1 : 0;
  const size_t cnt = f.var ? (size_t)g.nt : (size_t)nm;
  f.l64.alloc(cnt);
  f.r64.alloc(cnt);
  if (want_f32) {
    f.l32.alloc(cnt);
    f.r32.alloc(cnt);
  }
  const long long lines = f.var ? g.nt / nm : 1;
  long long blocks = (lines + 127) / 128;
  factor_dim_kernel<<<(unsigned)blocks, 128, 0, st>>>(g.dim, g.n[0], g.n[1], g.dim == 3 ? g.n[2] : 1, m, a_nodal,
                                                      c_over_M, tau, f.l64.p, f.r64.p, want_f32 ? f.l32.p : nullptr,
                                                      want_f32 ? f.r32.p : nullptr, lines, f.var);
  PS_CUDA(cudaGetLastError());
}

template <typename Tin, typename Tout>
void sweep_dim(const Geom& g, int nslices, const LineFactors& f, bool fp32, const Tin* in, Tout* out,
               const SourceArgs& sa, const CorrArgs& ca, double* tmp, cudaStream_t st) {
  if (fp32) {
    PS_REQUIRE(f.l32.p != nullptr, "FP32 factors missing");
    PS_REQUIRE(tmp == nullptr && ca.mode != 1, "FP32 sweeps carry only the initial or increment-form epilogue");
    dispatch<Tin, Tout, float>(g, nslices, f, f.l32.p, f.r32.p, in, out, sa, ca, nullptr, st);
  } else {
    if constexpr (sizeof(Tout) == 8) {
      dispatch<Tin, Tout, double>(g, nslices, f, f.l64.p, f.r64.p, in, out, sa, ca, reinterpret_cast<Tout*>(tmp), st);
    } else {
      throw Error(PS_ERR_INVALID, "an FP64 sweep needs an FP64 output");
    }
  }
}

template void sweep_dim<double, double>(const Geom&, int, const LineFactors&, bool, const double*, double*,
                                        const SourceArgs&, const CorrArgs&, double*, cudaStream_t);
template void sweep_dim<double, float>(const Geom&, int, const LineFactors&, bool, const double*, float*,
                                       const SourceArgs&, const CorrArgs&, double*, cudaStream_t);
template void sweep_dim<float, float>(const Geom&, int, const LineFactors&, bool, const float*, float*,
                                      const SourceArgs&, const CorrArgs&, double*, cudaStream_t);
template void sweep_dim<float, double>(const Geom&, int, const LineFactors&, bool, const float*, double*,
                                       const SourceArgs&, const CorrArgs&, double*, cudaStream_t);

template <typename Tin, typename T>
void sweep_x_warp(const Geom& g, const LineFactors& f, const Tin* in, T* out, const SourceArgs& sa, cudaStream_t st) {
  const T* lt = sizeof(T) == 4 ? reinterpret_cast<const T*>(f.lt32.p) : reinterpret_cast<const T*>(f.lt64.p);
  const T* rt = sizeof(T) == 4 ? reinterpret_cast<const T*>(f.rt32.p) : reinterpret_cast<const T*>(f.rt64.p);
  PS_REQUIRE(f.m == 0 && lt && rt, "the warp x-sweep needs line-major x factors of its precision");
  const int nx = g.n[0];
  const long long rows = g.nt / nx;
  const int m = ((nx + 31) / 32 + 1) & ~1;  // even: the skewed pitch m + 1 is odd
  const int span = nx + nx / m + 2;
  const int Lp = (nx + 3) & ~3;
  const int threads = 256;
  const size_t smem = (size_t)(threads / 32) * 3 * span * sizeof(T);
  PS_REQUIRE(smem <= (size_t)max_dyn_smem(), "x-line too long for the warp x-sweep");
  int dev = 0, sms = 0;
  PS_CUDA(cudaGetDevice(&dev));
  PS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const long long want = (rows + threads / 32 - 1) / (threads / 32);
  const unsigned grid = (unsigned)std::min<long long>(want, (long long)sms * 8);
  auto launch = [&](auto kern) {
    PS_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<grid, threads, smem, st>>>(in, out, rows, nx, m, span, lt, rt, Lp, sa);
  };
  if (sa.src) launch(sweep_x_warp_kernel<T, Tin, true>);
  else launch(sweep_x_warp_kernel<T, Tin, false>);
  PS_CUDA(cudaGetLastError());
}
template void sweep_x_warp<float, float>(const Geom&, const LineFactors&, const float*, float*, const SourceArgs&,
                                         cudaStream_t);
template void sweep_x_warp<double, float>(const Geom&, const LineFactors&, const double*, float*, const SourceArgs&,
                                          cudaStream_t);
template void sweep_x_warp<double, double>(const Geom&, const LineFactors&, const double*, double*,
                                           const SourceArgs&, cudaStream_t);

int max_dyn_smem_public() { return max_dyn_smem(); }

int coarse_y_grouped_lines() { return SC_T; }

void coarse_y_grouped(bool var, int epi, const CoarseJob* jobs, const WorkSeg* segs, const int* nseg, int grid,
                      cudaStream_t st, int axis) {
  auto go = [&](auto kern) { kern<<<grid, SC_T, kScSmem, st>>>(jobs, segs, nseg); };
  if (axis == 1) {
    if (var) {
      if (epi == 1) go(sweep_y_grouped_kernel<true, 1, 1>);
      else if (epi == 2) go(sweep_y_grouped_kernel<true, 2, 1>);
      else go(sweep_y_grouped_kernel<true, 0, 1>);
    } else {
      if (epi == 1) go(sweep_y_grouped_kernel<false, 1, 1>);
      else if (epi == 2) go(sweep_y_grouped_kernel<false, 2, 1>);
      else go(sweep_y_grouped_kernel<false, 0, 1>);
    }
  } else {
    if (var) {
      if (epi == 1) go(sweep_y_grouped_kernel<true, 1, 2>);
      else go(sweep_y_grouped_kernel<true, 2, 2>);
    } else {
      if (epi == 1) go(sweep_y_grouped_kernel<false, 1, 2>);
      else go(sweep_y_grouped_kernel<false, 2, 2>);
    }
  }
  PS_CUDA(cudaGetLastError());
}
void coarse_x32_grouped(const XWarpJob* jobs, const WorkSeg* segs, const int* nseg, int grid, int span_max,
                        cudaStream_t st) {
  const size_t smem = (size_t)(kThreads / 32) * 3 * span_max * sizeof(float);
  PS_CUDA(cudaFuncSetAttribute(sweep_x32_grouped_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  sweep_x32_grouped_kernel<<<grid, kThreads, smem, st>>>(jobs, segs, nseg, span_max);
  PS_CUDA(cudaGetLastError());
}
void coarse_y32_grouped(bool var, int epi, const CoarseJob* jobs, const WorkSeg* segs, const int* nseg, int grid,
                        cudaStream_t st, int axis) {
  // twice the CTAs of 128 lines: as many resident lines as the other grouped launches' 256-thread CTAs
  auto go = [&](auto kern) { kern<<<grid * 2, SC_T, 0, st>>>(jobs, segs, nseg); };
  if (axis == 1) {
    if (var) {
      if (epi == 3) go(sweep_y32_grouped_kernel<true, 3, 1>);
      else if (epi == 2) go(sweep_y32_grouped_kernel<true, 2, 1>);
      else go(sweep_y32_grouped_kernel<true, 0, 1>);
    } else {
      if (epi == 3) go(sweep_y32_grouped_kernel<false, 3, 1>);
      else if (epi == 2) go(sweep_y32_grouped_kernel<false, 2, 1>);
      else go(sweep_y32_grouped_kernel<false, 0, 1>);
    }
  } else {
    if (var) {
      if (epi == 3) go(sweep_y32_grouped_kernel<true, 3, 2>);
      else go(sweep_y32_grouped_kernel<true, 2, 2>);
    } else {
      if (epi == 3) go(sweep_y32_grouped_kernel<false, 3, 2>);
      else go(sweep_y32_grouped_kernel<false, 2, 2>);
    }
  }
  PS_CUDA(cudaGetLastError());
}
void copy_inc_grouped(const CoarseJob* jobs, const WorkSeg* segs, const int* nseg, int grid, cudaStream_t st) {
  copy_inc_grouped_kernel<<<grid, kThreads, 0, st>>>(jobs, segs, nseg);
  PS_CUDA(cudaGetLastError());
}

void copy_with_increment(long long nt, const double* src, double* dst, unsigned long long* inc, int* nonfinite,
                         unsigned long long* slice_stats, float* dout, cudaStream_t st) {
  long long blocks = std::min<long long>((nt + 255) / 256, 152 * 8);
  copy_inc_kernel<<<(unsigned)blocks, 256, 0, st>>>(nt, src, dst, inc, nonfinite, slice_stats, dout);
  PS_CUDA(cudaGetLastError());
}

}  // namespace ps
