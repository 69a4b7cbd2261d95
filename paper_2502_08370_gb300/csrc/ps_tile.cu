// ps_tile.cu -- the fine propagator's batched line solves on the slice-interleaved layout.
//
// During a fine phase every time slice advances with the same step size, so all slices
// share the substep factors.  The fine working state is kept interleaved,
//     W[z][y][x][s]   (slice index fastest, S_pad slots),
// which turns every direction x, y, z into a batch of strided lines whose 32 consecutive
// slices form one warp: a warp walks 32 lines that share every factor (one broadcast
// load) and whose elements at one line position are one 128-/256-byte row.
//
// A CTA owns a tile of TS slices x P positions of a second axis x the whole line (L nodes).
// The tile moves between HBM and shared memory by TMA (cp.async.bulk.tensor, one load and
// one store per 256-node chunk of the line), its factors and source are staged in shared
// memory, and TS*P threads run the two recurrences of the L D L^T solve in shared memory:
//     forward   y_i = b_i - l_i y_{i-1}
//     backward  x_i = r_i y_i - l_{i+1} x_{i+1}
// so each element is read from and written to HBM exactly once per substep.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

#include "ps_async.h"
#include "ps_tile.h"

namespace ps {
namespace {

constexpr int kPipeStages = 3;  // shared-memory stages of the persistent tile kernel

__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, uint64_t* bar, int c0, int c1, int c2,
                                            int c3) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5, %6}], "
      "[%2];" ::"r"(smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_addr(bar)), "r"(c0), "r"(c1), "r"(c2), "r"(c3)
      : "memory");
}
__device__ __forceinline__ void tma_store_4d(const CUtensorMap* map, const void* src, int c0, int c1, int c2, int c3) {
  asm volatile("cp.async.bulk.tensor.4d.global.shared::cta.tile.bulk_group [%0, {%2, %3, %4, %5}], [%1];" ::"l"(
                   reinterpret_cast<uint64_t>(map)),
               "r"(smem_addr(src)), "r"(c0), "r"(c1), "r"(c2), "r"(c3)
               : "memory");
}
__device__ __forceinline__ void tma_store_commit_and_drain() {
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
  asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}

// Tile geometry shared by host and device.
struct TileArgs {
  int axis;          // 0 = x, 1 = y, 2 = z: direction of the lines
  int L;             // line length (n_axis)
  int nb;            // extent of the paired axis b (P positions per tile)
  int P, TS;         // positions and slices per tile
  int n[3];          // nx, ny, nz
  int s_lo, s_hi;    // slice groups [s_lo, s_hi) of TS slots each
  int nbt;           // tiles along b
  int chunks;        // TMA chunks along the line (box extent <= 256)
  int chunk;         // nodes per chunk
  int var;           // factors per node (1) or shared by all lines (0)
  long long rows_x;  // ny*nz: leading dimension of the transposed x-factors
  const void* fl;       // factor rows l of every line: [line][Lp], line = c * nb + b
  const void* fr;       // factor rows r, same layout
  const void* srcrow;   // source rows (x-lines of a step's first substep) [line][Lp] or null
  int Lp;               // row length: L rounded up to 4, zero padded
  const double* src;    // non-null when the source is added
  const double* src_t;  // time factors or null
  int t_first, t_slice; // time index of slot s: t_first + s * t_slice
  int src_t_len;
  double tau;
  int* err;
};

// One (problem, direction) of a grouped launch, and a run of its tiles.
struct alignas(64) TileJob {
  CUtensorMap map;
  TileArgs a;
};

// Offset of element i of line (slot-in-tile s, position p) in the tile's shared memory,
// which mirrors the TMA box order (slice fastest, then x, y, z of the box).
__device__ __forceinline__ int tile_off(const TileArgs& a, int s, int p, int i) {
  return a.axis == 0 ? (p * a.L + i) * a.TS + s : (i * a.P + p) * a.TS + s;
}

// Bytes the factor (and source) rows of a tile add to its barrier's transaction count.
template <typename T, bool SRC>
__device__ __forceinline__ uint32_t side_bytes(const TileArgs& a, int nvalid) {
  return (uint32_t)((SRC ? 3 : 2) * nvalid * a.Lp * (int)sizeof(T));
}
// Factor (and source) rows of the tile's valid positions: nvalid consecutive lines.
template <typename T, bool SRC>
__device__ __forceinline__ void issue_side_loads(const TileArgs& a, int b0, int c, int nvalid, T* fl_s, T* fr_s,
                                                 T* src_s, uint64_t* bar) {
  const long long row = (long long)c * a.nb + b0;
  const uint32_t bytes = (uint32_t)(nvalid * a.Lp * (int)sizeof(T));
  bulk_load(fl_s, reinterpret_cast<const T*>(a.fl) + row * a.Lp, bytes, bar);
  bulk_load(fr_s, reinterpret_cast<const T*>(a.fr) + row * a.Lp, bytes, bar);
  if (SRC) bulk_load(src_s, reinterpret_cast<const T*>(a.srcrow) + row * a.Lp, bytes, bar);
}
// tau * src_t at the end time of the step, for interleaved slot `slot`.
template <typename T>
__device__ __forceinline__ T slot_time_factor(const TileArgs& a, int slot, int t_first) {
  const int ti = t_first + slot * a.t_slice;
  const double f = a.src_t ? (ti >= 0 && ti < a.src_t_len ? a.src_t[ti] : 0.0) : 1.0;
  return (T)(a.tau * f);
}

// V adjacent slots of one line position, as one vector access (V * sizeof(T) bytes).
template <typename T, int V>
struct alignas(sizeof(T) * V) VecT {
  T v[V];
};
// Four consecutive factors (16- or 32-byte aligned rows, padded with zeros past L).
template <typename T>
struct alignas(sizeof(T) * 4) Quad {
  T q[4];
};

// The three roundings of a node, written as explicit FMAs so that every kernel that solves a
// line (one tile per CTA, pipelined chunks, persistent, grouped) computes the same bits:
//     b + f * ft (source),   y = b - l y,   x = r y - l' x
template <typename T>
__device__ __forceinline__ T fmat(T a, T b, T c) {
  if constexpr (sizeof(T) == 4) return fmaf(a, b, c);
  else return fma(a, b, c);
}
template <typename T>
__device__ __forceinline__ T rhs_node(T b, T f, T ft) { return fmat(f, ft, b); }
template <typename T>
__device__ __forceinline__ T fwd_node(T y, T b, T l) { return fmat(-l, y, b); }
template <typename T>
__device__ __forceinline__ T bwd_node(T x, T yv, T r, T ln) { return fmat(-ln, x, r * yv); }

// The two recurrences of the L D L^T solve for V lines (adjacent slots, one thread) held
// in shared memory, element i of the V lines at x + i*st.  Factors are shared by the V
// lines and read four at a time; l_0 = 0 and the zero padding past L make the first and
// last steps uniform:
//     forward   y_i = b_i - l_i y_{i-1}            (y_{-1} = 0)
//     backward  x_i = r_i y_i - l_{i+1} x_{i+1}    (x_L = 0, l_L = 0)
// The source, when present, enters the right-hand side: b_i += src_i * ft[v].
template <typename T, int V, bool SRC>
__device__ __forceinline__ void line_solve(T* x, int st, int L, const T* Lf, const T* Rf, const T* S, const T* ft) {
  using VT = VecT<T, V>;
  using QT = Quad<T>;
  // Each chunk of four nodes is loaded one chunk ahead, into registers, before the previous
  // chunk is stored: the compiler cannot move those loads above the stores itself (it does
  // not know that st > 0), and without them every chunk would wait a full shared-memory
  // latency before its dependent FMAs.  The arithmetic is the same in every order.
  T y[V];
#pragma unroll
  for (int v = 0; v < V; ++v) y[v] = T(0);
  const int nq = L / 4;
  QT l4n{}, s4n{};
  VT bn[4];
  if (nq > 0) {
    l4n = *reinterpret_cast<const QT*>(Lf);
    if (SRC) s4n = *reinterpret_cast<const QT*>(S);
#pragma unroll
    for (int u = 0; u < 4; ++u) bn[u] = *reinterpret_cast<const VT*>(x + u * st);
  }
  for (int c = 0; c < nq; ++c) {
    const int i0 = 4 * c;
    const QT l4 = l4n;
    const QT s4 = s4n;
    VT b[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) b[u] = bn[u];
    if (c + 1 < nq) {
      l4n = *reinterpret_cast<const QT*>(Lf + i0 + 4);
      if (SRC) s4n = *reinterpret_cast<const QT*>(S + i0 + 4);
#pragma unroll
      for (int u = 0; u < 4; ++u) bn[u] = *reinterpret_cast<const VT*>(x + (i0 + 4 + u) * st);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
#pragma unroll
      for (int v = 0; v < V; ++v) {
        T bb = b[u].v[v];
        if (SRC) bb = rhs_node(bb, s4.q[u], ft[v]);
        y[v] = fwd_node(y[v], bb, l4.q[u]);
        b[u].v[v] = y[v];
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) *reinterpret_cast<VT*>(x + (i0 + u) * st) = b[u];
  }
  for (int i = 4 * nq; i < L; ++i) {
    VT b = *reinterpret_cast<const VT*>(x + i * st);
    const T li = Lf[i];
#pragma unroll
    for (int v = 0; v < V; ++v) {
      T bb = b.v[v];
      if (SRC) bb = rhs_node(bb, S[i], ft[v]);
      y[v] = fwd_node(y[v], bb, li);
      b.v[v] = y[v];
    }
    *reinterpret_cast<VT*>(x + i * st) = b;
  }
  T xn[V];
#pragma unroll
  for (int v = 0; v < V; ++v) xn[v] = T(0);
  T lnext = T(0);  // l_{i+1} for the step at i
  for (int i = L - 1; i >= 4 * nq; --i) {
    VT yy = *reinterpret_cast<const VT*>(x + i * st);
    const T ri = Rf[i];
#pragma unroll
    for (int v = 0; v < V; ++v) {
      xn[v] = bwd_node(xn[v], yy.v[v], ri, lnext);
      yy.v[v] = xn[v];
    }
    *reinterpret_cast<VT*>(x + i * st) = yy;
    lnext = Lf[i];
  }
  QT r4n{};
  VT yyn[4];
  if (nq > 0) {
    const int i0 = 4 * (nq - 1);
    r4n = *reinterpret_cast<const QT*>(Rf + i0);
    l4n = *reinterpret_cast<const QT*>(Lf + i0);
#pragma unroll
    for (int u = 0; u < 4; ++u) yyn[u] = *reinterpret_cast<const VT*>(x + (i0 + u) * st);
  }
  for (int c = nq - 1; c >= 0; --c) {
    const int i0 = 4 * c;
    const QT r4 = r4n;
    const QT l4 = l4n;
    VT yy[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) yy[u] = yyn[u];
    if (c > 0) {
      r4n = *reinterpret_cast<const QT*>(Rf + i0 - 4);
      l4n = *reinterpret_cast<const QT*>(Lf + i0 - 4);
#pragma unroll
      for (int u = 0; u < 4; ++u) yyn[u] = *reinterpret_cast<const VT*>(x + (i0 - 4 + u) * st);
    }
#pragma unroll
    for (int u = 3; u >= 0; --u) {
      const T l1 = u == 3 ? lnext : l4.q[u + 1];
#pragma unroll
      for (int v = 0; v < V; ++v) {
        xn[v] = bwd_node(xn[v], yy[u].v[v], r4.q[u], l1);
        yy[u].v[v] = xn[v];
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) *reinterpret_cast<VT*>(x + (i0 + u) * st) = yy[u];
    lnext = l4.q[0];
  }
}

// Tile t -> (first slot, first paired position, fixed coordinate).
__device__ __forceinline__ void tile_coords(const TileArgs& a, int t, int* s0, int* b0, int* c) {
  const int ngroups = a.s_hi - a.s_lo;
  *s0 = (a.s_lo + t % ngroups) * a.TS;
  t /= ngroups;
  *b0 = (t % a.nbt) * a.P;
  *c = t / a.nbt;
}

// One tile: TMA load of the slots x positions x line block (and the line-major factor /
// source rows by bulk copies) completing on `bar` (phase `parity`), the recurrences in
// shared memory, TMA store back.  Thread 0 alone polls the barrier within its time limit
// and shares the outcome.  Returns false (after setting *a.err) when the load timed out.
// Shared memory from `tile` (128-byte aligned): [tile data | factors l | factors r | source].
template <typename T, int V, bool SRC>
__device__ __forceinline__ bool tile_body(const CUtensorMap* map, const TileArgs& a, int t, T* tile, uint64_t* bar,
                                          uint32_t parity, int t_first) {
  __shared__ int s_ok;
  const int lines = a.TS * a.P;
  const int Lp = a.Lp;
  T* fl_s = reinterpret_cast<T*>((reinterpret_cast<uintptr_t>(tile + (size_t)lines * a.L) + 31) & ~(uintptr_t)31);
  T* fr_s = fl_s + (size_t)a.P * Lp;
  T* src_s = fr_s + (size_t)a.P * Lp;
  int s0, b0, c;
  tile_coords(a, t, &s0, &b0, &c);
  const int tid = threadIdx.x;
  const int nvalid = min(a.P, a.nb - b0);  // positions of this tile inside the grid
  if (tid == 0) {
    if (a.axis == 0) {
      // x-lines: one box (TS slots x chunk nodes) per position and chunk
      mbar_expect_tx(bar, (uint32_t)(nvalid * a.L * a.TS * (int)sizeof(T)) + side_bytes<T, SRC>(a, nvalid));
      issue_side_loads<T, SRC>(a, b0, c, nvalid, fl_s, fr_s, src_s, bar);
      for (int p = 0; p < nvalid; ++p)
        for (int k = 0; k < a.chunks; ++k) {
          const int i0 = k * a.chunk;
          tma_load_4d(tile + ((size_t)p * a.L + i0) * a.TS, map, bar, s0, i0, b0 + p, c);
        }
    } else {
      // y/z-lines: one box (TS slots x P positions x chunk nodes) per chunk
      mbar_expect_tx(bar, (uint32_t)(lines * a.L * (int)sizeof(T)) + side_bytes<T, SRC>(a, nvalid));
      issue_side_loads<T, SRC>(a, b0, c, nvalid, fl_s, fr_s, src_s, bar);
      for (int k = 0; k < a.chunks; ++k) {
        const int i0 = k * a.chunk;
        T* dst = tile + (size_t)i0 * a.P * a.TS;
        if (a.axis == 1) tma_load_4d(dst, map, bar, s0, b0, i0, c);
        else tma_load_4d(dst, map, bar, s0, b0, c, i0);
      }
    }
    s_ok = mbar_wait(bar, parity) ? 1 : 0;
    if (!s_ok) atomicExch(a.err, 1);
  }
  __syncthreads();
  if (!s_ok) return false;
  if (tid != 0) mbar_wait(bar, parity);  // completed: acquires the tile's bytes
  const int per_row = a.TS / V;          // threads per line position
  const int s = (tid % per_row) * V, p = tid / per_row;
  if (p < a.P && b0 + p < a.nb) {
    T ft[V];
#pragma unroll
    for (int v = 0; v < V; ++v) ft[v] = SRC ? slot_time_factor<T>(a, s0 + s + v, t_first) : T(0);
    line_solve<T, V, SRC>(tile + tile_off(a, s, p, 0), a.axis == 0 ? a.TS : a.P * a.TS, a.L, fl_s + p * Lp,
                          fr_s + p * Lp, src_s + p * Lp, ft);
  }
  fence_async_smem();
  __syncthreads();
  if (tid == 0) {
    if (a.axis == 0) {
      for (int p = 0; p < nvalid; ++p)
        for (int k = 0; k < a.chunks; ++k) {
          const int i0 = k * a.chunk;
          tma_store_4d(map, tile + ((size_t)p * a.L + i0) * a.TS, s0, i0, b0 + p, c);
        }
    } else {
      for (int k = 0; k < a.chunks; ++k) {
        const int i0 = k * a.chunk;
        const T* srcp = tile + (size_t)i0 * a.P * a.TS;
        if (a.axis == 1) tma_store_4d(map, srcp, s0, b0, i0, c);
        else tma_store_4d(map, srcp, s0, b0, c, i0);
      }
    }
    tma_store_commit_and_drain();
  }
  __syncthreads();
  return true;
}

// Shared memory of a tile kernel: [barrier (128 bytes) | tile ...].
template <typename T, int V, bool SRC>
__global__ void tile_sweep_kernel(const __grid_constant__ CUtensorMap map, TileArgs a) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw);
  T* tile = reinterpret_cast<T*>(smem_raw + 128);
  __shared__ int s_abort;
  const int tid = threadIdx.x;
  if (tid == 0) {
    // once a tile has timed out the launch is abandoned: later tiles start no copies
    s_abort = *reinterpret_cast<volatile int*>(a.err);
    // TMA tensor copies need 128-byte aligned shared-memory destinations
    if (smem_addr(tile) & 127) {
      atomicExch(a.err, 2);
      s_abort = 1;
    }
    if (!s_abort) {
      mbar_init(bar, 1);
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
  }
  __syncthreads();
  if (s_abort) return;
  tile_body<T, V, SRC>(&map, a, blockIdx.x, tile, bar, 0, a.t_first);
}

// Grouped, persistent form: many problems' tiles in one launch.  jobs[j] holds one
// (problem, direction)'s tensor map and tile arguments (in global memory, 64-byte aligned);
// the first *nseg segments of `segs` list which tiles of which job run, with running
// prefix counts.  Each CTA walks the items t = blockIdx.x, blockIdx.x + gridDim.x, ...
// Jobs with a source (x tiles of problems with f != 0) add tau f at the end of fine step
// `step` of each slot: time index step + 1 + slot * t_slice.
template <typename T, int V>
__global__ void tile_sweep_grouped_kernel(const TileJob* __restrict__ jobs, const WorkSeg* __restrict__ segs,
                                          const int* __restrict__ nseg_ptr, int* err, int step) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw);
  T* tile = reinterpret_cast<T*>(smem_raw + 128);
  __shared__ int s_abort;
  const int nseg = *nseg_ptr;
  if (nseg <= 0) return;
  const long long total = (long long)segs[nseg - 1].prefix + segs[nseg - 1].count;
  if (threadIdx.x == 0) {
    s_abort = *reinterpret_cast<volatile int*>(err);
    if (smem_addr(tile) & 127) {
      atomicExch(err, 2);
      s_abort = 1;
    }
    if (!s_abort) {
      mbar_init(bar, 1);
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
  }
  __syncthreads();
  if (s_abort) return;
  uint32_t parity = 0;
  for (long long it = blockIdx.x; it < total; it += gridDim.x) {
    // segment of item `it`: the last segment whose prefix is <= it
    int lo = 0, hi = nseg - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (segs[mid].prefix <= it) lo = mid;
      else hi = mid - 1;
    }
    const WorkSeg sg = segs[lo];
    const TileJob& job = jobs[sg.job];
    // the tensor map lives in global memory (written by a host copy): acquire it for the
    // tensormap proxy before TMA reads it
    if (threadIdx.x == 0)
      asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(&job.map) : "memory");
    const int tt = sg.first + (int)(it - sg.prefix);
    const bool ok = job.a.src ? tile_body<T, V, true>(&job.map, job.a, tt, tile, bar, parity, step + 1)
                              : tile_body<T, V, false>(&job.map, job.a, tt, tile, bar, parity, 0);
    if (!ok) return;
    parity ^= 1u;
  }
}


template <typename T, bool SRC>
__device__ __forceinline__ void issue_tile_load(const CUtensorMap* map, const TileArgs& a, T* buf, T* fl_s, T* fr_s,
                                                T* src_s, uint64_t* bar, int t) {
  int s0, b0, c;
  tile_coords(a, t, &s0, &b0, &c);
  const int nvalid = min(a.P, a.nb - b0);
  if (a.axis == 0) {
    mbar_expect_tx(bar, (uint32_t)(nvalid * a.L * a.TS * (int)sizeof(T)) + side_bytes<T, SRC>(a, nvalid));
    issue_side_loads<T, SRC>(a, b0, c, nvalid, fl_s, fr_s, src_s, bar);
    for (int p = 0; p < nvalid; ++p)
      for (int k = 0; k < a.chunks; ++k) {
        const int i0 = k * a.chunk;
        tma_load_4d(buf + ((size_t)p * a.L + i0) * a.TS, map, bar, s0, i0, b0 + p, c);
      }
  } else {
    mbar_expect_tx(bar, (uint32_t)(a.TS * a.P * a.L * (int)sizeof(T)) + side_bytes<T, SRC>(a, nvalid));
    issue_side_loads<T, SRC>(a, b0, c, nvalid, fl_s, fr_s, src_s, bar);
    for (int k = 0; k < a.chunks; ++k) {
      const int i0 = k * a.chunk;
      T* dst = buf + (size_t)i0 * a.P * a.TS;
      if (a.axis == 1) tma_load_4d(dst, map, bar, s0, b0, i0, c);
      else tma_load_4d(dst, map, bar, s0, b0, c, i0);
    }
  }
}

template <typename T>
__device__ __forceinline__ void issue_tile_store(const CUtensorMap* map, const TileArgs& a, const T* buf, int t) {
  int s0, b0, c;
  tile_coords(a, t, &s0, &b0, &c);
  const int nvalid = min(a.P, a.nb - b0);
  if (a.axis == 0) {
    for (int p = 0; p < nvalid; ++p)
      for (int k = 0; k < a.chunks; ++k) {
        const int i0 = k * a.chunk;
        tma_store_4d(map, buf + ((size_t)p * a.L + i0) * a.TS, s0, i0, b0 + p, c);
      }
  } else {
    for (int k = 0; k < a.chunks; ++k) {
      const int i0 = k * a.chunk;
      const T* srcp = buf + (size_t)i0 * a.P * a.TS;
      if (a.axis == 1) tma_store_4d(map, srcp, s0, b0, i0, c);
      else tma_store_4d(map, srcp, s0, b0, c, i0);
    }
  }
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}

// Persistent form: each CTA walks tiles t = blockIdx.x, blockIdx.x + gridDim.x, ... through a
// ring of kPipeStages shared-memory stages.  While tile k is solved, the loads of tiles
// k+1 .. k+kPipeStages-2 are in flight and the store of tile k-1 drains; the stage of tile
// k-1 is refilled once its store has been read out (wait_group.read 1 leaves only tile k's
// store pending), so no thread waits on a store it has just issued.  Thread 0 alone polls a
// stage's barrier (bounded by kWaitNs) and shares the outcome; on a timeout the CTA records
// the error, drains the loads it has in flight (bounded) and returns.
template <typename T, int V, bool SRC>
__global__ void tile_sweep_pipe_kernel(const __grid_constant__ CUtensorMap map, TileArgs a, int ntiles) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  constexpr int R = kPipeStages;
  const int lines = a.TS * a.P;
  const int Lp = a.Lp;
  const size_t tile_elems = (size_t)lines * a.L;
  const size_t side = (size_t)a.P * Lp;
  T* buf0 = reinterpret_cast<T*>(smem_raw);
  // per stage: l, r (and source) of the tile's positions, rows of Lp entries, 32-byte aligned
  T* fac0 = reinterpret_cast<T*>((reinterpret_cast<uintptr_t>(buf0 + R * tile_elems) + 31) & ~(uintptr_t)31);
  const size_t fac_stride = SRC ? 3 * side : 2 * side;
  uint64_t* bars = reinterpret_cast<uint64_t*>(
      (reinterpret_cast<uintptr_t>(fac0 + R * fac_stride) + 15) & ~(uintptr_t)15);
  __shared__ int s_ok;
  const int tid = threadIdx.x;
  auto stage_load = [&](int stage, int t) {
    T* fl = fac0 + stage * fac_stride;
    issue_tile_load<T, SRC>(&map, a, buf0 + stage * tile_elems, fl, fl + side, fl + 2 * side, &bars[stage], t);
  };
  if (tid == 0) {
    s_ok = *reinterpret_cast<volatile int*>(a.err) ? 0 : 1;
    if (smem_addr(buf0) & 127) {  // TMA tensor destinations must be 128-byte aligned
      atomicExch(a.err, 2);
      s_ok = 0;
    }
    if (s_ok) {
      for (int q = 0; q < R; ++q) mbar_init(&bars[q], 1);
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
      for (int q = 0; q < R - 1; ++q)
        if (blockIdx.x + q * (int)gridDim.x < ntiles) stage_load(q, blockIdx.x + q * gridDim.x);
    }
  }
  __syncthreads();
  if (!s_ok) return;
  int k = 0;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++k) {
    const int stage = k % R;
    const uint32_t parity = (uint32_t)((k / R) & 1);
    T* buf = buf0 + stage * tile_elems;
    T* fl_s = fac0 + stage * fac_stride;
    T* fr_s = fl_s + side;
    T* src_s = fr_s + side;
    int s0, b0, c;
    tile_coords(a, t, &s0, &b0, &c);
    if (tid == 0) s_ok = mbar_wait(&bars[stage], parity) ? 1 : 0;
    __syncthreads();
    if (!s_ok) {
      if (tid == 0) {
        atomicExch(a.err, 1);
        // this tile's load and those issued for the next tiles land in this CTA's shared
        // memory: wait for them (bounded)
        for (int q = 0; q < R - 1; ++q)
          if (t + q * (int)gridDim.x < ntiles) mbar_wait(&bars[(k + q) % R], (uint32_t)(((k + q) / R) & 1));
        asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
      }
      return;
    }
    if (tid != 0) mbar_wait(&bars[stage], parity);  // completed: acquires the tile's bytes
    const int per_row = a.TS / V;
    const int s = (tid % per_row) * V, p = tid / per_row;
    if (p < a.P && b0 + p < a.nb) {
      T ft[V];
#pragma unroll
      for (int v = 0; v < V; ++v) ft[v] = SRC ? slot_time_factor<T>(a, s0 + s + v, a.t_first) : T(0);
      line_solve<T, V, SRC>(buf + tile_off(a, s, p, 0), a.axis == 0 ? a.TS : a.P * a.TS, a.L, fl_s + p * Lp,
                            fr_s + p * Lp, src_s + p * Lp, ft);
    }
    fence_async_smem();
    __syncthreads();
    if (tid == 0) {
      issue_tile_store(&map, a, buf, t);  // commits one bulk group
      const int tn = t + (R - 1) * (int)gridDim.x;
      if (tn < ntiles) {
        // the refilled stage held tile k-1 (or is unused yet): its store group must be read out
        asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
        stage_load((k + R - 1) % R, tn);
      }
    }
  }
  if (tid == 0) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}

// U (slice-major, FP64, slices [s_first, s_first+nsl)) <-> W (interleaved, S_pad slots).
template <typename T>
__global__ void to_interleaved_kernel(const double* __restrict__ U, T* __restrict__ W, long long nt, int S_pad,
                                      int s_first, int nsl, int rev) {
  __shared__ double tile[32][33];
  const long long pos0 = (long long)blockIdx.x * 32;
  const int sl0 = blockIdx.y * 32;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int sl = sl0 + r;
    const long long pos = pos0 + threadIdx.x;
    const long long src = rev ? (long long)(nsl - 1 - sl) : (long long)sl;  // slot s_first + sl <- state src
    tile[r][threadIdx.x] = (sl < nsl && pos < nt) ? U[src * nt + pos] : 0.0;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const long long pos = pos0 + r;
    const int sl = sl0 + threadIdx.x;
    if (sl < nsl && pos < nt) W[pos * S_pad + s_first + sl] = (T)tile[threadIdx.x][r];
  }
}
template <typename T>
__global__ void from_interleaved_kernel(const T* __restrict__ W, double* __restrict__ U, long long nt, int S_pad,
                                        int s_first, int nsl) {
  __shared__ double tile[32][33];
  const long long pos0 = (long long)blockIdx.x * 32;
  const int sl0 = blockIdx.y * 32;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const long long pos = pos0 + r;
    const int sl = sl0 + threadIdx.x;
    tile[r][threadIdx.x] = (sl < nsl && pos < nt) ? (double)W[pos * S_pad + s_first + sl] : 0.0;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int sl = sl0 + r;
    const long long pos = pos0 + threadIdx.x;
    if (sl < nsl && pos < nt) U[(long long)sl * nt + pos] = tile[threadIdx.x][r];
  }
}

// Grouped pack / unpack of many problems' slices (FP64 slice-major <-> FP32 interleaved).
__device__ __forceinline__ int pack_segment(const WorkSeg* segs, int nseg, long long it) {
  int lo = 0, hi = nseg - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (segs[mid].prefix <= it) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}
template <bool TO>
__global__ void pack_grouped_kernel(const PackJob* __restrict__ jobs, const WorkSeg* __restrict__ segs,
                                    const int* __restrict__ nseg_ptr) {
  __shared__ double tile[32][33];
  const int nseg = *nseg_ptr;
  if (nseg <= 0) return;
  const long long total = (long long)segs[nseg - 1].prefix + segs[nseg - 1].count;
  for (long long it = blockIdx.x; it < total; it += gridDim.x) {
    const WorkSeg sg = segs[pack_segment(segs, nseg, it)];
    const PackJob& j = jobs[sg.job];
    const long long b = sg.first + (it - sg.prefix);
    const int nsb = (j.nsl + 31) / 32;
    const long long pos0 = (b / nsb) * 32;
    const int sl0 = (int)(b % nsb) * 32;
    if (TO) {
      for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int sl = sl0 + r;
        const long long pos = pos0 + threadIdx.x;
        tile[r][threadIdx.x] = (sl < j.nsl && pos < j.nt) ? j.U[(long long)sl * j.nt + pos] : 0.0;
      }
      __syncthreads();
      for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const long long pos = pos0 + r;
        const int sl = sl0 + threadIdx.x;
        if (sl < j.nsl && pos < j.nt) j.W[pos * j.S_pad + j.s_first + sl] = (float)tile[threadIdx.x][r];
      }
    } else {
      for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const long long pos = pos0 + r;
        const int sl = sl0 + threadIdx.x;
        tile[r][threadIdx.x] = (sl < j.nsl && pos < j.nt) ? (double)j.W[pos * j.S_pad + j.s_first + sl] : 0.0;
      }
      __syncthreads();
      for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int sl = sl0 + r;
        const long long pos = pos0 + threadIdx.x;
        if (sl < j.nsl && pos < j.nt) j.U[(long long)sl * j.nt + pos] = tile[threadIdx.x][r];
      }
    }
    __syncthreads();
  }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    cudaDriverEntryPointQueryResult q;
    void* f = nullptr;
    PS_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q));
    if (q != cudaDriverEntryPointSuccess || !f) throw Error(PS_ERR_CUDA, "cuTensorMapEncodeTiled unavailable");
    fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
  }
  return fn;
}

}  // namespace

// Chooses the tile shape of one direction and encodes its tensor map.
void tile_plan(const Geom& g, int S_pad, int elem, int axis, TilePlan& tp, void* W, int positions, int pipe,
               int slots, int vec) {
  const int L = g.n[axis];
  tp.axis = axis;
  tp.L = L;
  // slots per tile by default: 32 (128-byte rows in FP32, 256-byte rows in FP64)
  tp.TS = S_pad % 32 == 0 ? 32 : 128 / elem;
  bool short_rows = false;
  if (slots > 0) {
    // requested slots per tile: a divisor of S_pad whose rows are a multiple of 128 bytes, so
    // that every TMA destination in the tile (rows, positions, chunks) is 128-byte aligned as
    // tensor copies require -- or shorter rows (16-byte multiples) for tiles of a single box
    // (one position, lines of at most 256 nodes), whose only destination is the tile's start
    int ts = slots;
    while (ts > 1 && S_pad % ts != 0) ts /= 2;
    if (S_pad % ts == 0 && (ts * elem) % 128 == 0) {
      tp.TS = ts;
    } else if (S_pad % ts == 0 && (ts * elem) % 16 == 0 && L <= 256 && positions <= 1 && pipe != 1) {
      tp.TS = ts;
      short_rows = true;
    }
  }
  PS_REQUIRE((tp.TS * elem) % 128 == 0 || short_rows, "tile rows must be a multiple of 128 bytes");
  tp.pipe = pipe < 0 ? 1 : pipe;
  {
    // long lines: fewer slots per tile (down to 128-byte rows) until one tile fits in shared memory
    int dev = 0, maxsm = 0;
    PS_CUDA(cudaGetDevice(&dev));
    PS_CUDA(cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    const int Lp4 = (L + 3) & ~3;
    const int st = tp.pipe ? kPipeStages : 1;
    while (!short_rows && tp.TS * elem > 128 && S_pad % (tp.TS / 2) == 0 &&
           (size_t)st * ((size_t)tp.TS * L * elem + 3 * (size_t)Lp4 * elem + 64) + 512 > (size_t)maxsm)
      tp.TS /= 2;
  }
  const int stages = tp.pipe ? kPipeStages : 1;
  // per CTA, so that 2 (ring of stages) or 2-3 (one tile) CTAs share an SM
  const size_t budget = tp.pipe ? 110 * 1024 : 96 * 1024;
  const int nb = g.n[axis == 0 ? 1 : 0];  // the paired axis: y for x-lines, x otherwise
  if (short_rows) {
    tp.P = 1;  // one box per tile
  } else if (positions > 0) {
    tp.P = positions >= 4 ? 4 : (positions >= 2 ? 2 : 1);
    // fewer positions when the paired axis is short or the stages would not fit in shared memory
    while (tp.P > 1 && (tp.P > nb || (size_t)stages * tp.TS * tp.P * L * elem > 200 * 1024)) tp.P /= 2;
  } else if (elem == 4) {
    // FP32: one position per tile (34 KB at 255-node lines), so that six tiles share an SM and
    // their loads, solves and stores overlap (measured best at 127^3 and 255^3, 64 slices)
    tp.P = 1;
  } else {
    tp.P = 1;
    while (tp.P < 4 && tp.P * 2 <= nb && (size_t)stages * tp.TS * (tp.P * 2) * L * elem <= budget) tp.P *= 2;
  }
  // lines per thread: one by default (more threads per tile); FP32 threads can take two
  // adjacent lines (paired 8-byte shared-memory accesses) when asked for
  tp.V = (elem == 4 && tp.TS >= 32 && vec == 2) ? 2 : 1;
  // a TMA box extent is at most 256: split the line into the fewest equal chunks
  tp.chunks = (L + 255) / 256;
  while (L % tp.chunks) ++tp.chunks;
  tp.chunk = L / tp.chunks;
  // globals: dims (S_pad, nx, ny, nz), strides in bytes of dims 1..3
  cuuint64_t dims[4] = {(cuuint64_t)S_pad, (cuuint64_t)g.n[0], (cuuint64_t)g.n[1], (cuuint64_t)g.n[2]};
  cuuint64_t strides[3] = {(cuuint64_t)S_pad * elem, (cuuint64_t)S_pad * elem * g.n[0],
                           (cuuint64_t)S_pad * elem * g.n[0] * g.n[1]};
  cuuint32_t box[4] = {(cuuint32_t)tp.TS, 1, 1, 1};
  cuuint32_t estr[4] = {1, 1, 1, 1};
  if (axis == 0) {
    box[1] = tp.chunk;
  } else if (axis == 1) {
    box[1] = tp.P;
    box[2] = tp.chunk;
  } else {
    box[1] = tp.P;
    box[3] = tp.chunk;
  }
  CUresult r = encode_fn()(&tp.map, elem == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 4, W,
                           dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) throw Error(PS_ERR_CUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
  r = encode_fn()(&tp.map_grp, elem == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 4, W, dims,
                  strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) throw Error(PS_ERR_CUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
  const int lines = tp.TS * tp.P;
  const int Lp = (L + 3) & ~3;
  // stages x (tile + factor rows l, r) + alignment + barriers; the source, when added, takes
  // one more factor row per position and stage
  tp.smem = (size_t)stages * ((size_t)lines * L * elem + 2 * (size_t)tp.P * Lp * elem + 64) + 64 + 128;
  tp.threads = lines / tp.V;
  int dev = 0, maxsm = 0;
  PS_CUDA(cudaGetDevice(&dev));
  PS_CUDA(cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  // the x-sweep of a step's first substep also stages the source: P * L more per stage
  if (tp.smem + (size_t)stages * tp.P * Lp * elem + 256 > (size_t)maxsm)
    throw Error(PS_ERR_UNSUPPORTED, "fine line tile does not fit in shared memory (line too long)");
}

template <typename T>
void tile_sweep(const Geom& g, const TilePlan& tp, const LineFactors& f, int S_pad, int s_first, int nsl,
                const SourceArgs& sa, const T* srcrow, int* err, cudaStream_t st, bool part_of_slots) {
  const CUtensorMap& map = part_of_slots ? tp.map_grp : tp.map;
  TileArgs a{};
  a.axis = tp.axis;
  a.L = tp.L;
  a.P = tp.P;
  a.TS = tp.TS;
  a.n[0] = g.n[0];
  a.n[1] = g.n[1];
  a.n[2] = g.n[2];
  const int other[3][2] = {{1, 2}, {0, 2}, {0, 1}};  // (b, c) axes per line axis
  const int bax = other[tp.axis][0], cax = other[tp.axis][1];
  a.nb = g.n[bax];
  a.nbt = (a.nb + tp.P - 1) / tp.P;
  a.s_lo = s_first / tp.TS;
  a.s_hi = (s_first + nsl + tp.TS - 1) / tp.TS;
  a.chunks = tp.chunks;
  a.chunk = tp.chunk;
  a.var = f.var;
  a.rows_x = (long long)g.n[1] * g.n[2];
  a.Lp = (tp.L + 3) & ~3;
  if (sizeof(T) == 4) {
    a.fl = f.lt32.p;
    a.fr = f.rt32.p;
  } else {
    a.fl = f.lt64.p;
    a.fr = f.rt64.p;
  }
  a.src = sa.src;
  a.srcrow = srcrow;
  a.src_t = sa.src_t;
  a.t_first = sa.t0;
  a.t_slice = sa.tstride;
  a.src_t_len = sa.src_t_len;
  PS_REQUIRE(a.fl && a.fr, "line-major factors of the sweep's precision are missing");
  PS_REQUIRE(!sa.src || srcrow, "line-major source rows are missing");
  a.tau = sa.tau;
  a.err = err;
  const long long tiles = (long long)(a.s_hi - a.s_lo) * a.nbt * g.n[cax];
  const bool src = sa.src != nullptr;
  PS_REQUIRE(!src || tp.axis == 0, "the source enters with the x-substep");
  const int stages = tp.pipe ? kPipeStages : 1;
  const int Lp = (tp.L + 3) & ~3;
  const size_t smem = tp.smem + (src ? (size_t)stages * tp.P * Lp * sizeof(T) : 0);
  if (!tp.pipe) {
    auto kern = tp.V == 2 ? (src ? tile_sweep_kernel<T, 2, true> : tile_sweep_kernel<T, 2, false>)
                          : (src ? tile_sweep_kernel<T, 1, true> : tile_sweep_kernel<T, 1, false>);
    PS_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<(unsigned)tiles, tp.threads, smem, st>>>(map, a);
  } else {
    auto kern = tp.V == 2 ? (src ? tile_sweep_pipe_kernel<T, 2, true> : tile_sweep_pipe_kernel<T, 2, false>)
                          : (src ? tile_sweep_pipe_kernel<T, 1, true> : tile_sweep_pipe_kernel<T, 1, false>);
    PS_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0, dev = 0, sms = 0;
    PS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, tp.threads, smem));
    PS_CUDA(cudaGetDevice(&dev));
    PS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    per_sm = std::max(per_sm, 1);
    const long long grid = std::min<long long>(tiles, (long long)per_sm * sms);
    kern<<<(unsigned)grid, tp.threads, smem, st>>>(map, a, (int)tiles);
  }
  PS_CUDA(cudaGetLastError());
}

template void tile_sweep<float>(const Geom&, const TilePlan&, const LineFactors&, int, int, int, const SourceArgs&,
                                const float*, int*, cudaStream_t, bool);
template void tile_sweep<double>(const Geom&, const TilePlan&, const LineFactors&, int, int, int, const SourceArgs&,
                                 const double*, int*, cudaStream_t, bool);

// Line-major copies [line][Lp] (zero padded) of a direction's factors, in the tile's
// precision.  Line numbering: c * n_b + b, with (b, c) = (y, z) for x-lines, (x, z) for
// y-lines, (x, y) for z-lines.
template <typename T>
__global__ void line_major_kernel(const T* __restrict__ l, const T* __restrict__ r, T* __restrict__ lt,
                                  T* __restrict__ rt, int axis, int nx, int ny, int nz, long long lines, int L, int Lp,
                                  int var) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= lines * Lp) return;
  const long long line = e / Lp;
  const int i = (int)(e - line * Lp);
  T lv = T(0), rv = T(0);
  if (i < L) {
    long long idx;
    if (!var) idx = i;
    else if (axis == 0) idx = (long long)i * lines + line;  // transposed x-factors: [i][z*ny + y]
    else if (axis == 1) {
      const long long z = line / nx, x = line % nx;
      idx = (z * ny + i) * nx + x;
    } else {
      const long long y = line / nx, x = line % nx;
      idx = ((long long)i * ny + y) * nx + x;
    }
    lv = l[idx];
    rv = r[idx];
  }
  lt[e] = lv;
  rt[e] = rv;
}
__global__ void src_rows_kernel(const double* __restrict__ src, void* out, int elem, long long rows, int nx, int Lp) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= rows * Lp) return;
  const long long row = e / Lp;
  const int i = (int)(e - row * Lp);
  const double v = i < nx ? src[row * nx + i] : 0.0;
  if (elem == 4) reinterpret_cast<float*>(out)[e] = (float)v;
  else reinterpret_cast<double*>(out)[e] = v;
}

void factor_lines(const Geom& g, LineFactors& f, bool fp32, cudaStream_t st) {
  const int m = f.m, L = g.n[m], Lp = (L + 3) & ~3;
  const long long lines = g.nt / L;
  const long long total = lines * Lp;
  const unsigned blocks = (unsigned)((total + 255) / 256);
  if (fp32) {
    f.lt32.alloc((size_t)total);
    f.rt32.alloc((size_t)total);
    line_major_kernel<float><<<blocks, 256, 0, st>>>(f.l32.p, f.r32.p, f.lt32.p, f.rt32.p, m, g.n[0], g.n[1], g.n[2],
                                                     lines, L, Lp, f.var);
  } else {
    f.lt64.alloc((size_t)total);
    f.rt64.alloc((size_t)total);
    line_major_kernel<double><<<blocks, 256, 0, st>>>(f.l64.p, f.r64.p, f.lt64.p, f.rt64.p, m, g.n[0], g.n[1],
                                                      g.n[2], lines, L, Lp, f.var);
  }
  PS_CUDA(cudaGetLastError());
}

long long tile_job_fill(const Geom& g, const TilePlan& tp, const LineFactors& f, int S_pad, int s_first, int nsl,
                        int* err, void* job_out, const SourceArgs& sa, const float* srcrow) {
  TileJob* job = reinterpret_cast<TileJob*>(job_out);
  std::memset(job, 0, sizeof(TileJob));
  job->map = tp.map;
  TileArgs& a = job->a;
  a.axis = tp.axis;
  a.L = tp.L;
  a.P = tp.P;
  a.TS = tp.TS;
  a.n[0] = g.n[0];
  a.n[1] = g.n[1];
  a.n[2] = g.n[2];
  const int other[3][2] = {{1, 2}, {0, 2}, {0, 1}};
  const int bax = other[tp.axis][0], cax = other[tp.axis][1];
  a.nb = g.n[bax];
  a.nbt = (a.nb + tp.P - 1) / tp.P;
  a.s_lo = s_first / tp.TS;
  a.s_hi = (s_first + nsl + tp.TS - 1) / tp.TS;
  a.chunks = tp.chunks;
  a.chunk = tp.chunk;
  a.var = f.var;
  a.rows_x = (long long)g.n[1] * g.n[2];
  a.Lp = (tp.L + 3) & ~3;
  a.fl = f.lt32.p;
  a.fr = f.rt32.p;
  a.err = err;
  PS_REQUIRE(a.fl && a.fr, "line-major FP32 factors missing");
  if (sa.src && tp.axis == 0) {
    PS_REQUIRE(srcrow, "line-major source rows missing");
    a.src = sa.src;
    a.srcrow = srcrow;
    a.src_t = sa.src_t;
    a.t_slice = sa.tstride;
    a.src_t_len = sa.src_t_len;
    a.tau = sa.tau;
  }
  return (long long)(a.s_hi - a.s_lo) * a.nbt * g.n[cax];
}
size_t tile_job_bytes() { return sizeof(TileJob); }

size_t tile_grouped_smem(const TilePlan& tp, bool src) {
  return tp.smem + (src ? (size_t)tp.P * ((tp.L + 3) & ~3) * sizeof(float) + 64 : 0);
}

int tile_grouped_ctas_per_sm(int threads, size_t smem) {
  auto kern = tile_sweep_grouped_kernel<float, 1>;
  PS_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int n = 0;
  PS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, threads, smem));
  return n;
}

void tile_sweep_grouped(const void* jobs, const WorkSeg* segs, const int* nseg, int grid, int threads, size_t smem,
                        int* err, int step, cudaStream_t st) {
  auto kern = tile_sweep_grouped_kernel<float, 1>;  // one line per thread, as the default single-problem plan
  PS_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  kern<<<grid, threads, smem, st>>>(reinterpret_cast<const TileJob*>(jobs), segs, nseg, err, step);
  PS_CUDA(cudaGetLastError());
}

void pack_grouped(bool to_interleaved_dir, const PackJob* jobs, const WorkSeg* segs, const int* nseg, int grid,
                  cudaStream_t st) {
  if (to_interleaved_dir) pack_grouped_kernel<true><<<grid, dim3(32, 8), 0, st>>>(jobs, segs, nseg);
  else pack_grouped_kernel<false><<<grid, dim3(32, 8), 0, st>>>(jobs, segs, nseg);
  PS_CUDA(cudaGetLastError());
}

void source_rows(const Geom& g, const double* src, void* out, int elem, cudaStream_t st) {
  const int Lp = (g.n[0] + 3) & ~3;
  const long long rows = g.nt / g.n[0];
  const long long total = rows * Lp;
  src_rows_kernel<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(src, out, elem, rows, g.n[0], Lp);
  PS_CUDA(cudaGetLastError());
}

template <typename T>
void to_interleaved(const Geom& g, const double* U, T* W, int S_pad, int s_first, int nsl, cudaStream_t st, bool rev) {
  dim3 grid((unsigned)((g.nt + 31) / 32), (unsigned)((nsl + 31) / 32));
  to_interleaved_kernel<T><<<grid, dim3(32, 8), 0, st>>>(U, W, g.nt, S_pad, s_first, nsl, rev ? 1 : 0);
  PS_CUDA(cudaGetLastError());
}
template <typename T>
void from_interleaved(const Geom& g, const T* W, double* U, int S_pad, int s_first, int nsl, cudaStream_t st) {
  dim3 grid((unsigned)((g.nt + 31) / 32), (unsigned)((nsl + 31) / 32));
  from_interleaved_kernel<T><<<grid, dim3(32, 8), 0, st>>>(W, U, g.nt, S_pad, s_first, nsl);
  PS_CUDA(cudaGetLastError());
}
template void to_interleaved<float>(const Geom&, const double*, float*, int, int, int, cudaStream_t, bool);
template void to_interleaved<double>(const Geom&, const double*, double*, int, int, int, cudaStream_t, bool);
template void from_interleaved<float>(const Geom&, const float*, double*, int, int, int, cudaStream_t);
template void from_interleaved<double>(const Geom&, const double*, double*, int, int, int, cudaStream_t);

}  // namespace ps
