// ps_internal.h -- internal declarations of the CUDA library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <cstdint>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/ps.h"

namespace ps {

// Error carried from a failing call to the C boundary, which turns it into a status.
struct Error : std::runtime_error {
  int code;
  Error(int c, const std::string& m) : std::runtime_error(m), code(c) {}
};

#define PS_CUDA(call)                                                                          \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess)                                                                     \
      throw ::ps::Error(e_ == cudaErrorMemoryAllocation ? PS_ERR_OOM : PS_ERR_CUDA,             \
                        std::string(#call) + ": " + cudaGetErrorString(e_));                    \
  } while (0)
#define PS_REQUIRE(cond, msg) \
  do {                        \
    if (!(cond)) throw ::ps::Error(PS_ERR_INVALID, msg); \
  } while (0)

// Device buffer owned by a handle.
template <typename T>
struct DevBuf {
  T* p = nullptr;
  size_t n = 0;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  DevBuf(DevBuf&& o) noexcept : p(o.p), n(o.n) {
    o.p = nullptr;
    o.n = 0;
  }
  DevBuf& operator=(DevBuf&& o) noexcept {
    if (this != &o) {
      reset();
      p = o.p;
      n = o.n;
      o.p = nullptr;
      o.n = 0;
    }
    return *this;
  }
  ~DevBuf() { reset(); }
  void alloc(size_t count) {
    reset();
    if (count == 0) return;
    PS_CUDA(cudaMalloc(&p, count * sizeof(T)));
    n = count;
  }
  void reset() {
    if (p) cudaFree(p);
    p = nullptr;
    n = 0;
  }
};

// Factors of one dimensional substep (I - tau A_m) = L D L^T along every line of direction m:
// l[i] = L_{i,i-1} (l at the first node of a line is 0), r[i] = 1/D_i.
// var = 0: all lines share one factor vector of length n_m (constant coefficients);
// var = 1: one value per interior node, in the state layout for m = 1, 2 and transposed
// for m = 0 (entry (line, i) at i * (nt / nx) + line, line = z*ny + y), so that the threads
// of a warp, which walk consecutive x-lines, read consecutive addresses.
struct LineFactors {
  int m = 0;
  int var = 0;
  DevBuf<double> l64, r64;
  DevBuf<float> l32, r32;
  // line-major copies [line][L rounded up to 4] for the fine propagator's tile sweeps
  DevBuf<double> lt64, rt64;
  DevBuf<float> lt32, rt32;
};

// Geometry of a state on the grid (x fastest).
struct Geom {
  int dim = 2;
  int n[3] = {1, 1, 1};
  long long nt = 0;
  long long stride(int m) const { return m == 0 ? 1LL : (m == 1 ? (long long)n[0] : (long long)n[0] * n[1]); }
};

// Source term f = src(x) * src_t(t_j) handed to the sweeps that form the right-hand side.
struct SourceArgs {
  const double* src = nullptr;    // interior field or null (no source)
  const double* src_t = nullptr;  // device table of time factors or null (factor 1)
  int t0 = 0;                     // time index of the first slice of the launch
  int tstride = 0;                // added per slice of the launch
  int src_t_len = 0;              // entries of src_t
  double tau = 0.0;
  const double* src2 = nullptr;   // second separable term src2(x) * src2_t(t_j) (DD and DR paths), or null
  const double* src2_t = nullptr; // its time factors (same time index as src_t) or null (factor 1)
};

// Epilogue of the last sweep of a coarse step (the parareal correction, Sec. 3).
struct CorrArgs {
  // 0 none; 1 correction U_{n+1} = Fout + (g - Gold), Gold <- g; 2 initial sweep U_{n+1} = g
  // (and Gold = g when Gold is set); 3 increment form U_{n+1} = Fout + g with g = G applied
  // to the increment of U_n, writing the new increment of U_{n+1} to dnext
  int mode = 0;
  double* U_next = nullptr;          // U_{n+1}: old value in, new value out
  const double* Fout = nullptr;      // F(U_n^{k-1})
  double* Gold = nullptr;            // G(U_n^{k-1}) in, G(U_n^k) out
  unsigned long long* inc = nullptr; // running max |U^k - U^{k-1}| as bits of a nonnegative double
  int* nonfinite = nullptr;          // set to 1 when a non-finite value appears
  unsigned long long* slice_stats = nullptr;  // optional {max |U^k - U^{k-1}|, max |U^k|} of this slice
  float* dnext = nullptr;            // mode 3: U_{n+1}^k - U_{n+1}^{k-1}, rounded to FP32
};

// A run of work items of a grouped (batched) launch: items [prefix, prefix + count) are
// blocks/tiles first .. first + count - 1 of job `job`.
struct WorkSeg {
  int job;
  int first;
  int count;
  int prefix;
};

// One batched problem's coarse step n (2-D, FP64): the x-sweep reads xin (U_n) into xout
// (the coarse scratch state) in blocks of R rows; the y-sweep solves xout in place and
// applies the correction `ca` (mode 1) or the initial-sweep epilogue (mode 2).  The
// slice-k copy reads xin (F result) into xout (U_k) with the increment in `ca`.
struct CoarseJob {
  const double* xin;
  double* xout;
  long long rows, nt;  // rows = x-lines (ny * nz)
  int nx, ny, nz;      // nz = 1 in 2-D
  const double* lx;
  const double* rx;
  const double* ly;
  const double* ry;
  const double* lz;    // 3-D: z factors
  const double* rz;
  CorrArgs ca;
  SourceArgs sa;  // the coarse step's source (added on the x-sweep), or sa.src == null
  // FP32 increment form: the y-sweep runs in place on g32 with the FP32 factors
  float* g32;
  const float* ly32;
  const float* ry32;
  const float* lz32;
  const float* rz32;
};

// One batched problem's FP32 x-sweep of coarse step n (increment form): rows of the FP64 state
// (in64, initial sweep, with the source sa) or of the FP32 increment (in32) into out.
struct XWarpJob {
  const double* in64;
  const float* in32;
  float* out;
  long long rows;
  int nx, m, span, Lp;
  const float* lt;
  const float* rt;
  SourceArgs sa;
};

// Launchers (ps_dim.cu).  `in` and `out` may alias (in-place sweeps).  nslices states of
// geometry g are stored back to back.  Tin/Tout are double or float; the recurrences run in
// double when fp32 == false and in float otherwise.
void factor_dim(const Geom& g, int m, const double* a_nodal, double c_over_M, double tau, LineFactors& f,
                bool want_f32, cudaStream_t st);
template <typename Tin, typename Tout>
void sweep_dim(const Geom& g, int nslices, const LineFactors& f, bool fp32, const Tin* in, Tout* out,
               const SourceArgs& srcargs, const CorrArgs& corr, double* tmp, cudaStream_t st);
// Coarse x-substep in FP32 on one slice, one warp per row (segmented scans of the two
// recurrences); needs the line-major FP32 factors of direction x (factor_lines).
// T = double: the same segmented scans in FP64 (line-major FP64 x factors, factor_lines).
template <typename Tin, typename T = float>
void sweep_x_warp(const Geom& g, const LineFactors& f, const Tin* in, T* out, const SourceArgs& sa,
                  cudaStream_t st);
// FP64 x-substep of nslices states (in may alias out), Thomas per thread in warp-private
// chunks through shared memory (ps_coarse.cu), bitwise equal to the whole-row sweep.  Returns
// false (nothing launched) for rows shorter than 16 nodes or without FP64 x factors.
bool sweep_x_chunked(const Geom& g, int nslices, const LineFactors& f, const double* in, double* out,
                     const SourceArgs& sa, cudaStream_t st);
// CTAs per SM that the chunked FP64 sweeps (x warp chunks, strided chunks) may keep resident
// on the calling host thread: 0 = as many as fit (one launch wave); > 0 = a persistent grid of
// that many CTAs per SM, each walking its share of the work.  Set while the coarse chain runs
// beside the fine phase, so that the fine tiles keep most of every SM's shared memory.
// Host-side trace range (NVTX; free when no tool is attached): one per parareal phase, and
// one around each batched run.
struct TraceRange {
  explicit TraceRange(const char* name) { nvtxRangePushA(name); }
  ~TraceRange() { nvtxRangePop(); }
  TraceRange(const TraceRange&) = delete;
  TraceRange& operator=(const TraceRange&) = delete;
};
extern thread_local int chain_ctas_per_sm;
struct ChainResidency {
  int saved;
  explicit ChainResidency(int cap) : saved(chain_ctas_per_sm) { chain_ctas_per_sm = cap; }
  ~ChainResidency() { chain_ctas_per_sm = saved; }
};
// Coarse-propagator sweep of direction f.m on ONE slice, staged through shared memory
// (ps_coarse.cu); in may alias out.  T = double: x, y, z (x carries the source, y/z the
// epilogues of CorrArgs modes 0-2); T = float: y, z with modes 0, 2, 3.  Returns false (nothing
// launched) when the shape does not fit the kernels' shared-memory budget; the caller then runs
// sweep_dim.
template <typename T>
bool coarse_sweep_staged(const Geom& g, const LineFactors& f, const T* in, T* out, const SourceArgs& sa,
                         const CorrArgs& ca, cudaStream_t st);
// Coarse x-substep in FP32 on one slice by parallel cyclic reduction, one warp per row (rows
// of at most 256 nodes; returns false otherwise).  et/dt: line-major FP32 rows of the
// sub-diagonal and diagonal of (I - tau A_x), built by tridiag_x_rows.
template <typename Tin>
bool sweep_x_pcr(const Geom& g, const float* et, const float* dt, const Tin* in, float* out, const SourceArgs& sa,
                 cudaStream_t st);
void tridiag_x_rows(const Geom& g, const double* a_nodal, double c_over_M, double tau, DevBuf<float>& et,
                    DevBuf<float>& dt, cudaStream_t st);
// Douglas-Rachford fine step in increment form (ps_dr.cu), nsl consecutive states of the
// natural layout: w = tau (A u + f) (A with reaction c, f from sa at t0 + slice * tstride);
// out = u + w (out may alias u).
void dr_increment(const Geom& g, int nsl, const double* a_nodal, double c, double tau, const double* u, double* w,
                  const SourceArgs& sa, cudaStream_t st);
// Same for the full diffusion tensor D = [[a, d12], [d12, a]] in 2-D: A is the cell-based
// nine-point operator (the sum of the DD suboperators of ps_dd.cu, with rho = 1).
void dr_increment_tensor(const Geom& g, int nsl, const double* a_nodal, const double* d12_nodal, double c, double tau,
                         const double* u, double* w, const SourceArgs& sa, cudaStream_t st);
void dr_add(const Geom& g, int nsl, const double* u, const double* w, double* out, cudaStream_t st);
// dst <- src with the increment max |src - dst| (and per-slice stats); when dout is set it
// also receives src - dst rounded to FP32 (the increment the coarse increment form propagates).
void copy_with_increment(long long nt, const double* src, double* dst, unsigned long long* inc, int* nonfinite,
                         unsigned long long* slice_stats, float* dout, cudaStream_t st);
// Grouped coarse-step launches (persistent grids of `grid` CTAs; *nseg work segments).
// x (ps_coarse.cu): a work item is coarse_x_grouped_rows() rows of one job, warp-private
// Thomas chunks as the single-problem FP64 x-sweep; y: an item is coarse_y_grouped_lines()
// lines (FP64: pipelined as the single-problem strided sweeps; FP32: one chunk ahead).
int coarse_x_grouped_rows();
int coarse_y_grouped_lines();
void coarse_x_grouped(bool var, const CoarseJob* jobs, const WorkSeg* segs, const int* nseg, int grid,
                      cudaStream_t st);
// axis 1: the y-lines (nx * nz of them), axis 2: the z-lines (nx * ny); epi: the correction
// epilogue of the last sweep (0 on a 3-D problem's y-sweep)
void coarse_y_grouped(bool var, int epi, const CoarseJob* jobs, const WorkSeg* segs, const int* nseg, int grid,
                      cudaStream_t st, int axis = 1);
void copy_inc_grouped(const CoarseJob* jobs, const WorkSeg* segs, const int* nseg, int grid, cudaStream_t st);
void coarse_x32_grouped(const XWarpJob* jobs, const WorkSeg* segs, const int* nseg, int grid, int span_max,
                        cudaStream_t st);
void coarse_y32_grouped(bool var, int epi, const CoarseJob* jobs, const WorkSeg* segs, const int* nseg, int grid,
                        cudaStream_t st, int axis = 1);
int max_dyn_smem_public();

}  // namespace ps
