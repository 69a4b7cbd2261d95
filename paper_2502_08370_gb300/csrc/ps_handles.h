// ps_handles.h -- definitions of the opaque handles of include/ps.h (internal).
#pragma once

#include <cuda_runtime.h>

#include <memory>
#include <string>
#include <vector>

#include "ps_dd.h"
#include "ps_tile.h"

struct ps_grid {
  ps::Geom g;
};
struct ps_operator {
  const ps_grid* grid = nullptr;
  ps::DevBuf<double> a;
  ps::DevBuf<double> d12;     // off-diagonal diffusion (full tensor, 2-D DD only), nodal
  ps::DevBuf<double> src;
  ps::DevBuf<double> src_t;
  int src_t_len = 0;
  ps::DevBuf<double> src2;    // second separable source term
  ps::DevBuf<double> src2_t;
  int src2_t_len = 0;
  double c = 0.0;
};

struct ps_splitting {
  const ps_operator* op = nullptr;
  int kind = PS_SPLIT_DIM;
  ps_dd_params dd{};
  int M = 0;
};


namespace ps {

// One propagator: `steps` FIE steps of size tau per slice; step q of slice n ends at fine
// time index n*s + (q+1)*tstride.
struct Prop {
  const ps_splitting* sp = nullptr;
  double tau = 0.0;
  int steps = 1;
  int tstride = 1;
  bool f32 = false;
  std::vector<std::unique_ptr<LineFactors>> dim;
  std::unique_ptr<DDFactors> dd;
  TilePlan tiles[3];  // fine propagator, dimensional splitting: one TMA plan per direction
};

// Per-launch CUDA events around the library's kernels (params.timing == 2), resolved at
// the host synchronisation points and summed per kernel kind.
struct KernelTimer {
  struct Kind {
    std::string name;
    int launches = 0;
    double ms = 0.0, bytes = 0.0, flops = 0.0;
  };
  bool on = false;
  std::vector<cudaEvent_t> pool;
  struct Mark {
    int kind;
    double bytes, flops;
  };
  std::vector<Mark> marks;
  std::vector<Kind> kinds;
  cudaStream_t st = nullptr;
  ~KernelTimer() {
    for (auto e : pool) cudaEventDestroy(e);
  }
  int kind_id(const std::string& name) {
    for (size_t i = 0; i < kinds.size(); ++i)
      if (kinds[i].name == name) return (int)i;
    kinds.push_back(Kind{name});
    return (int)kinds.size() - 1;
  }
  void begin(cudaStream_t s) {
    if (!on) return;
    st = s;
    size_t need = 2 * (marks.size() + 1);
    while (pool.size() < need) {
      cudaEvent_t e;
      PS_CUDA(cudaEventCreate(&e));
      pool.push_back(e);
    }
    PS_CUDA(cudaEventRecord(pool[2 * marks.size()], s));
  }
  void end(const std::string& name, double bytes, double flops) {
    if (!on) return;
    PS_CUDA(cudaEventRecord(pool[2 * marks.size() + 1], st));
    marks.push_back(Mark{kind_id(name), bytes, flops});
  }
  // call after the stream was synchronised
  void resolve() {
    for (size_t i = 0; i < marks.size(); ++i) {
      float ms = 0.f;
      PS_CUDA(cudaEventElapsedTime(&ms, pool[2 * i], pool[2 * i + 1]));
      Kind& k = kinds[marks[i].kind];
      k.launches++;
      k.ms += ms;
      k.bytes += marks[i].bytes;
      k.flops += marks[i].flops;
    }
    marks.clear();
  }
  void reset() {
    marks.clear();
    kinds.clear();
  }
};


}  // namespace ps

struct ps_problem {
  const ps_splitting* fine = nullptr;
  const ps_splitting* coarse = nullptr;
  const ps_operator* op = nullptr;
  ps::Geom g;
  double T = 1.0;
  int N = 1, gs = 1, fs = 1;
  ps_params prm{};
  ps::Prop F, G;
  ps::DevBuf<double> U, Fout, Gold, gtmp;
  bool delta32 = false;       // coarse increment form in FP32 (PS_COARSE_DELTA32); no Gold then
  bool dr = false;            // fine propagator: Douglas-Rachford steps (PS_FINE_DR)
  bool coarse_staged = false;  // coarse sweeps staged through shared memory (ps_coarse.cu), else streamed
  bool coarse_split = false;   // FP64 coarse correction as its own pass after the last sweep (same values)
  int xsched = PS_SCHED_HYBRID;  // schedule of the FP32 increment form's coarse x-sweep
  ps::DevBuf<float> pcr_e, pcr_d;  // its tridiagonal rows for the PCR schedule (line-major FP32)
  struct TuneEntry {
    std::string name;
    double ms;
    int chosen;
  };
  std::vector<TuneEntry> tune_log;  // the last ps_autotune's timings
  ps::DevBuf<double> dr_W;    // its increments U_{n,j} - U_n, N states
  ps::DevBuf<float> d32, g32; // its increment U_n^k - U_n^{k-1} and coarse working state
  ps::DevBuf<float> W;      // fine working state, slice-interleaved (FP32 line solves)
  ps::DevBuf<double> W64;   // same for FP64 line solves
  int S_pad = 0;        // slots of the interleaved layout
  ps::DevBuf<int> tmo;      // set by a kernel whose bounded wait ran out
  ps::DevBuf<float> srcrow32;   // fine source rows along x, line-major (tile sweeps)
  ps::DevBuf<double> srcrow64;
  ps::DevBuf<unsigned long long> sstats;  // per slice {max |U^k - U^{k-1}|, max |U^k|}, slices 0..N
  unsigned long long* h_sstats = nullptr;
  bool transposed = false;  // propagate with the transposed steps (substeps reversed, no source)
  int batched = 0;          // batches holding this problem (their grouped kernels run one line per
                            // thread, one tile per work item: the autotuner keeps to such shapes)
  bool have_forward = false;
  bool resumable = false;   // U, Gold and the history hold a forward run's iterate (or a loaded checkpoint)
  // adjoint workspaces (allocated by the first ps_adjoint_vjp with a coefficient gradient)
  ps::DevBuf<double> Uchk, snap, Lam, gedge[3];
  ps::TilePlan adj_tiles[3];
  bool adj_ready = false;
  ps::DevBuf<unsigned long long> inc;
  ps::DevBuf<int> flag;
  ps::DevBuf<double> jpart;  // per-block partial sums of the loss of ps_adjoint, then J
  unsigned long long* h_inc = nullptr;
  int* h_flag = nullptr;
  std::vector<double> hist;
  int iters = 0;
  double updates = 0.0;
  int launches = 0;
  float ms_total = 0, ms_fine = 0, ms_coarse = 0;
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
  // overlap of the fine phase (side stream, slot group by slot group) with the coarse chain:
  // per group, an event after its pack (its inputs U^{k-1} have been read) and after its unpack
  // (its F results are in Fout)
  cudaStream_t side = nullptr;
  cudaStream_t hi = nullptr;  // high-priority stream of the coarse chain beside the fine phase
  std::vector<cudaEvent_t> ev_pack, ev_done;
  cudaEvent_t ev_fine[2] = {nullptr, nullptr};
  bool overlap = false;  // run the fine phase beside the chain when it spans several slot groups
  ps::KernelTimer kt;
  ~ps_problem() {
    if (h_sstats) cudaFreeHost(h_sstats);
    if (h_inc) cudaFreeHost(h_inc);
    if (h_flag) cudaFreeHost(h_flag);
    for (auto& e : ev)
      if (e) cudaEventDestroy(e);
    for (auto& e : ev_fine)
      if (e) cudaEventDestroy(e);
    for (auto e : ev_pack) cudaEventDestroy(e);
    for (auto e : ev_done) cudaEventDestroy(e);
    if (side) cudaStreamDestroy(side);
    if (hi) cudaStreamDestroy(hi);
  }
};

