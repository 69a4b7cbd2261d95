// ps_capi.cu -- handles, the parareal host loop and the C ABI declared in include/ps.h.
//
// Parareal (Sec. 3) with FIE propagators (Sec. 2.2, eq. FIE_method):
//   U_0 = u0,  U_{n+1}^0 = G(U_n^0),
//   U_{n+1}^k = F(U_n^{k-1}) + (G(U_n^k) - G(U_n^{k-1})),  k = 1, 2, ...
// F of every slice runs in one batched launch per substep (all slices at once); the
// coarse chain runs slice after slice with the correction fused into its last sweep.
// Finite termination (Sec. 3): U_n^k = U_n^{k-1} for n <= k-1, so the correction of
// slice k-1 has an exactly zero bracket and slices n < k-1 are unchanged; the host loop
// skips that work, which leaves every value bitwise as the full iteration computes it.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>
#include <mutex>
#include <string>
#include <vector>


#include "ps_adjoint.h"
#include "ps_async.h"
#include "ps_handles.h"

using namespace ps;

namespace {

thread_local std::string g_last_error;

int fail(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

template <typename F>
int guarded(F&& f) {
  try {
    f();
    return PS_OK;
  } catch (const Error& e) {
    return fail(e.code, e.what());
  } catch (const std::bad_alloc&) {
    return fail(PS_ERR_OOM, "host allocation failed");
  } catch (const std::exception& e) {
    return fail(PS_ERR_INVALID, e.what());
  }
}

inline cudaStream_t S(uintptr_t s) { return reinterpret_cast<cudaStream_t>(s); }

}  // namespace

namespace {

void build_prop(ps_problem* p, Prop& P, const ps_splitting* sp, double tau, int steps, int tstride, bool f32,
                cudaStream_t st) {
  P.sp = sp;
  P.tau = tau;
  P.steps = steps;
  P.tstride = tstride;
  P.f32 = f32;
  const ps_operator* op = sp->op;
  if (sp->kind == PS_SPLIT_DIM) {
    for (int m = 0; m < p->g.dim; ++m) {
      auto f = std::make_unique<LineFactors>();
      factor_dim(p->g, m, op->a.p, op->c / p->g.dim, tau, *f, f32, st);
      P.dim.push_back(std::move(f));
    }
  } else {
    if (f32) throw Error(PS_ERR_UNSUPPORTED, "DD splitting runs in FP64 only");
    P.dd = std::make_unique<DDFactors>();
    dd_factor(p->g, sp->dd, op->a.p, op->d12.p, op->c, tau, *P.dd, st);
  }
}

SourceArgs source_for(const ps_problem* p, const Prop& P, int t0, int tslice) {
  SourceArgs sa;
  if (!p->op->src.p || p->transposed) return sa;  // the transposed (adjoint) steps carry no source
  sa.src = p->op->src.p;
  sa.src_t = p->op->src_t.p;
  sa.t0 = t0;
  sa.tstride = tslice;
  sa.src_t_len = p->op->src_t_len;
  sa.tau = P.tau;
  sa.src2 = p->op->src2.p;
  sa.src2_t = p->op->src2_t.p;
  return sa;
}

// One FP64 FIE step of propagator P on nsl consecutive states: in -> out (out may alias in).
// The source of slice j of the launch is taken at fine time index t0 + j*tslice.  When
// corr.mode != 0 the last sweep of the step carries the parareal correction instead of
// writing out.
const char* kAxis[3] = {"x", "y", "z"};

// Algorithmic bytes and flops of one sweep launch: read the right-hand side, write the
// result (bytes_in + bytes_out per unknown), read the factors once (they are shared by all
// slices of the launch), read the source when it is added, and for the fused correction
// read Fout, Gold and U_{n+1} and write Gold and U_{n+1}.  Flops: 5 per unknown (FMA
// forward, MUL + FMA backward, FMA = 2) plus 2 for the source.
void sweep_cost(const ps_problem* p, const LineFactors& f, int nsl, int bin, int bout, int bc, bool src, int corr,
                double* bytes, double* flops) {
  const double nt = (double)p->g.nt;
  double b = nsl * nt * (bin + bout);
  b += (f.var ? nt : (double)p->g.n[f.m]) * 2.0 * bc;
  if (src) b += nt * 8.0;
  if (corr == 1) b += nt * 40.0 - nsl * nt * bout;
  if (corr == 2) b += nt * 16.0 - nsl * nt * bout;
  *bytes = b;
  *flops = nsl * nt * (5.0 + (src ? 2.0 : 0.0));
}

// DD step: right-hand side (and copy in -> out), the colour solves in place, and the
// correction as a separate pass over the slice (it touches every node, not only boxes).
void fie_step_dd(ps_problem* p, Prop& P, int nsl, const double* in, double* out, int t0, int tslice,
                 const CorrArgs& corr, cudaStream_t st, const char* phase) {
  const int M = P.sp->M;
  const double nt = (double)p->g.nt;
  SourceArgs sa = source_for(p, P, t0, tslice);
  if (in != out || sa.src) {
    p->kt.begin(st);
    dd_rhs(p->g, nsl, in, out, sa, st);
    if (p->kt.on) p->kt.end(std::string(phase) + ".rhs.f64", nsl * nt * 16.0 + (sa.src ? nt * 8.0 : 0.0), 0.0);
    p->launches++;
  }
  const int spb = p->prm.dd_slices_per_block > 0 ? p->prm.dd_slices_per_block : 2;
  for (int q = 0; q < M; ++q) {
    const int c = p->transposed ? M - 1 - q : q;
    p->kt.begin(st);
    dd_solve(p->g, nsl, *P.dd, c, out, spb, p->tmo.p, st);
    if (p->kt.on) {
      const auto& pl = P.dd->plan;
      // per box node and slice: w FMAs forward and w backward (w = line length of the box)
      const double w = pl.nodes[c] > 0 ? pl.fac_entries[c] / (2.0 * pl.nodes[c]) - 0.5 : 0.0;
      p->kt.end(std::string(phase) + ".dd" + std::to_string(c) + ".f64", nsl * pl.nodes[c] * 16.0 + pl.fac_entries[c] * 8.0,
                nsl * pl.nodes[c] * 4.0 * w);
    }
    p->launches++;
  }
  if (corr.mode != 0) {
    p->kt.begin(st);
    dd_correct(p->g, out, corr, st);
    if (p->kt.on) p->kt.end(std::string(phase) + (corr.mode == 1 ? ".corr.f64" : ".init.f64"), nt * 48.0, 0.0);
    p->launches++;
  }
}

// One FP64 sweep of the coarse propagator on one slice: staged through shared memory when the
// shape fits (ps_coarse.cu), else the streaming sweeps of ps_dim.cu.
void coarse_sweep64(ps_problem* p, const LineFactors& f, const double* in, double* out, const SourceArgs& sa,
                    const CorrArgs& corr, cudaStream_t st) {
  if (f.m == 0 && p->xsched == PS_SCHED_HYBRID && f.lt64.p && corr.mode == 0) {
    sweep_x_warp<double, double>(p->g, f, in, out, sa, st);
    return;
  }
  if (p->coarse_staged && coarse_sweep_staged<double>(p->g, f, in, out, sa, corr, st)) return;
  if (f.m == 0 && corr.mode == 0 && sweep_x_chunked(p->g, 1, f, in, out, sa, st)) return;
  sweep_dim<double, double>(p->g, 1, f, false, in, out, sa, corr, corr.mode != 0 ? out : nullptr, st);
}

void fie_step64(ps_problem* p, Prop& P, int nsl, const double* in, double* out, int t0, int tslice,
                const CorrArgs& corr, cudaStream_t st, const char* phase) {
  if (P.sp->kind == PS_SPLIT_DD) {
    fie_step_dd(p, P, nsl, in, out, t0, tslice, corr, st, phase);
    return;
  }
  const int M = P.sp->M;
  const bool tr = p->transposed;
  // the transposed step ends with the x-substep, whose kernel carries no epilogue: then the
  // correction runs as its own pass over the slice
  const bool fuse = corr.mode != 0 && !tr;
  for (int q = 0; q < M; ++q) {
    const int m = tr ? M - 1 - q : q;
    SourceArgs sa = q == 0 ? source_for(p, P, t0, tslice) : SourceArgs{};
    const double* src_state = q == 0 ? in : out;
    const bool epi = (q == M - 1 && fuse);
    double bytes = 0, flops = 0;
    if (p->kt.on) sweep_cost(p, *P.dim[m], nsl, 8, 8, 8, sa.src != nullptr, epi ? corr.mode : 0, &bytes, &flops);
    p->kt.begin(st);
    if (&P == &p->G && nsl == 1 && epi && p->coarse_split) {
      // the last sweep without the epilogue, then the correction as one coalesced pass over the
      // slice: the same expressions as the fused epilogue, so the same values
      coarse_sweep64(p, *P.dim[m], src_state, out, sa, CorrArgs{}, st);
      if (p->kt.on) {
        sweep_cost(p, *P.dim[m], nsl, 8, 8, 8, sa.src != nullptr, 0, &bytes, &flops);
        p->kt.end(std::string(phase) + "." + kAxis[m] + ".f64", bytes, flops);
      }
      p->launches++;
      p->kt.begin(st);
      dd_correct(p->g, out, corr, st);
      if (p->kt.on) p->kt.end(std::string(phase) + (corr.mode == 1 ? ".corr.f64" : ".init.f64"), p->g.nt * 48.0, 0.0);
      p->launches++;
      continue;
    }
    if (&P == &p->G && nsl == 1)
      coarse_sweep64(p, *P.dim[m], src_state, out, sa, epi ? corr : CorrArgs{}, st);
    else if (epi)
      sweep_dim<double, double>(p->g, nsl, *P.dim[m], false, src_state, out, sa, corr, out, st);
    else
      sweep_dim<double, double>(p->g, nsl, *P.dim[m], false, src_state, out, sa, CorrArgs{}, nullptr, st);
    if (p->kt.on)
      p->kt.end(std::string(phase) + "." + kAxis[m] + ".f64" + (epi ? (corr.mode == 1 ? "+corr" : "+init") : ""),
                bytes, flops);
    p->launches++;
  }
  if (corr.mode != 0 && !fuse) {
    p->kt.begin(st);
    dd_correct(p->g, out, corr, st);
    if (p->kt.on) p->kt.end(std::string(phase) + (corr.mode == 1 ? ".corr.f64" : ".init.f64"), p->g.nt * 48.0, 0.0);
    p->launches++;
  }
}

// F (s fine steps) on nsl consecutive slices starting at absolute slice n_first.  With the
// dimensional splitting the slices are packed into the interleaved working state, every
// substep is one TMA tile sweep over all of them, and the result is unpacked into `out`.
template <typename T>
void run_F_tiles(ps_problem* p, int n_first, int nsl, const double* in, double* out, cudaStream_t st,
                 cudaEvent_t after_pack = nullptr, bool part_of_slots = false) {
  Prop& P = p->F;
  const int M = P.sp->M;
  T* W = sizeof(T) == 4 ? reinterpret_cast<T*>(p->W.p) : reinterpret_cast<T*>(p->W64.p);
  const double nt = (double)p->g.nt;
  const char* tn = sizeof(T) == 4 ? "f32" : "f64";
  p->kt.begin(st);
  to_interleaved<T>(p->g, in, W, p->S_pad, n_first, nsl, st);
  if (p->kt.on) p->kt.end(std::string("F.pack.") + tn, nsl * nt * (8.0 + sizeof(T)), 0.0);
  p->launches++;
  if (after_pack) PS_CUDA(cudaEventRecord(after_pack, st));
  for (int j = 0; j < P.steps; ++j) {
    for (int q = 0; q < M; ++q) {
      const int m = p->transposed ? M - 1 - q : q;
      SourceArgs sa = q == 0 ? source_for(p, P, j + 1, p->fs) : SourceArgs{};
      const LineFactors& f = *P.dim[m];
      double bytes = 0, flops = 0;
      if (p->kt.on) sweep_cost(p, f, nsl, sizeof(T), sizeof(T), sizeof(T), sa.src != nullptr, 0, &bytes, &flops);
      p->kt.begin(st);
      const T* srow = sizeof(T) == 4 ? reinterpret_cast<const T*>(p->srcrow32.p) : reinterpret_cast<const T*>(p->srcrow64.p);
      tile_sweep<T>(p->g, P.tiles[m], f, p->S_pad, n_first, nsl, sa, srow, p->tmo.p, st, part_of_slots);
      if (p->kt.on) p->kt.end(std::string("F.") + kAxis[m] + "." + tn, bytes, flops);
      p->launches++;
    }
  }
  p->kt.begin(st);
  from_interleaved<T>(p->g, W, out, p->S_pad, n_first, nsl, st);
  if (p->kt.on) p->kt.end(std::string("F.unpack.") + tn, nsl * nt * (8.0 + sizeof(T)), 0.0);
  p->launches++;
}

// F as s Douglas-Rachford steps (eq. DR_method) on nsl consecutive slices of the natural
// layout, in increment form: W_0 = tau (A U_n + f), the M substep solves (I - tau A_j) in
// place on W (the printed right-hand sides U_{n,j-1} - tau A_j U_n minus (I - tau A_j) U_n),
// then U_{n+1} = U_n + W_M.  The stencil pass is the same for both splittings: the DD
// suboperators sum to A exactly (rho_j sums to 1 at every edge midpoint and node), so only
// the substep solves differ (line sweeps, or colour j's box solves).
void run_F_dr(ps_problem* p, int n_first, int nsl, const double* in, double* out, cudaStream_t st) {
  Prop& P = p->F;
  const int M = P.sp->M;
  const double nt = (double)p->g.nt;
  const double dnt = (double)nsl * nt;
  double* W = p->dr_W.p;
  for (int q = 0; q < P.steps; ++q) {
    const double* u = q == 0 ? in : out;
    SourceArgs sa = source_for(p, P, n_first * p->fs + (q + 1) * P.tstride, p->fs);
    p->kt.begin(st);
    if (p->op->d12.p)
      dr_increment_tensor(p->g, nsl, p->op->a.p, p->op->d12.p, p->op->c, P.tau, u, W, sa, st);
    else
      dr_increment(p->g, nsl, p->op->a.p, p->op->c, P.tau, u, W, sa, st);
    if (p->kt.on)
      p->kt.end("F.drW.f64", dnt * 16.0 + (p->op->a.p ? nt * 8.0 : 0.0) + (sa.src ? nt * 8.0 : 0.0),
                dnt * (1.0 + 6.0 * M + (sa.src ? 3.0 : 0.0)));
    p->launches++;
    for (int j = 0; j < M; ++j) {
      if (P.sp->kind == PS_SPLIT_DD) {
        // colour j's box solves on W (identity outside its boxes, like the FIE substep)
        const int spb = p->prm.dd_slices_per_block > 0 ? p->prm.dd_slices_per_block : 2;
        p->kt.begin(st);
        dd_solve(p->g, nsl, *P.dd, j, W, spb, p->tmo.p, st);
        if (p->kt.on) {
          const auto& pl = P.dd->plan;
          const double w = pl.nodes[j] > 0 ? pl.fac_entries[j] / (2.0 * pl.nodes[j]) - 0.5 : 0.0;
          p->kt.end("F.dd" + std::to_string(j) + ".f64", nsl * pl.nodes[j] * 16.0 + pl.fac_entries[j] * 8.0,
                    nsl * pl.nodes[j] * 4.0 * w);
        }
        p->launches++;
        continue;
      }
      double bytes = 0, flops = 0;
      if (p->kt.on) sweep_cost(p, *P.dim[j], nsl, 8, 8, 8, false, 0, &bytes, &flops);
      p->kt.begin(st);
      sweep_dim<double, double>(p->g, nsl, *P.dim[j], false, W, W, SourceArgs{}, CorrArgs{}, nullptr, st);
      if (p->kt.on) p->kt.end(std::string("F.") + kAxis[j] + ".f64", bytes, flops);
      p->launches++;
    }
    p->kt.begin(st);
    dr_add(p->g, nsl, u, W, out, st);
    if (p->kt.on) p->kt.end("F.dradd.f64", dnt * 24.0, dnt);
    p->launches++;
  }
  p->updates += (double)nsl * P.steps * (double)p->g.nt;
}

void run_F(ps_problem* p, int n_first, int nsl, const double* in, double* out, cudaStream_t st) {
  Prop& P = p->F;
  if (p->dr) {
    run_F_dr(p, n_first, nsl, in, out, st);
    return;
  }
  if (P.sp->kind == PS_SPLIT_DIM) {
    if (P.f32) run_F_tiles<float>(p, n_first, nsl, in, out, st);
    else run_F_tiles<double>(p, n_first, nsl, in, out, st);
  } else {
    for (int j = 0; j < P.steps; ++j)
      fie_step64(p, P, nsl, j == 0 ? in : out, out, n_first * p->fs + (j + 1) * P.tstride, p->fs, CorrArgs{}, st,
                 "F");
  }
  p->updates += (double)nsl * P.steps * (double)p->g.nt;
}

// G on slice n from `in`; the last sweep carries `corr` (mode 0: result left in gtmp).
void run_G(ps_problem* p, int n, const double* in, const CorrArgs& corr, cudaStream_t st) {
  Prop& P = p->G;
  for (int q = 0; q < P.steps; ++q) {
    CorrArgs c = (q == P.steps - 1) ? corr : CorrArgs{};
    fie_step64(p, P, 1, q == 0 ? in : p->gtmp.p, p->gtmp.p, n * p->fs + (q + 1) * P.tstride, 0, c, st, "G");
  }
  p->updates += (double)P.steps * (double)p->g.nt;
}

// The FP32 coarse x-sweep of the increment form on one slice, in the installed schedule:
// hybrid (one warp per row, segmented scans), PCR (one warp per row), or Thomas (one thread
// per row, rows staged in shared memory by sweep_dim).
template <typename Tin>
void coarse_x32(ps_problem* p, const Tin* in, float* out, const SourceArgs& sa, cudaStream_t st) {
  const LineFactors& f = *p->G.dim[0];
  if (p->xsched == PS_SCHED_PCR && sweep_x_pcr<Tin>(p->g, p->pcr_e.p, p->pcr_d.p, in, out, sa, st)) return;
  if (p->xsched == PS_SCHED_THOMAS) {
    sweep_dim<Tin, float>(p->g, 1, f, true, in, out, sa, CorrArgs{}, nullptr, st);
    return;
  }
  sweep_x_warp<Tin>(p->g, f, in, out, sa, st);
}

// G's one FIE step in FP32 line solves for the coarse increment form (PS_COARSE_DELTA32):
// init = true:  U_{n+1}^0 = G(U_n^0) on the state, source included (x-sweep reads FP64 U_n);
// init = false: U_{n+1}^k = Fout_n + B d_n with d_n = U_n^k - U_n^{k-1} (FP32, in d32), no
// source (it cancels); the last sweep's epilogue writes the new increment d_{n+1} to d32.
void run_G32(ps_problem* p, int n, bool init, cudaStream_t st) {
  Prop& P = p->G;
  const int M = P.sp->M;
  const long long nt = p->g.nt;
  const double dnt = (double)nt;
  PS_REQUIRE(P.steps == 1, "the FP32 coarse increment form takes one coarse step per slice");
  CorrArgs c;
  c.mode = init ? 2 : 3;
  c.U_next = p->U.p + (n + 1) * nt;
  c.nonfinite = p->flag.p;
  if (!init) {
    c.Fout = p->Fout.p + n * nt;
    c.inc = p->inc.p;
    c.slice_stats = p->sstats.p + 2 * (n + 1);
    c.dnext = p->d32.p;
  }
  for (int m = 0; m < M; ++m) {
    const bool last = m == M - 1;
    SourceArgs sa = (init && m == 0) ? source_for(p, P, n * p->fs + P.tstride, 0) : SourceArgs{};
    p->kt.begin(st);
    double bytes = 0;
    if (m == 0) {
      // x-lines are contiguous rows: the schedule of ps_params.schedule (or the autotuner's)
      if (init) coarse_x32(p, p->U.p + n * nt, p->g32.p, sa, st);
      else coarse_x32(p, p->d32.p, p->g32.p, SourceArgs{}, st);
      bytes = dnt * ((init ? 8 : 4) + 4 + 8 + (sa.src ? 8 : 0));
    } else {
      const float* in = m == 0 ? p->d32.p : p->g32.p;
      const CorrArgs cm = last ? c : CorrArgs{};
      if (!(p->coarse_staged && coarse_sweep_staged<float>(p->g, *P.dim[m], in, p->g32.p, SourceArgs{}, cm, st)))
        sweep_dim<float, float>(p->g, 1, *P.dim[m], true, in, p->g32.p, SourceArgs{}, cm, nullptr, st);
      bytes = dnt * (4 + 4 + 8) + (last ? dnt * (init ? 8.0 : 28.0) : 0.0);
    }
    if (p->kt.on)
      p->kt.end(std::string("G.") + kAxis[m] + ".f32" + (last ? (init ? "+init" : "+dcorr") : ""), bytes,
                dnt * 5.0);
    p->launches++;
  }
  p->updates += dnt;
}

CorrArgs corr_args(ps_problem* p, int mode, int n) {
  CorrArgs c;
  c.mode = mode;
  const long long nt = p->g.nt;
  c.U_next = p->U.p + (n + 1) * nt;
  c.Fout = p->Fout.p + n * nt;
  c.Gold = p->Gold.p + n * nt;
  c.inc = p->inc.p;
  c.nonfinite = p->flag.p;
  c.slice_stats = p->sstats.p + 2 * (n + 1);
  return c;
}

// The tile kernels abandon their work once the flag `tmo` holds an error (1: a bounded TMA wait
// ran out, 2: a misaligned shared-memory destination), so every entry point that launches them
// zeroes it first and reads it back after its last launch.
void tile_flag_reset(ps_problem* p, cudaStream_t st) { PS_CUDA(cudaMemsetAsync(p->tmo.p, 0, sizeof(int), st)); }

void tile_flag_throw(int v) {
  if (v == 2) throw Error(PS_ERR_CUDA, "a tile's shared-memory buffer was not 128-byte aligned");
  if (v) throw Error(PS_ERR_DEVICE_TIMEOUT, "an asynchronous copy into shared memory did not arrive within its wait limit");
}

void tile_flag_check(ps_problem* p, cudaStream_t st) {
  int v = 0;
  PS_CUDA(cudaMemcpyAsync(&v, p->tmo.p, sizeof(int), cudaMemcpyDeviceToHost, st));
  PS_CUDA(cudaStreamSynchronize(st));
  tile_flag_throw(v);
}

void require_slices(const ps_problem* p) {
  PS_REQUIRE(p->N >= 1, "the problem has no slices (its last ps_problem_set_slices failed)");
}

void check_state_len(const ps_problem* p, int slice) {
  require_slices(p);
  PS_REQUIRE(slice >= 0 && slice <= p->N, "slice out of range");
}

// resume_k < 0: a new run from u0.  resume_k >= 0: continue after iteration resume_k from the
// problem's states U^k, coarse values Gold and history (a stopped run, or a loaded checkpoint).
void do_run(ps_problem* p, const double* u0, double tol, int max_iter, cudaStream_t st, int* iters_out,
            int resume_k = -1) {
  TraceRange whole(p->transposed ? "ps.adjoint_parareal" : "ps.parareal");
  require_slices(p);
  const long long nt = p->g.nt;
  const int N = p->N;
  if (max_iter <= 0 || max_iter > N) max_iter = N;
  const bool resume = resume_k >= 0;
  if (!resume) p->hist.clear();
  p->resumable = false;
  p->updates = 0;
  p->launches = 0;
  p->ms_total = p->ms_fine = p->ms_coarse = 0;
  const bool timing = p->prm.timing != 0;
  p->kt.on = p->prm.timing >= 2;
  p->kt.reset();
  if (timing) PS_CUDA(cudaEventRecord(p->ev[0], st));
  if (!resume) PS_CUDA(cudaMemcpyAsync(p->U.p, u0, sizeof(double) * nt, cudaMemcpyDeviceToDevice, st));
  PS_CUDA(cudaMemsetAsync(p->flag.p, 0, sizeof(int), st));
  tile_flag_reset(p, st);
  // k = 0: sequential coarse sweep, U_{n+1}^0 = G(U_n^0), Gold_n = G(U_n^0)
  if (!resume) {
    TraceRange r("ps.coarse_initial");
    for (int n = 0; n < N; ++n) {
      if (p->delta32) run_G32(p, n, true, st);
      else run_G(p, n, p->U.p + n * nt, corr_args(p, 2, n), st);
    }
  }
  int k = resume ? resume_k : 0;
  // a resumed run that had already met its stopping rule stays where it stopped
  const bool done = resume && k > 0 && ((int)p->hist.size() == k && p->hist[k - 1] < tol);
  while (k < max_iter && !done) {
    ++k;
    const int nlo = k - 1;
    PS_CUDA(cudaMemsetAsync(p->inc.p, 0, sizeof(unsigned long long), st));
    PS_CUDA(cudaMemsetAsync(p->sstats.p, 0, sizeof(unsigned long long) * 2 * (N + 1), st));
    // Fine phase beside the chain: F needs only U^{k-1}, and the chain's step n needs only F of
    // slice n, so F runs slot group by slot group on the side stream while the chain follows the
    // groups as they finish.  Only the ordering changes; every value is computed as before.
    std::vector<int> bounds;  // slot groups [bounds[g], bounds[g+1]) of this iteration's fine phase
    if (p->overlap && p->side && !p->dr && !p->transposed && p->F.sp->kind == PS_SPLIT_DIM) {
      const int TS = p->F.tiles[0].TS;
      bounds.push_back(nlo);
      for (int b = (nlo / TS + 1) * TS; b < N; b += TS) bounds.push_back(b);
      bounds.push_back(N);
      if (bounds.size() < 3 || (int)bounds.size() - 1 > (int)p->ev_done.size()) bounds.clear();
    }
    if (!bounds.empty()) {
      TraceRange r("ps.fine_and_chain_overlapped");
      const int ng = (int)bounds.size() - 1;
      PS_CUDA(cudaEventRecord(p->ev_fine[0], st));  // U^{k-1} complete (the initial sweep, or the last chain)
      PS_CUDA(cudaStreamWaitEvent(p->side, p->ev_fine[0], 0));
      if (timing) PS_CUDA(cudaEventRecord(p->ev[1], p->side));
      for (int g = 0; g < ng; ++g) {
        const int a = bounds[g], nsl = bounds[g + 1] - bounds[g];
        if (p->F.f32)
          run_F_tiles<float>(p, a, nsl, p->U.p + a * nt, p->Fout.p + a * nt, p->side, p->ev_pack[g], true);
        else
          run_F_tiles<double>(p, a, nsl, p->U.p + a * nt, p->Fout.p + a * nt, p->side, p->ev_pack[g], true);
        p->updates += (double)nsl * p->F.steps * (double)nt;
        PS_CUDA(cudaEventRecord(p->ev_done[g], p->side));
      }
      if (timing) PS_CUDA(cudaEventRecord(p->ev[2], p->side));
      TraceRange r2("ps.coarse_chain_correction");
      // the chain runs on a high-priority stream, its FP64 sweeps on a persistent grid of two CTAs
      // per SM, so that its CTAs are scheduled ahead of the fine tiles' and leave them most of
      // every SM
      cudaStream_t cs = p->hi ? p->hi : st;
      if (cs != st) PS_CUDA(cudaStreamWaitEvent(cs, p->ev_fine[0], 0));
      ChainResidency residency(2);
      auto group_of = [&](int slice) {
        int g = 0;
        while (g + 1 < ng && slice >= bounds[g + 1]) ++g;
        return g;
      };
      int waited_done = -1, waited_pack = 0;
      // before the chain reads F of slice n: its group has been unpacked
      auto need_F = [&](int n) {
        const int g = group_of(n);
        while (waited_done < g) PS_CUDA(cudaStreamWaitEvent(cs, p->ev_done[++waited_done], 0));
      };
      // before the chain writes U_j: the group holding slice j has read its U^{k-1} (packed)
      auto writes_U = [&](int j) {
        if (j >= N) return;
        const int g = group_of(j);
        while (waited_pack < g && waited_done < g) PS_CUDA(cudaStreamWaitEvent(cs, p->ev_pack[++waited_pack], 0));
      };
      need_F(nlo);
      writes_U(k);
      copy_with_increment(nt, p->Fout.p + nlo * nt, p->U.p + k * nt, p->inc.p, p->flag.p, p->sstats.p + 2 * k,
                          p->delta32 ? p->d32.p : nullptr, cs);
      p->launches++;
      for (int n = k; n < N; ++n) {
        need_F(n);
        writes_U(n + 1);
        if (p->delta32) run_G32(p, n, false, cs);
        else run_G(p, n, p->U.p + n * nt, corr_args(p, 1, n), cs);
      }
      // the side stream's last group is part of this iteration: the chain ends after it
      while (waited_done < ng - 1) PS_CUDA(cudaStreamWaitEvent(cs, p->ev_done[++waited_done], 0));
      if (cs != st) {
        PS_CUDA(cudaEventRecord(p->ev_fine[1], cs));
        PS_CUDA(cudaStreamWaitEvent(st, p->ev_fine[1], 0));
      }
    } else {
    if (timing) PS_CUDA(cudaEventRecord(p->ev[1], st));
    {
      TraceRange r("ps.fine_all_slices");
      run_F(p, nlo, N - nlo, p->U.p + nlo * nt, p->Fout.p + nlo * nt, st);
    }
    if (timing) PS_CUDA(cudaEventRecord(p->ev[2], st));
    {
      TraceRange r("ps.coarse_chain_correction");
      // slice k-1: U_k^k = F(U_{k-1}^{k-1}) exactly (its G bracket is zero)
      copy_with_increment(nt, p->Fout.p + nlo * nt, p->U.p + k * nt, p->inc.p, p->flag.p, p->sstats.p + 2 * k,
                          p->delta32 ? p->d32.p : nullptr, st);
      p->launches++;
      for (int n = k; n < N; ++n) {
        if (p->delta32) run_G32(p, n, false, st);
        else run_G(p, n, p->U.p + n * nt, corr_args(p, 1, n), st);
      }
    }
    }
    if (timing) PS_CUDA(cudaEventRecord(p->ev[3], st));
    TraceRange test("ps.increment_test");
    PS_CUDA(cudaMemcpyAsync(p->h_inc, p->inc.p, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
    PS_CUDA(cudaMemcpyAsync(p->h_flag, p->flag.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    PS_CUDA(cudaMemcpyAsync(p->h_flag + 1, p->tmo.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    if (p->prm.tol_mode == 1)
      PS_CUDA(cudaMemcpyAsync(p->h_sstats, p->sstats.p, sizeof(unsigned long long) * 2 * (N + 1),
                              cudaMemcpyDeviceToHost, st));
    PS_CUDA(cudaStreamSynchronize(st));
    if (p->h_flag[1]) {
      p->iters = k;
      tile_flag_throw(p->h_flag[1]);
    }
    p->kt.resolve();
    if (timing) {
      float a = 0, b = 0;
      PS_CUDA(cudaEventElapsedTime(&a, p->ev[1], p->ev[2]));
      PS_CUDA(cudaEventElapsedTime(&b, p->ev[2], p->ev[3]));
      p->ms_fine += a;
      p->ms_coarse += b;
    }
    double inc;
    unsigned long long bits = *p->h_inc;
    std::memcpy(&inc, &bits, sizeof inc);
    if (p->prm.tol_mode == 1) {
      // per-slice relative increments: max_n ||U_n^k - U_n^{k-1}|| / ||U_n^k||
      inc = 0.0;
      for (int j = 1; j <= N; ++j) {
        double d, u;
        std::memcpy(&d, &p->h_sstats[2 * j], sizeof d);
        std::memcpy(&u, &p->h_sstats[2 * j + 1], sizeof u);
        const double r = u > 0.0 ? d / u : (d > 0.0 ? HUGE_VAL : 0.0);
        if (r > inc || r != r) inc = r;
      }
    }
    p->hist.push_back(inc);
    if (*p->h_flag) {
      p->iters = k;
      throw Error(PS_ERR_NONFINITE, "non-finite value in the parareal correction at iteration " + std::to_string(k));
    }
    if (inc < tol) break;
  }
  if (timing) {
    PS_CUDA(cudaEventRecord(p->ev[1], st));
    PS_CUDA(cudaEventSynchronize(p->ev[1]));
    PS_CUDA(cudaEventElapsedTime(&p->ms_total, p->ev[0], p->ev[1]));
  }
  p->iters = k;
  if (!p->transposed) {
    p->have_forward = true;
    p->resumable = true;
  }
  if (iters_out) *iters_out = k;
}

}  // namespace

namespace {
// Slice count N, coarse steps g and fine steps f per slice (Sec. 3: G = g FIE steps of
// DeltaT/g, F = f FIE steps of DeltaT/f, DeltaT = T/N).  Builds the substep factors of both
// propagators for their step sizes and (re)allocates every per-slice buffer; the previous
// run's states, history and adjoint workspaces are dropped.  The arguments are checked
// before anything is released; if an allocation fails afterwards the problem is left with
// no slices (N = 0) and every run refuses it until a later call succeeds.
void configure_slices(ps_problem* p, int N, int g_steps, int f_steps, cudaStream_t st) {
  PS_REQUIRE(N >= 1 && g_steps >= 1 && f_steps >= 1, "N, g_steps, f_steps must be >= 1");
  PS_REQUIRE(f_steps % g_steps == 0, "f_steps must be a multiple of g_steps");
  if (p->op->src_t.p)
    PS_REQUIRE(p->op->src_t_len >= (long long)N * f_steps + 1, "src_t must cover the fine times 0..N*f_steps");
  if (p->op->src2_t.p)
    PS_REQUIRE(p->op->src2_t_len >= (long long)N * f_steps + 1, "src2_t must cover the fine times 0..N*f_steps");
  PS_REQUIRE((long long)(N + 1) * p->g.nt * 8 < (1LL << 46), "slice states too large");
  const ps_splitting* fine = p->fine;
  const ps_splitting* coarse = p->coarse;
  // drop everything that depends on N or on the step sizes
  p->N = 0;
  p->iters = 0;
  p->hist.clear();
  p->have_forward = false;
  p->resumable = false;
  p->adj_ready = false;
  for (auto* b : {&p->U, &p->Fout, &p->Gold, &p->gtmp, &p->dr_W, &p->W64, &p->srcrow64, &p->Uchk, &p->snap, &p->Lam})
    b->reset();
  for (auto& b : p->gedge) b.reset();
  for (auto* b : {&p->d32, &p->g32, &p->W, &p->srcrow32, &p->pcr_e, &p->pcr_d}) b->reset();
  p->sstats.reset();
  if (p->h_sstats) {
    cudaFreeHost(p->h_sstats);
    p->h_sstats = nullptr;
  }
  p->F = Prop{};
  p->G = Prop{};
  const bool mixed = p->prm.precision == PS_PREC_MIXED;
  const double T = p->T;
  build_prop(p, p->F, fine, T / N / f_steps, f_steps, 1, mixed, st);
  build_prop(p, p->G, coarse, T / N / g_steps, g_steps, f_steps / g_steps, p->delta32, st);
  if (p->delta32) {
    Geom g3 = p->g;
    if (g3.dim == 2) g3.n[2] = 1;
    factor_lines(g3, *p->G.dim[0], true, st);  // line-major x factors of the warp x-sweep
    // rows of (I - DeltaT/g A_x) for the PCR schedule of that sweep
    if (p->g.n[0] <= 256) tridiag_x_rows(p->g, p->op->a.p, p->op->c / p->g.dim, p->G.tau, p->pcr_e, p->pcr_d, st);
  } else if (coarse->kind == PS_SPLIT_DIM) {
    Geom g3 = p->g;
    if (g3.dim == 2) g3.n[2] = 1;
    factor_lines(g3, *p->G.dim[0], false, st);  // line-major FP64 x factors of the hybrid x-sweep
  }
  const long long nt = p->g.nt;
  p->U.alloc((size_t)(N + 1) * nt);
  p->Fout.alloc((size_t)N * nt);
  if (p->delta32) {
    p->d32.alloc((size_t)nt);
    p->g32.alloc((size_t)nt);
  } else {
    p->Gold.alloc((size_t)N * nt);
  }
  p->gtmp.alloc((size_t)nt);
  if (p->dr) p->dr_W.alloc((size_t)N * nt);
  p->sstats.alloc((size_t)2 * (N + 1));
  PS_CUDA(cudaMallocHost(&p->h_sstats, sizeof(unsigned long long) * 2 * (N + 1)));
  p->S_pad = 0;
  if (fine->kind == PS_SPLIT_DIM) {
    const int elem = mixed ? 4 : 8;
    const int TS = mixed ? 32 : 16;
    p->S_pad = (N + TS - 1) / TS * TS;
    void* W = nullptr;
    if (mixed) {
      p->W.alloc((size_t)p->S_pad * nt);
      W = p->W.p;
    } else {
      p->W64.alloc((size_t)p->S_pad * nt);
      W = p->W64.p;
    }
    PS_CUDA(cudaMemsetAsync(W, 0, (size_t)p->S_pad * nt * elem, st));
    Geom g3 = p->g;
    if (g3.dim == 2) g3.n[2] = 1;
    for (int m = 0; m < p->g.dim; ++m) {
      tile_plan(g3, p->S_pad, elem, m, p->F.tiles[m], W, p->prm.tile_positions,
                p->prm.tile_pipeline == 1 ? 1 : 0, p->prm.tile_slots,
                p->prm.tile_lines_per_thread);
      factor_lines(g3, *p->F.dim[m], mixed, st);
    }
    if (p->op->src.p) {
      const size_t rows = (size_t)(nt / g3.n[0]) * ((g3.n[0] + 3) & ~3);
      void* out;
      if (mixed) {
        p->srcrow32.alloc(rows);
        out = p->srcrow32.p;
      } else {
        p->srcrow64.alloc(rows);
        out = p->srcrow64.p;
      }
      source_rows(g3, p->op->src.p, out, elem, st);
    }
  }
  // events of the overlapped fine phase: one pair per slot group
  const int groups = p->S_pad > 0 ? p->S_pad / std::max(1, p->F.tiles[0].TS) + 1 : 0;
  while ((int)p->ev_done.size() < groups) {
    cudaEvent_t a, b;
    PS_CUDA(cudaEventCreateWithFlags(&a, cudaEventDisableTiming));
    PS_CUDA(cudaEventCreateWithFlags(&b, cudaEventDisableTiming));
    p->ev_pack.push_back(a);
    p->ev_done.push_back(b);
  }
  PS_CUDA(cudaStreamSynchronize(st));
  p->N = N;
  p->gs = g_steps;
  p->fs = f_steps;
}
}  // namespace

// ---------------------------------------------------------------------------------------
// Coarse sequential solution without device allocation (ps_run_coarse_sequential_noalloc).
// The working state of each coarse step lives in this file-scope array instead of the
// problem's workspace.  Host code must not take its address directly: the symbol's host
// stand-in is not a device address, so the device address is looked up once per device.
static __device__ __align__(256) double g_noalloc_work[PS_NOALLOC_MAX_UNKNOWNS];

namespace {
std::mutex g_noalloc_mu;
double* g_noalloc_ptr[64] = {};

double* noalloc_work_ptr() {
  int dev = 0;
  PS_CUDA(cudaGetDevice(&dev));
  PS_REQUIRE(dev >= 0 && dev < 64, "device index out of range");
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* ptr = nullptr;
    PS_CUDA(cudaGetSymbolAddress(&ptr, g_noalloc_work));
    g_noalloc_ptr[dev] = static_cast<double*>(ptr);
  }
  return g_noalloc_ptr[dev];
}

// One coarse step from `in` into `work`: the same launches as the allocating coarse step,
// without the kernel timer (whose events it would otherwise create).
void coarse_step_into(ps_problem* p, int n, int q, const double* in, double* work, cudaStream_t st) {
  Prop& P = p->G;
  const int t_end = n * p->fs + (q + 1) * P.tstride;
  const int M = P.sp->M;
  if (P.sp->kind == PS_SPLIT_DD) {
    SourceArgs sa = source_for(p, P, t_end, 0);
    dd_rhs(p->g, 1, in, work, sa, st);
    const int spb = p->prm.dd_slices_per_block > 0 ? p->prm.dd_slices_per_block : 2;
    for (int c = 0; c < M; ++c) dd_solve(p->g, 1, *P.dd, c, work, spb, p->tmo.p, st);
    return;
  }
  for (int m = 0; m < M; ++m) {
    SourceArgs sa = m == 0 ? source_for(p, P, t_end, 0) : SourceArgs{};
    coarse_sweep64(p, *P.dim[m], m == 0 ? in : work, work, sa, CorrArgs{}, st);
  }
}
// The bounded wait of the tile and DD kernels, on a barrier that nothing arrives at: the wait
// must run out after limit_ns, set the flag and return (ps_selftest_wait_timeout).
__global__ void wait_selftest_kernel(int* err, unsigned long long limit_ns) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    if (!mbar_wait_ns(&bar, 0, limit_ns)) atomicExch(err, 1);
  }
}
}  // namespace

namespace {
// Deterministic loss of ps_adjoint: g = U_N - target and per-block sums of g^2 (fixed grid),
// then one block adds the partial sums in a fixed order; out[0] = J = 1/2 sum g^2.
constexpr int kLossBlocks = 512;
__global__ void __launch_bounds__(256) loss_residual_kernel(const double* __restrict__ uN,
                                                          const double* __restrict__ tgt, double* __restrict__ g,
                                                          long long n, double* __restrict__ part) {
  __shared__ double red[256];
  double acc = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double d = uN[i] - tgt[i];
    g[i] = d;
    acc = fma(d, d, acc);
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}
__global__ void __launch_bounds__(256) loss_sum_kernel(const double* __restrict__ part, int nb, double* out) {
  __shared__ double red[256];
  double acc = 0.0;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) acc += part[i];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = 0.5 * red[0];
}

}  // namespace

extern "C" {

int ps_selftest_wait_timeout(int limit_us, uintptr_t stream) {
  return guarded([&] {
    PS_REQUIRE(limit_us >= 1 && limit_us <= 1000000, "limit_us must be in [1, 1e6]");
    cudaStream_t st = S(stream);
    DevBuf<int> flag;
    flag.alloc(1);
    PS_CUDA(cudaMemsetAsync(flag.p, 0, sizeof(int), st));
    wait_selftest_kernel<<<1, 32, 0, st>>>(flag.p, 1000ULL * (unsigned long long)limit_us);
    PS_CUDA(cudaGetLastError());
    int h = 0;
    PS_CUDA(cudaMemcpyAsync(&h, flag.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    PS_CUDA(cudaStreamSynchronize(st));
    if (h) throw Error(PS_ERR_DEVICE_TIMEOUT, "self-test: the bounded wait ran out as designed");
  });
}

const char* ps_last_error(void) { return g_last_error.c_str(); }
int ps_version(void) { return PS_VERSION; }

int ps_grid_create(int dim, const int n[3], ps_grid** out) {
  return guarded([&] {
    PS_REQUIRE(out && n, "null argument");
    PS_REQUIRE(dim == 2 || dim == 3, "dim must be 2 or 3");
    auto g = std::make_unique<ps_grid>();
    g->g.dim = dim;
    long long nt = 1;
    for (int d = 0; d < 3; ++d) {
      int v = d < dim ? n[d] : 1;
      PS_REQUIRE(v >= 1 && v <= (1 << 20), "grid size out of range");
      g->g.n[d] = v;
      nt *= v;
    }
    g->g.nt = nt;
    *out = g.release();
  });
}

int ps_grid_destroy(ps_grid* g) {
  delete g;
  return PS_OK;
}

int ps_operator_create_ex(const ps_grid* g, const ps_operator_desc* d, uintptr_t stream, ps_operator** out) {
  return guarded([&] {
    PS_REQUIRE(g && d && out, "null argument");
    PS_REQUIRE(d->c >= 0.0 && std::isfinite(d->c), "c must be finite and >= 0");
    PS_REQUIRE(!d->src_t_host || d->src_t_len > 0, "src_t_len must be positive");
    PS_REQUIRE(!d->src2_t_host || d->src2_t_len > 0, "src2_t_len must be positive");
    PS_REQUIRE(!d->src2_dev || d->src_dev, "a second source term needs the first");
    const Geom& G = g->g;
    if (d->d12_nodal_dev && G.dim != 2)
      throw Error(PS_ERR_UNSUPPORTED, "the full diffusion tensor is implemented in 2-D");
    auto op = std::make_unique<ps_operator>();
    op->grid = g;
    op->c = d->c;
    cudaStream_t st = S(stream);
    const long long na = (long long)(G.n[0] + 2) * (G.n[1] + 2) * (G.dim == 3 ? G.n[2] + 2 : 1);
    auto copy_dev = [&](DevBuf<double>& b, const double* src, long long n) {
      b.alloc(n);
      PS_CUDA(cudaMemcpyAsync(b.p, src, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
    };
    auto copy_host = [&](DevBuf<double>& b, const double* src, int n) {
      b.alloc(n);
      PS_CUDA(cudaMemcpyAsync(b.p, src, sizeof(double) * n, cudaMemcpyHostToDevice, st));
    };
    if (d->a_nodal_dev) copy_dev(op->a, d->a_nodal_dev, na);
    if (d->d12_nodal_dev) copy_dev(op->d12, d->d12_nodal_dev, na);
    if (d->src_dev) {
      copy_dev(op->src, d->src_dev, G.nt);
      if (d->src_t_host) {
        copy_host(op->src_t, d->src_t_host, d->src_t_len);
        op->src_t_len = d->src_t_len;
      }
    }
    if (d->src2_dev) {
      copy_dev(op->src2, d->src2_dev, G.nt);
      if (d->src2_t_host) {
        copy_host(op->src2_t, d->src2_t_host, d->src2_t_len);
        op->src2_t_len = d->src2_t_len;
      }
    }
    PS_CUDA(cudaStreamSynchronize(st));
    *out = op.release();
  });
}

int ps_operator_create(const ps_grid* g, const double* a_nodal_dev, double c, const double* src_dev,
                       const double* src_t_host, int src_t_len, uintptr_t stream, ps_operator** out) {
  ps_operator_desc d{};
  d.a_nodal_dev = a_nodal_dev;
  d.c = c;
  d.src_dev = src_dev;
  d.src_t_host = src_t_host;
  d.src_t_len = src_t_len;
  return ps_operator_create_ex(g, &d, stream, out);
}

int ps_operator_destroy(ps_operator* op) {
  delete op;
  return PS_OK;
}

int ps_splitting_create(const ps_operator* op, int kind, const ps_dd_params* dd, ps_splitting** out) {
  return guarded([&] {
    PS_REQUIRE(op && out, "null argument");
    auto sp = std::make_unique<ps_splitting>();
    sp->op = op;
    sp->kind = kind;
    const Geom& G = op->grid->g;
    if (kind == PS_SPLIT_DIM) {
      if (op->d12.p)
        throw Error(PS_ERR_UNSUPPORTED, "the full diffusion tensor's mixed derivatives need the DD splitting (Sec. 2.1)");
      sp->M = G.dim;
    } else if (kind == PS_SPLIT_DD) {
      PS_REQUIRE(dd, "DD splitting needs ps_dd_params");
      if (G.dim != 2) throw Error(PS_ERR_UNSUPPORTED, "DD splitting is implemented in 2-D");
      PS_REQUIRE(dd->boxes[0] >= 1 && dd->boxes[1] >= 1, "boxes must be >= 1");
      PS_REQUIRE(dd->overlap >= 0.0, "overlap must be >= 0");
      sp->dd = *dd;
      sp->M = (dd->boxes[0] > 1 ? 2 : 1) * (dd->boxes[1] > 1 ? 2 : 1);
    } else {
      throw Error(PS_ERR_INVALID, "unknown splitting kind");
    }
    *out = sp.release();
  });
}

int ps_splitting_destroy(ps_splitting* sp) {
  delete sp;
  return PS_OK;
}

int ps_problem_create(const ps_splitting* fine, const ps_splitting* coarse, double T, int N, int g_steps,
                      int f_steps, const ps_params* params, uintptr_t stream, ps_problem** out) {
  return guarded([&] {
    PS_REQUIRE(fine && out, "null argument");
    if (!coarse) coarse = fine;
    PS_REQUIRE(coarse->op == fine->op, "coarse and fine splittings must share the operator");
    PS_REQUIRE(T > 0 && std::isfinite(T), "T must be positive");
    auto p = std::make_unique<ps_problem>();
    p->fine = fine;
    p->coarse = coarse;
    p->op = fine->op;
    p->g = fine->op->grid->g;
    p->T = T;
    if (params) p->prm = *params;
    PS_REQUIRE(p->prm.precision == PS_PREC_FP64 || p->prm.precision == PS_PREC_MIXED, "unknown precision");
    PS_REQUIRE(p->prm.schedule >= PS_SCHED_AUTO && p->prm.schedule <= PS_SCHED_HYBRID, "unknown schedule");
    PS_REQUIRE(p->prm.coarse == PS_COARSE_FP64 || p->prm.coarse == PS_COARSE_DELTA32, "unknown coarse mode");
    PS_REQUIRE(p->prm.fine_method == PS_FINE_FIE || p->prm.fine_method == PS_FINE_DR, "unknown fine method");
    PS_REQUIRE(p->prm.tol_mode == 0 || p->prm.tol_mode == 1, "tol_mode must be 0 or 1");
    PS_REQUIRE(p->prm.coarse_sweep >= PS_COARSE_SWEEP_AUTO && p->prm.coarse_sweep <= PS_COARSE_SWEEP_STREAMED,
               "unknown coarse sweep schedule");
    p->coarse_staged = p->prm.coarse_sweep == PS_COARSE_SWEEP_STAGED;
    PS_REQUIRE(p->prm.overlap_phases == 0 || p->prm.overlap_phases == 1, "overlap_phases must be 0 or 1");
    p->overlap = p->prm.overlap_phases == 1;
    p->dr = p->prm.fine_method == PS_FINE_DR;
    if (p->dr && p->prm.precision != PS_PREC_FP64)
      throw Error(PS_ERR_UNSUPPORTED, "the Douglas-Rachford fine propagator runs in FP64");
    if (p->op->src2.p && (fine->kind != PS_SPLIT_DD || coarse->kind != PS_SPLIT_DD))
      throw Error(PS_ERR_UNSUPPORTED, "a second source term is implemented with the DD splitting");
    p->delta32 = p->prm.coarse == PS_COARSE_DELTA32;
    p->xsched = p->prm.schedule != PS_SCHED_AUTO ? p->prm.schedule
                                                 : (p->delta32 ? PS_SCHED_HYBRID : PS_SCHED_THOMAS);
    if (p->xsched == PS_SCHED_PCR && !p->delta32)
      throw Error(PS_ERR_UNSUPPORTED, "the PCR schedule is built for the FP32 coarse increment form's x-sweep");
    if (p->delta32 && (fine->kind != PS_SPLIT_DIM || coarse->kind != PS_SPLIT_DIM))
      throw Error(PS_ERR_UNSUPPORTED, "the FP32 coarse increment form needs the dimensional splitting");
    cudaStream_t st = S(stream);
    PS_CUDA(cudaMallocHost(&p->h_inc, sizeof(unsigned long long)));
    PS_CUDA(cudaMallocHost(&p->h_flag, 2 * sizeof(int)));
    for (auto& e : p->ev) PS_CUDA(cudaEventCreate(&e));
    for (auto& e : p->ev_fine) PS_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    PS_CUDA(cudaStreamCreateWithFlags(&p->side, cudaStreamNonBlocking));
    {
      int least = 0, greatest = 0;
      PS_CUDA(cudaDeviceGetStreamPriorityRange(&least, &greatest));
      PS_CUDA(cudaStreamCreateWithPriority(&p->hi, cudaStreamNonBlocking, greatest));
    }
    p->inc.alloc(1);
    p->tmo.alloc(1);
    p->flag.alloc(1);
    p->jpart.alloc(kLossBlocks + 1);
    PS_CUDA(cudaMemset(p->tmo.p, 0, sizeof(int)));
    configure_slices(p.get(), N, g_steps, f_steps, st);
    *out = p.release();
  });
}

int ps_problem_set_slices(ps_problem* p, int N, int g_steps, int f_steps, uintptr_t stream) {
  return guarded([&] {
    PS_REQUIRE(p, "null argument");
    PS_REQUIRE(p->batched == 0, "the problem belongs to a batch: destroy the batch before changing its slices");
    configure_slices(p, N, g_steps, f_steps, S(stream));
  });
}

int ps_problem_destroy(ps_problem* p) {
  delete p;
  return PS_OK;
}

int ps_run_parareal(ps_problem* p, const double* u0_dev, double tol, int max_iter, uintptr_t stream,
                    int* iters_out) {
  return guarded([&] {
    PS_REQUIRE(p && u0_dev, "null argument");
    do_run(p, u0_dev, tol, max_iter, S(stream), iters_out);
  });
}

int ps_run_parareal_host(ps_problem* p, const double* u0_host, double* uN_host, double tol, int max_iter,
                         uintptr_t stream, int* iters_out) {
  return guarded([&] {
    PS_REQUIRE(p && u0_host && uN_host, "null argument");
    require_slices(p);
    cudaStream_t st = S(stream);
    const long long nt = p->g.nt;
    // u0 is staged in the coarse scratch state, which the run copies to U_0 before using it
    PS_CUDA(cudaMemcpyAsync(p->gtmp.p, u0_host, sizeof(double) * nt, cudaMemcpyHostToDevice, st));
    do_run(p, p->gtmp.p, tol, max_iter, st, iters_out);
    PS_CUDA(cudaMemcpyAsync(uN_host, p->U.p + (long long)p->N * nt, sizeof(double) * nt, cudaMemcpyDeviceToHost, st));
    PS_CUDA(cudaStreamSynchronize(st));
  });
}

int ps_get_state(const ps_problem* p, int slice, double* out_dev, uintptr_t stream) {
  return guarded([&] {
    PS_REQUIRE(p && out_dev, "null argument");
    check_state_len(p, slice);
    const long long nt = p->g.nt;
    PS_CUDA(cudaMemcpyAsync(out_dev, p->U.p + slice * nt, sizeof(double) * nt, cudaMemcpyDeviceToDevice, S(stream)));
  });
}

int ps_set_state(ps_problem* p, int slice, const double* in_dev, uintptr_t stream) {
  return guarded([&] {
    PS_REQUIRE(p && in_dev, "null argument");
    check_state_len(p, slice);
    const long long nt = p->g.nt;
    PS_CUDA(cudaMemcpyAsync(p->U.p + slice * nt, in_dev, sizeof(double) * nt, cudaMemcpyDeviceToDevice, S(stream)));
    p->resumable = false;  // a state edited by hand is not an iterate of the run
  });
}

namespace {
// Checkpoint layout (host memory, native byte order): this header, the history (hist_len
// doubles), U^k ((N+1) states), and Gold (N states) when the coarse propagator is FP64.
struct CkptHeader {
  char magic[8];
  int version, N, dim, n[3], k, delta32, has_gold, hist_len, pad;
  long long nt;
};
constexpr char kCkptMagic[8] = {'P', 'S', 'C', 'K', 'P', 'T', '1', 0};
size_t ckpt_bytes(const ps_problem* p) {
  const size_t nt = (size_t)p->g.nt;
  return sizeof(CkptHeader) + sizeof(double) * ((size_t)p->N + (size_t)(p->N + 1) * nt +
                                                (p->delta32 ? 0 : (size_t)p->N * nt));
}
}  // namespace

int ps_checkpoint_bytes(const ps_problem* p, size_t* bytes) {
  return guarded([&] {
    PS_REQUIRE(p && bytes, "null argument");
    require_slices(p);
    *bytes = ckpt_bytes(p);
  });
}

int ps_checkpoint_save(const ps_problem* p, void* host_buf, size_t bytes, uintptr_t stream) {
  return guarded([&] {
    PS_REQUIRE(p && host_buf, "null argument");
    require_slices(p);
    PS_REQUIRE(p->resumable, "no parareal iterate to save: run ps_run_parareal first");
    PS_REQUIRE(bytes >= ckpt_bytes(p), "checkpoint buffer too small (ps_checkpoint_bytes)");
    cudaStream_t st = S(stream);
    CkptHeader h{};
    std::memcpy(h.magic, kCkptMagic, sizeof h.magic);
    h.version = PS_VERSION;
    h.N = p->N;
    h.dim = p->g.dim;
    for (int d = 0; d < 3; ++d) h.n[d] = p->g.n[d];
    h.k = p->iters;
    h.delta32 = p->delta32 ? 1 : 0;
    h.has_gold = p->delta32 ? 0 : 1;
    h.hist_len = (int)p->hist.size();
    h.nt = p->g.nt;
    char* out = static_cast<char*>(host_buf);
    std::memcpy(out, &h, sizeof h);
    double* hist = reinterpret_cast<double*>(out + sizeof h);
    for (int i = 0; i < p->N; ++i) hist[i] = i < h.hist_len ? p->hist[i] : 0.0;
    double* U = hist + p->N;
    const size_t nt = (size_t)p->g.nt;
    PS_CUDA(cudaMemcpyAsync(U, p->U.p, sizeof(double) * (p->N + 1) * nt, cudaMemcpyDeviceToHost, st));
    if (h.has_gold)
      PS_CUDA(cudaMemcpyAsync(U + (size_t)(p->N + 1) * nt, p->Gold.p, sizeof(double) * p->N * nt,
                              cudaMemcpyDeviceToHost, st));
    PS_CUDA(cudaStreamSynchronize(st));
  });
}

int ps_checkpoint_load(ps_problem* p, const void* host_buf, size_t bytes, uintptr_t stream) {
  return guarded([&] {
    PS_REQUIRE(p && host_buf, "null argument");
    require_slices(p);
    PS_REQUIRE(bytes >= sizeof(CkptHeader), "checkpoint too short");
    CkptHeader h;
    std::memcpy(&h, host_buf, sizeof h);
    PS_REQUIRE(std::memcmp(h.magic, kCkptMagic, sizeof h.magic) == 0, "not a parareal checkpoint");
    PS_REQUIRE(h.version == PS_VERSION, "checkpoint written by another ABI version");
    PS_REQUIRE(h.N == p->N && h.dim == p->g.dim && h.n[0] == p->g.n[0] && h.n[1] == p->g.n[1] &&
                   h.n[2] == p->g.n[2] && h.nt == p->g.nt,
               "checkpoint of another grid or slice count");
    PS_REQUIRE(h.delta32 == (p->delta32 ? 1 : 0), "checkpoint of another coarse propagator form");
    PS_REQUIRE(h.k >= 0 && h.k <= p->N && h.hist_len == h.k, "corrupt checkpoint header");
    PS_REQUIRE(bytes >= ckpt_bytes(p), "checkpoint truncated");
    const double* hist = reinterpret_cast<const double*>(static_cast<const char*>(host_buf) + sizeof h);
    const double* U = hist + p->N;
    const size_t nt = (size_t)p->g.nt;
    cudaStream_t st = S(stream);
    PS_CUDA(cudaMemcpyAsync(p->U.p, U, sizeof(double) * (p->N + 1) * nt, cudaMemcpyHostToDevice, st));
    if (h.has_gold)
      PS_CUDA(cudaMemcpyAsync(p->Gold.p, U + (size_t)(p->N + 1) * nt, sizeof(double) * p->N * nt,
                              cudaMemcpyHostToDevice, st));
    PS_CUDA(cudaStreamSynchronize(st));
    p->hist.assign(hist, hist + h.k);
    p->iters = h.k;
    p->have_forward = h.k > 0;
    p->resumable = true;
  });
}

int ps_resume_parareal(ps_problem* p, double tol, int max_iter, uintptr_t stream, int* iters_out) {
  return guarded([&] {
    PS_REQUIRE(p, "null argument");
    require_slices(p);
    PS_REQUIRE(p->resumable, "nothing to resume: no stopped run or loaded checkpoint on this problem");
    do_run(p, nullptr, tol, max_iter, S(stream), iters_out, p->iters);
  });
}

int ps_get_history(const ps_problem* p, double* inc_host, int cap, int* len) {
  return guarded([&] {
    PS_REQUIRE(p && len, "null argument");
    int n = std::min<int>(cap, (int)p->hist.size());
    for (int i = 0; i < n; ++i) inc_host[i] = p->hist[i];
    *len = n;
  });
}

int ps_run_fine_sequential(ps_problem* p, const double* u0_dev, double* U_out_dev, uintptr_t stream) {
  return guarded([&] {
    PS_REQUIRE(p && u0_dev && U_out_dev, "null argument");
    require_slices(p);
    cudaStream_t st = S(stream);
    const long long nt = p->g.nt;
    p->updates = 0;
    p->launches = 0;
    tile_flag_reset(p, st);
    PS_CUDA(cudaMemcpyAsync(U_out_dev, u0_dev, sizeof(double) * nt, cudaMemcpyDeviceToDevice, st));
    for (int n = 0; n < p->N; ++n) run_F(p, n, 1, U_out_dev + n * nt, U_out_dev + (n + 1) * nt, st);
    tile_flag_check(p, st);
  });
}

int ps_run_coarse_sequential(ps_problem* p, const double* u0_dev, double* U_out_dev, uintptr_t stream) {
  return guarded([&] {
    PS_REQUIRE(p && u0_dev && U_out_dev, "null argument");
    require_slices(p);
    cudaStream_t st = S(stream);
    const long long nt = p->g.nt;
    tile_flag_reset(p, st);
    PS_CUDA(cudaMemcpyAsync(U_out_dev, u0_dev, sizeof(double) * nt, cudaMemcpyDeviceToDevice, st));
    for (int n = 0; n < p->N; ++n) {
      run_G(p, n, U_out_dev + n * nt, CorrArgs{}, st);
      PS_CUDA(cudaMemcpyAsync(U_out_dev + (n + 1) * nt, p->gtmp.p, sizeof(double) * nt, cudaMemcpyDeviceToDevice, st));
    }
    tile_flag_check(p, st);
  });
}

int ps_substep_solve(ps_problem* p, int which, int m, double* x_dev, uintptr_t stream) {
  return guarded([&] {
    PS_REQUIRE(p && x_dev, "null argument");
    require_slices(p);
    PS_REQUIRE(which == 0 || which == 1, "which must be 0 (fine) or 1 (coarse)");
    Prop& P = which == 0 ? p->F : p->G;
    PS_REQUIRE(m >= 0 && m < P.sp->M, "substep out of range");
    if (P.sp->kind == PS_SPLIT_DD) {
      tile_flag_reset(p, S(stream));
      dd_solve(p->g, 1, *P.dd, m, x_dev, 1, p->tmo.p, S(stream));
      tile_flag_check(p, S(stream));
      return;
    }
    sweep_dim<double, double>(p->g, 1, *P.dim[m], P.f32, x_dev, x_dev, SourceArgs{}, CorrArgs{}, nullptr, S(stream));
  });
}

int ps_propagate(ps_problem* p, int which, int nsteps, int t0, int tstride, double* x_dev, uintptr_t stream) {
  return guarded([&] {
    PS_REQUIRE(p && x_dev && nsteps >= 0, "bad argument");
    require_slices(p);
    PS_REQUIRE(which == 0 || which == 1, "which must be 0 (fine) or 1 (coarse)");
    Prop& P = which == 0 ? p->F : p->G;
    if (p->op->src_t.p)
      PS_REQUIRE(t0 >= 0 && t0 + (long long)nsteps * tstride < p->op->src_t_len, "time index outside src_t");
    if (p->op->src2_t.p)
      PS_REQUIRE(t0 >= 0 && t0 + (long long)nsteps * tstride < p->op->src2_t_len, "time index outside src2_t");
    cudaStream_t st = S(stream);
    tile_flag_reset(p, st);
    for (int q = 0; q < nsteps; ++q) {
      const int te = t0 + (q + 1) * tstride;
      if (!P.f32) {
        fie_step64(p, P, 1, x_dev, x_dev, te, 0, CorrArgs{}, st, which == 0 ? "F" : "G");
      } else {
        for (int m = 0; m < P.sp->M; ++m) {
          SourceArgs sa = m == 0 ? source_for(p, P, te, 0) : SourceArgs{};
          sweep_dim<double, double>(p->g, 1, *P.dim[m], true, x_dev, x_dev, sa, CorrArgs{}, nullptr, st);
        }
      }
    }
    tile_flag_check(p, st);
  });
}

int ps_problem_stats(const ps_problem* p, ps_stats* out) {
  return guarded([&] {
    PS_REQUIRE(p && out, "null argument");
    out->iterations = p->iters;
    out->unknown_updates = p->updates;
    out->ms_total = p->ms_total;
    out->ms_fine = p->ms_fine;
    out->ms_coarse = p->ms_coarse;
    out->kernel_launches = p->launches;
  });
}

namespace {
// Tile plans of the fine propagator for a schedule (slots per tile, positions, pipeline).
void rebuild_tiles(ps_problem* p, int slots, int positions, int pipe, int vec) {
  if (p->F.sp->kind != PS_SPLIT_DIM) return;
  Geom g3 = p->g;
  if (g3.dim == 2) g3.n[2] = 1;
  const bool mixed = p->prm.precision == PS_PREC_MIXED;
  void* W = mixed ? static_cast<void*>(p->W.p) : static_cast<void*>(p->W64.p);
  TilePlan tmp[3];
  for (int m = 0; m < p->g.dim; ++m)
    tile_plan(g3, p->S_pad, mixed ? 4 : 8, m, tmp[m], W, positions, pipe, slots, vec);
  for (int m = 0; m < p->g.dim; ++m) p->F.tiles[m] = tmp[m];
  p->prm.tile_slots = slots;
  p->prm.tile_positions = positions;
  p->prm.tile_pipeline = pipe == 1 ? 1 : 2;
  p->prm.tile_lines_per_thread = vec;
}
}  // namespace

int ps_autotune(ps_problem* p, int budget_ms, uintptr_t stream, int* choice_out) {
  return guarded([&] {
    PS_REQUIRE(p, "null argument");
    require_slices(p);
    if (choice_out) *choice_out = 0;
    if (p->F.sp->kind != PS_SPLIT_DIM) {
      // DD: time slices per CTA of the fine colour solves (1, 2, 4) on all slices at once, in the
      // F-result buffer (recomputed by every run); each slice's arithmetic does not depend on it
      p->tune_log.clear();
      cudaStream_t st = S(stream);
      if (p->dr) return;
      tile_flag_reset(p, st);
      cudaEvent_t e0, e1;
      PS_CUDA(cudaEventCreate(&e0));
      PS_CUDA(cudaEventCreate(&e1));
      float best = 1e30f;
      int bestS = p->prm.dd_slices_per_block > 0 ? p->prm.dd_slices_per_block : 2;
      try {
        for (int spb : {1, 2, 4}) {
          auto solve = [&] {
            for (int c = 0; c < p->F.sp->M; ++c) dd_solve(p->g, p->N, *p->F.dd, c, p->Fout.p, spb, p->tmo.p, st);
          };
          solve();
          PS_CUDA(cudaEventRecord(e0, st));
          solve();
          PS_CUDA(cudaEventRecord(e1, st));
          PS_CUDA(cudaEventSynchronize(e1));
          float ms = 0.f;
          PS_CUDA(cudaEventElapsedTime(&ms, e0, e1));
          p->tune_log.push_back({"dd:" + std::to_string(spb) + "-slices-per-cta", ms, 0});
          if (ms < best) {
            best = ms;
            bestS = spb;
          }
        }
      } catch (...) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        throw;
      }
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      p->prm.dd_slices_per_block = bestS;
      for (auto& e : p->tune_log)
        if (e.name == "dd:" + std::to_string(bestS) + "-slices-per-cta") e.chosen = 1;
      tile_flag_check(p, st);
      if (choice_out) *choice_out = bestS;
      return;
    }
    cudaStream_t st = S(stream);
    const bool mixed = p->prm.precision == PS_PREC_MIXED;
    struct Cand {
      int slots, positions, pipe, vec;
    };
    // slots per tile, line positions per tile, persistent double-buffered CTAs, lines per thread
    // pipe: 0 one tile per CTA, 1 persistent ring of stages
    std::vector<Cand> cands = {{32, 2, 0, 2}, {32, 1, 0, 2}, {32, 1, 0, 1}, {32, 2, 0, 1}, {64, 1, 0, 2},
                               {16, 1, 0, 1}, {32, 1, 1, 2}, {32, 1, 1, 1}};
    // the grouped kernels of a batch run one tile per item, one line per thread, and every item
    // of a launch with the largest shared-memory tile of the batch: one line position per tile
    // keeps six tiles per SM for all of them (a single problem on two positions would halve that)
    if (p->batched > 0)
      cands.erase(std::remove_if(cands.begin(), cands.end(),
                                 [](const Cand& c) { return c.pipe || c.vec == 2 || c.positions != 1; }),
                  cands.end());
    // FP32 tiles of 16 slots (64-byte rows) are valid for one-box tiles but measured far slower
    // on GB300 (the z-sweep's 64-byte rows): not timed
    if (mixed)
      cands.erase(std::remove_if(cands.begin(), cands.end(), [](const Cand& c) { return c.slots * 4 < 128; }),
                  cands.end());
    auto cand_name = [](const Cand& c) {
      return "fine:" + std::to_string(c.slots) + "x" + std::to_string(c.positions) + "/v" + std::to_string(c.vec) +
             (c.pipe == 1 ? "/ring" : "/tile");
    };
    tile_flag_reset(p, st);
    p->tune_log.clear();
    cudaEvent_t e0, e1;
    PS_CUDA(cudaEventCreate(&e0));
    PS_CUDA(cudaEventCreate(&e1));
    Geom g3 = p->g;
    if (g3.dim == 2) g3.n[2] = 1;
    const int M = p->g.dim;
    float best = 1e30f;
    Cand bestc{0, 0, 0, 0};
    const double per_cand_ms = std::max(1.0, (double)budget_ms / cands.size());
    const int old_slots = p->prm.tile_slots, old_pos = p->prm.tile_positions, old_pipe = p->prm.tile_pipeline,
              old_vec = p->prm.tile_lines_per_thread;
    try {
      for (const Cand& c : cands) {
        try {
          rebuild_tiles(p, c.slots, c.positions, c.pipe, c.vec);
        } catch (const Error&) {
          continue;  // shape does not fit this grid / precision
        }
        if (p->F.tiles[0].TS != c.slots) continue;  // the plan could not take these slots: a duplicate
        auto sweep_all = [&]() {
          for (int m = 0; m < M; ++m) {
            if (mixed)
              tile_sweep<float>(g3, p->F.tiles[m], *p->F.dim[m], p->S_pad, 0, p->N, SourceArgs{}, nullptr, p->tmo.p,
                                st);
            else
              tile_sweep<double>(g3, p->F.tiles[m], *p->F.dim[m], p->S_pad, 0, p->N, SourceArgs{}, nullptr, p->tmo.p,
                                 st);
          }
        };
        sweep_all();  // warm-up
        int reps = 1;
        float ms = 0.f;
        for (;;) {
          PS_CUDA(cudaEventRecord(e0, st));
          for (int r = 0; r < reps; ++r) sweep_all();
          PS_CUDA(cudaEventRecord(e1, st));
          PS_CUDA(cudaEventSynchronize(e1));
          PS_CUDA(cudaEventElapsedTime(&ms, e0, e1));
          if (ms * 4 >= per_cand_ms || reps >= 64) break;
          reps *= 2;
        }
        const float per = ms / reps;
        p->tune_log.push_back({cand_name(c),
                               per, 0});
        if (per < best) {
          best = per;
          bestc = c;
        }
      }
    } catch (...) {
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      throw;
    }
    // coarse line solves on one slice: staged through shared memory or streamed, timed on one
    // coarse step's sweeps of this problem (both schedules compute the same recurrences with the
    // same roundings, so the choice changes no result)
    int coarse_choice = 0;
    if (p->G.sp->kind == PS_SPLIT_DIM) {
      const int MG = p->g.dim;
      auto coarse_step = [&]() {
        for (int m = 0; m < MG; ++m) {
          if (p->delta32) {
            if (m == 0) {
              coarse_x32<float>(p, p->g32.p, p->g32.p, SourceArgs{}, st);
            } else if (!(p->coarse_staged &&
                         coarse_sweep_staged<float>(p->g, *p->G.dim[m], p->g32.p, p->g32.p, SourceArgs{}, CorrArgs{}, st))) {
              sweep_dim<float, float>(p->g, 1, *p->G.dim[m], true, p->g32.p, p->g32.p, SourceArgs{}, CorrArgs{}, nullptr,
                                      st);
            }
          } else {
            coarse_sweep64(p, *p->G.dim[m], m == 0 ? p->U.p : p->gtmp.p, p->gtmp.p, SourceArgs{}, CorrArgs{}, st);
          }
        }
      };
      auto time4 = [&](auto&& fn) {
        fn();  // warm-up
        PS_CUDA(cudaEventRecord(e0, st));
        for (int r = 0; r < 4; ++r) fn();
        PS_CUDA(cudaEventRecord(e1, st));
        PS_CUDA(cudaEventSynchronize(e1));
        float ms = 0.f;
        PS_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        return ms / 4.f;
      };
      // the coarse x-sweep's schedule: Thomas per row, PCR per warp (FP32 increment form) or the
      // hybrid segmented scans per warp.  In a batch, whose grouped kernels run Thomas, only Thomas
      // keeps the batched results bitwise equal to the problem's own runs.
      {
        const char* names[4] = {"", "thomas", "pcr", "hybrid"};
        const std::string pre = p->delta32 ? "coarse-x32:" : "coarse-x64:";
        float xbest = 1e30f;
        int xchoice = p->xsched;
        std::string xname;
        for (int sc = PS_SCHED_THOMAS; sc <= PS_SCHED_HYBRID; ++sc) {
          if (sc == PS_SCHED_PCR && (!p->delta32 || !p->pcr_e.p)) continue;  // FP32 rows of <= 256 nodes
          // a batch's grouped kernels run Thomas (FP64 coarse) or the hybrid (increment form)
          if (p->batched > 0 && sc != (p->delta32 ? PS_SCHED_HYBRID : PS_SCHED_THOMAS)) continue;
          if (sc == PS_SCHED_HYBRID && !p->delta32 && !p->G.dim[0]->lt64.p) continue;
          p->xsched = sc;
          const float ms = p->delta32
                               ? time4([&] { coarse_x32<float>(p, p->g32.p, p->g32.p, SourceArgs{}, st); })
                               : time4([&] {
                                   coarse_sweep64(p, *p->G.dim[0], p->U.p, p->gtmp.p, SourceArgs{}, CorrArgs{}, st);
                                 });
          const std::string nm = pre + names[sc];
          p->tune_log.push_back({nm, ms, 0});
          if (ms < xbest) {
            xbest = ms;
            xchoice = sc;
            xname = nm;
          }
        }
        p->xsched = xchoice;
        p->prm.schedule = xchoice;
        for (auto& e : p->tune_log)
          if (e.name == xname) e.chosen = 1;
      }
      float tbest = 1e30f;
      const bool saved = p->coarse_staged;
      for (int sched = PS_COARSE_SWEEP_STAGED; sched <= PS_COARSE_SWEEP_STREAMED; ++sched) {
        p->coarse_staged = sched == PS_COARSE_SWEEP_STAGED;
        const float ms = time4(coarse_step);
        p->tune_log.push_back({sched == PS_COARSE_SWEEP_STAGED ? "coarse:staged" : "coarse:streamed", ms, 0});
        if (ms < tbest) {
          tbest = ms;
          coarse_choice = sched;
        }
      }
      p->coarse_staged = coarse_choice ? coarse_choice == PS_COARSE_SWEEP_STAGED : saved;
      if (coarse_choice) p->prm.coarse_sweep = coarse_choice;
      for (auto& e : p->tune_log)
        if (e.name == (coarse_choice == PS_COARSE_SWEEP_STAGED ? "coarse:staged" : "coarse:streamed")) e.chosen = 1;
      // FP64 coarse form: the correction fused into the last sweep, or as its own pass.  Timed on
      // the last sweep with an epilogue whose target is the scratch state (the values are
      // discarded; the next run clears the flags it may set)
      if (!p->delta32) {
        CorrArgs scratch;
        scratch.mode = 1;
        scratch.U_next = scratch.Gold = p->gtmp.p;
        scratch.Fout = p->gtmp.p;
        scratch.inc = p->inc.p;
        scratch.nonfinite = p->flag.p;
        const LineFactors& fz = *p->G.dim[MG - 1];
        float sbest = 1e30f;
        bool split_choice = p->coarse_split;
        for (int split = 0; split < 2; ++split) {
          const float ms = time4([&] {
            if (split) {
              coarse_sweep64(p, fz, p->gtmp.p, p->gtmp.p, SourceArgs{}, CorrArgs{}, st);
              dd_correct(p->g, p->gtmp.p, scratch, st);
            } else {
              coarse_sweep64(p, fz, p->gtmp.p, p->gtmp.p, SourceArgs{}, scratch, st);
            }
          });
          p->tune_log.push_back({split ? "coarse-corr:split" : "coarse-corr:fused", ms, 0});
          if (ms < sbest) {
            sbest = ms;
            split_choice = split != 0;
          }
        }
        p->coarse_split = split_choice;
        for (auto& e : p->tune_log)
          if (e.name == (split_choice ? "coarse-corr:split" : "coarse-corr:fused")) e.chosen = 1;
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (bestc.slots == 0) {
      rebuild_tiles(p, old_slots, old_pos, old_pipe == 1 ? 1 : 0, old_vec);
      if (choice_out) *choice_out = coarse_choice * 100000;
      return;
    }
    rebuild_tiles(p, bestc.slots, bestc.positions, bestc.pipe, bestc.vec);
    for (auto& e : p->tune_log)
      if (e.name == cand_name(bestc))
        e.chosen = 1;
    tile_flag_check(p, st);
    // choice code: coarse schedule, lines per thread, slots, positions, pipeline as decimal digits cvSSpq
    if (choice_out)
      *choice_out = coarse_choice * 100000 + bestc.vec * 10000 + bestc.slots * 100 + bestc.positions * 10 + bestc.pipe;
  });
}

int ps_autotune_record(const ps_problem* p, ps_tune_entry* out, int cap, int* len) {
  return guarded([&] {
    PS_REQUIRE(p && len && (out || cap == 0), "null argument");
    const int n = std::min<int>(cap, (int)p->tune_log.size());
    for (int i = 0; i < n; ++i) {
      const auto& e = p->tune_log[i];
      std::memset(out[i].name, 0, sizeof out[i].name);
      std::strncpy(out[i].name, e.name.c_str(), sizeof out[i].name - 1);
      out[i].ms = e.ms;
      out[i].chosen = e.chosen;
    }
    *len = n;
  });
}

int ps_copy_schedule(const ps_problem* src, ps_problem* dst) {
  return guarded([&] {
    PS_REQUIRE(src && dst, "null argument");
    rebuild_tiles(dst, src->prm.tile_slots, src->prm.tile_positions,
                  src->prm.tile_pipeline == 1 ? 1 : 0,
                  src->prm.tile_lines_per_thread);
    dst->coarse_staged = src->coarse_staged;
    dst->prm.coarse_sweep = src->prm.coarse_sweep;
    dst->xsched = src->xsched;
    dst->prm.schedule = src->prm.schedule;
    dst->coarse_split = src->coarse_split;
  });
}

int ps_problem_update_coefficients(ps_problem* p, const double* a_nodal_dev, uintptr_t stream) {
  return guarded([&] {
    PS_REQUIRE(p && a_nodal_dev, "null argument");
    require_slices(p);
    ps_operator* op = const_cast<ps_operator*>(p->op);
    PS_REQUIRE(op->a.p, "the operator was created with a = 1; create it with a nodal coefficient to update it");
    cudaStream_t st = S(stream);
    PS_CUDA(cudaMemcpyAsync(op->a.p, a_nodal_dev, sizeof(double) * op->a.n, cudaMemcpyDeviceToDevice, st));
    const bool mixed = p->prm.precision == PS_PREC_MIXED;
    Geom g3 = p->g;
    if (g3.dim == 2) g3.n[2] = 1;
    for (Prop* P : {&p->F, &p->G}) {
      const bool fine = P == &p->F;
      if (P->sp->kind == PS_SPLIT_DIM) {
        for (int m = 0; m < p->g.dim; ++m) {
          factor_dim(p->g, m, op->a.p, op->c / p->g.dim, P->tau, *P->dim[m], fine ? mixed : p->delta32, st);
          if (fine) factor_lines(g3, *P->dim[m], mixed, st);
          else if (p->delta32 && m == 0) {
            factor_lines(g3, *P->dim[m], true, st);
            if (p->g.n[0] <= 256) tridiag_x_rows(p->g, op->a.p, op->c / p->g.dim, P->tau, p->pcr_e, p->pcr_d, st);
          } else if (m == 0) {
            factor_lines(g3, *P->dim[m], false, st);
          }
        }
      } else {
        dd_factor(p->g, P->sp->dd, op->a.p, op->d12.p, op->c, P->tau, *P->dd, st);
      }
    }
    p->have_forward = false;
    p->resumable = false;
    PS_CUDA(cudaStreamSynchronize(st));
  });
}

namespace {
// Coefficient gradient: recompute every fine state of every slice from the checkpoints,
// then sweep backwards with the transposed substeps, accumulating the edge products.
void adjoint_coefficient_gradient(ps_problem* p, double* grad_a, cudaStream_t st) {
  Prop& F = p->F;
  const long long nt = p->g.nt;
  const int N = p->N, s = F.steps, M = p->g.dim, S_pad = p->S_pad;
  Geom g3 = p->g;
  if (g3.dim == 2) g3.n[2] = 1;
  const size_t wsz = (size_t)S_pad * nt;
  if (!p->adj_ready) {
    p->snap.alloc((size_t)s * M * wsz);
    p->Lam.alloc(wsz);
    PS_CUDA(cudaMemsetAsync(p->Lam.p, 0, wsz * sizeof(double), st));
    for (int m = 0; m < M; ++m) {
      p->gedge[m].alloc((size_t)edge_count(p->g, m));
      tile_plan(g3, S_pad, 8, m, p->adj_tiles[m], p->Lam.p, p->prm.tile_positions,
                p->prm.tile_pipeline == 1 ? 1 : 0, p->prm.tile_slots);
    }
    p->adj_ready = true;
  }
  // forward recomputation from U_0..U_{N-1}, every substep's result kept
  to_interleaved<double>(p->g, p->Uchk.p, p->W64.p, S_pad, 0, N, st);
  for (int q = 0; q < s; ++q)
    for (int m = 0; m < M; ++m) {
      SourceArgs sa = m == 0 ? source_for(p, F, q + 1, p->fs) : SourceArgs{};
      tile_sweep<double>(g3, F.tiles[m], *F.dim[m], S_pad, 0, N, sa, p->srcrow64.p, p->tmo.p, st);
      PS_CUDA(cudaMemcpyAsync(p->snap.p + ((size_t)q * M + m) * wsz, p->W64.p, wsz * sizeof(double),
                              cudaMemcpyDeviceToDevice, st));
    }
  // slot n <- lambda_{n+1} = (adjoint state N-1-n of the reversed-time run held in U)
  to_interleaved<double>(p->g, p->U.p, p->Lam.p, S_pad, 0, N, st, true);
  for (int m = 0; m < M; ++m) PS_CUDA(cudaMemsetAsync(p->gedge[m].p, 0, p->gedge[m].n * sizeof(double), st));
  for (int q = s - 1; q >= 0; --q)
    for (int m = M - 1; m >= 0; --m) {
      tile_sweep<double>(g3, p->adj_tiles[m], *F.dim[m], S_pad, 0, N, SourceArgs{}, nullptr, p->tmo.p, st);
      const double h = 1.0 / (p->g.n[m] + 1);
      grad_edges(g3, m, p->Lam.p, p->snap.p + ((size_t)q * M + m) * wsz, S_pad, N, F.tau / (h * h), p->gedge[m].p,
                 st);
    }
  const double* ge[3] = {p->gedge[0].p, p->gedge[1].p, M == 3 ? p->gedge[2].p : nullptr};
  combine_grad(g3, ge, grad_a, st);
}

// Body of ps_adjoint_vjp (see include/ps.h).
void adjoint_vjp(ps_problem* p, const double* gN_dev, double tol, int max_iter, double* grad_u0_dev,
                 double* grad_a_dev, cudaStream_t st, int* iters_out) {
  PS_REQUIRE(p->have_forward, "ps_adjoint_vjp needs a preceding ps_run_parareal on this problem");
  if (p->delta32) throw Error(PS_ERR_UNSUPPORTED, "the adjoint runs with the FP64 coarse propagator");
  if (p->dr) throw Error(PS_ERR_UNSUPPORTED, "the adjoint differentiates the FIE fine propagator");
  if (grad_a_dev) {
    if (p->F.sp->kind != PS_SPLIT_DIM || p->G.sp->kind != PS_SPLIT_DIM)
      throw Error(PS_ERR_UNSUPPORTED, "the coefficient gradient is implemented for the dimensional splitting");
    if (p->F.f32) throw Error(PS_ERR_UNSUPPORTED, "the coefficient gradient runs in FP64 (PS_PREC_FP64)");
    PS_REQUIRE(p->op->a.p, "the coefficient gradient needs an operator created with a nodal coefficient");
  }
  const long long nt = p->g.nt;
  const size_t ubytes = sizeof(double) * (size_t)(p->N + 1) * nt;
  if (!p->Uchk.p) p->Uchk.alloc((size_t)(p->N + 1) * nt);
  PS_CUDA(cudaMemcpyAsync(p->Uchk.p, p->U.p, ubytes, cudaMemcpyDeviceToDevice, st));
  const int saved_mode = p->prm.tol_mode;
  const std::vector<double> saved_hist = p->hist;
  const int saved_iters = p->iters;
  p->transposed = true;
  p->prm.tol_mode = 1;
  try {
    do_run(p, gN_dev, tol, max_iter, st, iters_out);
  } catch (...) {
    p->transposed = false;
    p->prm.tol_mode = saved_mode;
    throw;
  }
  p->transposed = false;
  p->prm.tol_mode = saved_mode;
  PS_CUDA(cudaMemcpyAsync(grad_u0_dev, p->U.p + (long long)p->N * nt, sizeof(double) * nt, cudaMemcpyDeviceToDevice,
                          st));
  if (grad_a_dev) adjoint_coefficient_gradient(p, grad_a_dev, st);
  // the problem's states are the forward ones again
  PS_CUDA(cudaMemcpyAsync(p->U.p, p->Uchk.p, ubytes, cudaMemcpyDeviceToDevice, st));
  p->hist = saved_hist;
  p->iters = saved_iters;
  p->have_forward = true;
  tile_flag_check(p, st);
}
}  // namespace

int ps_adjoint_vjp(ps_problem* p, const double* gN_dev, double tol, int max_iter, double* grad_u0_dev,
                   double* grad_a_dev, uintptr_t stream, int* iters_out) {
  return guarded([&] {
    PS_REQUIRE(p && gN_dev && grad_u0_dev, "null argument");
    require_slices(p);
    adjoint_vjp(p, gN_dev, tol, max_iter, grad_u0_dev, grad_a_dev, S(stream), iters_out);
  });
}

int ps_adjoint(ps_problem* p, const double* u_target_dev, double tol, int max_iter, double* grad_u0_dev,
               double* grad_a_dev, uintptr_t stream, double* J_out, int* iters_out) {
  return guarded([&] {
    PS_REQUIRE(p && u_target_dev && grad_u0_dev, "null argument");
    require_slices(p);
    PS_REQUIRE(p->have_forward, "ps_adjoint needs a preceding ps_run_parareal on this problem");
    cudaStream_t st = S(stream);
    const long long nt = p->g.nt;
    // g = U_N - u_target into the coarse scratch state (the adjoint run copies it to its U_0
    // before the scratch state is reused), and J = 1/2 |g|^2 summed in a fixed order
    loss_residual_kernel<<<kLossBlocks, 256, 0, st>>>(p->U.p + (long long)p->N * nt, u_target_dev, p->gtmp.p, nt,
                                                     p->jpart.p);
    PS_CUDA(cudaGetLastError());
    loss_sum_kernel<<<1, 256, 0, st>>>(p->jpart.p, kLossBlocks, p->jpart.p + kLossBlocks);
    PS_CUDA(cudaGetLastError());
    double J = 0.0;
    PS_CUDA(cudaMemcpyAsync(&J, p->jpart.p + kLossBlocks, sizeof(double), cudaMemcpyDeviceToHost, st));
    adjoint_vjp(p, p->gtmp.p, tol, max_iter, grad_u0_dev, grad_a_dev, st, iters_out);
    if (J_out) *J_out = J;  // the copy completed: adjoint_vjp synchronised the stream
  });
}

int ps_run_coarse_sequential_noalloc(ps_problem* p, const double* u0_dev, double* U_out_dev, uintptr_t stream) {
  return guarded([&] {
    PS_REQUIRE(p && u0_dev && U_out_dev, "null argument");
    require_slices(p);
    const long long nt = p->g.nt;
    if (nt > PS_NOALLOC_MAX_UNKNOWNS)
      throw Error(PS_ERR_INVALID, "grid has " + std::to_string(nt) + " unknowns; the no-allocation coarse solve holds at most " +
                                      std::to_string(PS_NOALLOC_MAX_UNKNOWNS));
    cudaStream_t st = S(stream);
    double* work = noalloc_work_ptr();
    tile_flag_reset(p, st);
    PS_CUDA(cudaMemcpyAsync(U_out_dev, u0_dev, sizeof(double) * nt, cudaMemcpyDeviceToDevice, st));
    for (int n = 0; n < p->N; ++n) {
      for (int q = 0; q < p->G.steps; ++q) coarse_step_into(p, n, q, q == 0 ? U_out_dev + n * nt : work, work, st);
      PS_CUDA(cudaMemcpyAsync(U_out_dev + (n + 1) * nt, work, sizeof(double) * nt, cudaMemcpyDeviceToDevice, st));
    }
    tile_flag_check(p, st);
  });
}

int ps_problem_kernel_times(const ps_problem* p, ps_kernel_time* out, int cap, int* len) {
  return guarded([&] {
    PS_REQUIRE(p && len && (out || cap == 0), "null argument");
    int n = std::min<int>(cap, (int)p->kt.kinds.size());
    for (int i = 0; i < n; ++i) {
      const auto& k = p->kt.kinds[i];
      std::memset(out[i].name, 0, sizeof out[i].name);
      std::strncpy(out[i].name, k.name.c_str(), sizeof out[i].name - 1);
      out[i].launches = k.launches;
      out[i].ms = k.ms;
      out[i].bytes = k.bytes;
      out[i].flops = k.flops;
    }
    *len = n;
  });
}

}  // extern "C"
