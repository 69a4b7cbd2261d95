// ps_batch.cu -- many independent parareal problems advanced together (batched launches,
// one CUDA graph per parareal iteration) and the tile-shape autotuner.
//
// All problems of a batch start together, so every unconverged problem is at the same
// parareal iteration k (Sec. 3).  One iteration of the whole batch is a fixed sequence of
// grouped persistent launches:
//   pack U_n -> interleaved FP32 (slices n >= k-1 of every problem)
//   for every fine step j and direction m: one tile-sweep launch over every problem with
//     s_p > j (the fine line solves of all slices of all problems)
//   unpack -> F results;  U_k <- F(U_{k-1}) (the finite-termination slice)
//   for every coarse step n: one x-sweep and one y-sweep-with-correction launch over every
//     problem with N_p > n >= k
// The launches read their work from device tables (which problems, which tiles or blocks),
// so the sequence is captured once as a CUDA graph and replayed every iteration; between
// replays the host only rewrites the tables (converged problems drop out) and reads back
// the per-problem increments.  The tile launches take the batch's own tile shapes (problems
// with shorter lines get more line positions per tile, batch_tile_plans).  Each problem's
// arithmetic is the same as in its own ps_run_parareal, so batched and individual results
// agree bitwise.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "ps_handles.h"

using namespace ps;

struct ps_batch {
  std::vector<ps_problem*> probs;
  int count = 0;
  int maxS = 0, maxN = 0;
  bool var = true;
  bool delta32 = false;             // the problems' coarse propagator: FP32 increment form
  DevBuf<XWarpJob> xjobs32;         // [maxN][count] x-sweeps of the increment form
  std::vector<XWarpJob> h_xjobs32;
  int span_max = 0;
  // device tables
  int dims = 2;                     // the problems' dimension (all the same)
  DevBuf<unsigned char> tile_jobs;  // [dims][count] TileJob
  DevBuf<WorkSeg> tile_segs;        // [dims][count]
  DevBuf<int> tile_nseg;            // [maxS][dims]
  DevBuf<PackJob> pack_jobs, unpack_jobs;
  DevBuf<WorkSeg> pack_segs, unpack_segs;
  DevBuf<CoarseJob> copy_jobs;
  DevBuf<WorkSeg> copy_segs;
  DevBuf<CoarseJob> cjobs;          // [maxN][count]
  DevBuf<WorkSeg> xsegs, ysegs, zsegs;  // [maxN][count]
  DevBuf<int> nseg_misc;            // [0] pack, [1] unpack, [2] copy, [3 + n] coarse step n
  DevBuf<unsigned long long> inc;   // per problem
  DevBuf<int> flag, tmo;
  std::vector<TilePlan> bplans;     // [count][dims] the batch's tile shapes (batch_tile_plans)
  size_t tile_smem = 0;
  int tile_threads = 0;
  int tile_grid = 0;                // CTAs of a grouped tile launch: one wave
  int sms = 152;
  cudaStream_t cs = nullptr;
  cudaGraphExec_t iter_graph = nullptr, init_graph = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  // host staging
  std::vector<unsigned char> h_tile_jobs;
  std::vector<WorkSeg> h_tile_segs, h_pack_segs, h_unpack_segs, h_copy_segs, h_xsegs, h_ysegs, h_zsegs;
  std::vector<int> h_tile_nseg, h_nseg_misc;
  std::vector<PackJob> h_pack, h_unpack;
  std::vector<CoarseJob> h_copy, h_cjobs;
  std::vector<unsigned long long> h_inc;
  std::vector<int> h_flag;
  double updates = 0.0;
  int launches_per_iter = 0, launches_init = 0, launches = 0;
  bool registered = false;  // counted in its problems' `batched`
  ~ps_batch() {
    if (registered)
      for (ps_problem* p : probs) --p->batched;
    if (iter_graph) cudaGraphExecDestroy(iter_graph);
    if (init_graph) cudaGraphExecDestroy(init_graph);
    if (ev_in) cudaEventDestroy(ev_in);
    if (ev_out) cudaEventDestroy(ev_out);
    if (cs) cudaStreamDestroy(cs);
  }
};

namespace {

thread_local std::string g_batch_error;
int bfail(int code, const std::string& m) {
  g_batch_error = m;
  return code;
}
template <typename F>
int bguarded(F&& f) {
  try {
    f();
    return PS_OK;
  } catch (const Error& e) {
    return bfail(e.code, e.what());
  } catch (const std::exception& e) {
    return bfail(PS_ERR_INVALID, e.what());
  }
}

CoarseJob coarse_job(ps_batch* b, int i, int n) {
  ps_problem* p = b->probs[i];
  CoarseJob j{};
  const long long nt = p->g.nt;
  j.xin = p->U.p + n * nt;
  j.xout = p->gtmp.p;
  j.nx = p->g.n[0];
  j.ny = p->g.n[1];
  j.nz = p->g.dim == 3 ? p->g.n[2] : 1;
  j.rows = (long long)j.ny * j.nz;
  j.nt = nt;
  j.lx = p->G.dim[0]->l64.p;
  j.rx = p->G.dim[0]->r64.p;
  j.ly = p->G.dim[1]->l64.p;
  j.ry = p->G.dim[1]->r64.p;
  if (p->g.dim == 3) {
    j.lz = p->G.dim[2]->l64.p;
    j.rz = p->G.dim[2]->r64.p;
  }
  j.ca.U_next = p->U.p + (n + 1) * nt;
  j.ca.Fout = p->Fout.p + n * nt;
  j.ca.Gold = p->Gold.p + n * nt;
  j.ca.inc = b->inc.p + i;
  j.ca.nonfinite = b->flag.p + i;
  j.ca.slice_stats = nullptr;
  if (p->op->src.p) {
    // as the problem's own coarse step n: the source at the step's end time, step DeltaT
    j.sa.src = p->op->src.p;
    j.sa.src_t = p->op->src_t.p;
    j.sa.t0 = n * p->fs + p->fs;
    j.sa.tstride = 0;
    j.sa.src_t_len = p->op->src_t_len;
    j.sa.tau = p->G.tau;
  }
  return j;
}

template <typename T>
void upload(DevBuf<T>& d, const std::vector<T>& h, cudaStream_t st) {
  PS_REQUIRE(h.size() <= d.n, "batch work table larger than its device buffer");
  if (!h.empty()) PS_CUDA(cudaMemcpyAsync(d.p, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice, st));
}

// Coarse tables for the initial sweep (mode 2) or iteration k (mode 1): for every step n,
// the problems with N_p > n (and n >= k) in order of decreasing N_p.
void fill_coarse_tables(ps_batch* b, const std::vector<int>& active, int k) {
  std::vector<int> order(active);
  std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return b->probs[a]->N > b->probs[c]->N; });
  const int P = b->count;
  for (int n = 0; n < b->maxN; ++n) {
    int cnt = 0, px = 0, py = 0, pz = 0;
    if (n >= k)
      for (int i : order) {
        ps_problem* p = b->probs[i];
        if (p->N <= n) break;
        b->h_cjobs[(size_t)n * P + cnt] = coarse_job(b, i, n);
        const long long xrows = b->h_cjobs[(size_t)n * P + cnt].rows;
        int bx = (int)((xrows + coarse_x_grouped_rows() - 1) / coarse_x_grouped_rows());
        if (b->delta32) {
          // the increment form, as the problem's own run_G32: x by warp rows (eight per item)
          // from U_n with the source (initial sweep) or from the FP32 increment, y in place on
          // g32 with the initial (mode 2) or increment (mode 3) epilogue
          const long long nt = p->g.nt;
          const int nx = p->g.n[0];
          XWarpJob xj{};
          xj.in64 = k == 0 ? p->U.p + n * nt : nullptr;
          xj.in32 = k == 0 ? nullptr : p->d32.p;
          xj.out = p->g32.p;
          xj.rows = xrows;
          xj.nx = nx;
          xj.m = ((nx + 31) / 32 + 1) & ~1;
          xj.span = nx + nx / xj.m + 2;
          xj.Lp = (nx + 3) & ~3;
          xj.lt = p->G.dim[0]->lt32.p;
          xj.rt = p->G.dim[0]->rt32.p;
          if (k == 0 && p->op->src.p) xj.sa = b->h_cjobs[(size_t)n * P + cnt].sa;
          b->h_xjobs32[(size_t)n * P + cnt] = xj;
          bx = (int)((xj.rows + 7) / 8);
          CoarseJob& cj = b->h_cjobs[(size_t)n * P + cnt];
          cj.g32 = p->g32.p;
          cj.ly32 = p->G.dim[1]->l32.p;
          cj.ry32 = p->G.dim[1]->r32.p;
          if (p->g.dim == 3) {
            cj.lz32 = p->G.dim[2]->l32.p;
            cj.rz32 = p->G.dim[2]->r32.p;
          }
          cj.ca.Gold = nullptr;
          if (k == 0) {
            cj.ca.mode = 2;
          } else {
            cj.ca.mode = 3;
            cj.ca.dnext = p->d32.p;
          }
        }
        const CoarseJob& cj0 = b->h_cjobs[(size_t)n * P + cnt];
        const long long ylines = (long long)cj0.nx * cj0.nz, zlines = (long long)cj0.nx * cj0.ny;
        const int by = (int)((ylines + coarse_y_grouped_lines() - 1) / coarse_y_grouped_lines());
        const int bz = (int)((zlines + coarse_y_grouped_lines() - 1) / coarse_y_grouped_lines());
        b->h_xsegs[(size_t)n * P + cnt] = WorkSeg{cnt, 0, bx, px};  // job index within step n
        b->h_ysegs[(size_t)n * P + cnt] = WorkSeg{cnt, 0, by, py};
        b->h_zsegs[(size_t)n * P + cnt] = WorkSeg{cnt, 0, bz, pz};
        px += bx;
        py += by;
        pz += bz;
        ++cnt;
      }
    b->h_nseg_misc[3 + n] = cnt;
  }
}

// Tables of iteration k: fine phase on slices k-1.. of every active problem, the slice-k
// copy, and the coarse chain.
void fill_iteration_tables(ps_batch* b, const std::vector<int>& active, int k) {
  const int P = b->count;
  const size_t jb = tile_job_bytes();
  // fine tiles, problems in order of decreasing s
  std::vector<int> order(active);
  std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return b->probs[a]->fs > b->probs[c]->fs; });
  const int D = b->dims;
  for (int m = 0; m < D; ++m) {
    int prefix = 0;
    for (size_t r = 0; r < order.size(); ++r) {
      ps_problem* p = b->probs[order[r]];
      const int nsl = p->N - (k - 1);
      Geom g3 = p->g;
      if (g3.dim == 2) g3.n[2] = 1;
      SourceArgs sa;
      if (p->op->src.p && m == 0) {
        sa.src = p->op->src.p;
        sa.src_t = p->op->src_t.p;
        sa.tstride = p->fs;
        sa.src_t_len = p->op->src_t_len;
        sa.tau = p->F.tau;
      }
      const long long tiles = tile_job_fill(g3, b->bplans[(size_t)order[r] * D + m], *p->F.dim[m], p->S_pad, k - 1,
                                            nsl, b->tmo.p,
                                            b->h_tile_jobs.data() + ((size_t)m * P + r) * jb, sa, p->srcrow32.p);
      b->h_tile_segs[(size_t)m * P + r] = WorkSeg{(int)r, 0, (int)tiles, prefix};  // job index within axis m
      prefix += (int)tiles;
    }
    for (int j = 0; j < b->maxS; ++j) {
      int cnt = 0;
      for (int i : order)
        if (b->probs[i]->fs > j) ++cnt;
      b->h_tile_nseg[(size_t)j * D + m] = cnt;
    }
  }
  // pack / unpack / copy, any order
  int pp = 0, cp = 0, cnt = 0;
  for (size_t r = 0; r < active.size(); ++r) {
    ps_problem* p = b->probs[active[r]];
    const int nsl = p->N - (k - 1);
    const long long nt = p->g.nt;
    b->h_pack[r] = PackJob{p->U.p + (k - 1) * nt, p->W.p, nt, p->S_pad, k - 1, nsl, 0};
    b->h_unpack[r] = PackJob{p->Fout.p + (k - 1) * nt, p->W.p, nt, p->S_pad, k - 1, nsl, 0};
    const int blocks = (int)(((nt + 31) / 32) * ((nsl + 31) / 32));
    b->h_pack_segs[r] = WorkSeg{(int)r, 0, blocks, pp};
    b->h_unpack_segs[r] = WorkSeg{(int)r, 0, blocks, pp};
    pp += blocks;
    CoarseJob cj{};
    cj.xin = p->Fout.p + (k - 1) * nt;
    cj.xout = p->U.p + k * nt;
    cj.nt = nt;
    cj.ca.inc = b->inc.p + active[r];
    cj.ca.nonfinite = b->flag.p + active[r];
    cj.ca.dnext = b->delta32 ? p->d32.p : nullptr;
    b->h_copy[r] = cj;
    const int cb = (int)((nt + 255) / 256);
    b->h_copy_segs[r] = WorkSeg{(int)r, 0, cb, cp};
    cp += cb;
    ++cnt;
  }
  b->h_nseg_misc[0] = b->h_nseg_misc[1] = b->h_nseg_misc[2] = cnt;
  fill_coarse_tables(b, active, k);
}

void upload_tables(ps_batch* b, cudaStream_t st) {
  PS_REQUIRE(b->h_tile_jobs.size() <= b->tile_jobs.n, "batch tile table larger than its device buffer");
  PS_CUDA(cudaMemcpyAsync(b->tile_jobs.p, b->h_tile_jobs.data(), b->h_tile_jobs.size(), cudaMemcpyHostToDevice, st));
  upload(b->tile_segs, b->h_tile_segs, st);
  upload(b->tile_nseg, b->h_tile_nseg, st);
  upload(b->pack_jobs, b->h_pack, st);
  upload(b->unpack_jobs, b->h_unpack, st);
  upload(b->pack_segs, b->h_pack_segs, st);
  upload(b->unpack_segs, b->h_unpack_segs, st);
  upload(b->copy_jobs, b->h_copy, st);
  upload(b->copy_segs, b->h_copy_segs, st);
  upload(b->cjobs, b->h_cjobs, st);
  if (b->delta32) upload(b->xjobs32, b->h_xjobs32, st);
  upload(b->xsegs, b->h_xsegs, st);
  upload(b->ysegs, b->h_ysegs, st);
  upload(b->zsegs, b->h_zsegs, st);
  upload(b->nseg_misc, b->h_nseg_misc, st);
}

// The launch sequence of one iteration (mode 1) or of the initial coarse sweep (mode 2).
int enqueue_sequence(ps_batch* b, int mode, cudaStream_t st) {
  const int P = b->count;
  const int grid = b->sms * 8;
  int n_launch = 0;
  if (mode == 1) {
    pack_grouped(true, b->pack_jobs.p, b->pack_segs.p, b->nseg_misc.p + 0, grid, st);
    ++n_launch;
    for (int j = 0; j < b->maxS; ++j)
      for (int m = 0; m < b->dims; ++m) {
        tile_sweep_grouped(b->tile_jobs.p + (size_t)m * P * tile_job_bytes(), b->tile_segs.p + (size_t)m * P,
                           b->tile_nseg.p + (size_t)j * b->dims + m, b->tile_grid, b->tile_threads, b->tile_smem,
                           b->tmo.p,
                           j, st);
        ++n_launch;
      }
    pack_grouped(false, b->unpack_jobs.p, b->unpack_segs.p, b->nseg_misc.p + 1, grid, st);
    copy_inc_grouped(b->copy_jobs.p, b->copy_segs.p, b->nseg_misc.p + 2, grid, st);
    n_launch += 2;
  }
  for (int n = 0; n < b->maxN; ++n) {
    if (b->delta32) {
      coarse_x32_grouped(b->xjobs32.p + (size_t)n * P, b->xsegs.p + (size_t)n * P, b->nseg_misc.p + 3 + n, grid,
                         b->span_max, st);
      const int epi32 = mode == 2 ? 2 : 3;  // the last sweep carries the epilogue
      coarse_y32_grouped(b->var, b->dims == 3 ? 0 : epi32, b->cjobs.p + (size_t)n * P, b->ysegs.p + (size_t)n * P,
                         b->nseg_misc.p + 3 + n, grid, st, 1);
      n_launch += 2;
      if (b->dims == 3) {
        coarse_y32_grouped(b->var, epi32, b->cjobs.p + (size_t)n * P, b->zsegs.p + (size_t)n * P,
                           b->nseg_misc.p + 3 + n, grid, st, 2);
        ++n_launch;
      }
      continue;
    }
    coarse_x_grouped(b->var, b->cjobs.p + (size_t)n * P, b->xsegs.p + (size_t)n * P, b->nseg_misc.p + 3 + n, grid,
                     st);
    coarse_y_grouped(b->var, b->dims == 3 ? 0 : mode, b->cjobs.p + (size_t)n * P, b->ysegs.p + (size_t)n * P,
                     b->nseg_misc.p + 3 + n, grid, st, 1);
    n_launch += 2;
    if (b->dims == 3) {
      coarse_y_grouped(b->var, mode, b->cjobs.p + (size_t)n * P, b->zsegs.p + (size_t)n * P, b->nseg_misc.p + 3 + n,
                       grid, st, 2);
      ++n_launch;
    }
  }
  return n_launch;
}

cudaGraphExec_t capture(ps_batch* b, int mode) {
  cudaGraph_t g = nullptr;
  PS_CUDA(cudaStreamBeginCapture(b->cs, cudaStreamCaptureModeThreadLocal));
  int n = 0;
  try {
    n = enqueue_sequence(b, mode, b->cs);
  } catch (...) {
    cudaStreamEndCapture(b->cs, &g);
    if (g) cudaGraphDestroy(g);
    throw;
  }
  PS_CUDA(cudaStreamEndCapture(b->cs, &g));
  cudaGraphExec_t ex = nullptr;
  cudaError_t e = cudaGraphInstantiate(&ex, g, 0);
  cudaGraphDestroy(g);
  PS_CUDA(e);
  if (mode == 1) b->launches_per_iter = n;
  else b->launches_init = n;
  return ex;
}

// Problem i of a batch must run the batch's form (see include/ps.h, ps_batch_create).
void batch_check(const ps_batch* b, const ps_problem* p) {
  PS_REQUIRE(p, "null problem");
  PS_REQUIRE(p->N >= 1, "the problem has no slices");
  if (p->fine->kind != PS_SPLIT_DIM || p->coarse->kind != PS_SPLIT_DIM)
    throw Error(PS_ERR_UNSUPPORTED, "batches hold problems with dimensional splitting");
  if (p->prm.precision != PS_PREC_MIXED)
    throw Error(PS_ERR_UNSUPPORTED, "batches run the FP32 line-solve form (PS_PREC_MIXED)");
  if (p->gs != 1) throw Error(PS_ERR_UNSUPPORTED, "batches use one coarse step per slice");
  if (p->delta32 && p->g.n[0] > 1024) throw Error(PS_ERR_UNSUPPORTED, "increment-form batches take rows of <= 1024 nodes");
  // the grouped coarse x-sweep runs the hybrid (increment form) or Thomas (FP64 coarse)
  if (p->xsched != (p->delta32 ? PS_SCHED_HYBRID : PS_SCHED_THOMAS))
    throw Error(PS_ERR_UNSUPPORTED, "batches run the coarse x-sweep with the default schedule of the coarse form");
  if (p->dr) throw Error(PS_ERR_UNSUPPORTED, "batches run the FIE fine propagator");
  const bool var = p->op->a.p != nullptr;
  if (!b->probs.empty()) {
    PS_REQUIRE(var == (b->probs[0]->op->a.p != nullptr), "all problems of a batch need a nodal coefficient, or none");
    PS_REQUIRE(p->delta32 == b->probs[0]->delta32, "all problems of a batch need the same coarse propagator form");
    PS_REQUIRE(p->g.dim == b->probs[0]->g.dim, "all problems of a batch need the same dimension (2-D or 3-D)");
  }
  for (const ps_problem* q : b->probs) PS_REQUIRE(q != p, "a problem appears twice in the batch");
}

// The batch's tile shapes.  One grouped launch serves every problem, so every CTA reserves
// the largest tile of the batch (and at least what six tiles per SM take: one position of
// 255-node FP32 lines, the best single-problem shape).  A problem with shorter lines takes as
// many line positions per tile (up to 4) as fit in that reservation, so that its CTAs keep
// as many bytes in flight as those of the longest lines; with one position per tile a CTA of
// 63-node lines would move an eighth of them.  The number of positions per tile changes no
// line's arithmetic.  Each problem keeps its own plans for its own runs.  The grouped launch
// then takes one wave of CTAs (as many as fit on every SM): its CTAs walk equal shares of the
// tiles, so a second, partial wave would leave SMs idle at the end of each launch.
void batch_tile_plans(ps_batch* b) {
  const int D = b->dims;
  size_t budget = 0;
  for (ps_problem* p : b->probs)
    for (int m = 0; m < D; ++m)
      budget = std::max(budget, tile_grouped_smem(p->F.tiles[m], m == 0 && p->op->src.p != nullptr));
  int dev = 0, per_sm = 0;
  PS_CUDA(cudaGetDevice(&dev));
  PS_CUDA(cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
  budget = std::max(budget, (size_t)per_sm / 6 - 1024);
  b->bplans.assign(b->probs.size() * D, TilePlan{});
  b->tile_smem = 0;
  b->tile_threads = 0;
  for (size_t i = 0; i < b->probs.size(); ++i) {
    ps_problem* p = b->probs[i];
    Geom g3 = p->g;
    if (g3.dim == 2) g3.n[2] = 1;
    for (int m = 0; m < D; ++m) {
      const TilePlan& own = p->F.tiles[m];
      const bool src = m == 0 && p->op->src.p != nullptr;
      TilePlan tp = own;
      for (int q = 4; q > own.P; q /= 2) {
        TilePlan c;
        try {
          tile_plan(g3, p->S_pad, 4, m, c, p->W.p, q, 0, own.TS, 1);
        } catch (const Error&) {
          continue;  // no such shape for these lines: keep fewer positions
        }
        if (c.TS == own.TS && c.P > own.P && tile_grouped_smem(c, src) <= budget) {
          tp = c;
          break;
        }
      }
      b->bplans[i * D + m] = tp;
      b->tile_smem = std::max(b->tile_smem, tile_grouped_smem(tp, src));
      // the grouped kernel runs one line per thread, whatever the plan's own split
      b->tile_threads = std::max(b->tile_threads, tp.TS * tp.P);
    }
  }
  b->tile_threads = (b->tile_threads + 31) / 32 * 32;
  b->tile_grid = b->sms;
  if (b->tile_threads > 0) b->tile_grid *= std::max(1, tile_grouped_ctas_per_sm(b->tile_threads, b->tile_smem));
}

// Sizes of the batch's tables from its problems, and the device tables and host staging.
void batch_layout(ps_batch* b) {
  const int P = (int)b->probs.size();
  b->count = P;
  b->maxS = b->maxN = 0;
  b->var = P > 0 ? b->probs[0]->op->a.p != nullptr : true;
  b->delta32 = P > 0 && b->probs[0]->delta32;
  b->dims = P > 0 ? b->probs[0]->g.dim : 2;
  b->span_max = 0;
  for (ps_problem* p : b->probs) {
    const int nx = p->g.n[0], m = ((nx + 31) / 32 + 1) & ~1;
    b->span_max = std::max(b->span_max, nx + nx / m + 2);
  }
  for (ps_problem* p : b->probs) {
    b->maxS = std::max(b->maxS, p->fs);
    b->maxN = std::max(b->maxN, p->N);
  }
  batch_tile_plans(b);
  if (b->iter_graph) {
    cudaGraphExecDestroy(b->iter_graph);
    b->iter_graph = nullptr;
  }
  if (b->init_graph) {
    cudaGraphExecDestroy(b->init_graph);
    b->init_graph = nullptr;
  }
  const size_t Pz = (size_t)std::max(P, 1);
  b->tile_jobs.alloc((size_t)b->dims * Pz * tile_job_bytes());
  b->tile_segs.alloc((size_t)b->dims * Pz);
  b->tile_nseg.alloc((size_t)b->dims * std::max(b->maxS, 1));
  b->pack_jobs.alloc(Pz);
  b->unpack_jobs.alloc(Pz);
  b->pack_segs.alloc(Pz);
  b->unpack_segs.alloc(Pz);
  b->copy_jobs.alloc(Pz);
  b->copy_segs.alloc(Pz);
  b->cjobs.alloc((size_t)std::max(b->maxN, 1) * Pz);
  if (b->delta32) b->xjobs32.alloc((size_t)std::max(b->maxN, 1) * Pz);
  else b->xjobs32.reset();
  b->xsegs.alloc((size_t)std::max(b->maxN, 1) * Pz);
  b->ysegs.alloc((size_t)std::max(b->maxN, 1) * Pz);
  b->zsegs.alloc((size_t)std::max(b->maxN, 1) * Pz);
  b->nseg_misc.alloc((size_t)3 + b->maxN);
  b->inc.alloc(Pz);
  b->flag.alloc(Pz);
  b->tmo.alloc(1);
  PS_CUDA(cudaMemset(b->tmo.p, 0, sizeof(int)));
  b->h_tile_jobs.assign((size_t)b->dims * P * tile_job_bytes(), 0);
  b->h_tile_segs.assign((size_t)b->dims * P, WorkSeg{});
  b->h_tile_nseg.assign((size_t)b->dims * b->maxS, 0);
  b->h_pack.assign(P, PackJob{});
  b->h_unpack.assign(P, PackJob{});
  b->h_pack_segs.assign(P, WorkSeg{});
  b->h_unpack_segs.assign(P, WorkSeg{});
  b->h_copy.assign(P, CoarseJob{});
  b->h_copy_segs.assign(P, WorkSeg{});
  b->h_cjobs.assign((size_t)b->maxN * P, CoarseJob{});
  b->h_xjobs32.assign(b->delta32 ? (size_t)b->maxN * P : 0, XWarpJob{});
  b->h_xsegs.assign((size_t)b->maxN * P, WorkSeg{});
  b->h_ysegs.assign((size_t)b->maxN * P, WorkSeg{});
  b->h_zsegs.assign((size_t)b->maxN * P, WorkSeg{});
  b->h_nseg_misc.assign((size_t)3 + b->maxN, 0);
  b->h_inc.assign(P, 0);
  b->h_flag.assign(P, 0);
}

}  // namespace

extern "C" {

const char* ps_batch_last_error(void) { return g_batch_error.c_str(); }

int ps_batch_create(ps_problem* const* problems, int count, uintptr_t stream, ps_batch** out) {
  return bguarded([&] {
    PS_REQUIRE(out && count >= 0 && (problems || count == 0), "bad argument");
    auto b = std::make_unique<ps_batch>();
    int dev = 0;
    PS_CUDA(cudaGetDevice(&dev));
    PS_CUDA(cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev));
    PS_CUDA(cudaStreamCreateWithFlags(&b->cs, cudaStreamNonBlocking));
    PS_CUDA(cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming));
    PS_CUDA(cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming));
    for (int i = 0; i < count; ++i) {
      batch_check(b.get(), problems[i]);
      b->probs.push_back(problems[i]);
    }
    batch_layout(b.get());
    PS_CUDA(cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream)));
    for (ps_problem* p : b->probs) ++p->batched;
    b->registered = true;
    *out = b.release();
  });
}

int ps_batch_add(ps_batch* b, ps_problem* p, uintptr_t stream) {
  return bguarded([&] {
    PS_REQUIRE(b && p, "null argument");
    batch_check(b, p);
    b->probs.push_back(p);
    try {
      batch_layout(b);
    } catch (...) {
      b->probs.pop_back();
      batch_layout(b);
      throw;
    }
    ++p->batched;
    PS_CUDA(cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream)));
  });
}

int ps_batch_get_state(const ps_batch* b, int index, int slice, double* out_dev, uintptr_t stream) {
  return bguarded([&] {
    PS_REQUIRE(b && out_dev, "null argument");
    PS_REQUIRE(index >= 0 && index < b->count, "problem index out of range");
    const ps_problem* p = b->probs[index];
    PS_REQUIRE(slice >= 0 && slice <= p->N, "slice out of range");
    const long long nt = p->g.nt;
    PS_CUDA(cudaMemcpyAsync(out_dev, p->U.p + slice * nt, sizeof(double) * nt, cudaMemcpyDeviceToDevice,
                            reinterpret_cast<cudaStream_t>(stream)));
  });
}

int ps_batch_destroy(ps_batch* b) {
  delete b;
  return PS_OK;
}

int ps_batch_run(ps_batch* b, const double* const* u0_devs, double tol, int max_iter, uintptr_t stream,
                 int* iters_out) {
  return bguarded([&] {
    TraceRange whole("ps.batch");
    PS_REQUIRE(b && u0_devs, "null argument");
    PS_REQUIRE(b->count > 0, "the batch holds no problem");
    cudaStream_t ust = reinterpret_cast<cudaStream_t>(stream);
    cudaStream_t st = b->cs;
    const int P = b->count;
    // (re)capture the graphs: tile shapes may have changed (autotuner)
    if (b->iter_graph) {
      cudaGraphExecDestroy(b->iter_graph);
      b->iter_graph = nullptr;
    }
    if (b->init_graph) {
      cudaGraphExecDestroy(b->init_graph);
      b->init_graph = nullptr;
    }
    batch_tile_plans(b);
    b->init_graph = capture(b, 2);
    b->iter_graph = capture(b, 1);
    PS_CUDA(cudaEventRecord(b->ev_in, ust));
    PS_CUDA(cudaStreamWaitEvent(st, b->ev_in, 0));
    PS_CUDA(cudaMemsetAsync(b->flag.p, 0, sizeof(int) * P, st));
    PS_CUDA(cudaMemsetAsync(b->tmo.p, 0, sizeof(int), st));
    b->updates = 0;
    b->launches = 0;
    std::vector<int> active(P);
    std::iota(active.begin(), active.end(), 0);
    for (int i = 0; i < P; ++i) {
      ps_problem* p = b->probs[i];
      PS_REQUIRE(u0_devs[i], "null u0");
      PS_CUDA(cudaMemcpyAsync(p->U.p, u0_devs[i], sizeof(double) * p->g.nt, cudaMemcpyDeviceToDevice, st));
      p->hist.clear();
      p->iters = 0;
      b->updates += (double)p->N * p->g.nt;
    }
    // k = 0: coarse sweep of every problem
    fill_coarse_tables(b, active, 0);
    upload_tables(b, st);
    PS_CUDA(cudaGraphLaunch(b->init_graph, st));
    b->launches += b->launches_init;
    int k = 0;
    const int cap = max_iter <= 0 ? (1 << 30) : max_iter;
    while (!active.empty()) {
      ++k;
      fill_iteration_tables(b, active, k);
      upload_tables(b, st);
      PS_CUDA(cudaMemsetAsync(b->inc.p, 0, sizeof(unsigned long long) * P, st));
      PS_CUDA(cudaGraphLaunch(b->iter_graph, st));
      b->launches += b->launches_per_iter;
      PS_CUDA(cudaMemcpyAsync(b->h_inc.data(), b->inc.p, sizeof(unsigned long long) * P, cudaMemcpyDeviceToHost, st));
      PS_CUDA(cudaMemcpyAsync(b->h_flag.data(), b->flag.p, sizeof(int) * P, cudaMemcpyDeviceToHost, st));
      int tmo = 0;
      PS_CUDA(cudaMemcpyAsync(&tmo, b->tmo.p, sizeof(int), cudaMemcpyDeviceToHost, st));
      PS_CUDA(cudaStreamSynchronize(st));
      if (tmo) throw Error(PS_ERR_DEVICE_TIMEOUT, "a TMA tile load did not arrive within its wait limit");
      std::vector<int> next;
      for (int i : active) {
        ps_problem* p = b->probs[i];
        double inc;
        std::memcpy(&inc, &b->h_inc[i], sizeof inc);
        p->hist.push_back(inc);
        p->iters = k;
        b->updates += (double)(p->N - k + 1) * p->fs * p->g.nt + (double)(p->N - k) * p->g.nt;
        if (b->h_flag[i]) throw Error(PS_ERR_NONFINITE, "non-finite value in batch problem " + std::to_string(i));
        const bool done = inc < tol || k >= p->N || k >= cap;
        if (done) p->have_forward = true;
        else next.push_back(i);
      }
      active.swap(next);
    }
    if (iters_out)
      for (int i = 0; i < P; ++i) iters_out[i] = b->probs[i]->iters;
    PS_CUDA(cudaEventRecord(b->ev_out, st));
    PS_CUDA(cudaStreamWaitEvent(ust, b->ev_out, 0));
  });
}

int ps_batch_stats(const ps_batch* b, ps_stats* out) {
  return bguarded([&] {
    PS_REQUIRE(b && out, "null argument");
    std::memset(out, 0, sizeof *out);
    int kmax = 0;
    for (ps_problem* p : b->probs) kmax = std::max(kmax, p->iters);
    out->iterations = kmax;
    out->unknown_updates = b->updates;
    out->kernel_launches = b->launches;
  });
}

}  // extern "C"
