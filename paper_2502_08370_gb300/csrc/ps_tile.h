// ps_tile.h -- fine-propagator sweeps on the slice-interleaved layout (ps_tile.cu).
#pragma once

#include <cuda.h>

#include "ps_internal.h"

namespace ps {

// Tile shape and TMA tensor map of one sweep direction over W[z][y][x][S_pad].
struct TilePlan {
  CUtensorMap map;
  CUtensorMap map_grp;  // the same box with 128-byte L2 promotion: launches over part of the slots
  int axis = 0, L = 0, TS = 32, P = 1, chunks = 1, chunk = 0, threads = 0;
  int V = 1;         // adjacent slots (lines) per thread
  int pipe = 1;      // persistent double-buffered CTAs (1) or one tile per CTA (0)
  int ctas_per_sm = 1;
  size_t smem = 0;   // dynamic shared memory per CTA without the source staging
};

// positions: 1, 2 or 4 line positions per tile (0 = largest that fits); pipe: 1 persistent
// double-buffered, 0 one tile per CTA, -1 auto.
void tile_plan(const Geom& g, int S_pad, int elem, int axis, TilePlan& tp, void* W, int positions = 0, int pipe = -1,
               int slots = 0, int vec = 0);
// One substep along tp.axis on slots [s_first, s_first + nsl) (whole TS-slot groups are
// processed).  `err` is set when a tile's TMA load does not arrive within the wait limit.
// part_of_slots: the launch covers only some slot groups (the fine phase beside the chain):
// tiles use map_grp, whose L2 promotion fetches no neighbouring group's bytes.
template <typename T>
void tile_sweep(const Geom& g, const TilePlan& tp, const LineFactors& f, int S_pad, int s_first, int nsl,
                const SourceArgs& sa, const T* srcrow, int* err, cudaStream_t st, bool part_of_slots = false);
// Line-major, zero-padded copies of a direction's factors for the tile sweeps (f.lt*, f.rt*).
void factor_lines(const Geom& g, LineFactors& f, bool fp32, cudaStream_t st);
// Source rows along x, line-major [z*ny + y][Lp], in precision elem (4 or 8 bytes).
void source_rows(const Geom& g, const double* src, void* out, int elem, cudaStream_t st);
// Pack states U[0..nsl) into slots [s_first, s_first + nsl); rev = true takes them in reverse
// order (slot s_first + j <- U[nsl - 1 - j]).
template <typename T>
void to_interleaved(const Geom& g, const double* U, T* W, int S_pad, int s_first, int nsl, cudaStream_t st,
                    bool rev = false);
template <typename T>
void from_interleaved(const Geom& g, const T* W, double* U, int S_pad, int s_first, int nsl, cudaStream_t st);

// ---- grouped (batched) launches -------------------------------------------------------
// Pack job: slices [s_first, s_first + nsl) of one problem between U (FP64 slice-major,
// starting at slice s_first) and W (FP32 interleaved, S_pad slots).
struct PackJob {
  double* U;
  float* W;
  long long nt;
  int S_pad, s_first, nsl, pad;
};
// Fills one (problem, direction) job of a grouped FP32 tile launch (job_out must hold
// tile_job_bytes(), 64-byte aligned) and returns its tile count.
// sa/srcrow: the fine propagator's source (x tiles add it; sa.tstride = fine steps per slice),
// or sa.src == null.
long long tile_job_fill(const Geom& g, const TilePlan& tp, const LineFactors& f, int S_pad, int s_first, int nsl,
                        int* err, void* job_out, const SourceArgs& sa, const float* srcrow);
size_t tile_job_bytes();
size_t tile_grouped_smem(const TilePlan& tp, bool src);
// CTAs of the grouped tile kernel resident per SM at `threads` threads and `smem` bytes
int tile_grouped_ctas_per_sm(int threads, size_t smem);
// step: the fine step of the launch (the source's time index is step + 1 + slot * t_slice)
void tile_sweep_grouped(const void* jobs, const WorkSeg* segs, const int* nseg, int grid, int threads, size_t smem,
                        int* err, int step, cudaStream_t st);
void pack_grouped(bool to_interleaved_dir, const PackJob* jobs, const WorkSeg* segs, const int* nseg, int grid,
                  cudaStream_t st);

}  // namespace ps
