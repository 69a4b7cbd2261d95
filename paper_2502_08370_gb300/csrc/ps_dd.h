// ps_dd.h -- internal declarations of the domain-decomposition splitting (ps_dd.cu).
#pragma once

#include <vector>

#include "ps_internal.h"

namespace ps {

// One box of a colour: nodes [x0, x0+wx) x [y0, y0+wy) (1-based interior indices), ordered
// with the shorter extent fastest; lead = that extent = the half-bandwidth of its block.
struct DDBox {
  int bx, by;         // box indices; colour = (bx % 2) + (Bx > 1 ? 2 : 1) * (by % 2)
  int x0, y0;         // first node
  int xfast;          // 1: x fastest (lead = wx), 0: y fastest (lead = wy)
  int lead;           // half-bandwidth
  int n;              // nodes in the box
  int pad;
  long long offset;   // of the box's factors in DDFactors::fac (per line: S^{-1}, F, C; see ps_dd.cu)
};

struct DDGeomArgs {
  int nx, ny, Bx, By;
  const double* a;    // nodal coefficient (diagonal of D) or null (1)
  const double* d12;  // nodal off-diagonal of D, or null: full = 0
  double c, tau, overlap;
  int full;           // 1: cell-based nine-point operator of the full tensor (d12 given)
};

struct DDPlan {
  int M = 0;
  int max_lead = 0;
  int full = 0;       // full-tensor operator (line couplings C_k tridiagonal)
  long long fac_len = 0;
  std::vector<std::vector<DDBox>> colours;
  std::vector<double> nodes, fac_entries;  // per colour: box nodes, factor doubles
};

struct DDFactors {
  DDPlan plan;
  double tau = 0.0;
  DevBuf<double> fac;
  DevBuf<int> status;
  std::vector<DevBuf<DDBox>> dev_boxes;  // per colour
  DevBuf<DDBox> dev_all;                 // every box (factorisation launch)
  DDFactors() = default;
  DDFactors(const DDFactors&) = delete;
};

// full: plan for the full-tensor operator (its factors hold three coupling vectors per line).
void dd_plan(const Geom& g, const ps_dd_params& dd, bool full, DDPlan& plan);
// d12_nodal: off-diagonal diffusion on the nodal grid (boundary included), or null for D = a I.
void dd_factor(const Geom& g, const ps_dd_params& dd, const double* a_nodal, const double* d12_nodal, double c,
               double tau, DDFactors& f, cudaStream_t st);
// Colour `colour`'s substep on nslices consecutive states, in place.  err: device flag set to
// 1 when a bounded wait for a streamed factor chunk ran out (the launch is then abandoned);
// a launch does nothing while the flag is set.
void dd_solve(const Geom& g, int nslices, const DDFactors& f, int colour, double* state, int slices_per_block,
              int* err, cudaStream_t st);
void dd_rhs(const Geom& g, int nslices, const double* in, double* out, const SourceArgs& sa, cudaStream_t st);
void dd_correct(const Geom& g, const double* gstate, const CorrArgs& ca, cudaStream_t st);

}  // namespace ps
