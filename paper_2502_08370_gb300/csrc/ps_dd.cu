// ps_dd.cu -- domain-decomposition splitting (Sec. 2.1): partition of unity over
// overlapping boxes, banded subdomain factorisation and batched subdomain solves.
//
// Colour j's suboperator is L_j u = div(rho_j a grad u) - rho_j c u (Sec. 2.1).  With
// rho_j evaluated at edge midpoints, (I - tau A_j) is the identity outside the boxes of
// colour j and block diagonal over its boxes (Sec. 2.2: "q independent subsystems, one
// for each connected component").  Every box block is SPD and banded (half-bandwidth =
// the box's lead extent in its local ordering); it is factored once per step size as
// L L^T and the substeps solve  L y = b,  L^T x = y  for all time slices of a launch.
//
// Both triangular solves run column by column: when the pivot row's value p_j is final,
// the w rows below it receive  acc_r -= (L_{rj} / L_jj) p_j.  One warp owns one
// (box, slice) system; its 32 lanes share the w updates of each column and the running
// sums of the w+1 rows in flight live in a shared-memory ring.  The factors are stored
// pre-divided by the pivot (column-major for L, row-major for L^T), so no multiply sits
// on the critical path between two pivots.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

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

// Node (1-based interior indices) of box-local row r.
__device__ __forceinline__ long long box_node(const DDBox& bx, int nx, int r) {
  int slow = r / bx.lead, fast = r - slow * bx.lead;
  int gx, gy;
  if (bx.xfast) {
    gx = bx.x0 + fast;
    gy = bx.y0 + slow;
  } else {
    gx = bx.x0 + slow;
    gy = bx.y0 + fast;
  }
  return (long long)(gy - 1) * nx + (gx - 1);
}

// Assembled band row r of (I - tau A_j) restricted to the box, entries (r, r - d),
// d = 0..w: diagonal, and the couplings to the previous node in the lead direction
// (d = 1) and in the other direction (d = w).
struct RowEntries {
  double diag, lead, other;
};
__device__ RowEntries assemble_row(const DDBox& bx, const DDGeomArgs& ga, int r) {
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
  return e;
}

// Band row r: entry d = 0 is the diagonal, d = 1 the previous node in the lead direction,
// d = w the previous node in the other direction (both at d = 1 when w = 1).
__device__ __forceinline__ void store_row(double* row, const RowEntries& e, int w) {
  row[0] = e.diag;
  if (w >= 1) {
    row[1] = e.lead;
    row[w] += e.other;
  }
}

// ---------------------------------------------------------------------------------------
// a1 (DD): banded Cholesky of one box per CTA, right-looking, with the w+1 rows in flight
// in a shared-memory ring win[slot][d] = A(r, r - d), slot = r mod (w+1).  Writes
//   Lc[j*(w+1) + 0] = 1/L_jj,  Lc[j*(w+1) + d] = L_{j+d, j} / L_jj   (column j of L)
//   Lr[i*(w+1) + 0] = 1/L_ii,  Lr[i*(w+1) + d] = L_{i, i-d} / L_ii   (row i of L)
// Sets *status = 1 if a pivot is not positive (the matrix is SPD, so only on bad input).
__global__ void dd_factor_kernel(const DDBox* __restrict__ boxes, DDGeomArgs ga, double* __restrict__ fac,
                                 int* status) {
  const DDBox bx = boxes[blockIdx.x];
  const int w = bx.lead, W = w + 1, n = bx.n;
  extern __shared__ double win[];  // W*W ring + W column values
  double* col = win + (size_t)W * W;
  double* Lc = fac + bx.offset;
  double* Lr = Lc + (size_t)n * W;
  const int tid = threadIdx.x + threadIdx.y * blockDim.x, nthr = blockDim.x * blockDim.y;
  // load rows 0..min(w, n-1)
  for (int e = tid; e < W * W; e += nthr) win[e] = 0.0;
  __syncthreads();
  for (int r = tid; r < min(W, n); r += nthr) store_row(win + (size_t)(r % W) * W, assemble_row(bx, ga, r), w);
  __syncthreads();
  __shared__ double s_rinv;
  for (int k = 0; k < n; ++k) {
    double* rowk = win + (size_t)(k % W) * W;
    if (tid == 0) {
      const double piv = rowk[0];
      if (!(piv > 0.0)) atomicExch(status, 1);
      const double lkk = sqrt(piv > 0.0 ? piv : 1.0);
      s_rinv = 1.0 / lkk;
      rowk[0] = lkk;
    }
    __syncthreads();
    const double rinv = s_rinv;
    const int tmax = min(w, n - 1 - k);
    // column k: L_{k+t, k} = A(k+t, k) / L_kk
    for (int t = 1 + tid; t <= tmax; t += nthr) {
      double* rowi = win + (size_t)((k + t) % W) * W;
      const double lik = rowi[t] * rinv;
      rowi[t] = lik;
      col[t] = lik;
      Lc[(size_t)k * W + t] = lik * rinv;
    }
    if (tid == 0) Lc[(size_t)k * W] = rinv;
    for (int t = tmax + 1 + tid; t <= w; t += nthr) Lc[(size_t)k * W + t] = 0.0;
    __syncthreads();
    // trailing update of the rows in flight: A(i, j) -= L_ik L_jk, k < j <= i <= k + w
    for (int ti = 1 + threadIdx.y; ti <= tmax; ti += blockDim.y) {
      double* rowi = win + (size_t)((k + ti) % W) * W;
      const double lik = col[ti];
      for (int tj = 1 + threadIdx.x; tj <= ti; tj += blockDim.x) rowi[ti - tj] -= lik * col[tj];
    }
    __syncthreads();
    // row k is final: L_{k, k-d} for d = 1..w, and the pivot
    for (int d = tid; d <= w; d += nthr) {
      if (d == 0) Lr[(size_t)k * W] = rinv;
      else Lr[(size_t)k * W + d] = (k - d >= 0) ? rowk[d] * rinv : 0.0;
    }
    __syncthreads();
    // the slot of row k takes row k + W
    const int rn = k + W;
    if (rn < n) {
      for (int d = tid; d <= w; d += nthr) rowk[d] = 0.0;
      __syncthreads();
      if (tid == 0) store_row(rowk, assemble_row(bx, ga, rn), w);
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------------------
// a3 (DD): one warp solves one (box, slice) system in place in the state array:
// forward L y = b with the column-major factor, then backward L^T x = y with the
// row-major one.  The right-hand sides and factor columns are fetched kPre rows ahead.
constexpr int kRing = 256;  // running-sum ring, a power of two > w
constexpr int kPre = 4;     // prefetch distance in rows
constexpr int kPerLane = 8; // factor entries per lane per row: w + 1 <= 32 * kPerLane

template <bool BACKWARD>
__device__ __forceinline__ void dd_triangular(const DDBox& bx, int nx, const double* __restrict__ F,
                                              double* __restrict__ x, double* ring, int lane) {
  const int w = bx.lead, W = w + 1, n = bx.n;
  for (int e = lane; e < kRing; e += 32) ring[e] = 0.0;
  __syncwarp();
  double cf[kPre][kPerLane];
  double rhs[kPre];
#pragma unroll
  for (int u = 0; u < kPre; ++u) {
    const int j = BACKWARD ? n - 1 - u : u;
    const bool ok = BACKWARD ? j >= 0 : j < n;
    rhs[u] = ok ? x[box_node(bx, nx, j)] : 0.0;
#pragma unroll
    for (int t = 0; t < kPerLane; ++t) {
      const int d = lane + 32 * t;
      cf[u][t] = (ok && d <= w) ? F[(size_t)j * W + d] : 0.0;
    }
  }
  for (int j0 = 0; j0 < n; j0 += kPre) {
#pragma unroll
    for (int u = 0; u < kPre; ++u) {
      const int step = j0 + u;
      if (step < n) {
        const int j = BACKWARD ? n - 1 - step : step;
        const int slot = j & (kRing - 1);
        const double p = ring[slot] + rhs[u];  // final value of row j
        __syncwarp();
        if (lane == 0) {
          ring[slot] = 0.0;
          x[box_node(bx, nx, j)] = p * cf[u][0];
        }
#pragma unroll
        for (int t = 0; t < kPerLane; ++t) {
          const int d = lane + 32 * t;
          if (d >= 1 && d <= w) {
            const int r = BACKWARD ? j - d : j + d;
            if (BACKWARD ? r >= 0 : r < n) ring[r & (kRing - 1)] -= cf[u][t] * p;
          }
        }
        // prefetch row j -/+ kPre
        const int sn = step + kPre;
        const int jn = BACKWARD ? n - 1 - sn : sn;
        const bool ok = sn < n;
        rhs[u] = ok ? x[box_node(bx, nx, jn)] : 0.0;
#pragma unroll
        for (int t = 0; t < kPerLane; ++t) {
          const int d = lane + 32 * t;
          cf[u][t] = (ok && d <= w) ? F[(size_t)jn * W + d] : 0.0;
        }
        __syncwarp();
      }
    }
  }
  __syncwarp();
}

__global__ void dd_solve_kernel(const DDBox* __restrict__ boxes, int nx, long long nt, const double* __restrict__ fac,
                                double* state, int nslices, int slices_per_block) {
  __shared__ double rings[8][kRing];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const DDBox bx = boxes[blockIdx.x];
  const int sl = blockIdx.y * slices_per_block + warp;
  if (warp >= slices_per_block || sl >= nslices) return;
  double* x = state + (long long)sl * nt;
  const double* Lc = fac + bx.offset;
  const double* Lr = Lc + (size_t)bx.n * (bx.lead + 1);
  dd_triangular<false>(bx, nx, Lc, x, rings[warp], lane);
  dd_triangular<true>(bx, nx, Lr, x, rings[warp], lane);
}

// out = in + tau * src * src_t (all nodes, nslices states); out may alias in.
__global__ void dd_rhs_kernel(const double* in, double* out, long long total, long long nt, SourceArgs sa) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    double v = in[i];
    if (sa.src) {
      const long long sl = i / nt;
      const double ft = sa.src_t ? sa.src_t[sa.t0 + sl * sa.tstride] : 1.0;
      v = v + sa.tau * sa.src[i - sl * nt] * ft;
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

void dd_plan(const Geom& g, const ps_dd_params& dd, DDPlan& plan) {
  PS_REQUIRE(g.dim == 2, "DD splitting is 2-D");
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
      PS_REQUIRE(b.lead + 1 <= 32 * 8, "DD box too wide (lead extent must be < 256)");
      b.offset = off;
      off += 2LL * b.n * (b.lead + 1);
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
      plan.fac_entries[c] += 2.0 * b.n * (b.lead + 1);
    }
}

void dd_factor(const Geom& g, const ps_dd_params& dd, const double* a_nodal, double c, double tau, DDFactors& f,
               cudaStream_t st) {
  dd_plan(g, dd, f.plan);
  f.tau = tau;
  f.fac.alloc((size_t)f.plan.fac_len);
  f.status.alloc(1);
  PS_CUDA(cudaMemsetAsync(f.status.p, 0, sizeof(int), st));
  f.dev_boxes.resize(f.plan.M);
  DDGeomArgs ga;
  ga.nx = g.n[0];
  ga.ny = g.n[1];
  ga.a = a_nodal;
  ga.c = c;
  ga.tau = tau;
  ga.Bx = dd.boxes[0];
  ga.By = dd.boxes[1];
  ga.overlap = dd.overlap;
  const int W = f.plan.max_lead + 1;
  const size_t smem = ((size_t)W * W + W) * sizeof(double);
  int dev = 0, maxsm = 0;
  PS_CUDA(cudaGetDevice(&dev));
  PS_CUDA(cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  // the kernel also holds one static double
  if ((int)smem + 64 > maxsm) throw Error(PS_ERR_UNSUPPORTED, "DD box too wide for the shared-memory factorisation");
  PS_CUDA(cudaFuncSetAttribute(dd_factor_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  for (int c = 0; c < f.plan.M; ++c) {
    auto& boxes = f.plan.colours[c];
    f.dev_boxes[c].alloc(boxes.size());
    if (boxes.empty()) continue;
    PS_CUDA(cudaMemcpyAsync(f.dev_boxes[c].p, boxes.data(), sizeof(DDBox) * boxes.size(), cudaMemcpyHostToDevice,
                            st));
    dd_factor_kernel<<<(unsigned)boxes.size(), dim3(32, 16), smem, st>>>(f.dev_boxes[c].p, ga, f.fac.p,
                                                                          f.status.p);
    PS_CUDA(cudaGetLastError());
  }
  int h = 0;
  PS_CUDA(cudaMemcpyAsync(&h, f.status.p, sizeof(int), cudaMemcpyDeviceToHost, st));
  PS_CUDA(cudaStreamSynchronize(st));
  if (h) throw Error(PS_ERR_INVALID, "DD factorisation met a non-positive pivot (is a > 0?)");
}

void dd_solve(const Geom& g, int nslices, const DDFactors& f, int colour, double* state, int slices_per_block,
              cudaStream_t st) {
  const auto& boxes = f.plan.colours[colour];
  if (boxes.empty()) return;
  slices_per_block = std::max(1, std::min(8, slices_per_block));
  dim3 grid((unsigned)boxes.size(), (unsigned)((nslices + slices_per_block - 1) / slices_per_block));
  dd_solve_kernel<<<grid, 32 * slices_per_block, 0, st>>>(f.dev_boxes[colour].p, g.n[0], g.nt, f.fac.p, state,
                                                         nslices, slices_per_block);
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
