// ps_dr.cu -- the Douglas-Rachford fine step (Sec. 2.2, eq. DR_method) for Parareal/FIE-DR
// (Sec. 4.2), on the natural layout, for nsl consecutive states at once.
//
// The step as printed:
//     U_{n,0} = (I + tau A) U_n + tau f(t_{n+1}),          A = A_1 + ... + A_M,
//     (I - tau A_j) U_{n,j} = U_{n,j-1} - tau A_j U_n,      j = 1..M,     U_{n+1} = U_{n,M}.
// Subtracting (I - tau A_j) U_n from both sides of substep j shows that the increments
// W_j = U_{n,j} - U_n obey
//     W_0 = tau (A U_n + f(t_{n+1})),   (I - tau A_j) W_j = W_{j-1},   U_{n+1} = U_n + W_M,
// the same line solves as an FIE step (eq. FIE_method) applied to W_0.  The GPU takes this
// form: one stencil pass for W_0, the M line sweeps of ps_dim.cu in place on W, one add.
// The M separate products tau A_j U_n of the printed form are never formed.
#include <cuda_runtime.h>

#include <algorithm>

#include "ps_internal.h"

namespace ps {
namespace {

constexpr int kThreads = 256;

// w = tau (A u + f) for the nsl states of u.  A = sum_j A_j, A_j the 3-point flux form along
// direction j, [a_{i+1/2}(u_{i+1} - u_i) - a_{i-1/2}(u_i - u_{i-1})] / h_j^2 - (c/M) u_i, with
// a_{i+1/2} = (a_i + a_{i+1}) / 2 from the nodal coefficient (boundary nodes included; VAR
// false: a = 1) and u = 0 outside the interior.  k_j = tau / h_j^2, ctau = tau c.
// One warp per grid row (lanes along x, coalesced); the face weights of a node are formed
// once and reused for the slices blockIdx.y, blockIdx.y + gridDim.y, ...
template <int M, bool VAR, bool SRC>
__global__ void __launch_bounds__(kThreads) dr_increment_kernel(int nx, int ny, int nz, int nsl, long long nt,
                                                                const double* __restrict__ a, double k0, double k1,
                                                                double k2, double ctau,
                                                                const double* __restrict__ u, double* __restrict__ w,
                                                                SourceArgs sa) {
  const int lane = threadIdx.x & 31;
  const long long rows = (long long)ny * nz;
  const long long wpb = kThreads / 32;
  const long long nwarps = (long long)gridDim.x * wpb;
  const long long nx2 = nx + 2, ny2 = ny + 2;
  const long long st[3] = {1LL, (long long)nx, (long long)nx * ny};
  const long long sa_[3] = {1LL, nx2, nx2 * ny2};
  const double k[3] = {k0, k1, k2};
  for (long long row = (long long)blockIdx.x * wpb + (threadIdx.x >> 5); row < rows; row += nwarps) {
    const int y = (int)(row % ny);
    const int z = (int)(row / ny);
    for (int x = lane; x < nx; x += 32) {
      const long long node = row * nx + x;
      const int c[3] = {x, y, z};
      const int n[3] = {nx, ny, nz};
      double wm[M], wp[M];
      if (VAR) {
        const long long i0 = (M == 3 ? (long long)(z + 1) * ny2 + (y + 1) : (long long)(y + 1)) * nx2 + (x + 1);
        const double a0 = a[i0];
#pragma unroll
        for (int j = 0; j < M; ++j) {
          wm[j] = k[j] * (0.5 * (a0 + a[i0 - sa_[j]]));
          wp[j] = k[j] * (0.5 * (a0 + a[i0 + sa_[j]]));
        }
      } else {
#pragma unroll
        for (int j = 0; j < M; ++j) wm[j] = wp[j] = k[j];
      }
      const double sv = SRC ? sa.src[node] : 0.0;
      for (int sl = blockIdx.y; sl < nsl; sl += gridDim.y) {
        const long long e = (long long)sl * nt + node;
        const double uc = u[e];
        double acc = -ctau * uc;
#pragma unroll
        for (int j = 0; j < M; ++j) {
          const double um = c[j] > 0 ? u[e - st[j]] : 0.0;
          const double up = c[j] < n[j] - 1 ? u[e + st[j]] : 0.0;
          acc = fma(wp[j], up - uc, acc);
          acc = fma(-wm[j], uc - um, acc);
        }
        if (SRC) {
          const long long ti = sa.t0 + (long long)sl * sa.tstride;
          const double ft = sa.src_t ? sa.src_t[ti] : 1.0;
          acc = fma(sa.tau, sv * ft, acc);
          if (sa.src2) acc = fma(sa.tau, sa.src2[node] * (sa.src2_t ? sa.src2_t[ti] : 1.0), acc);
        }
        w[e] = acc;
      }
    }
  }
}

// w = tau (A u + f) for the full tensor D = [[a, d12], [d12, a]] (2-D, Sec. 5.2): A is the
// cell-based nine-point operator, the sum of the colour suboperators of the DD splitting
// (their weights rho_j add up to 1 at every cell centre).  Cell (ci, cj) (lower-left node)
// contributes through ax = a/(2hx^2), ay = a/(2hy^2), g = d12/(hx hy), with a and d12 the means
// of its four nodal values; -(A u)_P = sum over the four cells at P of their rows at P:
//     diagonal  ax + ay + g/2 (cells SW, NE of P),  ax + ay - g/2 (SE, NW),
//     W, E      -ax of the two cells sharing that edge;  S, N  -ay likewise,
//     SW, NE    -g/2 of the cell between;  SE, NW  +g/2 of the cell between,
// plus c u_P; u = 0 on the boundary.  One thread per node; the slices of blockIdx.y.
__global__ void __launch_bounds__(kThreads) dr_increment_tensor_kernel(int nx, int ny, int nsl, long long nt,
                                                                       const double* __restrict__ a,
                                                                       const double* __restrict__ d12, double hx,
                                                                       double hy, double ctau,
                                                                       const double* __restrict__ u,
                                                                       double* __restrict__ w, SourceArgs sa) {
  const long long node = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (node >= nt) return;
  const int i = (int)(node % nx) + 1, j = (int)(node / nx) + 1;  // 1-based interior node
  const long long nx2 = nx + 2;
  // nodal values around P (boundary included): f[dy][dx] at (i + dx - 1, j + dy - 1)
  double av[3][3], bv[3][3];
#pragma unroll
  for (int dy = 0; dy < 3; ++dy)
#pragma unroll
    for (int dx = 0; dx < 3; ++dx) {
      const long long k = (long long)(j + dy - 1) * nx2 + (i + dx - 1);
      av[dy][dx] = a ? a[k] : 1.0;
      bv[dy][dx] = d12[k];
    }
  // cells: c = 0 SW, 1 SE, 2 NW, 3 NE; lower-left corner offset (cx, cy) in {0,1}^2
  double ax[4], ay[4], g[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const int cx = c & 1, cy = c >> 1;
    const double am = 0.25 * (av[cy][cx] + av[cy][cx + 1] + av[cy + 1][cx] + av[cy + 1][cx + 1]);
    const double bm = 0.25 * (bv[cy][cx] + bv[cy][cx + 1] + bv[cy + 1][cx] + bv[cy + 1][cx + 1]);
    ax[c] = am / (2.0 * hx * hx);
    ay[c] = am / (2.0 * hy * hy);
    g[c] = bm / (hx * hy);
  }
  const double dgl = (ax[0] + ay[0] + 0.5 * g[0]) + (ax[1] + ay[1] - 0.5 * g[1]) + (ax[2] + ay[2] - 0.5 * g[2]) +
                     (ax[3] + ay[3] + 0.5 * g[3]);
  const double eW = -(ax[0] + ax[2]), eE = -(ax[1] + ax[3]), eS = -(ay[0] + ay[1]), eN = -(ay[2] + ay[3]);
  const double eSW = -0.5 * g[0], eNE = -0.5 * g[3], eSE = 0.5 * g[1], eNW = 0.5 * g[2];
  const bool hasW = i > 1, hasE = i < nx, hasS = j > 1, hasN = j < ny;
  for (int sl = blockIdx.y; sl < nsl; sl += gridDim.y) {
    const double* us = u + (long long)sl * nt;
    const double uc = us[node];
    // sum of the row's entries times u (the negative of A u without reaction)
    double r = dgl * uc;
    if (hasW) r = fma(eW, us[node - 1], r);
    if (hasE) r = fma(eE, us[node + 1], r);
    if (hasS) r = fma(eS, us[node - nx], r);
    if (hasN) r = fma(eN, us[node + nx], r);
    if (hasS && hasW) r = fma(eSW, us[node - nx - 1], r);
    if (hasN && hasE) r = fma(eNE, us[node + nx + 1], r);
    if (hasS && hasE) r = fma(eSE, us[node - nx + 1], r);
    if (hasN && hasW) r = fma(eNW, us[node + nx - 1], r);
    double acc = sa.tau * (-r) - ctau * uc;
    if (sa.src) {
      const long long ti = sa.t0 + (long long)sl * sa.tstride;
      acc = fma(sa.tau, sa.src[node] * (sa.src_t ? sa.src_t[ti] : 1.0), acc);
      if (sa.src2) acc = fma(sa.tau, sa.src2[node] * (sa.src2_t ? sa.src2_t[ti] : 1.0), acc);
    }
    w[(long long)sl * nt + node] = acc;
  }
}

// out = u + w (out may alias u)
__global__ void dr_add_kernel(const double* u, const double* __restrict__ w, double* out, long long total) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x)
    out[e] = u[e] + w[e];
}

// SM count of the current device, queried per launch (the attribute query is cheap and a
// cached value would be wrong for a problem that lives on another device).
int sm_count() {
  int dev = 0, sms = 0;
  PS_CUDA(cudaGetDevice(&dev));
  PS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  return sms;
}

}  // namespace

void dr_increment(const Geom& g, int nsl, const double* a_nodal, double c, double tau, const double* u, double* w,
                  const SourceArgs& sa, cudaStream_t st) {
  const int nx = g.n[0], ny = g.n[1], nz = g.dim == 3 ? g.n[2] : 1;
  const long long rows = (long long)ny * nz;
  const long long want = (rows + kThreads / 32 - 1) / (kThreads / 32);
  const int sms = sm_count();
  const unsigned bx = (unsigned)std::min<long long>(want, (long long)sms * 16);
  // spread the slices over blockIdx.y until about 8 blocks per SM are in flight
  const long long by_want = ((long long)sms * 8 + bx - 1) / bx;
  const unsigned by = (unsigned)std::max<long long>(1, std::min<long long>({by_want, (long long)nsl, 65535LL}));
  const double h[3] = {1.0 / (g.n[0] + 1), 1.0 / (g.n[1] + 1), 1.0 / (nz + 1)};
  const double k0 = tau / (h[0] * h[0]), k1 = tau / (h[1] * h[1]), k2 = tau / (h[2] * h[2]);
  const dim3 grid(bx, by);
  const bool var = a_nodal != nullptr, src = sa.src != nullptr;
#define PS_DR_LAUNCH(M_, V_, S_) \
  dr_increment_kernel<M_, V_, S_><<<grid, kThreads, 0, st>>>(nx, ny, nz, nsl, g.nt, a_nodal, k0, k1, k2, tau * c, u, w, sa)
  if (g.dim == 3) {
    if (var) { if (src) PS_DR_LAUNCH(3, true, true); else PS_DR_LAUNCH(3, true, false); }
    else { if (src) PS_DR_LAUNCH(3, false, true); else PS_DR_LAUNCH(3, false, false); }
  } else {
    if (var) { if (src) PS_DR_LAUNCH(2, true, true); else PS_DR_LAUNCH(2, true, false); }
    else { if (src) PS_DR_LAUNCH(2, false, true); else PS_DR_LAUNCH(2, false, false); }
  }
#undef PS_DR_LAUNCH
  PS_CUDA(cudaGetLastError());
}

void dr_increment_tensor(const Geom& g, int nsl, const double* a_nodal, const double* d12_nodal, double c, double tau,
                         const double* u, double* w, const SourceArgs& sa, cudaStream_t st) {
  PS_REQUIRE(g.dim == 2 && d12_nodal, "the full-tensor stencil is 2-D with a d12 field");
  const int sms = sm_count();
  const unsigned bx = (unsigned)((g.nt + kThreads - 1) / kThreads);
  const long long by_want = ((long long)sms * 8 + bx - 1) / bx;
  const unsigned by = (unsigned)std::max<long long>(1, std::min<long long>({by_want, (long long)nsl, 65535LL}));
  dr_increment_tensor_kernel<<<dim3(bx, by), kThreads, 0, st>>>(g.n[0], g.n[1], nsl, g.nt, a_nodal, d12_nodal,
                                                                1.0 / (g.n[0] + 1), 1.0 / (g.n[1] + 1), tau * c, u, w, sa);
  PS_CUDA(cudaGetLastError());
}

void dr_add(const Geom& g, int nsl, const double* u, const double* w, double* out, cudaStream_t st) {
  const long long total = (long long)nsl * g.nt;
  const unsigned grid = (unsigned)std::min<long long>((total + 255) / 256, (long long)sm_count() * 16);
  dr_add_kernel<<<grid, 256, 0, st>>>(u, w, out, total);
  PS_CUDA(cudaGetLastError());
}

}  // namespace ps
