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
          const double ft = sa.src_t ? sa.src_t[sa.t0 + (long long)sl * sa.tstride] : 1.0;
          acc = fma(sa.tau, sv * ft, acc);
        }
        w[e] = acc;
      }
    }
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

void dr_add(const Geom& g, int nsl, const double* u, const double* w, double* out, cudaStream_t st) {
  const long long total = (long long)nsl * g.nt;
  const unsigned grid = (unsigned)std::min<long long>((total + 255) / 256, (long long)sm_count() * 16);
  dr_add_kernel<<<grid, 256, 0, st>>>(u, w, out, total);
  PS_CUDA(cudaGetLastError());
}

}  // namespace ps
