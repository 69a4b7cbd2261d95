// ps_dr.cu -- the Douglas-Rachford fine step (Sec. 2.2, eq. DR_method) for Parareal/FIE-DR
// (Sec. 4.2), on the natural layout, for nsl consecutive states at once:
//     U_{n,0} = (I + tau A) U_n + tau F_{n+1},          A = A_1 + ... + A_M,
//     (I - tau A_j) U_{n,j} = U_{n,j-1} - tau A_j U_n,   j = 1..M,
//     U_{n+1} = U_{n,M}.
// Dimensional splitting, FP64.  The substep solves are the line sweeps of ps_dim.cu; this
// file adds the operator products tau A_j U_n and the stage combinations.
#include <cuda_runtime.h>

#include <algorithm>

#include "ps_internal.h"

namespace ps {
namespace {

// out_j = tau A_j u for the nsl states of u (total = nsl * nt values), A_j the 3-point flux
// form along direction j: [a_{i+1/2}(u_{i+1} - u_i) - a_{i-1/2}(u_i - u_{i-1})] / h_j^2 - (c/M) u_i
// with a_{i+1/2} = (a_i + a_{i+1}) / 2 from the nodal coefficient (boundary nodes included;
// null: a = 1) and u = 0 outside the interior.
__global__ void apply_Aj_kernel(int dim, int nx, int ny, int nz, int j, const double* __restrict__ a, double c_over_M,
                                double tau, const double* __restrict__ u, double* __restrict__ out, long long nt,
                                long long total) {
  const int n[3] = {nx, ny, nz};
  const long long st = j == 0 ? 1LL : (j == 1 ? (long long)nx : (long long)nx * ny);
  const double h = 1.0 / (n[j] + 1);
  const double h2 = h * h;
  const long long nx2 = nx + 2, ny2 = ny + 2;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long r = e % nt;
    const int x = (int)(r % nx);
    const long long q = r / nx;
    const int y = (int)(q % ny);
    const int z = (int)(q / ny);
    const int c[3] = {x, y, z};
    const double uc = u[e];
    const double um = c[j] > 0 ? u[e - st] : 0.0;
    const double up = c[j] < n[j] - 1 ? u[e + st] : 0.0;
    double wm = 1.0, wp = 1.0;
    if (a) {
      // nodal index of interior node (x, y, z) in the (n+2)^d array: coordinates shifted by 1
      const long long zoff = dim == 3 ? (long long)(z + 1) * ny2 : 0;
      const long long i0 = (zoff + (y + 1)) * nx2 + (x + 1);
      const long long sa = j == 0 ? 1LL : (j == 1 ? nx2 : nx2 * ny2);
      const double a0 = a[i0];
      wm = 0.5 * (a0 + a[i0 - sa]);
      wp = 0.5 * (a0 + a[i0 + sa]);
    }
    out[e] = tau * ((wp * (up - uc) - wm * (uc - um)) / h2 - c_over_M * uc);
  }
}

// v = u + sum_j TA_j + tau f(t) for nsl states; TA_j at TA + j * total.  The source of slice
// sl of the launch is taken at time index sa.t0 + sl * sa.tstride.
__global__ void dr_stage0_kernel(const double* __restrict__ u, const double* __restrict__ TA, int M, long long total,
                                 long long nt, SourceArgs sa, double* v) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    double s = u[e];
    for (int j = 0; j < M; ++j) s += TA[(long long)j * total + e];
    if (sa.src) {
      const long long sl = e / nt;
      const double ft = sa.src_t ? sa.src_t[sa.t0 + sl * sa.tstride] : 1.0;
      s += sa.tau * sa.src[e - sl * nt] * ft;
    }
    v[e] = s;
  }
}

// v -= TA (the right-hand side U_{n,j-1} - tau A_j U_n of substep j)
__global__ void sub_kernel(double* v, const double* __restrict__ TA, long long total) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x)
    v[e] -= TA[e];
}

unsigned grid_for(long long total) { return (unsigned)std::min<long long>((total + 255) / 256, 152LL * 16); }

}  // namespace

void dr_apply_Aj(const Geom& g, int nsl, int j, const double* a_nodal, double c_over_M, double tau, const double* u,
                 double* out, cudaStream_t st) {
  const long long total = (long long)nsl * g.nt;
  apply_Aj_kernel<<<grid_for(total), 256, 0, st>>>(g.dim, g.n[0], g.n[1], g.dim == 3 ? g.n[2] : 1, j, a_nodal,
                                                    c_over_M, tau, u, out, g.nt, total);
  PS_CUDA(cudaGetLastError());
}

void dr_stage0(const Geom& g, int nsl, const double* u, const double* TA, int M, const SourceArgs& sa, double* v,
               cudaStream_t st) {
  const long long total = (long long)nsl * g.nt;
  dr_stage0_kernel<<<grid_for(total), 256, 0, st>>>(u, TA, M, total, g.nt, sa, v);
  PS_CUDA(cudaGetLastError());
}

void dr_subtract(const Geom& g, int nsl, double* v, const double* TA, cudaStream_t st) {
  const long long total = (long long)nsl * g.nt;
  sub_kernel<<<grid_for(total), 256, 0, st>>>(v, TA, total);
  PS_CUDA(cudaGetLastError());
}

}  // namespace ps
