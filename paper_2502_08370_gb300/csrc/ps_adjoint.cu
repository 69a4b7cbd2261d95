// ps_adjoint.cu -- kernels of the discrete adjoint (gradient w.r.t. the nodal coefficient).
//
// No counterpart in the paper: the gradient of a loss of U_N through every FIE step.  One
// substep solves w = (I - tau A_m)^{-1} v with A_m the flux form along direction m, whose
// edge coefficient is a_e = (a_P + a_Q) / 2 on the edge P -> Q = P + e_m.  With the
// adjoint nu = (I - tau A_m)^{-T} lambda (the matrix is symmetric), the substep adds
//     dJ/da_e += tau nu^T (dA_m / da_e) w = -tau (nu_Q - nu_P)(w_Q - w_P) / h_m^2,
// half to a_P and half to a_Q; boundary values of nu and w are zero.  All time slices are
// processed at once in the slice-interleaved layout, so one warp sums an edge's products
// over the slices with a fixed-order reduction (deterministic, no atomics).
#include <cuda_runtime.h>

#include <algorithm>

#include "ps_adjoint.h"

namespace ps {
namespace {

// Edge e of direction m (t = 0..n_m joins 0-based interior coordinates t-1 and t along m).
__device__ __forceinline__ void edge_coords(int m, long long e, int nx, int ny, int* i, int* j, int* k, int* t) {
  if (m == 0) {
    *t = (int)(e % (nx + 1));
    const long long r = e / (nx + 1);
    *j = (int)(r % ny);
    *k = (int)(r / ny);
    *i = 0;
  } else if (m == 1) {
    *i = (int)(e % nx);
    const long long r = e / nx;
    *t = (int)(r % (ny + 1));
    *k = (int)(r / (ny + 1));
    *j = 0;
  } else {
    *i = (int)(e % nx);
    const long long r = e / nx;
    *j = (int)(r % ny);
    *t = (int)(r / ny);
    *k = 0;
  }
}

__global__ void grad_edges_kernel(int m, int nx, int ny, int nz, const double* __restrict__ lam,
                                  const double* __restrict__ w, int S_pad, int nsl, double coef,
                                  double* __restrict__ gedge, long long nedges) {
  const long long e = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (e >= nedges) return;
  int i, j, k, t;
  edge_coords(m, e, nx, ny, &i, &j, &k, &t);
  const int nm = m == 0 ? nx : (m == 1 ? ny : nz);
  int cP[3] = {i, j, k}, cQ[3] = {i, j, k};
  cP[m] = t - 1;
  cQ[m] = t;
  const bool vP = t >= 1, vQ = t <= nm - 1;
  const long long posP = ((long long)cP[2] * ny + cP[1]) * nx + cP[0];
  const long long posQ = ((long long)cQ[2] * ny + cQ[1]) * nx + cQ[0];
  double sum = 0.0;
  for (int s = lane; s < nsl; s += 32) {
    const double nP = vP ? lam[posP * S_pad + s] : 0.0, nQ = vQ ? lam[posQ * S_pad + s] : 0.0;
    const double wP = vP ? w[posP * S_pad + s] : 0.0, wQ = vQ ? w[posQ * S_pad + s] : 0.0;
    sum += (nQ - nP) * (wQ - wP);
  }
  for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
  if (lane == 0) gedge[e] += -coef * sum;
}

// grad_a at every node of the (n+2)^d grid: half of each incident edge's accumulated value.
__global__ void combine_kernel(int dim, int nx, int ny, int nz, const double* __restrict__ g0,
                               const double* __restrict__ g1, const double* __restrict__ g2, double* __restrict__ ga,
                               long long nnodes) {
  const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= nnodes) return;
  const int I = (int)(id % (nx + 2));
  const long long r = id / (nx + 2);
  const int J = (int)(r % (ny + 2));
  const int K = dim == 3 ? (int)(r / (ny + 2)) : 1;
  const bool inI = I >= 1 && I <= nx, inJ = J >= 1 && J <= ny, inK = dim == 2 || (K >= 1 && K <= nz);
  double v = 0.0;
  // x-edges through node I: t = I - 1 (node is Q) and t = I (node is P), rows (J, K) interior
  if (inJ && inK) {
    const long long row = (long long)(K - 1) * ny + (J - 1);
    if (I >= 1) v += g0[row * (nx + 1) + (I - 1)];
    if (I <= nx) v += g0[row * (nx + 1) + I];
  }
  if (inI && inK) {
    const long long base = (long long)(K - 1) * (ny + 1);
    if (J >= 1) v += g1[(base + (J - 1)) * nx + (I - 1)];
    if (J <= ny) v += g1[(base + J) * nx + (I - 1)];
  }
  if (dim == 3 && inI && inJ) {
    if (K >= 1) v += g2[((long long)(K - 1) * ny + (J - 1)) * nx + (I - 1)];
    if (K <= nz) v += g2[((long long)K * ny + (J - 1)) * nx + (I - 1)];
  }
  ga[id] = 0.5 * v;
}

}  // namespace

long long edge_count(const Geom& g, int m) {
  long long c = 1;
  for (int d = 0; d < g.dim; ++d) c *= (d == m) ? (long long)g.n[d] + 1 : (long long)g.n[d];
  return c;
}

void grad_edges(const Geom& g, int m, const double* lam, const double* w, int S_pad, int nsl, double coef,
                double* gedge, cudaStream_t st) {
  const long long ne = edge_count(g, m);
  const int warps = 8;
  const long long blocks = (ne + warps - 1) / warps;
  grad_edges_kernel<<<(unsigned)blocks, 32 * warps, 0, st>>>(m, g.n[0], g.n[1], g.dim == 3 ? g.n[2] : 1, lam, w,
                                                             S_pad, nsl, coef, gedge, ne);
  PS_CUDA(cudaGetLastError());
}

void combine_grad(const Geom& g, const double* const gedge[3], double* grad_a, cudaStream_t st) {
  const long long nn = (long long)(g.n[0] + 2) * (g.n[1] + 2) * (g.dim == 3 ? g.n[2] + 2 : 1);
  combine_kernel<<<(unsigned)((nn + 255) / 256), 256, 0, st>>>(g.dim, g.n[0], g.n[1], g.dim == 3 ? g.n[2] : 1,
                                                              gedge[0], gedge[1], g.dim == 3 ? gedge[2] : gedge[1],
                                                              grad_a, nn);
  PS_CUDA(cudaGetLastError());
}

}  // namespace ps
