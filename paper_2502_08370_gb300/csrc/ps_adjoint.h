// ps_adjoint.h -- gradient kernels of the discrete adjoint (ps_adjoint.cu).
#pragma once

#include "ps_internal.h"

namespace ps {

// Edges of direction m: (n_m + 1) x prod_{d != m} n_d, boundary edges included.
long long edge_count(const Geom& g, int m);
// gedge[e] += -coef * sum_{slots < nsl} (lam_Q - lam_P)(w_Q - w_P) over the edges of direction m;
// lam and w are slice-interleaved states with S_pad slots.
void grad_edges(const Geom& g, int m, const double* lam, const double* w, int S_pad, int nsl, double coef,
                double* gedge, cudaStream_t st);
// grad_a (nodal, boundary included) = half the sum of the incident edges' values.
void combine_grad(const Geom& g, const double* const gedge[3], double* grad_a, cudaStream_t st);

}  // namespace ps
