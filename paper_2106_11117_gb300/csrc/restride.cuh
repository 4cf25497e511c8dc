// Narrowing the row stride of a ragged batch.
//
// Every per-node and per-edge array of a batch is sample-major [row][S].
// When the draws still stepping in a ragged batch are the prefix [0, S_act)
// with S_act far below S, each row still spans S draws and a DRAM sector of
// it carries a fraction of useful values (a 2-draw row of a 64-draw stride
// uses 8 of 32 bytes).  The loop then copies the arrays it still needs to a
// smaller stride S' >= S_act and steps on; the QoI of the draws that finish
// later is read with the new stride.
#pragma once
#include "kernels.cuh"

namespace lflts {

// dst[r][s] = src[r][s] for s < S_new (rows of stride S_old -> S_new).
template <typename Real>
__global__ void k_restride(const Real* __restrict__ src, Real* __restrict__ dst, int64_t n_rows, int S_old,
                           int S_new) {
  const int64_t n = n_rows * S_new;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = k / S_new;
    const int s = static_cast<int>(k - r * S_new);
    dst[k] = src[r * S_old + s];
  }
}

// QoI stage 1 (k_qoi_partial's arithmetic and order) on a state of row
// stride S_u, the partials kept at the batch's stride S_ps.
template <typename Real>
__global__ void k_qoi_partial_rs(const Real* __restrict__ u, int S_u, const int* __restrict__ idx,
                                 const double* __restrict__ gw, int nnz, int chunk, double* __restrict__ ps,
                                 double* __restrict__ pc, int S_ps, int s_lo, int s_hi) {
  const int s = s_lo + blockIdx.y * blockDim.x + threadIdx.x;
  if (s >= s_hi) return;
  const int c = blockIdx.x;
  const int k0 = c * chunk, k1 = min(nnz, k0 + chunk);
  Neumaier acc;
  for (int k = k0; k < k1; ++k) acc.add(__dmul_rn(gw[k], (double)u[(size_t)idx[k] * S_u + s]));
  ps[(size_t)c * S_ps + s] = acc.s;
  pc[(size_t)c * S_ps + s] = acc.c;
}

}  // namespace lflts
