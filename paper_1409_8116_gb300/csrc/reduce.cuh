// Deterministic grid-wide reductions shared by the iterative solvers.
#pragma once

#include <cuda_runtime.h>

namespace pf {

constexpr int kReduceBlock = 256;  // threads per block of every kernel that reduces

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Deterministic grid-wide sums of K values per thread.  Each block writes its
// K partial sums to part[k * gridDim.x + block]; the last block to finish
// (counted with one atomic) adds the partials in a fixed order and stores the
// totals to dst[k], then resets the counter.  The result does not depend on
// the order in which blocks run, so repeated solves are bitwise identical.
struct Reduce {
  double* part;     // K * gridDim.x doubles
  unsigned* count;  // zero between kernels
};

template <int K>
__device__ __forceinline__ void grid_sum(const double (&v)[K], Reduce R, double* const (&dst)[K]) {
  __shared__ double sh[K][kReduceBlock / 32];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < K; k++) {
    const double w = warp_sum(v[k]);
    if (lane == 0) sh[k][warp] = w;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < K; k++) {
      double t = 0.0;
      for (int w = 0; w < kReduceBlock / 32; w++) t += sh[k][w];
      R.part[(size_t)k * gridDim.x + blockIdx.x] = t;
    }
    __threadfence();
    last = atomicAdd(R.count, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
#pragma unroll
  for (int k = 0; k < K; k++) {
    double t = 0.0;
    for (unsigned b = threadIdx.x; b < gridDim.x; b += kReduceBlock) t += __ldcg(&R.part[(size_t)k * gridDim.x + b]);
    t = warp_sum(t);
    __syncthreads();
    if (lane == 0) sh[k][warp] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
      double u = 0.0;
      for (int w = 0; w < kReduceBlock / 32; w++) u += sh[k][w];
      *dst[k] = u;
    }
  }
  if (threadIdx.x == 0) *R.count = 0u;
}

}  // namespace pf
