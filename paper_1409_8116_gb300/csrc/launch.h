// Host-side launchers of the sweep kernels (defined in sweep_kernels.cu).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include "internal.h"

namespace pf {
namespace fast {
struct FastStridedArgs;
struct FastXArgs;
}  // namespace fast
}  // namespace pf

namespace pf {

template <typename T>
cudaError_t launch_x_sweep(const XArgs& a, unsigned grid, size_t smem, cudaStream_t s);

template <typename T>
cudaError_t launch_strided_sweep(const CUtensorMap& map, const StridedArgs& a, unsigned grid, size_t smem,
                                 cudaStream_t s);

template <typename T>
cudaError_t launch_pair_divide(const PairDivideArgs& a, cudaStream_t s);

// Specialised FP32 two-pass kernels (fast_f32.cu) for line lengths M in
// {64, 128, 256, 512, 1024}: radices R1 x R2 and the tile width W.
bool fast_shape(int M, int* R1, int* R2, int* W);
cudaError_t launch_fast_strided(int M, int W, int mode, int kind, const CUtensorMap& map,
                                const fast::FastStridedArgs& a, unsigned grid, size_t smem, cudaStream_t s);
cudaError_t launch_fast_x(int M, int mode, int kx, const fast::FastXArgs& a, unsigned grid, size_t smem,
                          cudaStream_t s);

}  // namespace pf
