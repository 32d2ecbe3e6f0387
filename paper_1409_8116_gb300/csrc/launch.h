// Host-side launchers of the sweep kernels (defined in sweep_kernels.cu).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include "internal.h"

namespace pf {

template <typename T>
cudaError_t launch_x_sweep(const XArgs& a, unsigned grid, size_t smem, cudaStream_t s);

template <typename T>
cudaError_t launch_strided_sweep(const CUtensorMap& map, const StridedArgs& a, unsigned grid, size_t smem,
                                 cudaStream_t s);

}  // namespace pf
