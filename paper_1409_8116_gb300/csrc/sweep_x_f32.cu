// x-sweep kernel instantiation (float).
#include "launch.h"
#include "sweep_kernels.cuh"

namespace pf {
template cudaError_t launch_x_sweep<float>(const XArgs&, unsigned, size_t, cudaStream_t);
}  // namespace pf
