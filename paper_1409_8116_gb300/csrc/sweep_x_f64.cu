// x-sweep kernel instantiation (double).
#include "launch.h"
#include "sweep_kernels.cuh"

namespace pf {
template cudaError_t launch_x_sweep<double>(const XArgs&, unsigned, size_t, cudaStream_t);
}  // namespace pf
