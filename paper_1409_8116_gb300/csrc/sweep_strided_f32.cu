// Strided (TMA-staged) sweep kernel instantiation (float).
#include "launch.h"
#include "sweep_kernels.cuh"

namespace pf {
template cudaError_t launch_strided_sweep<float>(const CUtensorMap&, const StridedArgs&, unsigned, size_t, cudaStream_t);
template cudaError_t launch_pair_divide<float>(const PairDivideArgs&, cudaStream_t);
template cudaError_t launch_batch_phase<float>(int, const BatchItem*, const int*, int, int, int*, int, unsigned,
                                                size_t, cudaStream_t, int*);
}  // namespace pf
