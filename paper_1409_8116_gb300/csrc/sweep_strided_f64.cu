// Strided (TMA-staged) sweep kernel instantiation (double).
#include "launch.h"
#include "sweep_kernels.cuh"

namespace pf {
template cudaError_t launch_strided_sweep<double>(const CUtensorMap&, const StridedArgs&, unsigned, size_t, cudaStream_t);
template cudaError_t launch_pair_divide<double>(const PairDivideArgs&, cudaStream_t);
template cudaError_t launch_batch_phase<double>(int, const BatchItem*, const int*, int, int, int*, int, unsigned,
                                                size_t, cudaStream_t, int*);
}  // namespace pf
