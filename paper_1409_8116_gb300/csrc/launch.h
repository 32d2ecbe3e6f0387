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
namespace tc {
struct TcStridedArgs;
}  // namespace tc
}  // namespace pf

namespace pf {

template <typename T>
cudaError_t launch_x_sweep(const XArgs& a, unsigned grid, size_t smem, cudaStream_t s);

template <typename T>
cudaError_t launch_strided_sweep(const CUtensorMap& map, const StridedArgs& a, unsigned grid, size_t smem,
                                 cudaStream_t s);

template <typename T>
cudaError_t launch_pair_divide(const PairDivideArgs& a, cudaStream_t s);

// Persistent batch phase (sweep_kernels.cuh); occ != nullptr: no launch,
// *occ = resident CTAs per SM for `smem`.
template <typename T>
cudaError_t launch_batch_phase(int kind, const BatchItem* items, const int* first, int nitems, int total,
                               int* counter, int bar_off, unsigned grid, size_t smem, cudaStream_t s, int* occ);

// Specialised FP32 two-pass kernels (fast_f32.cu) for line lengths M in
// {64, 128, 256, 512, 1024}: radices R1 x R2 and the tile width W.
bool fast_shape(int M, int* R1, int* R2, int* W);
cudaError_t launch_fast_strided(int M, int W, int mode, int kind, const CUtensorMap& map,
                                const fast::FastStridedArgs& a, unsigned grid, size_t smem, cudaStream_t s);
cudaError_t launch_fast_x(int M, int mode, int kx, const fast::FastXArgs& a, unsigned grid, size_t smem,
                          cudaStream_t s);

// Tensor-core sweeps of 1024-point strided axes (tc_f32.cu): mode and kind
// as for launch_fast_strided (FM_FWD / FM_INV with FK_DFT; FM_FUSED with
// FK_DFT or FK_DCT); persistent grid, fixed block and shared memory.
cudaError_t launch_tc_strided(int mode, int kind, const CUtensorMap& map, const tc::TcStridedArgs& a, unsigned grid,
                              cudaStream_t s);
size_t tc_smem_bytes();
// The four B operands F_hi, F_lo, G_hi, G_lo of the tensor-core sweeps as
// bf16 bit patterns in their shared-memory layout (tc_f32.cu, host only).
void tc_build_bmat(uint16_t* out);

}  // namespace pf
