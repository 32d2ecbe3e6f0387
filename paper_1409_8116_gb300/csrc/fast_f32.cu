// Instantiations and dispatch of the specialised two-pass FP32 kernels.
#include "fast_kernels.cuh"
#include "launch.h"

namespace pf {

namespace {

template <int R1, int R2, int W, int MODE, int KIND>
cudaError_t run_strided(const CUtensorMap& map, const fast::FastStridedArgs& a, unsigned grid, size_t smem,
                        cudaStream_t s) {
  void (*k)(const CUtensorMap, const fast::FastStridedArgs);
  if constexpr (MODE == fast::FM_FUSED)
    k = fast::fast_fused_kernel<R1, R2, W, KIND>;
  else
    k = fast::fast_strided_kernel<R1, R2, W, MODE, KIND>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
  if (e != cudaSuccess) return e;
  k<<<grid, W * fast::Shape<R1, R2>::RMAX, smem, s>>>(map, a);
  return cudaGetLastError();
}

template <int R1, int R2, int W>
cudaError_t run_strided_mk(int mode, int kind, const CUtensorMap& map, const fast::FastStridedArgs& a, unsigned grid,
                           size_t smem, cudaStream_t s) {
  using namespace fast;
  if (kind == FK_DFT) {
    if (mode == FM_FWD) return run_strided<R1, R2, W, FM_FWD, FK_DFT>(map, a, grid, smem, s);
    if (mode == FM_INV) return run_strided<R1, R2, W, FM_INV, FK_DFT>(map, a, grid, smem, s);
    return run_strided<R1, R2, W, FM_FUSED, FK_DFT>(map, a, grid, smem, s);
  }
  if (mode == FM_FWD) return run_strided<R1, R2, W, FM_FWD, FK_DCT>(map, a, grid, smem, s);
  if (mode == FM_INV) return run_strided<R1, R2, W, FM_INV, FK_DCT>(map, a, grid, smem, s);
  if (kind == FK_DCT_PAIR) return run_strided<R1, R2, W, FM_FUSED, FK_DCT_PAIR>(map, a, grid, smem, s);
  return run_strided<R1, R2, W, FM_FUSED, FK_DCT>(map, a, grid, smem, s);
}

template <int R1, int R2, int MODE, int KX>
cudaError_t run_x(const fast::FastXArgs& a, unsigned grid, size_t smem, cudaStream_t s) {
  auto k = fast::fast_x_kernel<R1, R2, MODE, KX>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
  if (e != cudaSuccess) return e;
  k<<<grid, 256, smem, s>>>(a);
  return cudaGetLastError();
}

template <int R1, int R2>
cudaError_t run_x_m(int mode, int kx, const fast::FastXArgs& a, unsigned grid, size_t smem, cudaStream_t s) {
  using namespace fast;
  if (kx == FX_DCT)
    return mode == FM_FWD ? run_x<R1, R2, FM_FWD, FX_DCT>(a, grid, smem, s) : run_x<R1, R2, FM_INV, FX_DCT>(a, grid, smem, s);
  return mode == FM_FWD ? run_x<R1, R2, FM_FWD, FX_R2C>(a, grid, smem, s) : run_x<R1, R2, FM_INV, FX_R2C>(a, grid, smem, s);
}

}  // namespace

// Tile widths measured on GB300 (W = 4 and 16 were slower for these sizes).
bool fast_shape(int M, int* R1, int* R2, int* W) {
  switch (M) {
    case 64: *R1 = 8; *R2 = 8; *W = 32; return true;
    case 128: *R1 = 16; *R2 = 8; *W = 16; return true;
    case 256: *R1 = 16; *R2 = 16; *W = 8; return true;
    case 512: *R1 = 32; *R2 = 16; *W = 8; return true;
    case 1024: *R1 = 32; *R2 = 32; *W = 8; return true;
    default: return false;
  }
}

cudaError_t launch_fast_strided(int M, int W, int mode, int kind, const CUtensorMap& map,
                                const fast::FastStridedArgs& a, unsigned grid, size_t smem, cudaStream_t s) {
  switch (M * 64 + W) {
    case 64 * 64 + 32: return run_strided_mk<8, 8, 32>(mode, kind, map, a, grid, smem, s);
    case 128 * 64 + 16: return run_strided_mk<16, 8, 16>(mode, kind, map, a, grid, smem, s);
    case 256 * 64 + 8: return run_strided_mk<16, 16, 8>(mode, kind, map, a, grid, smem, s);
    case 512 * 64 + 8: return run_strided_mk<32, 16, 8>(mode, kind, map, a, grid, smem, s);
    case 1024 * 64 + 8: return run_strided_mk<32, 32, 8>(mode, kind, map, a, grid, smem, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_fast_x(int M, int mode, int kx, const fast::FastXArgs& a, unsigned grid, size_t smem,
                          cudaStream_t s) {
  switch (M) {
    case 64: return run_x_m<8, 8>(mode, kx, a, grid, smem, s);
    case 128: return run_x_m<16, 8>(mode, kx, a, grid, smem, s);
    case 256: return run_x_m<16, 16>(mode, kx, a, grid, smem, s);
    case 512: return run_x_m<32, 16>(mode, kx, a, grid, smem, s);
    case 1024: return run_x_m<32, 32>(mode, kx, a, grid, smem, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace pf
