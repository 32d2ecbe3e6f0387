// Instantiations and dispatch of the tensor-core strided sweeps, and the
// host construction of their DFT-matrix operands.
#include <math.h>
#include <string.h>

#include "launch.h"
#include "tc_kernels.cuh"

namespace pf {

namespace {

template <int MODE, int KIND>
cudaError_t run_tc(const CUtensorMap& map, const tc::TcStridedArgs& a, unsigned grid, cudaStream_t s) {
  auto k = tc::tc_strided_kernel<MODE, KIND>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc::kSmemBytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
  if (e != cudaSuccess) return e;
  k<<<grid, tc::kThreadsTc, tc::kSmemBytes, s>>>(map, a);
  return cudaGetLastError();
}

// round-to-nearest-even of a finite float to bfloat16 (bit pattern)
uint16_t bf16_bits(float f) {
  uint32_t u;
  memcpy(&u, &f, 4);
  u += 0x7FFFu + ((u >> 16) & 1u);
  return (uint16_t)(u >> 16);
}
float bf16_value(uint16_t b) {
  const uint32_t u = (uint32_t)b << 16;
  float f;
  memcpy(&f, &u, 4);
  return f;
}

}  // namespace

size_t tc_smem_bytes() { return tc::kSmemBytes; }

cudaError_t launch_tc_strided(int mode, int kind, const CUtensorMap& map, const tc::TcStridedArgs& a, unsigned grid,
                              cudaStream_t s) {
  using namespace fast;
  if (mode == FM_FWD && kind == FK_DFT) return run_tc<FM_FWD, FK_DFT>(map, a, grid, s);
  if (mode == FM_INV && kind == FK_DFT) return run_tc<FM_INV, FK_DFT>(map, a, grid, s);
  if (mode == FM_FUSED && kind == FK_DFT) return run_tc<FM_FUSED, FK_DFT>(map, a, grid, s);
  if (mode == FM_FUSED && kind == FK_DCT) return run_tc<FM_FUSED, FK_DCT>(map, a, grid, s);
  return cudaErrorInvalidValue;
}

// B operand of pass p: 64 x 64 real matrix of the 32-point DFT (sign -1,
// F) or its inverse (sign +1, G), rows n = 2 s + {re, im}, columns
// k = 2 q + {re, im}: [[Re, -Im], [Im, Re]] of exp(sign 2 pi i q s / 32),
// angles reduced exactly (q s mod 32).  hi = bf16(v), lo = bf16(v - hi).
// Layout: canonical K-major without swizzle, element (n, k) at
// (n/8) 1024 + (k/8) 128 + (n%8) 16 + (k%8) 2 bytes.
void tc_build_bmat(uint16_t* out) {
  for (int m = 0; m < 2; m++) {
    const double sign = m == 0 ? -1.0 : 1.0;
    uint16_t* hi = out + (size_t)m * 2 * 4096;
    uint16_t* lo = hi + 4096;
    for (int s = 0; s < 32; s++)
      for (int q = 0; q < 32; q++) {
        const double ang = 2.0 * M_PI * (double)((q * s) % 32) / 32.0;
        const double re = cos(ang), im = sign * sin(ang);
        const double v[2][2] = {{re, -im}, {im, re}};
        for (int a = 0; a < 2; a++)
          for (int b = 0; b < 2; b++) {
            const int n = 2 * s + a, k = 2 * q + b;
            const size_t idx = ((size_t)(n / 8) * 1024 + (size_t)(k / 8) * 128 + (size_t)(n % 8) * 16 + (size_t)(k % 8) * 2) / 2;
            const uint16_t h = bf16_bits((float)v[a][b]);
            hi[idx] = h;
            lo[idx] = bf16_bits((float)(v[a][b] - (double)bf16_value(h)));
          }
      }
  }
}

}  // namespace pf
