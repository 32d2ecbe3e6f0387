// Tensor-core (tcgen05) strided sweeps for 1024-point axes: the radix-32
// DFT blocks of the two-pass factorisation 1024 = 32 x 32 run as GEMMs on
// the 5th-generation tensor cores, in BF16 with FP32 accumulation.
//
// Factorisation (n = j + 32 q, k = s + 32 k2, w = exp(-2 pi i / 1024),
// w32 = w^32):
//   X[s + 32 k2] = sum_j w32^(j k2) [ w^(j s) sum_q x[j + 32 q] w32^(q s) ]
// pass 1: D1[(j,c), s]  = sum_q  x[j + 32 q; c] F[s, q]       (F = w32^(q s))
// twiddle by w^(j s)
// pass 2: D2[(s,c), k2] = sum_j  D1'[(j,c), s] F[k2, j]
// and the inverse (G = conj F, output n = a + 32 b):
// pass 3: D3[(s,c), a]  = sum_k2 V[s + 32 k2; c] G[a, k2]
// twiddle by conj(w^(a s))
// pass 4: D4[(a,c), b]  = sum_s  D3'[(s,c), a] G[b, s]
// Each pass is one GEMM of M = 256 rows (8 columns c x 32 butterflies) by
// N = 64 (32 complex outputs, real and imaginary parts interleaved) by
// K = 64 (32 complex inputs, interleaved): the complex product is written
// in real form, B[2s][2q] = Re F, B[2s][2q+1] = -Im F, B[2s+1][2q] = Im F,
// B[2s+1][2q+1] = Re F.
//
// Precision: every operand v is split into v_hi = bf16(v) and
// v_lo = bf16(v - v_hi) (16 significant bits together); a pass accumulates
// X_hi F_hi + X_lo F_hi + X_hi F_lo in FP32 (one GEMM with K = 192), which
// drops only the X_lo F_lo term.  The relative error of a pass is about
// 2^-17, against 2^-24 for the FP32 butterflies.
//
// Operands live in shared memory in the canonical K-major layout without
// swizzle (8-row x 16-byte core matrices, K-adjacent core matrices 128 B
// apart, 8-row groups 1024 B apart); the accumulator lives in tensor memory
// (lanes = rows, columns = N), one M = 128 half per 64 columns, and is read
// back with tcgen05.ld so that thread t holds row t.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "fast_kernels.cuh"
#include "fft_engine.cuh"

namespace pf {
namespace tc {

constexpr int kM = 1024;          // line length (32 x 32)
constexpr int kW = 8;             // columns per tile
constexpr int kParts = 1;         // threads per GEMM row (2 measured slower: 4.17 against 3.93 ms)
constexpr int kPer = 32 / kParts;
constexpr int kThreadsTc = 256 * kParts;
constexpr uint32_t kTileBytes = kM * kW * 8;          // FP32 complex tile = bf16 hi | lo operand
constexpr uint32_t kHalf = kTileBytes / 2;            // lo part offset
constexpr uint32_t kBmatBytes = 4 * 64 * 64 * 2;      // F_hi, F_lo, G_hi, G_lo
constexpr uint32_t kTwStride = 33;                    // padded twiddle rows (complex)
constexpr uint32_t kTwBytes = 32 * kTwStride * 8;
constexpr uint32_t kSmemBytes = kTileBytes + kBmatBytes + kTwBytes + 64;
constexpr uint32_t kTmemCols = 128;                   // two M = 128 halves x N = 64

struct TcStridedArgs {
  fast::FastStridedArgs f;  // tables, eigenvalues, layout (the FP32 kernel's)
  const uint4* bmat;        // F_hi | F_lo | G_hi | G_lo, canonical K-major (kBmatBytes)
  int ntiles;               // ntile_c * number of outer rows
  int* counter;             // next tile to take (zero before the launch)
};

// ---------------------------------------------------------------------------
// PTX wrappers (tcgen05, shared-memory descriptors)
// ---------------------------------------------------------------------------
// Shared-memory matrix descriptor: start address, leading-dimension byte
// offset (K direction), stride byte offset (M/N direction), descriptor
// version 1, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((addr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}
// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t instr_desc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void umma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
               "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
               "l"(a), "l"(b), "r"(idesc), "r"(acc)
               : "memory");
}
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tmem_alloc(uint32_t* holder, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(holder)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
// 16 consecutive accumulator columns of this thread's lane
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
#pragma unroll
  for (int i = 0; i < 16; i++) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// This thread's part of its row's accumulator: complex outputs
// [kPer * part, kPer * part + kPer) of row 128 h + 32 (warp % 4) + lane.
__device__ __forceinline__ void tmem_row(uint32_t tmem, int h, int part, float2* y) {
  const int warp = threadIdx.x >> 5;
  const uint32_t t = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + 64u * (uint32_t)h + 2u * kPer * (uint32_t)part;
  float* f = reinterpret_cast<float*>(y);
#pragma unroll
  for (int i = 0; i < 2 * kPer; i += 16) tmem_ld16(t + i, f + i);
  tmem_wait_ld();
}

// ---------------------------------------------------------------------------
// BF16 hi/lo split and operand stores
// ---------------------------------------------------------------------------
// (re, im) -> bf16x2 hi = rn(v), lo = rn(v - hi); re in the low half (the
// even K index).
__device__ __forceinline__ void split2(float2 v, uint32_t& hi, uint32_t& lo) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(v.x, v.y);
  const uint32_t hb = *reinterpret_cast<const uint32_t*>(&h);
  const float hx = __uint_as_float(hb << 16), hy = __uint_as_float(hb & 0xffff0000u);
  const __nv_bfloat162 l = __floats2bfloat162_rn(v.x - hx, v.y - hy);
  hi = hb;
  lo = *reinterpret_cast<const uint32_t*>(&l);
}
// Operand row r, K = 2i + {re, im} for i = kPer * part + (0..kPer-1), from
// v[0..kPer-1]: 16-byte stores of four complex values (consecutive rows of
// a warp fill whole 128-byte core matrices).
__device__ __forceinline__ void store_row(unsigned char* T, int r, int part, const float2* v) {
  unsigned char* base = T + (r >> 3) * 1024 + (r & 7) * 16 + part * (kPer / 4) * 128;
#pragma unroll
  for (int g = 0; g < kPer / 4; g++) {
    uint4 h, l;
    split2(v[4 * g + 0], h.x, l.x);
    split2(v[4 * g + 1], h.y, l.y);
    split2(v[4 * g + 2], h.z, l.z);
    split2(v[4 * g + 3], h.w, l.w);
    *reinterpret_cast<uint4*>(base + g * 128) = h;
    *reinterpret_cast<uint4*>(base + kHalf + g * 128) = l;
  }
}
// Transposed store: this thread's v[i] (index I = kPer * part + i) goes to
// operand row (I, c) at K index 2m + {re, im}, i.e. element (row I*8 + c,
// K = 2m).  A warp's 32 threads (m in 4 consecutive values, c = 0..7) fill
// one 128-byte core-matrix row block per I without bank conflicts.
__device__ __forceinline__ void store_transposed(unsigned char* T, int m, int c, int part, const float2* v) {
  unsigned char* base = T + (m >> 2) * 128 + c * 16 + (m & 3) * 4 + part * kPer * 1024;
#pragma unroll
  for (int i = 0; i < kPer; i++) {
    uint32_t h, l;
    split2(v[i], h, l);
    *reinterpret_cast<uint32_t*>(base + i * 1024) = h;
    *reinterpret_cast<uint32_t*>(base + kHalf + i * 1024) = l;
  }
}

// One GEMM pass (issued by one thread): two M = 128 halves, each
// K = 3 x 64 (hi.hi, lo.hi, hi.lo), accumulator columns [64 h, 64 h + 64).
__device__ __forceinline__ void issue_pass(uint32_t tmem, uint32_t aT, uint32_t bh, uint32_t bl, uint64_t* bar) {
  tc_fence_after();
  constexpr uint32_t idesc = instr_desc(128, 64);
#pragma unroll
  for (int h = 0; h < 2; h++) {
    const uint32_t d = tmem + 64u * h;
    const uint32_t ah = aT + h * 16384, al = ah + kHalf;
#pragma unroll
    for (int kc = 0; kc < 4; kc++)
      umma(d, smem_desc(ah + kc * 256, 128, 1024), smem_desc(bh + kc * 256, 128, 1024), idesc, kc > 0);
#pragma unroll
    for (int kc = 0; kc < 4; kc++)
      umma(d, smem_desc(al + kc * 256, 128, 1024), smem_desc(bh + kc * 256, 128, 1024), idesc, 1);
#pragma unroll
    for (int kc = 0; kc < 4; kc++)
      umma(d, smem_desc(ah + kc * 256, 128, 1024), smem_desc(bl + kc * 256, 128, 1024), idesc, 1);
  }
  umma_commit(bar);
}

// ---------------------------------------------------------------------------
// the sweep kernel (persistent: every CTA loops over tiles)
// ---------------------------------------------------------------------------
// MODE (fast::FastMode): FM_FWD forward transform along the axis (passes 1,
// 2), FM_INV backward (passes 3, 4), FM_FUSED forward, eigenvalue divide,
// zero mode and backward (passes 1-4).  KIND (fast::FastKind): FK_DFT, or
// FK_DCT for the fused sweep of a DCT-II / DST-II axis stored in Makhoul's
// order (the fused step pairs k with M - k, as in the FP32 kernel).
// Shared memory: the 64 KB tile (TMA destination, then the bf16 operand of
// every pass, then the FP32 exchange buffer of the DCT step), the four
// 8 KB B operands, the padded twiddle table and two mbarriers.  Two CTAs
// per SM; each holds 128 tensor-memory columns.  Every GEMM row is shared
// by kParts threads (the tensor-memory lane quarter of a warp is its index
// mod 4), which keeps the per-thread chain of dependent work short.
template <int MODE, int KIND>
__global__ void __launch_bounds__(kThreadsTc, 2)
    tc_strided_kernel(const __grid_constant__ CUtensorMap tmap, const TcStridedArgs A) {
  const fast::FastStridedArgs& a = A.f;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* T = smem_raw;
  float2* T2 = reinterpret_cast<float2*>(smem_raw);
  unsigned char* Bm = smem_raw + kTileBytes;
  float2* tws = reinterpret_cast<float2*>(Bm + kBmatBytes);
  uint64_t* bars = reinterpret_cast<uint64_t*>(Bm + kBmatBytes + kTwBytes);  // [0] TMA, [1] MMA
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(bars + 2);
  int* s_next = reinterpret_cast<int*>(bars + 3);  // the tile thread 0 took last

  const int tid = threadIdx.x, warp = tid >> 5;
  // GEMM row of this thread: 128 h + 32 (warp % 4) + lane (tensor-memory
  // lane quarters follow warp % 4); `part` selects its half of the row
  const int h = (warp >> 2) & 1, part = warp >> 3;
  const int row = 128 * h + 32 * (warp & 3) + (tid & 31);
  const int hi3 = row >> 3, c = row & 7;
  const int i0 = kPer * part;

  // ---- set-up: B operands, twiddles, barriers, tensor memory
  {
    uint4* dst = reinterpret_cast<uint4*>(Bm);
    for (int e = tid; e < (int)(kBmatBytes / 16); e += kThreadsTc) dst[e] = __ldg(&A.bmat[e]);
    for (int e = tid; e < kM; e += kThreadsTc) tws[(e >> 5) * kTwStride + (e & 31)] = __ldg(&a.tw[e]);
  }
  fence_proxy_async();
  if (tid == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    fence_mbar_init();
  }
  if (warp == 0) tmem_alloc(tmem_holder, kTmemCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_holder;
  const uint32_t aT = smem_u32(T);
  const uint32_t bF = smem_u32(Bm), bFl = bF + 8192, bG = bF + 16384, bGl = bF + 24576;

  uint32_t tma_phase = 0, mma_phase = 0;
  bool tma_pending = false, mma_pending = false, bad = false;

  auto issue_tma = [&](int tile) {
    const int tcol = tile % a.ntile_c, outer = tile / a.ntile_c;
    mbar_arrive_expect_tx(&bars[0], kTileBytes);
    for (int b = 0; b < a.nbox; b++) {
      float2* dst = T2 + (size_t)b * a.box_h * kW;
      if (a.axis_dim == 1)
        tma_load_3d(dst, &tmap, &bars[0], 2 * tcol * kW, b * a.box_h, outer);
      else
        tma_load_3d(dst, &tmap, &bars[0], 2 * tcol * kW, outer, b * a.box_h);
    }
  };
  // all threads: wait for the pending GEMM pass; uniform result
  auto wait_mma = [&]() -> bool {
    const bool ok = mbar_wait_bounded(&bars[1], mma_phase);
    mma_phase ^= 1;
    const bool any_bad = __syncthreads_or(!ok);
    if (!any_bad) mma_pending = false;
    tc_fence_after();
    return !any_bad;
  };
  // all threads: operand stores done -> one thread issues the pass
  auto run_pass = [&](uint32_t bh, uint32_t bl) {
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    if (tid == 0) issue_pass(tmem, aT, bh, bl, &bars[1]);
    mma_pending = true;
  };

  // Tiles are taken from a global counter in order, so the tiles in flight
  // stay contiguous in memory (statically strided persistent CTAs drift
  // apart and lose DRAM page locality).  Thread 0 takes the next tile and
  // starts its load as soon as the shared tile is free; the others read
  // its index after the end-of-tile barrier.  tma_pending is thread 0's.
  auto take_next = [&]() {
    const int nx = atomicAdd(A.counter, 1);
    *s_next = nx;
    tma_pending = nx < A.ntiles;
    if (tma_pending) issue_tma(nx);
  };
  if (tid == 0) take_next();
  __syncthreads();
  int tile = *s_next;
  while (tile < A.ntiles) {
    const bool ok = mbar_wait_bounded(&bars[0], tma_phase);
    tma_phase ^= 1;
    if (__syncthreads_or(!ok)) { bad = true; break; }
    tma_pending = false;
    const int tcol = tile % a.ntile_c, outer = tile / a.ntile_c;
    const int c0 = tcol * kW;
    const int col = c0 + c;
    const bool col_ok = col < a.ncols;
    float2* out = a.data + (size_t)outer * a.s_outer + c0 + c;
    float2 v[kPer];  // indices i0 + i of this thread's row

    if (MODE == fast::FM_FWD || MODE == fast::FM_FUSED) {
      // pass 1: row (j = hi3, c), K = q
#pragma unroll
      for (int i = 0; i < kPer; i++) v[i] = T2[(hi3 + 32 * (i0 + i)) * kW + c];
      __syncthreads();
      store_row(T, row, part, v);
      run_pass(bF, bFl);
      if (!wait_mma()) { bad = true; break; }
      // twiddle w^(j s), transpose to rows (s, c), K = j
      tmem_row(tmem, h, part, v);
#pragma unroll
      for (int i = 0; i < kPer; i++) v[i] = cmul<float>(v[i], tws[(i0 + i) * kTwStride + hi3]);
      store_transposed(T, hi3, c, part, v);
      run_pass(bF, bFl);
      if (!wait_mma()) { bad = true; break; }
      tmem_row(tmem, h, part, v);  // row (s = hi3, c): X[s + 32 k2] in v[k2 - i0]
      if (MODE == fast::FM_FWD) {
        if (tid == 0) take_next();
        if (col_ok) {
#pragma unroll
          for (int i = 0; i < kPer; i++) out[(size_t)(hi3 + 32 * (i0 + i)) * a.s_axis] = v[i];
        }
        tc_fence_before();
        __syncthreads();  // every row read before the next tile's pass 1 overwrites the accumulator
        tile = *s_next;
        continue;
      }
      // ---- eigenvalue divide (and the DCT-II / DCT-III pair step)
      const float lam_xo = (col_ok ? __ldg(&a.lam_in[col]) : 0.f) + __ldg(&a.lam_out[outer]);
      const bool zero_row = a.singular && col == 0 && outer == 0;
      const int s = hi3;
      if (KIND == fast::FK_DFT) {
#pragma unroll
        for (int i = 0; i < kPer; i++) {
          const int k = s + 32 * (i0 + i);
          float f = __fdividef(a.scale, lam_xo + __ldg(&a.lam_ax[k]));
          if (zero_row && k == 0) f = 0.f;
          v[i] = make_float2(v[i].x * f, v[i].y * f);
        }
      } else {
        // exchange through the tile: E[k2][row]
#pragma unroll
        for (int i = 0; i < kPer; i++) T2[(i0 + i) * 256 + row] = v[i];
        __syncthreads();
        const int sp = (32 - s) & 31;
#pragma unroll
        for (int i = 0; i < kPer; i++) {
          const int k2 = i0 + i;
          const int k = s + 32 * k2;
          const int k2p = s == 0 ? (32 - k2) & 31 : 31 - k2;
          const float2 yp = T2[k2p * 256 + sp * 8 + c];
          const float4 t = __ldg(&a.pk[k]);
          // DCT-II post-processing, divide and DCT-III pre-processing in one
          // step, as in the FP32 kernel: V_k = (f_k + f_{M-k}) Y_k +
          // (f_k - f_{M-k}) e^{i pi k/M} Y_{M-k}, t = (lam[k], lam[M-k],
          // cos(pi k/M), sin(pi k/M))
          float fk = __fdividef(a.scale, lam_xo + t.x);
          if (zero_row && k == 0) fk = 0.f;
          const float fm = k == 0 ? fk : __fdividef(a.scale, lam_xo + t.y);
          const float2 cyp = make_float2(t.z * yp.x - t.w * yp.y, t.z * yp.y + t.w * yp.x);
          const float al = fk + fm, be = fk - fm;
          v[i] = make_float2(al * v[i].x + be * cyp.x, al * v[i].y + be * cyp.y);
        }
        __syncthreads();  // partners read before the operand overwrites the tile
      }
      store_row(T, row, part, v);  // rows (s, c), K = k2
    } else {
      // backward only: V in natural order in the tile; row (s, c), K = k2
#pragma unroll
      for (int i = 0; i < kPer; i++) v[i] = T2[(hi3 + 32 * (i0 + i)) * kW + c];
      __syncthreads();
      store_row(T, row, part, v);
    }
    // pass 3: D3[(s,c), a] = sum_k2 V G[a, k2]
    run_pass(bG, bGl);
    if (!wait_mma()) { bad = true; break; }
    tmem_row(tmem, h, part, v);
#pragma unroll
    for (int i = 0; i < kPer; i++) v[i] = cmulc<float>(v[i], tws[hi3 * kTwStride + i0 + i]);
    store_transposed(T, hi3, c, part, v);  // rows (a, c), K = s
    run_pass(bG, bGl);
    if (!wait_mma()) { bad = true; break; }
    if (tid == 0) take_next();
    tmem_row(tmem, h, part, v);  // row (a = hi3, c): x[a + 32 b] in v[b - i0]
    if (col_ok) {
#pragma unroll
      for (int i = 0; i < kPer; i++) out[(size_t)(hi3 + 32 * (i0 + i)) * a.s_axis] = v[i];
    }
    tc_fence_before();
    __syncthreads();
    tile = *s_next;
  }

  // ---- clean-up: nothing of ours may be in flight when tensor memory is freed
  if (bad) {
    if (tid == 0) atomicExch(a.err, 1);
    // a wait flips its phase before it is checked: the pending one is the other
    if (tid == 0 && tma_pending) mbar_wait_bounded(&bars[0], tma_phase ^ 1);
    if (tid == 0 && mma_pending) mbar_wait_bounded(&bars[1], mma_phase ^ 1);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, kTmemCols);
}

}  // namespace tc
}  // namespace pf
