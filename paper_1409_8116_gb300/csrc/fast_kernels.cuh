// Specialised sweep kernels for two-pass power-of-two lines (FP32).
//
// Line length M = R1 * R2 with R1, R2 in {8, 16, 32} (M = 64 ... 1024).
// Forward transforms are decimation in frequency (DIF), backward transforms
// decimation in time (DIT), so no pass reorders data:
//   DIF pass 1 (radix R1): butterfly j < R2 takes points j + R2*q, DFT,
//     twiddle exp(-2 pi i j s / M) on output s, stores it at block s, row j.
//   DIF pass 2 (radix R2): butterfly b < R1 takes block b; its output s2 is
//     the DFT coefficient k = b + R1*s2 (digit-reversed arrangement).
//   DIT pass A (radix R2) consumes that arrangement block by block, DIT pass B
//     (radix R1, twiddle before the butterfly) returns natural order.
// After pass 1 the tile sits in a padded layout (min(W, 8) complex after
// every block of R2 rows) so that pass 2 reads whole blocks without bank
// conflicts.
//
// Axes with DCT-II / DCT-III (Neumann staggered) and DST-II / DST-III
// (Dirichlet staggered) use the even/odd reordering of Makhoul (1980): the
// x sweeps store grid plane j of such an axis at plane position
// j/2 (j even) or n-1-(j-1)/2 (j odd), times (-1)^j for DST-II, so the
// strided sweep sees the reordered sequence directly; the backward sweep
// leaves its result in that order and the x backward sweep reads it back.
// The spectrum of those axes is stored in DCT-II index order (for DST-II the
// eigenvalue table is reversed accordingly).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "fft_engine.cuh"
#include "internal.h"

namespace pf {
namespace fast {

// FK_DCT_PAIR: DCT axis whose complex columns pack two real x columns
// (x itself DCT-II / DST-II); only the fused sweep differs (per-part divide).
enum FastKind : int { FK_DFT = 0, FK_DCT = 1, FK_DCT_PAIR = 2 };
// x transform of the contiguous sweep: real-to-complex DFT (periodic x) or
// DCT-II / DST-II by the reordering of Makhoul (Neumann / Dirichlet
// staggered x).
enum FastXKind : int { FX_R2C = 0, FX_DCT = 1 };
enum FastMode : int { FM_FWD = 0, FM_INV = 1, FM_FUSED = 2 };

struct FastStridedArgs {
  const float2* tw;        // tw[s * R2 + j] = exp(-2 pi i j s / M), s < R1, j < R2
  const float2* mk;        // exp(-i pi k / (2M)), k < M (DCT axes)
  const float4* pk;        // fused DCT axes: (lam_ax[k], lam_ax[(M-k) mod M], cos(pi k/M), sin(pi k/M))
  const float* lam_in;     // x eigenvalues by column (FK_DCT_PAIR: by real x index, 2 per column)
  const float* lam_ax;     // swept-axis eigenvalues in storage order
  const float* lam_out;    // outer-axis eigenvalues in storage order
  float scale;
  int singular;
  int ncols;               // valid complex columns
  int ntile_c;
  int box_h, nbox;
  int axis_dim;            // 1: y, 2: z (tensor-map dimension of the swept axis)
  long long s_axis, s_outer;
  float2* data;
  int* err;
};

struct FastXArgs {
  const float2* tw;        // as above for the x line
  const float2* mk;        // FX_DCT: exp(-i pi k / (2M)), k < M
  int xsign;               // FX_DCT: 1 for DST-II / DST-III (Dirichlet staggered x)
  int nx;                  // = M
  int lines;               // line pairs per CTA
  long long nrows;         // ny * nz
  int ny, nz;
  int perm_y, perm_z;      // 1: plane reordering along that axis (DCT/DST axes)
  int sign_y, sign_z;      // 1: (-1)^j sign along that axis (DST axes)
  long long ws_ld;         // workspace row stride (complex)
  const float* g;
  float* phi;
  float2* ws;
  long long g_sy, g_sz;    // element strides of g between y rows and z planes
  long long phi_sy, phi_sz;
  int stage_g;             // forward, M = 1024: rows of g are 16-byte aligned and staged by bulk copies
  int stage_phi;           // backward, M = 1024: rows of phi are 16-byte aligned and written by bulk copies
  int* err;                // bounded-wait timeout flag
};

// position of grid plane j in the even/odd reordering of an axis of length n
__device__ __forceinline__ int makhoul_pos(int j, int n) { return (j & 1) ? n - 1 - (j >> 1) : (j >> 1); }

template <int R1, int R2>
struct Shape {
  static constexpr int M = R1 * R2;
  static constexpr int RMAX = R1 > R2 ? R1 : R2;
};

// ---------------------------------------------------------------------------
// strided sweep
// ---------------------------------------------------------------------------
// Tile: W columns x M rows.  Thread t: column c = t % W, butterfly index
// t / W.  Smem: TMA layout row*W + c, then padded layout
// block*(R2*W + pad) + row*W + c.
// Forward (FM_FWD) or backward (FM_INV) transform of the swept axis, three
// CTAs per SM (768 threads); the fused sweep is fast_fused_kernel.
// Padding after every block of R2 rows in the padded layout (complex):
// shifts consecutive blocks across the smem banks for narrow tiles.
template <int W> struct BlockPad { static constexpr int value = W < 8 ? W : 8; };

// Write the tile staged in shared memory in the TMA box layout (row * W +
// column) back with tensor stores, one per box; called by every thread of
// the CTA (the fence and barrier make the staged values visible to the copy
// engine), thread 0 issues the stores and waits until they have read the
// tile.
template <int W>
__device__ __forceinline__ void store_tile(const CUtensorMap& tmap, const FastStridedArgs& a, const float2* sm,
                                           int c0, int outer) {
  fence_proxy_async();
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int b = 0; b < a.nbox; b++) {
      const float2* src = sm + (size_t)b * a.box_h * W;
      if (a.axis_dim == 1)
        tma_store_3d(&tmap, src, 2 * c0, b * a.box_h, outer);
      else
        tma_store_3d(&tmap, src, 2 * c0, outer, b * a.box_h);
    }
    bulk_commit_group();
    bulk_wait_group_read0();
  }
}

template <int R1, int R2, int W, int MODE, int KIND>
__global__ void __launch_bounds__(W * Shape<R1, R2>::RMAX, 768 / (W * Shape<R1, R2>::RMAX))
    fast_strided_kernel(const __grid_constant__ CUtensorMap tmap, const FastStridedArgs a) {
  constexpr int M = R1 * R2;
  static_assert(MODE == FM_FWD || MODE == FM_INV, "fused sweeps run fast_fused_kernel");
  constexpr bool DCT = KIND != FK_DFT;
  constexpr int BS = R2 * W + BlockPad<W>::value;  // padded block stride (complex)
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  float2* sm = reinterpret_cast<float2*>(smem_raw);
  constexpr int TILE_C = (R1 * BS > M * W) ? R1 * BS : M * W;
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw + ((TILE_C * 8 + 15) / 16) * 16);

  const int tid = threadIdx.x;
  const int c = tid % W;
  const int bi = tid / W;  // butterfly index within the column
  const int tcol = blockIdx.x % a.ntile_c;
  const int outer = blockIdx.x / a.ntile_c;
  const int c0 = tcol * W;

  if (tid == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (tid == 0) {
    const uint32_t box_bytes = (uint32_t)(2 * W * a.box_h * sizeof(float));
    mbar_arrive_expect_tx(bar, box_bytes * a.nbox);
    for (int b = 0; b < a.nbox; b++) {
      float2* dst = sm + (size_t)b * a.box_h * W;
      if (a.axis_dim == 1)
        tma_load_3d(dst, &tmap, bar, 2 * c0, b * a.box_h, outer);
      else
        tma_load_3d(dst, &tmap, bar, 2 * c0, outer, b * a.box_h);
    }
  }
  const bool ok = mbar_wait_bounded(bar, 0);
  if (__syncthreads_or(!ok)) {
    if (tid == 0) atomicExch(a.err, 1);
    return;
  }

  float2* out = a.data + (size_t)outer * a.s_outer + c0;
  const bool col_ok = c0 + c < a.ncols;

  if (MODE == FM_FWD) {
    // ---- DIF pass 1 from the TMA layout
    float2 u[R1];
    const bool act1 = bi < R2;
    const int j = bi;
    if (act1) {
#pragma unroll
      for (int q = 0; q < R1; q++) u[q] = sm[(j + R2 * q) * W + c];
    }
    __syncthreads();
    if (act1) {
      Dft<float, R1, false>::run(u);
      if (j != 0) {
#pragma unroll
        for (int s = 1; s < R1; s++) u[s] = cmul<float>(u[s], __ldg(&a.tw[s * R2 + j]));
      }
#pragma unroll
      for (int s = 0; s < R1; s++) sm[s * BS + j * W + c] = u[s];
    }
    __syncthreads();

    // ---- DIF pass 2: thread b holds coefficient k = b + R1*s2 in y[s2]
    float2 y[R2];
    const bool act2 = bi < R1;
    const int b = bi;
    if (act2) {
#pragma unroll
      for (int q = 0; q < R2; q++) y[q] = sm[b * BS + q * W + c];
      Dft<float, R2, false>::run(y);
    }

    if (DCT) {
      // DCT-II post-processing needs Y_{M-k}: exchange through smem
      if (act2) {
#pragma unroll
        for (int s2 = 0; s2 < R2; s2++) sm[b * BS + s2 * W + c] = y[s2];
      }
      __syncthreads();
    }

    if (M == 1024) {
      // 1024-point lines: the output tile goes back through shared memory in
      // the TMA box layout and out by tensor stores (columns beyond the
      // valid ones are clipped by the tensor map)
      if (act2) {
#pragma unroll
        for (int s2 = 0; s2 < R2; s2++) {
          const int k = b + R1 * s2;
          if (DCT) {
            const int kp = k == 0 ? 0 : M - k;
            const float2 yp = sm[(kp % R1) * BS + (kp / R1) * W + c];
            const float2 w = __ldg(&a.mk[k]);
            y[s2] = cadd<float>(cmul<float>(w, y[s2]), cmulc<float>(yp, w));  // X_k = w Y_k + conj(w) Y_{M-k}
          }
        }
      }
      __syncthreads();  // the staged output overwrites the coefficients
      if (act2) {
#pragma unroll
        for (int s2 = 0; s2 < R2; s2++) sm[(b + R1 * s2) * W + c] = y[s2];
      }
      store_tile<W>(tmap, a, sm, c0, outer);
      return;
    }
    if (act2 && col_ok) {
#pragma unroll
      for (int s2 = 0; s2 < R2; s2++) {
        const int k = b + R1 * s2;
        float2 x = y[s2];
        if (DCT) {
          const int kp = k == 0 ? 0 : M - k;
          const float2 yp = sm[(kp % R1) * BS + (kp / R1) * W + c];
          const float2 w = __ldg(&a.mk[k]);
          x = cadd<float>(cmul<float>(w, x), cmulc<float>(yp, w));  // X_k = w Y_k + conj(w) Y_{M-k}
        }
        out[(size_t)k * a.s_axis + c] = x;
      }
    }
    return;
  } else {
    // ---- backward only: DIT pass A from the TMA layout (natural order input)
    float2 y[R2];
    const bool act2 = bi < R1;
    const int b = bi;
    if (act2) {
#pragma unroll
      for (int q = 0; q < R2; q++) {
        const int k = b + R1 * q;
        float2 x = sm[k * W + c];
        if (DCT) {
          // V_k = conj(w_k) (X_k - i X_{M-k}), X_M = 0
          const float2 xm = k == 0 ? make_float2(0.f, 0.f) : sm[(M - k) * W + c];
          x = cmulc<float>(make_float2(x.x + xm.y, x.y - xm.x), __ldg(&a.mk[k]));
        }
        y[q] = x;
      }
      Dft<float, R2, true>::run(y);
    }
    __syncthreads();
    if (act2) {
#pragma unroll
      for (int s = 0; s < R2; s++) sm[b * BS + s * W + c] = y[s];
    }
    __syncthreads();
  }

  // ---- DIT pass B (radix R1): natural-order output j + R2*s
  if (M == 1024) {
    // staged in shared memory and written by tensor stores (see above)
    float2 u[R1];
    const int j = bi;
    if (bi < R2) {
#pragma unroll
      for (int q = 0; q < R1; q++) u[q] = sm[q * BS + j * W + c];
      if (j != 0) {
#pragma unroll
        for (int q = 1; q < R1; q++) u[q] = cmulc<float>(u[q], __ldg(&a.tw[q * R2 + j]));
      }
      Dft<float, R1, true>::run(u);
    }
    __syncthreads();  // the staged output overwrites the padded tile
    if (bi < R2) {
#pragma unroll
      for (int s = 0; s < R1; s++) sm[(j + R2 * s) * W + c] = u[s];
    }
    store_tile<W>(tmap, a, sm, c0, outer);
  } else {
    float2 u[R1];
    const int j = bi;
    if (bi < R2 && col_ok) {
#pragma unroll
      for (int q = 0; q < R1; q++) u[q] = sm[q * BS + j * W + c];
      if (j != 0) {
#pragma unroll
        for (int q = 1; q < R1; q++) u[q] = cmulc<float>(u[q], __ldg(&a.tw[q * R2 + j]));
      }
      Dft<float, R1, true>::run(u);
#pragma unroll
      for (int s = 0; s < R1; s++) out[(size_t)(j + R2 * s) * a.s_axis + c] = u[s];
    }
  }
}

// ---------------------------------------------------------------------------
// fused sweep, divide as a pass of its own
// ---------------------------------------------------------------------------
// Forward transform of the swept axis (DIF passes 1 and 2), the divide by
// the eigenvalue sums with the zero-mode fix, and the backward transform
// (DIT passes A and B) in one launch.  No step keeps more than one radix
// block of values in registers: the
// forward pass 2 writes its coefficients back in place, the divide runs as a
// separate pass in which one thread takes the coefficient pair (k, M-k) of a
// column (both outputs of the pair step from both inputs, so every
// coefficient is read and written once and the eigenvalue factors of the
// pair are computed once), and the backward pass A reads the result.  At 80
// registers three CTAs fit on an SM instead of two.
//
// Pair step per kind, with Y the forward spectrum of the swept axis,
// f_j = scale / (lambda_other + lambda_axis[j]) and t = (c, s) =
// (cos, sin)(pi k / M):
//   FK_DFT:      V_k = f_k Y_k, V_{M-k} = f_{M-k} Y_{M-k};
//   FK_DCT:      with al = f_k + f_{M-k}, be = f_k - f_{M-k},
//                V_k     = al Y_k     + be e^{+i pi k/M} Y_{M-k},
//                V_{M-k} = al Y_{M-k} + be e^{-i pi k/M} Y_k;
//   FK_DCT_PAIR: Y = Yu + i Yv with Yu, Yv Hermitian; each part takes the
//                FK_DCT step with its own x eigenvalue, and since each part's
//                result is Hermitian, V_{M-k} = conj(Vu_k) + i conj(Vv_k).
// k = 0 and k = M/2 pair with themselves (be = 0; both writes agree).
//
// Shared memory: the tile (M x W complex) without padding; between the
// passes block b, row q sits at row q ^ (b & 1) of the block, which spreads
// the four blocks a warp touches at once over both halves of the banks.
// The pair table pk[0 .. M/2] follows the tile, copied in by the bulk-copy
// engine together with the tile.  Pass twiddles w^(j s), s = s0 + D s1
// (D = 8 for R1 = 32, 4 for R1 = 16), are applied as the two factors
// w^(j s0) and w^(j D s1), so a thread loads R1/D - 1 + D - 1 table values
// instead of R1 - 1 (one more rounding where both factors apply).
template <int R1> struct TwSplit { static constexpr int D = R1; };

// u[s] *= w^(j s) (INV: conj), s = 1 .. R1 - 1, with tw[s * R2 + j] = w^(j s):
// factor w^(j s0) on every s with s0 = s mod D > 0, then w^(j D s1) on every
// s with s1 = s / D > 0 (one table value live at a time).
template <int R1, int R2, bool INV>
__device__ __forceinline__ void apply_pass_twiddles(float2* u, const float2* __restrict__ tw, int j) {
  constexpr int D = TwSplit<R1>::D;
  constexpr int NB = R1 / D;
#pragma unroll
  for (int s0 = 1; s0 < D; s0++) {
    const float2 w = __ldg(&tw[s0 * R2 + j]);
#pragma unroll
    for (int s1 = 0; s1 < NB; s1++) u[s0 + D * s1] = INV ? cmulc<float>(u[s0 + D * s1], w) : cmul<float>(u[s0 + D * s1], w);
  }
#pragma unroll
  for (int s1 = 1; s1 < NB; s1++) {
    const float2 w = __ldg(&tw[D * s1 * R2 + j]);
#pragma unroll
    for (int s0 = 0; s0 < D; s0++) u[s0 + D * s1] = INV ? cmulc<float>(u[s0 + D * s1], w) : cmul<float>(u[s0 + D * s1], w);
  }
}

// Per-column constants of the pair step: lambda_other = lambda_x(column) +
// lambda_outer (FK_DCT_PAIR: one per packed real column) and whether the
// column holds the zero mode of a singular problem.
struct PairCol {
  float lam_xo, lam_xo0, lam_xo1;
  bool zero_row;
};
template <int KIND>
__device__ __forceinline__ PairCol pair_col(const FastStridedArgs& a, int col, int outer) {
  PairCol pc;
  const bool cin = col < a.ncols;
  const float lam_o = __ldg(&a.lam_out[outer]);
  pc.lam_xo = KIND == FK_DCT_PAIR ? 0.f : (cin ? __ldg(&a.lam_in[col]) : 0.f) + lam_o;
  pc.lam_xo0 = KIND == FK_DCT_PAIR ? (cin ? __ldg(&a.lam_in[2 * col]) : 0.f) + lam_o : 0.f;
  pc.lam_xo1 = KIND == FK_DCT_PAIR ? (cin ? __ldg(&a.lam_in[2 * col + 1]) : 0.f) + lam_o : 0.f;
  pc.zero_row = a.singular && col == 0 && outer == 0;
  return pc;
}
// Outputs (vk, vm) of the pair step for the coefficients (yk, ym) = (Y_k,
// Y_{M-k}); t = pk[k] = (lambda_axis[k], lambda_axis[M-k], cos, sin)(pi k/M).
template <int KIND>
__device__ __forceinline__ void pair_values(const float4 t, float scale, const PairCol& pc, int k, float2 yk,
                                            float2 ym, float2& vk, float2& vm) {
  if (KIND == FK_DFT) {
    float fk = __fdividef(scale, pc.lam_xo + t.x);
    float fm = __fdividef(scale, pc.lam_xo + t.y);
    if (pc.zero_row && k == 0) fk = fm = 0.f;
    vk = make_float2(fk * yk.x, fk * yk.y);
    vm = make_float2(fm * ym.x, fm * ym.y);
  } else if (KIND == FK_DCT_PAIR) {
    const float2 Yu = make_float2(0.5f * (yk.x + ym.x), 0.5f * (yk.y - ym.y));
    const float2 Yv = make_float2(0.5f * (yk.y + ym.y), 0.5f * (ym.x - yk.x));
    float f0k = __fdividef(scale, pc.lam_xo0 + t.x);
    float f0m = k == 0 ? f0k : __fdividef(scale, pc.lam_xo0 + t.y);
    if (pc.zero_row && k == 0) f0k = f0m = 0.f;
    const float f1k = __fdividef(scale, pc.lam_xo1 + t.x);
    const float f1m = k == 0 ? f1k : __fdividef(scale, pc.lam_xo1 + t.y);
    const float2 cu = make_float2(t.z * Yu.x + t.w * Yu.y, t.w * Yu.x - t.z * Yu.y);
    const float2 cv = make_float2(t.z * Yv.x + t.w * Yv.y, t.w * Yv.x - t.z * Yv.y);
    const float al0 = f0k + f0m, be0 = f0k - f0m, al1 = f1k + f1m, be1 = f1k - f1m;
    const float2 Vu = make_float2(al0 * Yu.x + be0 * cu.x, al0 * Yu.y + be0 * cu.y);
    const float2 Vv = make_float2(al1 * Yv.x + be1 * cv.x, al1 * Yv.y + be1 * cv.y);
    vk = make_float2(Vu.x - Vv.y, Vu.y + Vv.x);
    vm = make_float2(Vu.x + Vv.y, Vv.x - Vu.y);
  } else {
    float fk = __fdividef(scale, pc.lam_xo + t.x);
    float fm = k == 0 ? fk : __fdividef(scale, pc.lam_xo + t.y);
    if (pc.zero_row && k == 0) fk = fm = 0.f;
    const float al = fk + fm, be = fk - fm;
    // e^{+i pi k/M} Y_{M-k} and e^{-i pi k/M} Y_k
    const float2 rm = make_float2(t.z * ym.x - t.w * ym.y, t.z * ym.y + t.w * ym.x);
    const float2 rk = make_float2(t.z * yk.x + t.w * yk.y, t.z * yk.y - t.w * yk.x);
    vk = make_float2(al * yk.x + be * rm.x, al * yk.y + be * rm.y);
    vm = make_float2(al * ym.x + be * rk.x, al * ym.y + be * rk.y);
  }
}

template <int R1, int R2, int W, int KIND>
__global__ void __launch_bounds__(W * Shape<R1, R2>::RMAX, 768 / (W * Shape<R1, R2>::RMAX))
    fast_fused_kernel(const __grid_constant__ CUtensorMap tmap, const FastStridedArgs a) {
  constexpr int M = R1 * R2;
  constexpr int NT = W * Shape<R1, R2>::RMAX;
  constexpr int KSTEP = NT / W;  // pair indices handled per column per sweep
  constexpr int KIT = (M / 2) / KSTEP;
  constexpr bool PAIR = KIND == FK_DCT_PAIR;
  constexpr int BS = R2 * W;  // block stride (complex), no padding
  constexpr uint32_t PK_BYTES = (M / 2 + 1) * 16;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  float2* sm = reinterpret_cast<float2*>(smem_raw);
  float4* pks = reinterpret_cast<float4*>(smem_raw + (size_t)M * W * 8);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw + (size_t)M * W * 8 + PK_BYTES);

  const int tid = threadIdx.x;
  const int c = tid % W;
  const int bi = tid / W;
  const int tcol = blockIdx.x % a.ntile_c;
  const int outer = blockIdx.x / a.ntile_c;
  const int c0 = tcol * W;
  // position of (block b, row q, column c) between the passes
  auto bpos = [&](int b, int q) { return b * BS + ((q ^ (b & 1)) * W) + c; };

  if (tid == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (tid == 0) {
    const uint32_t box_bytes = (uint32_t)(2 * W * a.box_h * sizeof(float));
    mbar_arrive_expect_tx(bar, box_bytes * a.nbox + PK_BYTES);
    bulk_load_1d(pks, a.pk, PK_BYTES, bar);
    for (int b = 0; b < a.nbox; b++) {
      float2* dst = sm + (size_t)b * a.box_h * W;
      if (a.axis_dim == 1)
        tma_load_3d(dst, &tmap, bar, 2 * c0, b * a.box_h, outer);
      else
        tma_load_3d(dst, &tmap, bar, 2 * c0, outer, b * a.box_h);
    }
  }
  const bool ok = mbar_wait_bounded(bar, 0);
  if (__syncthreads_or(!ok)) {
    if (tid == 0) atomicExch(a.err, 1);
    return;
  }

  // ---- DIF pass 1 (radix R1) from the TMA layout into the block layout
  {
    float2 u[R1];
    const int j = bi;
    if (bi < R2) {
#pragma unroll
      for (int q = 0; q < R1; q++) u[q] = sm[(j + R2 * q) * W + c];
    }
    __syncthreads();
    if (bi < R2) {
      Dft<float, R1, false>::run(u);
      if (j != 0) apply_pass_twiddles<R1, R2, false>(u, a.tw, j);
#pragma unroll
      for (int s = 0; s < R1; s++) sm[bpos(s, j)] = u[s];
    }
    __syncthreads();
  }
  // ---- DIF pass 2 (radix R2) in place: coefficient k at block k % R1, row k / R1
  if (bi < R1) {
    float2 y[R2];
#pragma unroll
    for (int q = 0; q < R2; q++) y[q] = sm[bpos(bi, q)];
    Dft<float, R2, false>::run(y);
#pragma unroll
    for (int s2 = 0; s2 < R2; s2++) sm[bpos(bi, s2)] = y[s2];
  }
  __syncthreads();

  // ---- divide: coefficient pairs (k, M - k) of column c
  {
    const PairCol pc = pair_col<KIND>(a, c0 + c, outer);
    auto pair_step = [&](int k) {
      const int km = (M - k) & (M - 1);
      float2* pk_ = sm + bpos(k % R1, k / R1);
      float2* pm_ = sm + bpos(km % R1, km / R1);
      float2 vk, vm;
      pair_values<KIND>(pks[k], a.scale, pc, k, *pk_, *pm_, vk, vm);
      *pk_ = vk;
      *pm_ = vm;
    };
#pragma unroll 4
    for (int i = 0; i < KIT; i++) pair_step(bi + KSTEP * i);
    if (bi == 0) pair_step(M / 2);
  }
  __syncthreads();

  // ---- DIT pass A (radix R2) in place
  if (bi < R1) {
    float2 y[R2];
#pragma unroll
    for (int q = 0; q < R2; q++) y[q] = sm[bpos(bi, q)];
    Dft<float, R2, true>::run(y);
#pragma unroll
    for (int s = 0; s < R2; s++) sm[bpos(bi, s)] = y[s];
  }
  __syncthreads();

  // ---- DIT pass B (radix R1): natural-order output j + R2*s
  if (M == 1024) {
    // 1024-point lines: staged in the TMA box layout, written by tensor stores
    float2 u[R1];
    const int j = bi;
    if (bi < R2) {
#pragma unroll
      for (int q = 0; q < R1; q++) u[q] = sm[bpos(q, j)];
      if (j != 0) apply_pass_twiddles<R1, R2, true>(u, a.tw, j);
      Dft<float, R1, true>::run(u);
    }
    __syncthreads();  // the staged output overwrites the tile
    if (bi < R2) {
#pragma unroll
      for (int s = 0; s < R1; s++) sm[(j + R2 * s) * W + c] = u[s];
    }
    store_tile<W>(tmap, a, sm, c0, outer);
    return;
  }
  float2* out = a.data + (size_t)outer * a.s_outer + c0;
  if (bi < R2 && c0 + c < a.ncols) {
    float2 u[R1];
    const int j = bi;
#pragma unroll
    for (int q = 0; q < R1; q++) u[q] = sm[bpos(q, j)];
    if (j != 0) apply_pass_twiddles<R1, R2, true>(u, a.tw, j);
    Dft<float, R1, true>::run(u);
#pragma unroll
    for (int s = 0; s < R1; s++) out[(size_t)(j + R2 * s) * a.s_axis + c] = u[s];
  }
}

// ---------------------------------------------------------------------------
// contiguous (x) sweep, periodic x: R2C / C2R of two rows per complex line
// ---------------------------------------------------------------------------
// Thread t: line l = t / RMAX, butterfly index t % RMAX.  Smem per line:
// R1 blocks of R2 + 1 complex (padded).
template <int R1, int R2>
__device__ __forceinline__ int xpos(int k) {  // padded smem position of coefficient k
  return (k % R1) * (R2 + 1) + k / R1;
}

__device__ __forceinline__ void ws_row_of(const FastXArgs& a, long long r, long long& wr, float& sg) {
  int y = (int)(r % a.ny);
  int z = (int)(r / a.ny);
  sg = 1.f;
  if (a.sign_y && (y & 1)) sg = -sg;
  if (a.sign_z && (z & 1)) sg = -sg;
  if (a.perm_y) y = makhoul_pos(y, a.ny);
  if (a.perm_z) z = makhoul_pos(z, a.nz);
  wr = (long long)z * a.ny + y;
}

// FX_DCT: two real rows a, b form one complex line.  Forward: the line
// holds v_m = x_{2m} (m < M/2), v_m = x_{2M-1-2m} (m >= M/2), times -1 on the
// odd samples for DST-II; after the FFT Z = V_a + i V_b, and
//   X_a,k = Re(w_k Z_k) + Re(w_k conj(Z_{M-k})),
//   X_b,k = Im(w_k Z_k) - Im(w_k conj(Z_{M-k})),  w_k = exp(-i pi k / 2M),
// the DCT-II (2 sum x_n cos(pi k (2n+1) / 2M)) of each row, stored as M
// reals per workspace row (two x coefficients per complex column).
// Backward: V_k = conj(w_k) (X_k - i X_{M-k}), V_{M-k} = w_k (X_k + i X_{M-k})
// (X_M = 0) for each row, Z = V_a + i V_b, inverse FFT, and the samples go
// back to x_{2m} / x_{2M-1-2m} (DCT-III; DST-III with the odd samples
// negated).
//
// Input staging: the CTA's 2 * LPC rows are copied whole into shared memory
// by the bulk-copy engine (one copy per row, completing on one mbarrier),
// and the first step reads them there.  Backward: the workspace rows (R2C:
// M/2 + 2 complex per row, the row with its first padding element, so that
// every copy is a multiple of 16 bytes; DCT: M reals), 1024^3: 1.87 -> 1.56
// ms.  Forward: the rows of g (M reals), only for M = 1024 and 16-byte
// aligned rows (a.stage_g): 1024^3 1.92 -> 1.78 ms, while shorter lines
// were slower staged (512^3: 0.31 -> 0.34 ms) and read g straight into
// registers.  The staging area is the same memory as the line buffer, so a
// barrier separates the last staged read from the first line write.
template <int M, int MODE, int KX> struct XStageRow {
  // elements of 4 bytes per staged row
  static constexpr int value = (MODE == FM_INV && KX == FX_R2C) ? 2 * (M / 2 + 2) : M;
};

template <int R1, int R2, int MODE, int KX>
__global__ void __launch_bounds__(256, MODE == 0 ? 2 : 3) fast_x_kernel(const FastXArgs a) {
  constexpr int M = R1 * R2;
  constexpr int RMAX = Shape<R1, R2>::RMAX;
  constexpr int LS = R1 * (R2 + 1);  // padded line stride (complex)
  constexpr int LPC = 256 / RMAX;    // lines per CTA
  constexpr int SR = XStageRow<M, MODE, KX>::value;
  static_assert(2 * LPC * SR <= 2 * LPC * LS, "staged rows fit in the line buffer");
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  float2* sm = reinterpret_cast<float2*>(smem_raw);
  float* stage = reinterpret_cast<float*>(smem_raw);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw + (size_t)LPC * LS * 8);
  const int tid = threadIdx.x;
  const int l = tid / RMAX;
  const int bi = tid % RMAX;
  float2* line = sm + l * LS;
  const long long r0 = (long long)blockIdx.x * LPC * 2;
  const long long ra = r0 + 2 * l;
  const long long rb = ra + 1;
  const bool va = ra < a.nrows, vb = rb < a.nrows;
  long long wa = 0, wb = 0;
  float sa = 1.f, sb = 1.f;
  if (va) ws_row_of(a, ra, wa, sa);
  if (vb) ws_row_of(a, rb, wb, sb);
  const bool bulk = MODE == FM_INV || (M == 1024 && a.stage_g);

  if (bulk) {
    if (tid == 0) {
      mbar_init(bar, 1);
      fence_mbar_init();
    }
    __syncthreads();
    const int nr = (int)(a.nrows - r0 < 2 * LPC ? a.nrows - r0 : 2 * LPC);
    if (tid == 0) mbar_arrive_expect_tx(bar, (uint32_t)(nr * SR * 4));
    if (tid < nr) {
      const long long r = r0 + tid;
      const void* src;
      if (MODE == FM_FWD) {
        src = a.g + (r % a.ny) * a.g_sy + (r / a.ny) * a.g_sz;
      } else {
        long long wr;
        float sg;
        ws_row_of(a, r, wr, sg);
        src = a.ws + wr * a.ws_ld;
      }
      bulk_load_1d(stage + (size_t)tid * SR, src, (uint32_t)(SR * 4), bar);
    }
    const bool ok = mbar_wait_bounded(bar, 0);
    if (__syncthreads_or(!ok)) {
      if (tid == 0) atomicExch(a.err, 1);
      return;
    }
  }

  if (MODE == FM_FWD) {
    // DIF pass 1 from rows a, b (staged, or straight from global memory)
    float2 u[R1];
    const int j = bi;
    if (bi < R2) {
      const float* ga = bulk ? stage + (size_t)(2 * l) * SR : a.g + (ra % a.ny) * a.g_sy + (ra / a.ny) * a.g_sz;
      const float* gb = bulk ? stage + (size_t)(2 * l + 1) * SR : a.g + (rb % a.ny) * a.g_sy + (rb / a.ny) * a.g_sz;
#pragma unroll
      for (int q = 0; q < R1; q++) {
        const int m = j + R2 * q;
        if (KX == FX_R2C) {
          u[q] = make_float2(va ? ga[m] : 0.f, vb ? gb[m] : 0.f);
        } else {
          const bool odd = q >= R1 / 2;  // m >= M/2
          const int src = odd ? 2 * M - 1 - 2 * m : 2 * m;
          const float sg = (odd && a.xsign) ? -1.f : 1.f;
          u[q] = make_float2(va ? sg * ga[src] : 0.f, vb ? sg * gb[src] : 0.f);
        }
      }
    }
    if (bulk) __syncthreads();  // the line buffer overwrites the staged rows
    if (bi < R2) {
      Dft<float, R1, false>::run(u);
      if (j != 0) {
#pragma unroll
        for (int s = 1; s < R1; s++) u[s] = cmul<float>(u[s], __ldg(&a.tw[s * R2 + j]));
      }
#pragma unroll
      for (int s = 0; s < R1; s++) line[s * (R2 + 1) + j] = u[s];
    }
    __syncthreads();
    if (bi < R1) {
      const int b = bi;
      float2 y[R2];
#pragma unroll
      for (int q = 0; q < R2; q++) y[q] = line[b * (R2 + 1) + q];
      Dft<float, R2, false>::run(y);
#pragma unroll
      for (int s = 0; s < R2; s++) line[b * (R2 + 1) + s] = y[s];
    }
    __syncthreads();
    if (KX == FX_R2C && M == 1024) {
      // split Z into the half spectra of rows a and b, staged in shared memory
      // (M/2 + 2 complex per row: the row and its first padding element, set
      // to zero) and written back by one bulk copy per row
      constexpr int NH = M / 2 + 1, OW = M / 2 + 2, NK = (NH + RMAX - 1) / RMAX;
      float2 A[NK], B[NK];
#pragma unroll
      for (int i = 0; i < NK; i++) {
        const int k = bi + i * RMAX;
        if (k < NH) {
          const float2 z1 = line[xpos<R1, R2>(k)];
          const float2 z2 = line[xpos<R1, R2>(k == 0 ? 0 : M - k)];
          A[i] = make_float2(sa * 0.5f * (z1.x + z2.x), sa * 0.5f * (z1.y - z2.y));
          B[i] = make_float2(sb * 0.5f * (z1.y + z2.y), sb * 0.5f * (z2.x - z1.x));
        }
      }
      __syncthreads();  // the staged rows overwrite the line buffer
      float2* oa = sm + (size_t)(2 * l) * OW;
      float2* ob = oa + OW;
#pragma unroll
      for (int i = 0; i < NK; i++) {
        const int k = bi + i * RMAX;
        if (k < NH) {
          oa[k] = A[i];
          ob[k] = B[i];
        }
      }
      if (bi == 0) oa[NH] = ob[NH] = make_float2(0.f, 0.f);
      fence_proxy_async();
      __syncthreads();
      const int nr = (int)(a.nrows - r0 < 2 * LPC ? a.nrows - r0 : 2 * LPC);
      if (tid < nr) {
        long long wr;
        float sg;
        ws_row_of(a, r0 + tid, wr, sg);
        bulk_store_1d(a.ws + wr * a.ws_ld, sm + (size_t)tid * OW, (uint32_t)(OW * 8));
        bulk_commit_group();
        bulk_wait_group_read0();
      }
    } else if (KX == FX_R2C) {
      // split Z into the half spectra of rows a and b
      constexpr int NH = M / 2 + 1;
      float2* da = a.ws + wa * a.ws_ld;
      float2* db = a.ws + wb * a.ws_ld;
      for (int k = bi; k < NH; k += RMAX) {
        const float2 z1 = line[xpos<R1, R2>(k)];
        const float2 z2 = line[xpos<R1, R2>(k == 0 ? 0 : M - k)];
        const float2 A = make_float2(0.5f * (z1.x + z2.x), 0.5f * (z1.y - z2.y));
        const float2 B = make_float2(0.5f * (z1.y + z2.y), 0.5f * (z2.x - z1.x));
        if (va) da[k] = make_float2(sa * A.x, sa * A.y);
        if (vb) db[k] = make_float2(sb * B.x, sb * B.y);
      }
    } else {
      float* da = reinterpret_cast<float*>(a.ws + wa * a.ws_ld);
      float* db = reinterpret_cast<float*>(a.ws + wb * a.ws_ld);
      for (int k = bi; k < M; k += RMAX) {
        const float2 z1 = line[xpos<R1, R2>(k)];
        const float2 z2 = line[xpos<R1, R2>(k == 0 ? 0 : M - k)];
        const float2 w = __ldg(&a.mk[k]);
        const float2 p1 = cmul<float>(w, z1);
        const float2 p2 = cmul<float>(w, make_float2(z2.x, -z2.y));
        if (va) da[k] = sa * (p1.x + p2.x);
        if (vb) db[k] = sb * (p1.y - p2.y);
      }
    }
  } else {
    constexpr int NH = M / 2 + 1;
    constexpr int NK = (NH + RMAX - 1) / RMAX;
    if (KX == FX_R2C) {
      // C2R assembly into the digit-reversed arrangement (all loads first)
      const float2* sa_p = reinterpret_cast<const float2*>(stage + (size_t)(2 * l) * SR);
      const float2* sb_p = reinterpret_cast<const float2*>(stage + (size_t)(2 * l + 1) * SR);
      float2 Av[NK], Bv[NK];
#pragma unroll
      for (int i = 0; i < NK; i++) {
        const int k = bi + i * RMAX;
        Av[i] = (va && k < NH) ? sa_p[k] : make_float2(0.f, 0.f);
        Bv[i] = (vb && k < NH) ? sb_p[k] : make_float2(0.f, 0.f);
      }
      __syncthreads();  // the line buffer overwrites the staged rows
#pragma unroll
      for (int i = 0; i < NK; i++) {
        const int k = bi + i * RMAX;
        if (k >= NH) break;
        const float2 A = make_float2(sa * Av[i].x, sa * Av[i].y);
        const float2 B = make_float2(sb * Bv[i].x, sb * Bv[i].y);
        if (k == 0 || 2 * k == M) {
          line[xpos<R1, R2>(k)] = make_float2(A.x, B.x);
        } else {
          line[xpos<R1, R2>(k)] = make_float2(A.x - B.y, A.y + B.x);
          line[xpos<R1, R2>(M - k)] = make_float2(A.x + B.y, B.x - A.y);
        }
      }
    } else {
      // DCT-III pre-processing of rows a, b for k and M - k (all loads first)
      const float* sa_p = stage + (size_t)(2 * l) * SR;
      const float* sb_p = stage + (size_t)(2 * l + 1) * SR;
      float xa[NK], xam[NK], xb[NK], xbm[NK];
#pragma unroll
      for (int i = 0; i < NK; i++) {
        const int k = bi + i * RMAX;
        const bool in = k < NH;
        xa[i] = (va && in) ? sa * sa_p[k] : 0.f;
        xb[i] = (vb && in) ? sb * sb_p[k] : 0.f;
        xam[i] = (va && in && k > 0) ? sa * sa_p[M - k] : 0.f;
        xbm[i] = (vb && in && k > 0) ? sb * sb_p[M - k] : 0.f;
      }
      __syncthreads();  // the line buffer overwrites the staged rows
#pragma unroll
      for (int i = 0; i < NK; i++) {
        const int k = bi + i * RMAX;
        if (k >= NH) break;
        const float2 w = __ldg(&a.mk[k]);
        // Z_k = conj(w) ((xa + xbm) + i (xb - xam)), Z_{M-k} = w ((xa - xbm) + i (xb + xam))
        line[xpos<R1, R2>(k)] = cmulc<float>(make_float2(xa[i] + xbm[i], xb[i] - xam[i]), w);
        if (k != 0 && 2 * k != M)
          line[xpos<R1, R2>(M - k)] = cmul<float>(w, make_float2(xa[i] - xbm[i], xb[i] + xam[i]));
      }
    }
    __syncthreads();
    if (bi < R1) {
      const int b = bi;
      float2 y[R2];
#pragma unroll
      for (int q = 0; q < R2; q++) y[q] = line[b * (R2 + 1) + q];
      Dft<float, R2, true>::run(y);
#pragma unroll
      for (int s = 0; s < R2; s++) line[b * (R2 + 1) + s] = y[s];
    }
    __syncthreads();
    if (M == 1024 && a.stage_phi) {
      // rows a, b of phi staged in shared memory (M reals each, over the line
      // buffer) and written back by one bulk copy per row
      float2 u[R1];
      const int j = bi;
      if (bi < R2) {
#pragma unroll
        for (int q = 0; q < R1; q++) u[q] = line[q * (R2 + 1) + j];
        if (j != 0) {
#pragma unroll
          for (int q = 1; q < R1; q++) u[q] = cmulc<float>(u[q], __ldg(&a.tw[q * R2 + j]));
        }
        Dft<float, R1, true>::run(u);
      }
      __syncthreads();  // the staged rows overwrite the line buffer
      if (bi < R2) {
        float* oa = stage + (size_t)(2 * l) * M;
        float* ob = oa + M;
#pragma unroll
        for (int s = 0; s < R1; s++) {
          const int n = j + R2 * s;
          if (KX == FX_R2C) {
            oa[n] = u[s].x;
            ob[n] = u[s].y;
          } else {
            const bool odd = s >= R1 / 2;  // n >= M/2
            const int dst = odd ? 2 * M - 1 - 2 * n : 2 * n;
            const float sg = (odd && a.xsign) ? -1.f : 1.f;
            oa[dst] = sg * u[s].x;
            ob[dst] = sg * u[s].y;
          }
        }
      }
      fence_proxy_async();
      __syncthreads();
      const int nr = (int)(a.nrows - r0 < 2 * LPC ? a.nrows - r0 : 2 * LPC);
      if (tid < nr) {
        const long long r = r0 + tid;
        bulk_store_1d(a.phi + (r % a.ny) * a.phi_sy + (r / a.ny) * a.phi_sz, stage + (size_t)tid * M,
                      (uint32_t)(M * 4));
        bulk_commit_group();
        bulk_wait_group_read0();
      }
    } else if (bi < R2) {
      const int j = bi;
      float2 u[R1];
#pragma unroll
      for (int q = 0; q < R1; q++) u[q] = line[q * (R2 + 1) + j];
      if (j != 0) {
#pragma unroll
        for (int q = 1; q < R1; q++) u[q] = cmulc<float>(u[q], __ldg(&a.tw[q * R2 + j]));
      }
      Dft<float, R1, true>::run(u);
      float* pa = a.phi + (ra % a.ny) * a.phi_sy + (ra / a.ny) * a.phi_sz;
      float* pb = a.phi + (rb % a.ny) * a.phi_sy + (rb / a.ny) * a.phi_sz;
#pragma unroll
      for (int s = 0; s < R1; s++) {
        const int n = j + R2 * s;
        if (KX == FX_R2C) {
          if (va) pa[n] = u[s].x;
          if (vb) pb[n] = u[s].y;
        } else {
          const bool odd = s >= R1 / 2;  // n >= M/2
          const int dst = odd ? 2 * M - 1 - 2 * n : 2 * n;
          const float sg = (odd && a.xsign) ? -1.f : 1.f;
          if (va) pa[dst] = sg * u[s].x;
          if (vb) pb[dst] = sg * u[s].y;
        }
      }
    }
  }
}

}  // namespace fast
}  // namespace pf
