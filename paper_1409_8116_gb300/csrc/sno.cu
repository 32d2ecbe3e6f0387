// Spectral neural operator for the learned initial guess of the PCG.
//
// The paper (Sec. 1) names the fast Poisson solve as a preconditioner for
// div(a grad phi) = g; the network here is this library's addition on top of
// that PCG.  It maps three per-cell features of a problem to a correction of
// the FFT-Poisson solution:
//   v_0 = P f + p;  for l < L: vhat = S(v_l), uhat[o,m] = sum_i R_l[m,o,i] vhat[i,m],
//   pre_l = W_l v_l + b_l + S_inv(uhat), v_{l+1} = gelu(pre_l) (identity for the last);
//   y = Q v_L + q.
// S / S_inv are the truncated sine transforms (DST-II basis, K modes per
// axis) with S[m,j] = (2/n) sin(pi(m+1)(2j+1)/2n), S_inv[j,m] = sin(...):
// resolution-independent coefficients, S S_inv = I.  Weights are stored in
// bfloat16 (an FP32 master copy is kept for the optimiser); activations and
// every accumulation are FP32, and the cross-block sums of the weight
// gradients are FP64 in a fixed order (repeatable results).
//
// Layouts: activations [B][C][nz][ny][nx] (x fastest); truncated
// intermediates [B][C][nz][ny][K], [B][C][nz][K][K], [B][C][K][K][K].  The
// parameter vector is P (C x 3), p (C), per layer W (C x C), b (C),
// R (K^3 x C x C, mode m = (mz K + my) K + mx), then Q (C), q (1).
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "../../include/poisfft.h"
#include "reduce.cuh"

namespace {

constexpr int kT = 256;
constexpr int kMaxC = 32, kMaxK = 16, kMaxL = 8, kF = 3;
constexpr int kTileP = 64;  // points per smem tile of the weight-gradient reduction

struct Dims {
  int B, C, K, L, nx, ny, nz;
  long long N;  // cells per sample
};

struct Layout {
  long long P, p, W[kMaxL], b[kMaxL], R[kMaxL], Q, q, total;
};

Layout layout_of(int C, int K, int L) {
  Layout o{};
  long long at = 0;
  o.P = at; at += (long long)C * kF;
  o.p = at; at += C;
  for (int l = 0; l < L; l++) {
    o.W[l] = at; at += (long long)C * C;
    o.b[l] = at; at += C;
    o.R[l] = at; at += (long long)K * K * K * C * C;
  }
  o.Q = at; at += C;
  o.q = at; at += 1;
  o.total = at;
  return o;
}

__device__ __forceinline__ float gelu(float x) {
  const float t = tanhf(0.7978845608028654f * (x + 0.044715f * x * x * x));
  return 0.5f * x * (1.f + t);
}

__device__ __forceinline__ float gelu_grad(float x) {
  const float t = tanhf(0.7978845608028654f * (x + 0.044715f * x * x * x));
  return 0.5f * (1.f + t) + 0.5f * x * (1.f - t * t) * 0.7978845608028654f * (1.f + 3.f * 0.044715f * x * x);
}

__device__ __forceinline__ float wload(const __nv_bfloat16* w, long long i) { return __bfloat162float(w[i]); }

#define GRID_STRIDE_LL(i, N) \
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < (N); i += (long long)gridDim.x * blockDim.x)

// v0[b,c,p] = sum_f P[c,f] feats[b,f,p] + p[c]
__global__ void __launch_bounds__(kT) lift_kernel(const float* __restrict__ feats, const __nv_bfloat16* __restrict__ th,
                                                  long long oP, long long op, float* __restrict__ v0, Dims D) {
  __shared__ float sP[kMaxC * kF], sp[kMaxC];
  for (int i = threadIdx.x; i < D.C * kF; i += blockDim.x) sP[i] = wload(th, oP + i);
  for (int i = threadIdx.x; i < D.C; i += blockDim.x) sp[i] = wload(th, op + i);
  __syncthreads();
  GRID_STRIDE_LL(idx, (long long)D.B * D.N) {
    const long long b = idx / D.N, p = idx - b * D.N;
    float f[kF];
#pragma unroll
    for (int k = 0; k < kF; k++) f[k] = feats[(b * kF + k) * D.N + p];
    for (int c = 0; c < D.C; c++)
      v0[(b * D.C + c) * D.N + p] = sp[c] + sP[c * kF] * f[0] + sP[c * kF + 1] * f[1] + sP[c * kF + 2] * f[2];
  }
}

// out[row][m] = sum_j M[m][j] in[row][j] for rows of length n (one warp per
// row, lanes stride the row, Kout partial sums per lane reduced by shuffles).
__global__ void __launch_bounds__(kT) row_contract_kernel(const float* __restrict__ in, const float* __restrict__ M,
                                                          float* __restrict__ out, long long rows, int n, int Kout) {
  const int lane = threadIdx.x & 31;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long r = warp; r < rows; r += nwarps) {
    float acc[kMaxK];
#pragma unroll
    for (int m = 0; m < kMaxK; m++) acc[m] = 0.f;
    const float* src = in + r * n;
    for (int j = lane; j < n; j += 32) {
      const float x = src[j];
#pragma unroll
      for (int m = 0; m < kMaxK; m++)
        if (m < Kout) acc[m] += __ldg(&M[m * n + j]) * x;
    }
#pragma unroll
    for (int m = 0; m < kMaxK; m++) {
      if (m >= Kout) break;
      float v = acc[m];
      for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
      if (lane == 0) out[r * Kout + m] = v;
    }
  }
}

// out[o][k][i] = sum_j M[k][j] in[o][j][i]: in [outer][n][inner] -> out [outer][Kout][inner]
__global__ void __launch_bounds__(kT) axis_contract_kernel(const float* __restrict__ in, const float* __restrict__ M,
                                                           float* __restrict__ out, long long outer, int n, int Kout,
                                                           long long inner) {
  GRID_STRIDE_LL(idx, outer * Kout * inner) {
    const long long i = idx % inner;
    const long long t = idx / inner;
    const int k = (int)(t % Kout);
    const long long o = t / Kout;
    const float* src = in + o * n * inner + i;
    const float* row = M + (long long)k * n;
    float acc = 0.f;
    for (int j = 0; j < n; j++) acc += __ldg(&row[j]) * src[(long long)j * inner];
    out[idx] = acc;
  }
}

// uhat[b][o][m] = sum_i R[m][o][i] vhat[b][i][m]
__global__ void __launch_bounds__(kT) mix_kernel(const float* __restrict__ vh, const __nv_bfloat16* __restrict__ th,
                                                 long long oR, float* __restrict__ uh, int B, int C, int M3) {
  GRID_STRIDE_LL(idx, (long long)B * C * M3) {
    const int m = (int)(idx % M3);
    const long long t = idx / M3;
    const int o = (int)(t % C);
    const long long b = t / C;
    float acc = 0.f;
    for (int i = 0; i < C; i++) acc += wload(th, oR + ((long long)m * C + o) * C + i) * vh[(b * C + i) * M3 + m];
    uh[idx] = acc;
  }
}

// dvh[b][i][m] = sum_o R[m][o][i] duh[b][o][m]
__global__ void __launch_bounds__(kT) mix_t_kernel(const float* __restrict__ duh, const __nv_bfloat16* __restrict__ th,
                                                   long long oR, float* __restrict__ dvh, int B, int C, int M3) {
  GRID_STRIDE_LL(idx, (long long)B * C * M3) {
    const int m = (int)(idx % M3);
    const long long t = idx / M3;
    const int i = (int)(t % C);
    const long long b = t / C;
    float acc = 0.f;
    for (int o = 0; o < C; o++) acc += wload(th, oR + ((long long)m * C + o) * C + i) * duh[(b * C + o) * M3 + m];
    dvh[idx] = acc;
  }
}

// dR[m][o][i] = sum_b duh[b][o][m] vhat[b][i][m]  (one thread per weight)
__global__ void __launch_bounds__(kT) mix_grad_kernel(const float* __restrict__ duh, const float* __restrict__ vh,
                                                      float* __restrict__ gR, int B, int C, int M3) {
  GRID_STRIDE_LL(idx, (long long)M3 * C * C) {
    const int i = (int)(idx % C);
    const long long t = idx / C;
    const int o = (int)(t % C);
    const int m = (int)(t / C);
    double acc = 0.0;
    for (int b = 0; b < B; b++) acc += (double)duh[((long long)b * C + o) * M3 + m] * vh[((long long)b * C + i) * M3 + m];
    gR[idx] = (float)acc;
  }
}

// Layer output: pre = W v + b + sum_m E[x][m] U[b,o,z,y,m]; out = gelu(pre) or pre.
__global__ void __launch_bounds__(kT) point_kernel(const float* __restrict__ v, const float* __restrict__ U,
                                                   const float* __restrict__ E, const __nv_bfloat16* __restrict__ th,
                                                   long long oW, long long ob, float* __restrict__ pre_out,
                                                   float* __restrict__ out, int act, Dims D) {
  __shared__ float sW[kMaxC * kMaxC], sb[kMaxC];
  for (int i = threadIdx.x; i < D.C * D.C; i += blockDim.x) sW[i] = wload(th, oW + i);
  for (int i = threadIdx.x; i < D.C; i += blockDim.x) sb[i] = wload(th, ob + i);
  __syncthreads();
  const long long rows = (long long)D.nz * D.ny;
  GRID_STRIDE_LL(idx, (long long)D.B * D.N) {
    const long long b = idx / D.N, p = idx - b * D.N;
    const int x = (int)(p % D.nx);
    const long long zy = p / D.nx;
    float vin[kMaxC];
#pragma unroll
    for (int i = 0; i < kMaxC; i++)
      if (i < D.C) vin[i] = v[(b * D.C + i) * D.N + p];
    float e[kMaxK];
#pragma unroll
    for (int m = 0; m < kMaxK; m++)
      if (m < D.K) e[m] = __ldg(&E[x * D.K + m]);
    for (int o = 0; o < D.C; o++) {
      float acc = sb[o];
#pragma unroll
      for (int i = 0; i < kMaxC; i++)
        if (i < D.C) acc += sW[o * D.C + i] * vin[i];
      const float* u = U + ((b * D.C + o) * rows + zy) * D.K;
#pragma unroll
      for (int m = 0; m < kMaxK; m++)
        if (m < D.K) acc += e[m] * u[m];
      const long long at = (b * D.C + o) * D.N + p;
      if (pre_out) pre_out[at] = acc;
      out[at] = act ? gelu(acc) : acc;
    }
  }
}

// Specialised forms of row_contract_kernel and point_kernel for compile-time
// K and C (the inference configuration): the matrix sits in shared memory,
// the row loads are issued four at a time, and every loop over channels and
// modes is unrolled (vectorised loads of the expansion rows).
template <int K>
__global__ void __launch_bounds__(kT) row_contract_k_kernel(const float* __restrict__ in, const float* __restrict__ M,
                                                            float* __restrict__ out, long long rows, int n) {
  // Two rows per warp pass, so that the loads and the shuffle reductions of
  // one row overlap those of the other.
  extern __shared__ float sM[];  // K x n
  for (int i = threadIdx.x; i < K * n; i += blockDim.x) sM[i] = M[i];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long r = 2 * warp; r < rows; r += 2 * nwarps) {
    const bool two = r + 1 < rows;
    float a0[K], a1[K];
#pragma unroll
    for (int m = 0; m < K; m++) a0[m] = a1[m] = 0.f;
    const float* s0 = in + r * n;
    const float* s1 = in + (two ? r + 1 : r) * n;
    for (int j0 = lane; j0 < n; j0 += 64) {
      const int j1 = j0 + 32;
      const float x0 = s0[j0], y0 = s1[j0];
      const float x1 = j1 < n ? s0[j1] : 0.f, y1 = j1 < n ? s1[j1] : 0.f;
#pragma unroll
      for (int m = 0; m < K; m++) {
        const float c0 = sM[m * n + j0];
        a0[m] += c0 * x0;
        a1[m] += c0 * y0;
      }
      if (j1 < n) {
#pragma unroll
        for (int m = 0; m < K; m++) {
          const float c1 = sM[m * n + j1];
          a0[m] += c1 * x1;
          a1[m] += c1 * y1;
        }
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
      for (int m = 0; m < K; m++) {
        a0[m] += __shfl_down_sync(0xffffffffu, a0[m], o);
        a1[m] += __shfl_down_sync(0xffffffffu, a1[m], o);
      }
    }
    if (lane == 0) {
#pragma unroll
      for (int m = 0; m < K; m++) {
        out[r * K + m] = a0[m];
        if (two) out[(r + 1) * K + m] = a1[m];
      }
    }
  }
}

template <int C, int K>
__global__ void __launch_bounds__(kT) point_ck_kernel(const float* __restrict__ v, const float* __restrict__ U,
                                                      const float* __restrict__ E,
                                                      const __nv_bfloat16* __restrict__ th, long long oW,
                                                      long long ob, float* __restrict__ pre_out,
                                                      float* __restrict__ out, int act, Dims D) {
  // Blocks take whole x rows (R rows at a time when nx < 256) so that the
  // expansion rows U[b][o][z,y][0..K) of those rows are staged in shared
  // memory once: no global load remains inside the loop over outputs.
  static_assert(K % 4 == 0 && C % 4 == 0, "vectorised rows");
  constexpr int RMAX = 8;
  __shared__ __align__(16) float sW[C * C];
  __shared__ float sb[C];
  __shared__ __align__(16) float sU[RMAX][C * K];
  for (int i = threadIdx.x; i < C * C; i += blockDim.x) sW[i] = wload(th, oW + i);
  for (int i = threadIdx.x; i < C; i += blockDim.x) sb[i] = wload(th, ob + i);
  const int R = D.nx >= kT ? 1 : min(RMAX, kT / D.nx);
  const long long rows = (long long)D.nz * D.ny;   // rows per sample
  const long long all_rows = (long long)D.B * rows;
  const int lr = threadIdx.x / D.nx < R ? threadIdx.x / D.nx : R;  // this thread's row in the group
  const int x0 = D.nx >= kT ? threadIdx.x : threadIdx.x - lr * D.nx;
  const int xstep = D.nx >= kT ? kT : D.nx;
  for (long long r0 = (long long)blockIdx.x * R; r0 < all_rows; r0 += (long long)gridDim.x * R) {
    __syncthreads();  // previous group's rows are no longer read
    for (int e = threadIdx.x; e < R * C * K; e += blockDim.x) {
      const int g = e / (C * K), o = (e / K) % C, m = e % K;
      const long long row = r0 + g;
      float val = 0.f;
      if (row < all_rows) {
        const long long b = row / rows, zy = row - b * rows;
        val = U[((b * C + o) * rows + zy) * K + m];
      }
      sU[g][o * K + m] = val;
    }
    __syncthreads();
    const long long row = r0 + lr;
    if (lr >= R || row >= all_rows) continue;
    const long long b = row / rows, zy = row - b * rows;
    for (int x = x0; x < D.nx; x += xstep) {
      const long long p = zy * D.nx + x;
      float vin[C];
#pragma unroll
      for (int i = 0; i < C; i++) vin[i] = v[(b * C + i) * D.N + p];
      float e[K];
      const float4* e4 = reinterpret_cast<const float4*>(E + (long long)x * K);
#pragma unroll
      for (int q = 0; q < K / 4; q++) {
        const float4 t = __ldg(e4 + q);
        e[4 * q] = t.x;
        e[4 * q + 1] = t.y;
        e[4 * q + 2] = t.z;
        e[4 * q + 3] = t.w;
      }
#pragma unroll
      for (int o = 0; o < C; o++) {
        float acc = sb[o];
        const float4* w4 = reinterpret_cast<const float4*>(sW + o * C);
#pragma unroll
        for (int q = 0; q < C / 4; q++) {
          const float4 w = w4[q];
          acc += w.x * vin[4 * q] + w.y * vin[4 * q + 1] + w.z * vin[4 * q + 2] + w.w * vin[4 * q + 3];
        }
        const float4* u4 = reinterpret_cast<const float4*>(&sU[lr][o * K]);
#pragma unroll
        for (int q = 0; q < K / 4; q++) {
          const float4 u = u4[q];
          acc += e[4 * q] * u.x + e[4 * q + 1] * u.y + e[4 * q + 2] * u.z + e[4 * q + 3] * u.w;
        }
        const long long at = (b * C + o) * D.N + p;
        if (pre_out) pre_out[at] = acc;
        out[at] = act ? gelu(acc) : acc;
      }
    }
  }
}

// y[b,p] = sum_c Q[c] v[b,c,p] + q
__global__ void __launch_bounds__(kT) proj_kernel(const float* __restrict__ v, const __nv_bfloat16* __restrict__ th,
                                                  long long oQ, long long oq, float* __restrict__ y, Dims D) {
  __shared__ float sQ[kMaxC + 1];
  for (int i = threadIdx.x; i <= D.C; i += blockDim.x) sQ[i] = wload(th, (i < D.C ? oQ + i : oq));
  __syncthreads();
  GRID_STRIDE_LL(idx, (long long)D.B * D.N) {
    const long long b = idx / D.N, p = idx - b * D.N;
    float acc = sQ[D.C];
    for (int c = 0; c < D.C; c++) acc += sQ[c] * v[(b * D.C + c) * D.N + p];
    y[idx] = acc;
  }
}

// dv[b,c,p] = Q[c] dy[b,p]
__global__ void __launch_bounds__(kT) proj_bwd_kernel(const float* __restrict__ dy, const __nv_bfloat16* __restrict__ th,
                                                      long long oQ, float* __restrict__ dv, Dims D) {
  __shared__ float sQ[kMaxC];
  for (int i = threadIdx.x; i < D.C; i += blockDim.x) sQ[i] = wload(th, oQ + i);
  __syncthreads();
  GRID_STRIDE_LL(idx, (long long)D.B * D.N) {
    const long long b = idx / D.N, p = idx - b * D.N;
    const float d = dy[idx];
    for (int c = 0; c < D.C; c++) dv[(b * D.C + c) * D.N + p] = sQ[c] * d;
  }
}

// dpre = dv_next * gelu'(pre) (or dv_next); dv[b,i,p] = sum_o W[o,i] dpre[b,o,p]
__global__ void __launch_bounds__(kT) point_bwd_kernel(const float* __restrict__ dvn, const float* __restrict__ pre,
                                                       const __nv_bfloat16* __restrict__ th, long long oW, int act,
                                                       float* __restrict__ dpre, float* __restrict__ dv, Dims D) {
  __shared__ float sW[kMaxC * kMaxC];
  for (int i = threadIdx.x; i < D.C * D.C; i += blockDim.x) sW[i] = wload(th, oW + i);
  __syncthreads();
  GRID_STRIDE_LL(idx, (long long)D.B * D.N) {
    const long long b = idx / D.N, p = idx - b * D.N;
    float d[kMaxC];
#pragma unroll
    for (int o = 0; o < kMaxC; o++) {
      if (o < D.C) {
        const long long at = (b * D.C + o) * D.N + p;
        float g = dvn[at];
        if (act) g *= gelu_grad(pre[at]);
        d[o] = g;
        dpre[at] = g;
      }
    }
    for (int i = 0; i < D.C; i++) {
      float acc = 0.f;
#pragma unroll
      for (int o = 0; o < kMaxC; o++)
        if (o < D.C) acc += sW[o * D.C + i] * d[o];
      dv[(b * D.C + i) * D.N + p] = acc;
    }
  }
}

// out[b,c,p] += sum_m E[x][m] U[b,c,z,y,m]
__global__ void __launch_bounds__(kT) expand_add_kernel(const float* __restrict__ U, const float* __restrict__ E,
                                                        float* __restrict__ out, Dims D) {
  const long long rows = (long long)D.nz * D.ny;
  GRID_STRIDE_LL(idx, (long long)D.B * D.C * D.N) {
    const long long bc = idx / D.N, p = idx - bc * D.N;
    const int x = (int)(p % D.nx);
    const long long zy = p / D.nx;
    const float* u = U + (bc * rows + zy) * D.K;
    float acc = 0.f;
    for (int m = 0; m < D.K; m++) acc += __ldg(&E[x * D.K + m]) * u[m];
    out[idx] += acc;
  }
}

// Per-block partial sums of G[o][i] = sum_{b,p} A[b,o,p] Bm[b,i,p] (Bm null:
// ones), over tiles of kTileP points staged in shared memory.
__global__ void __launch_bounds__(kT) gemm_reduce_kernel(const float* __restrict__ A, int Ca,
                                                         const float* __restrict__ Bm, int Cb,
                                                         float* __restrict__ part, Dims D) {
  __shared__ float sa[kMaxC][kTileP + 1], sb[kMaxC][kTileP + 1];
  const long long total = (long long)D.B * D.N;
  const int pairs = Ca * Cb;
  float acc[(kMaxC * kMaxC + kT - 1) / kT];
#pragma unroll
  for (int k = 0; k < (kMaxC * kMaxC + kT - 1) / kT; k++) acc[k] = 0.f;
  for (long long t0 = (long long)blockIdx.x * kTileP; t0 < total; t0 += (long long)gridDim.x * kTileP) {
    __syncthreads();
    for (int e = threadIdx.x; e < kTileP * Ca; e += blockDim.x) {
      const int j = e % kTileP, o = e / kTileP;
      const long long q = t0 + j;
      float val = 0.f;
      if (q < total) {
        const long long b = q / D.N, p = q - b * D.N;
        val = A[(b * Ca + o) * D.N + p];
      }
      sa[o][j] = val;
    }
    for (int e = threadIdx.x; e < kTileP * Cb; e += blockDim.x) {
      const int j = e % kTileP, i = e / kTileP;
      const long long q = t0 + j;
      float val = 0.f;
      if (q < total) {
        const long long b = q / D.N, p = q - b * D.N;
        val = Bm ? Bm[(b * Cb + i) * D.N + p] : 1.f;
      }
      sb[i][j] = val;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < (kMaxC * kMaxC + kT - 1) / kT; k++) {
      const int pr = threadIdx.x + k * kT;
      if (pr < pairs) {
        const int o = pr / Cb, i = pr % Cb;
        float s = 0.f;
        for (int j = 0; j < kTileP; j++) s += sa[o][j] * sb[i][j];
        acc[k] += s;
      }
    }
  }
#pragma unroll
  for (int k = 0; k < (kMaxC * kMaxC + kT - 1) / kT; k++) {
    const int pr = threadIdx.x + k * kT;
    if (pr < pairs) part[(long long)blockIdx.x * pairs + pr] = acc[k];
  }
}

// grad[k] = sum over blocks of part[blk][k] (FP64, fixed order)
__global__ void __launch_bounds__(kT) sum_blocks_kernel(const float* __restrict__ part, int nblk, int pairs,
                                                        float* __restrict__ grad) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < pairs; k += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int b = 0; b < nblk; b++) s += part[(long long)b * pairs + k];
    grad[k] = (float)s;
  }
}

// Relative squared error: S[0] = sum t^2, S[1] = sum (y - t)^2
__global__ void __launch_bounds__(kT) loss_kernel(const float* __restrict__ y, const float* __restrict__ t,
                                                  long long n, pf::Reduce R, double* S) {
  double a = 0.0, b = 0.0;
  GRID_STRIDE_LL(i, n) {
    const double ti = t[i], d = (double)y[i] - ti;
    a += ti * ti;
    b += d * d;
  }
  const double v[2] = {a, b};
  double* const dst[2] = {&S[0], &S[1]};
  pf::grid_sum<2>(v, R, dst);
}

__global__ void __launch_bounds__(kT) loss_grad_kernel(const float* __restrict__ y, const float* __restrict__ t,
                                                       long long n, const double* S, float* __restrict__ dy) {
  const float s = (float)(2.0 / S[0]);
  GRID_STRIDE_LL(i, n) dy[i] = s * (y[i] - t[i]);
}

__global__ void __launch_bounds__(kT) adam_kernel(float* __restrict__ theta, __nv_bfloat16* __restrict__ thb,
                                                  float* __restrict__ m, float* __restrict__ v,
                                                  const float* __restrict__ g, long long n, float lr_t, float b1,
                                                  float b2, float eps) {
  GRID_STRIDE_LL(i, n) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float th = theta[i] - lr_t * mi / (sqrtf(vi) + eps);
    theta[i] = th;
    thb[i] = __float2bfloat16_rn(th);
  }
}

__global__ void __launch_bounds__(kT) to_bf16_kernel(const float* __restrict__ x, __nv_bfloat16* __restrict__ y,
                                                     long long n) {
  GRID_STRIDE_LL(i, n) y[i] = __float2bfloat16_rn(x[i]);
}

}  // namespace

struct poisfft_sno {
  Dims D{};
  Layout lay{};
  int train = 0;
  int sms = 0;
  float* theta = nullptr;         // FP32 master
  __nv_bfloat16* thb = nullptr;   // bfloat16 copy used by the kernels
  float *adam_m = nullptr, *adam_v = nullptr;
  // per-axis matrices: analysis S (K x n), synthesis S_inv (n x K), and the
  // transposes used by the backward pass: S^T (n x K), S_inv^T (K x n)
  float *Sa[3] = {nullptr, nullptr, nullptr}, *Si[3] = {nullptr, nullptr, nullptr};
  float *SaT[3] = {nullptr, nullptr, nullptr}, *SiT[3] = {nullptr, nullptr, nullptr};
  // activations: v[0..L], pre[0..L-1] when training; two buffers otherwise
  std::vector<float*> v, pre;
  float *T1 = nullptr, *T2 = nullptr;   // [B][C][nz][ny][K], [B][C][nz][K][K]
  std::vector<float*> vh;               // [B][C][K^3] per layer (one when not training)
  float *uh = nullptr, *dvh = nullptr;  // [B][C][K^3]
  float *dv = nullptr, *dv2 = nullptr, *dpre = nullptr;
  float *part = nullptr;                // gemm_reduce partials
  int nblk = 0;
  double* S = nullptr;                  // loss scalars
  double* rpart = nullptr;
  unsigned* rcount = nullptr;
  double* hS = nullptr;
};

namespace {

void free_sno(poisfft_sno* s) {
  if (!s) return;
  std::vector<void*> bufs = {s->theta, s->thb, s->adam_m, s->adam_v, s->T1, s->T2, s->uh, s->dvh, s->dv, s->dv2,
                             s->dpre, s->part, s->S, s->rpart, s->rcount};
  for (int a = 0; a < 3; a++) {
    bufs.push_back(s->Sa[a]);
    bufs.push_back(s->Si[a]);
    bufs.push_back(s->SaT[a]);
    bufs.push_back(s->SiT[a]);
  }
  for (float* p : s->v) bufs.push_back(p);
  for (float* p : s->pre) bufs.push_back(p);
  for (float* p : s->vh) bufs.push_back(p);
  for (void* b : bufs) cudaFree(b);
  if (s->hS) cudaFreeHost(s->hS);
  delete s;
}

unsigned grid_for(long long n, int sms) {
  return (unsigned)std::max<long long>(1, std::min<long long>((n + kT - 1) / kT, (long long)sms * 16));
}

// out[row][m] = sum_j M[m][j] in[row][j]; the K = 12 form stages M in smem.
void row_contract(poisfft_sno* s, const float* in, const float* M, float* out, long long rows, int n, int K,
                  cudaStream_t st) {
  const size_t smem = (size_t)K * n * sizeof(float);
  if (K == 12 && smem <= 48 * 1024) {
    row_contract_k_kernel<12><<<grid_for(rows * 32, s->sms), kT, smem, st>>>(in, M, out, rows, n);
  } else {
    row_contract_kernel<<<grid_for(rows * 32, s->sms), kT, 0, st>>>(in, M, out, rows, n, K);
  }
}

// Truncated sine analysis / synthesis along the three axes (forward pass).
void analysis(poisfft_sno* s, const float* v, float* vh, cudaStream_t st) {
  const Dims& D = s->D;
  const long long BC = (long long)D.B * D.C;
  const long long rows = BC * D.nz * D.ny;
  row_contract(s, v, s->Sa[0], s->T1, rows, D.nx, D.K, st);
  axis_contract_kernel<<<grid_for(BC * D.nz * D.K * D.K, s->sms), kT, 0, st>>>(s->T1, s->Sa[1], s->T2, BC * D.nz,
                                                                              D.ny, D.K, D.K);
  axis_contract_kernel<<<grid_for(BC * D.K * D.K * D.K, s->sms), kT, 0, st>>>(s->T2, s->Sa[2], vh, BC, D.nz, D.K,
                                                                             (long long)D.K * D.K);
}

// uhat -> U = [B][C][nz][ny][K] (z then y expansion; x is expanded by the consumer)
void synthesis_zy(poisfft_sno* s, const float* const* mz, const float* uhat, float* U, cudaStream_t st) {
  const Dims& D = s->D;
  const long long BC = (long long)D.B * D.C;
  axis_contract_kernel<<<grid_for(BC * D.nz * D.K * D.K, s->sms), kT, 0, st>>>(uhat, mz[2], s->T2, BC, D.K, D.nz,
                                                                              (long long)D.K * D.K);
  axis_contract_kernel<<<grid_for(BC * D.nz * D.ny * D.K, s->sms), kT, 0, st>>>(s->T2, mz[1], U, BC * D.nz, D.K,
                                                                               D.ny, D.K);
}

// Reduce A (x) Bm over all points into grad[0 .. Ca*Cb).
void weight_grad(poisfft_sno* s, const float* A, int Ca, const float* Bm, int Cb, float* grad, cudaStream_t st) {
  gemm_reduce_kernel<<<s->nblk, kT, 0, st>>>(A, Ca, Bm, Cb, s->part, s->D);
  sum_blocks_kernel<<<(Ca * Cb + kT - 1) / kT, kT, 0, st>>>(s->part, s->nblk, Ca * Cb, grad);
}

int upload_matrix(float** dst, const std::vector<double>& h) {
  std::vector<float> f(h.begin(), h.end());
  if (cudaMalloc(dst, f.size() * sizeof(float)) != cudaSuccess) return POISFFT_ERR_ALLOC;
  return cudaMemcpy(*dst, f.data(), f.size() * sizeof(float), cudaMemcpyHostToDevice) == cudaSuccess
             ? POISFFT_OK
             : POISFFT_ERR_CUDA;
}

}  // namespace

namespace {
template <typename T> bool aligned(const T* p) { return p == nullptr || (uintptr_t)p % sizeof(T) == 0; }
}  // namespace

extern "C" {

int64_t poisfft_sno_num_params(int channels, int modes, int layers) {
  if (channels < 1 || channels > kMaxC || modes < 1 || modes > kMaxK || layers < 1 || layers > kMaxL) return -1;
  return layout_of(channels, modes, layers).total;
}

int poisfft_sno_create(poisfft_sno** out, const int64_t n[3], int batch, int channels, int modes, int layers,
                       int train) {
  if (!out) return POISFFT_ERR_INVALID_ARG;
  *out = nullptr;
  if (!n || batch < 1 || channels < 1 || channels > kMaxC || modes < 1 || modes > kMaxK || layers < 1 ||
      layers > kMaxL)
    return POISFFT_ERR_INVALID_ARG;
  for (int d = 0; d < 3; d++)
    if (n[d] < modes || n[d] > (1 << 16)) return POISFFT_ERR_INVALID_ARG;
  poisfft_sno* s = new (std::nothrow) poisfft_sno();
  if (!s) return POISFFT_ERR_ALLOC;
  Dims& D = s->D;
  D.B = batch;
  D.C = channels;
  D.K = modes;
  D.L = layers;
  D.nx = (int)n[0];
  D.ny = (int)n[1];
  D.nz = (int)n[2];
  D.N = n[0] * n[1] * n[2];
  s->lay = layout_of(channels, modes, layers);
  s->train = train ? 1 : 0;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&s->sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    delete s;
    return POISFFT_ERR_CUDA;
  }
  const long long P = s->lay.total;
  const long long act = (long long)D.B * D.C * D.N;
  const long long K3 = (long long)D.K * D.K * D.K;
  bool ok = cudaMalloc(&s->theta, P * sizeof(float)) == cudaSuccess &&
            cudaMalloc(&s->thb, P * sizeof(__nv_bfloat16)) == cudaSuccess;
  const int nv = s->train ? D.L + 1 : 2;
  s->v.assign(nv, nullptr);
  for (auto& b : s->v) ok = ok && cudaMalloc(&b, act * sizeof(float)) == cudaSuccess;
  s->vh.assign(s->train ? D.L : 1, nullptr);
  for (auto& b : s->vh) ok = ok && cudaMalloc(&b, D.B * D.C * K3 * sizeof(float)) == cudaSuccess;
  ok = ok && cudaMalloc(&s->T1, (long long)D.B * D.C * D.nz * D.ny * D.K * sizeof(float)) == cudaSuccess;
  ok = ok && cudaMalloc(&s->T2, (long long)D.B * D.C * D.nz * D.K * D.K * sizeof(float)) == cudaSuccess;
  ok = ok && cudaMalloc(&s->uh, D.B * D.C * K3 * sizeof(float)) == cudaSuccess;
  if (s->train) {
    s->pre.assign(D.L, nullptr);
    for (auto& b : s->pre) ok = ok && cudaMalloc(&b, act * sizeof(float)) == cudaSuccess;
    ok = ok && cudaMalloc(&s->dv, act * sizeof(float)) == cudaSuccess &&
         cudaMalloc(&s->dv2, act * sizeof(float)) == cudaSuccess &&
         cudaMalloc(&s->dpre, act * sizeof(float)) == cudaSuccess &&
         cudaMalloc(&s->dvh, D.B * D.C * K3 * sizeof(float)) == cudaSuccess &&
         cudaMalloc(&s->adam_m, P * sizeof(float)) == cudaSuccess &&
         cudaMalloc(&s->adam_v, P * sizeof(float)) == cudaSuccess;
    s->nblk = (int)std::min<long long>(((long long)D.B * D.N + kTileP - 1) / kTileP, (long long)s->sms * 4);
    ok = ok && cudaMalloc(&s->part, (long long)s->nblk * kMaxC * kMaxC * sizeof(float)) == cudaSuccess;
  }
  const unsigned rblocks = grid_for((long long)D.B * D.N, s->sms);
  ok = ok && cudaMalloc(&s->S, 2 * sizeof(double)) == cudaSuccess &&
       cudaMalloc(&s->rpart, 2 * rblocks * sizeof(double)) == cudaSuccess &&
       cudaMalloc(&s->rcount, sizeof(unsigned)) == cudaSuccess &&
       cudaMallocHost(&s->hS, 2 * sizeof(double)) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    free_sno(s);
    return POISFFT_ERR_ALLOC;
  }
  // sine matrices from FP64 host arithmetic
  const int nn[3] = {D.nx, D.ny, D.nz};
  for (int a = 0; a < 3; a++) {
    const int na = nn[a], K = D.K;
    std::vector<double> Sa((size_t)K * na), Si((size_t)na * K), SaT((size_t)na * K), SiT((size_t)K * na);
    for (int m = 0; m < K; m++)
      for (int j = 0; j < na; j++) {
        // sin(pi (m+1)(2j+1) / (2n)) with the argument reduced exactly mod 4n
        const long long r = ((long long)(m + 1) * (2 * j + 1)) % (4LL * na);
        const double sv = sin(M_PI * (double)r / (2.0 * na));
        Sa[(size_t)m * na + j] = 2.0 / na * sv;
        SiT[(size_t)m * na + j] = sv;
        Si[(size_t)j * K + m] = sv;
        SaT[(size_t)j * K + m] = 2.0 / na * sv;
      }
    int rc;
    if ((rc = upload_matrix(&s->Sa[a], Sa)) != POISFFT_OK || (rc = upload_matrix(&s->Si[a], Si)) != POISFFT_OK ||
        (rc = upload_matrix(&s->SaT[a], SaT)) != POISFFT_OK || (rc = upload_matrix(&s->SiT[a], SiT)) != POISFFT_OK) {
      free_sno(s);
      return rc;
    }
  }
  if (cudaMemset(s->rcount, 0, sizeof(unsigned)) != cudaSuccess ||
      cudaMemset(s->theta, 0, P * sizeof(float)) != cudaSuccess ||
      cudaMemset(s->thb, 0, P * sizeof(__nv_bfloat16)) != cudaSuccess ||
      (s->train && (cudaMemset(s->adam_m, 0, P * sizeof(float)) != cudaSuccess ||
                    cudaMemset(s->adam_v, 0, P * sizeof(float)) != cudaSuccess))) {
    free_sno(s);
    return POISFFT_ERR_CUDA;
  }
  *out = s;
  return POISFFT_OK;
}

int poisfft_sno_set_params(poisfft_sno* s, const float* theta) {
  if (!s || !theta) return POISFFT_ERR_INVALID_ARG;
  const long long P = s->lay.total;
  if (cudaMemcpy(s->theta, theta, P * sizeof(float), cudaMemcpyDefault) != cudaSuccess) return POISFFT_ERR_CUDA;
  to_bf16_kernel<<<grid_for(P, s->sms), kT>>>(s->theta, s->thb, P);
  if (s->train && (cudaMemset(s->adam_m, 0, P * sizeof(float)) != cudaSuccess ||
                   cudaMemset(s->adam_v, 0, P * sizeof(float)) != cudaSuccess))
    return POISFFT_ERR_CUDA;
  return cudaDeviceSynchronize() == cudaSuccess ? POISFFT_OK : POISFFT_ERR_CUDA;
}

int poisfft_sno_get_params(const poisfft_sno* s, float* theta) {
  if (!s || !theta) return POISFFT_ERR_INVALID_ARG;
  return cudaMemcpy(theta, s->theta, s->lay.total * sizeof(float), cudaMemcpyDefault) == cudaSuccess
             ? POISFFT_OK
             : POISFFT_ERR_CUDA;
}

int poisfft_sno_forward(poisfft_sno* s, float* y, const float* feats, void* stream) {
  if (!s || !y || !feats) return POISFFT_ERR_INVALID_ARG;
  if (!aligned(y) || !aligned(feats)) return POISFFT_ERR_MISALIGNED;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const Dims& D = s->D;
  const Layout& O = s->lay;
  const long long pts = (long long)D.B * D.N;
  const unsigned gp = grid_for(pts, s->sms);
  float* cur = s->v[0];
  lift_kernel<<<gp, kT, 0, st>>>(feats, s->thb, O.P, O.p, cur, D);
  for (int l = 0; l < D.L; l++) {
    float* vh = s->train ? s->vh[l] : s->vh[0];
    float* nxt = s->train ? s->v[l + 1] : s->v[(l + 1) & 1];
    analysis(s, cur, vh, st);
    mix_kernel<<<grid_for((long long)D.B * D.C * D.K * D.K * D.K, s->sms), kT, 0, st>>>(
        vh, s->thb, O.R[l], s->uh, D.B, D.C, D.K * D.K * D.K);
    synthesis_zy(s, s->Si, s->uh, s->T1, st);
    float* pre = s->train ? s->pre[l] : nullptr;
    const int act = l < D.L - 1 ? 1 : 0;
    if (D.C == 16 && D.K == 12 && D.nx >= 32)
      point_ck_kernel<16, 12><<<grid_for((long long)D.B * D.nz * D.ny * 32, s->sms), kT, 0, st>>>(
          cur, s->T1, s->Si[0], s->thb, O.W[l], O.b[l], pre, nxt, act, D);
    else
      point_kernel<<<gp, kT, 0, st>>>(cur, s->T1, s->Si[0], s->thb, O.W[l], O.b[l], pre, nxt, act, D);
    cur = nxt;
  }
  proj_kernel<<<gp, kT, 0, st>>>(cur, s->thb, O.Q, O.q, y, D);
  return cudaGetLastError() == cudaSuccess ? POISFFT_OK : POISFFT_ERR_CUDA;
}

int poisfft_sno_backward(poisfft_sno* s, float* grad, const float* dy, const float* feats, void* stream) {
  if (!s || !grad || !dy || !feats) return POISFFT_ERR_INVALID_ARG;
  if (!s->train) return POISFFT_ERR_INVALID_ARG;
  if (!aligned(grad) || !aligned(dy) || !aligned(feats)) return POISFFT_ERR_MISALIGNED;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const Dims& D = s->D;
  const Layout& O = s->lay;
  const long long pts = (long long)D.B * D.N;
  const unsigned gp = grid_for(pts, s->sms);
  const int M3 = D.K * D.K * D.K;
  const long long BC = (long long)D.B * D.C;
  // projection
  weight_grad(s, dy, 1, s->v[D.L], D.C, grad + O.Q, st);
  weight_grad(s, dy, 1, nullptr, 1, grad + O.q, st);
  proj_bwd_kernel<<<gp, kT, 0, st>>>(dy, s->thb, O.Q, s->dv, D);
  float* dvn = s->dv;   // gradient of v_{l+1}
  float* dvc = s->dv2;  // gradient of v_l (being built)
  for (int l = D.L - 1; l >= 0; l--) {
    point_bwd_kernel<<<gp, kT, 0, st>>>(dvn, s->pre[l], s->thb, O.W[l], l < D.L - 1 ? 1 : 0, s->dpre, dvc, D);
    weight_grad(s, s->dpre, D.C, s->v[l], D.C, grad + O.W[l], st);
    weight_grad(s, s->dpre, D.C, nullptr, 1, grad + O.b[l], st);
    // spectral path: duh = S_inv^T(dpre)
    const long long rows = BC * D.nz * D.ny;
    row_contract(s, s->dpre, s->SiT[0], s->T1, rows, D.nx, D.K, st);
    axis_contract_kernel<<<grid_for(BC * D.nz * D.K * D.K, s->sms), kT, 0, st>>>(s->T1, s->SiT[1], s->T2,
                                                                                BC * D.nz, D.ny, D.K, D.K);
    axis_contract_kernel<<<grid_for(BC * M3, s->sms), kT, 0, st>>>(s->T2, s->SiT[2], s->uh, BC, D.nz, D.K,
                                                                  (long long)D.K * D.K);
    mix_grad_kernel<<<grid_for((long long)M3 * D.C * D.C, s->sms), kT, 0, st>>>(s->uh, s->vh[l], grad + O.R[l], D.B,
                                                                               D.C, M3);
    // dvh = R^T duh, then dv_l += S^T(dvh): expand z, then y, then x (added)
    mix_t_kernel<<<grid_for(BC * M3, s->sms), kT, 0, st>>>(s->uh, s->thb, O.R[l], s->dvh, D.B, D.C, M3);
    axis_contract_kernel<<<grid_for(BC * D.nz * D.K * D.K, s->sms), kT, 0, st>>>(s->dvh, s->SaT[2], s->T2, BC, D.K,
                                                                                D.nz, (long long)D.K * D.K);
    axis_contract_kernel<<<grid_for(BC * D.nz * D.ny * D.K, s->sms), kT, 0, st>>>(s->T2, s->SaT[1], s->T1,
                                                                                 BC * D.nz, D.K, D.ny, D.K);
    expand_add_kernel<<<grid_for(BC * D.N, s->sms), kT, 0, st>>>(s->T1, s->SaT[0], dvc, D);
    std::swap(dvn, dvc);
  }
  // lifting: dvn holds the gradient of v_0
  weight_grad(s, dvn, D.C, feats, kF, grad + O.P, st);
  weight_grad(s, dvn, D.C, nullptr, 1, grad + O.p, st);
  return cudaGetLastError() == cudaSuccess ? POISFFT_OK : POISFFT_ERR_CUDA;
}

int poisfft_sno_loss(poisfft_sno* s, const float* y, const float* t, float* dy, double* loss, void* stream) {
  if (!s || !y || !t) return POISFFT_ERR_INVALID_ARG;
  if (!aligned(y) || !aligned(t) || !aligned(dy)) return POISFFT_ERR_MISALIGNED;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const long long n = (long long)s->D.B * s->D.N;
  const unsigned gb = grid_for(n, s->sms);
  loss_kernel<<<gb, kT, 0, st>>>(y, t, n, pf::Reduce{s->rpart, s->rcount}, s->S);
  if (dy) loss_grad_kernel<<<gb, kT, 0, st>>>(y, t, n, s->S, dy);
  if (cudaGetLastError() != cudaSuccess) return POISFFT_ERR_CUDA;
  if (loss) {
    if (cudaMemcpyAsync(s->hS, s->S, 2 * sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return POISFFT_ERR_CUDA;
    *loss = s->hS[0] > 0.0 ? s->hS[1] / s->hS[0] : 0.0;
  }
  return POISFFT_OK;
}

int poisfft_sno_adam(poisfft_sno* s, const float* grad, double lr, double beta1, double beta2, double eps, int step,
                     void* stream) {
  if (!s || !grad || !s->train || step < 1) return POISFFT_ERR_INVALID_ARG;
  if (!aligned(grad)) return POISFFT_ERR_MISALIGNED;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const double lr_t = lr * sqrt(1.0 - pow(beta2, step)) / (1.0 - pow(beta1, step));
  const long long P = s->lay.total;
  adam_kernel<<<grid_for(P, s->sms), kT, 0, st>>>(s->theta, s->thb, s->adam_m, s->adam_v, grad, P, (float)lr_t,
                                                   (float)beta1, (float)beta2, (float)eps);
  return cudaGetLastError() == cudaSuccess ? POISFFT_OK : POISFFT_ERR_CUDA;
}

int poisfft_sno_info(const poisfft_sno* s, int64_t out[8]) {
  if (!s || !out) return POISFFT_ERR_INVALID_ARG;
  const int64_t v[8] = {s->D.nx, s->D.ny, s->D.nz, s->D.B, s->D.C, s->D.K, s->D.L, s->train};
  for (int i = 0; i < 8; i++) out[i] = v[i];
  return POISFFT_OK;
}

int poisfft_sno_destroy(poisfft_sno* s) {
  free_sno(s);
  return POISFFT_OK;
}

}  // extern "C"
