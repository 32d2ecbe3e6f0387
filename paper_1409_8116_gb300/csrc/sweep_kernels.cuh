// Sweep kernels of the direct Poisson solve (Sec. 2.1 algorithm, Sec. 2.3
// multi-D sequence of 1D transforms).
//
//   x_sweep        contiguous axis.  Two field rows per complex line.
//                  Periodic x: R2C / C2R through the two-for-one split
//                  A_k = (Z_k + conj Z_{n-k})/2, B_k = (Z_k - conj Z_{n-k})/(2i).
//   strided_sweep  y or z axis of the workspace.  The tile [axis x w columns]
//                  arrives in shared memory by TMA (cp.async.bulk.tensor, one
//                  box of up to 256 axis rows per copy, no multicast), is
//                  transformed in place and written back with coalesced
//                  row stores.  Mode 2 fuses forward transform, the eigenvalue
//                  divide of step 2 (with the zero-mode fix) and the backward
//                  transform, so the last axis costs one HBM round trip.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "fft_engine.cuh"
#include "internal.h"

namespace pf {

template <typename T> struct Emax;
template <> struct Emax<float> { static constexpr int value = 40; };
template <> struct Emax<double> { static constexpr int value = 16; };

// ---------------------------------------------------------------------------
// contiguous (x) sweep
// ---------------------------------------------------------------------------
// Three CTAs per SM (80 registers, a few hundred bytes of spills): the sweep
// waits on its loads, and the third CTA hides more of that latency than the
// spills cost (512^3, x forward 0.85 -> 0.69 ms before the cp.async staging).
// One CTA's work (line pairs bid * lines ...) of the contiguous sweep; the
// kernel below runs it for blockIdx.x, the batch phase kernel for the tiles
// it takes from its work list.
template <typename T>
__device__ __forceinline__ void x_sweep_body(const XArgs& a, const int bid) {
  constexpr int EMAX = Emax<T>::value;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  cx<T>* buf = reinterpret_cast<cx<T>*>(smem_raw);
  // padding shift of the row tiles: 16 float or 8 double complex values per bank sweep
  constexpr int PSH = sizeof(T) == 4 ? 4 : 3;
  const RowTile lay{a.ld, PSH};
  cx<T>* scratch = buf + (size_t)a.lines * a.ld;  // direct-DFT scratch or the Bluestein buffer
  const cx<T>* tables = reinterpret_cast<const cx<T>*>(a.tables);
  const cx<T>* mk = a.ax.mk_off >= 0 ? tables + a.ax.mk_off : nullptr;
  const int* perm = a.perm;
  const int nx = a.nx;
  const int M = a.ax.fft.M;
  const long long row0 = (long long)bid * 2 * a.lines;
  const int kind = a.mode == 0 ? a.ax.kfwd : a.ax.kinv;
  // field row r = y + ny*z of the CTA's first line; later rows by one 32-bit
  // fast division of (y0 + offset) by ny
  const long long z0 = row0 / a.ny;
  const int y0 = (int)(row0 - z0 * a.ny);
  auto field_offset = [&](int dr, long long sy, long long sz) {
    const uint32_t yy = (uint32_t)(y0 + dr);
    const uint32_t dz = fdiv(yy, a.dny);
    return (long long)(yy - dz * (uint32_t)a.ny) * sy + (z0 + dz) * sz;
  };

  // ---- stage A: bring the source lines into smem
  if (a.mode == 0 || !a.r2c) {
    // complex line (row a, row b) in source order
    const T* src = reinterpret_cast<const T*>(a.mode == 0 ? a.g : a.ws);
    const int total = a.lines * nx;
    // element copies straight into the real / imaginary slots (no register
    // round trip, every load of the tile in flight at once); rows past the
    // end are zero-filled
    for (int e = threadIdx.x; e < total; e += kThreads) {
      const int l = (int)fdiv((uint32_t)e, a.dnx);
      const int j = e - l * nx;
      const long long ra = row0 + 2 * l, rb = ra + 1;
      // g rows may sit inside a larger array (strides g_sy, g_sz)
      const long long oa = a.mode == 0 ? field_offset(2 * l, a.g_sy, a.g_sz) : ra * a.ws_ld;
      const long long ob = a.mode == 0 ? field_offset(2 * l + 1, a.g_sy, a.g_sz) : rb * a.ws_ld;
      T* d = reinterpret_cast<T*>(&buf[lay.idx(j, l)]);
      cp_async_elem<sizeof(T)>(d, ra < a.nrows ? src + oa + j : src, ra < a.nrows);
      cp_async_elem<sizeof(T)>(d + 1, rb < a.nrows ? src + ob + j : src, rb < a.nrows);
    }
    cp_async_wait_all();
  } else {
    // C2R assembly: Z_k = A_k + i B_k and Z_{n-k} = conj(A_k) + i conj(B_k)
    const cx<T>* src = reinterpret_cast<const cx<T>*>(a.ws);
    const int nh = nx / 2 + 1;
    const int total = a.lines * nh;
    for (int e = threadIdx.x; e < total; e += kThreads) {
      const int l = (int)fdiv((uint32_t)e, a.dnh);
      const int k = e - l * nh;
      const long long ra = row0 + 2 * l, rb = ra + 1;
      const cx<T> A = ra < a.nrows ? src[ra * a.ws_ld + k] : czero<T>();
      const cx<T> B = rb < a.nrows ? src[rb * a.ws_ld + k] : czero<T>();
      if (k == 0 || 2 * k == nx) {
        buf[lay.idx(k, l)] = mkc<T>(A.x, B.x);  // Hermitian: real parts only
      } else {
        buf[lay.idx(k, l)] = mkc<T>(A.x - B.y, A.y + B.x);
        buf[lay.idx(nx - k, l)] = mkc<T>(A.x + B.y, B.x - A.y);
      }
    }
  }
  __syncthreads();

  // ---- stage B/C: pre-processing gather and the FFT (in place, or Bluestein
  // from the source lines into the convolution buffer)
  cx<T>* res = buf;
  RowTile lres = lay;
  if (a.ax.blu) {
    lres = RowTile{M + (M >> PSH), PSH};
    bluestein_fft<T, EMAX>(buf, lay, scratch, lres, a.ax, kind, nx, a.lines, tables, mk);
    res = scratch;
  } else {
    pre_tile<T, EMAX>(buf, lay, kind, nx, a.ax.fft.dM, a.lines, mk);
    run_passes<T, EMAX>(buf, scratch, lay, a.ax.fft, a.lines, tables, kind_uses_inverse_fft(kind));
  }

  // ---- stage D: post-processing and store
  if (a.mode == 0 && a.r2c) {
    cx<T>* dst = reinterpret_cast<cx<T>*>(a.ws);
    const int nh = nx / 2 + 1;
    const int total = a.lines * nh;
    for (int e = threadIdx.x; e < total; e += kThreads) {
      const int l = (int)fdiv((uint32_t)e, a.dnh);
      const int k = e - l * nh;
      const long long ra = row0 + 2 * l, rb = ra + 1;
      const cx<T> z1 = res[lres.idx(perm[k], l)];
      const cx<T> z2 = res[lres.idx(perm[k == 0 ? 0 : nx - k], l)];
      // A = (z1 + conj z2)/2,  B = (z1 - conj z2)/(2i)
      const cx<T> A = mkc<T>(T(0.5) * (z1.x + z2.x), T(0.5) * (z1.y - z2.y));
      const cx<T> B = mkc<T>(T(0.5) * (z1.y + z2.y), T(0.5) * (z2.x - z1.x));
      if (ra < a.nrows) dst[ra * a.ws_ld + k] = A;
      if (rb < a.nrows) dst[rb * a.ws_ld + k] = B;
    }
  } else {
    T* dst = reinterpret_cast<T*>(a.mode == 0 ? a.ws : a.phi);
    const int total = a.lines * nx;
    with_kind(kind, [&](auto kc) {
      for (int e = threadIdx.x; e < total; e += kThreads) {
        const int l = (int)fdiv((uint32_t)e, a.dnx);
        const int k = e - l * nx;
        const long long ra = row0 + 2 * l, rb = ra + 1;
        const long long oa = a.mode == 0 ? ra * a.ws_ld : field_offset(2 * l, a.phi_sy, a.phi_sz);
        const long long ob = a.mode == 0 ? rb * a.ws_ld : field_offset(2 * l + 1, a.phi_sy, a.phi_sz);
        const cx<T> v = post_value<T>(res, lres, decltype(kc)::value, nx, k, l, mk, perm);
        if (ra < a.nrows) dst[oa + k] = v.x;
        if (rb < a.nrows) dst[ob + k] = v.y;
        // odd nx: the padding half of the last packed column starts every solve
        // at zero (a periodic y/z DFT would otherwise leave rounding noise there)
        if (a.mode == 0 && k == nx - 1 && (nx & 1)) {
          if (ra < a.nrows) dst[oa + nx] = T(0);
          if (rb < a.nrows) dst[ob + nx] = T(0);
        }
      }
    });
  }
}

template <typename T>
__global__ void __launch_bounds__(kThreads, 3) x_sweep_kernel(const XArgs a) {
  x_sweep_body<T>(a, blockIdx.x);
}

// ---------------------------------------------------------------------------
// strided (y / z) sweep with TMA-staged tiles
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T eigen_factor(const StridedArgs& a, const T* lin, const T* lax, const T* lout, int kx, int k,
                                          int o) {
  if (kx >= a.nx) return T(0);
  if (a.singular && kx == 0 && k == 0 && o == 0) return T(0);
  const T den = lin[kx] + lax[k] + lout[o];
  return T(a.scale) / den;
}

// Eigenvalue factors of one workspace column at outer index o: the real
// part (and, for packed real x columns, the imaginary part separately) of a
// spectral value at axis index k is multiplied by
// s / (lam_in[kx] + lam_ax[k] + lam_out[o]), 0 for padding columns and for the
// zero mode of a singular problem.
template <typename T>
struct ColumnDivide {
  const T* lax;
  T s, ba, bb;
  bool oka, okb, za, zb;
  __device__ __forceinline__ ColumnDivide(const StridedArgs& a, int col, int o) {
    const T* lin = reinterpret_cast<const T*>(a.lam_in);
    const T lo = reinterpret_cast<const T*>(a.lam_out)[o];
    lax = reinterpret_cast<const T*>(a.lam_ax);
    s = T(a.scale);
    const int kxa = a.packed ? 2 * col : col;
    const int kxb = a.packed ? 2 * col + 1 : col;
    oka = kxa < a.nx;
    okb = kxb < a.nx;
    ba = oka ? lin[kxa] + lo : T(1);
    bb = okb ? lin[kxb] + lo : T(1);
    za = a.singular && kxa == 0 && o == 0;
    zb = a.singular && kxb == 0 && o == 0;
  }
  __device__ __forceinline__ cx<T> operator()(cx<T> x, int k) const {
    const T l = lax[k];
    const T fa = (oka && !(za && k == 0)) ? s / (ba + l) : T(0);
    const T fb = (okb && !(zb && k == 0)) ? s / (bb + l) : T(0);
    return mkc<T>(x.x * fa, x.y * fb);
  }
};

// Fused middle step of the strided sweep in the digit-reversed layout left by
// the forward DIF passes: post-processing of the forward transform, the
// eigenvalue divide and pre-processing of the backward transform, computed
// in place for the pair of FFT indices that each output depends on, so that
// the backward FFT runs as DIT passes (digit-reversed input, natural output).
//   DCT-II -> DCT-III  (n points, pairs m, n-m):
//     P_j = w_j Y_j + conj(w_j) Y_{n-j}  (the DCT-II value j, w_j = exp(-i pi j/2n)),
//     V_m = conj(w_m) (d(m) P_m - i d(n-m) P_{n-m}),  d(n) P_n := 0
//   DST-II -> DST-III: the same with d(j) -> d(n-1-j) (DST-II output k is
//     DCT-II value n-1-k; DST-III input j is read at n-1-j)
//   DST-I (M = 2(n+1)): X_k = i Y_{k+1};  V_m = d(m-1) X_{m-1} = -V_{M-m}, V_0 = V_{n+1} = 0
//   DCT-I (M = 2(n-1)): X_k = Y_k;  V_m = V_{M-m} = d(m) Y_m
//   DFT / length 1: V_k = d(k) Y_k
// Ends with a barrier.
template <typename T, class LAY>
__device__ __forceinline__ void fused_divide_pairs(cx<T>* buf, const LAY lay, int kfwd, int n, int M, int c, int g0,
                                                   int G, const ColumnDivide<T>& D, const cx<T>* __restrict__ mk,
                                                   const int* __restrict__ perm) {
  switch (kfwd) {
    case TK_DCT2:
    case TK_DST2: {
      const bool ds = kfwd == TK_DST2;
      for (int m = g0; 2 * m <= n; m += G) {
        const int mp = m == 0 ? 0 : n - m;
        const int pm = perm[m], pp = perm[mp];
        const cx<T> ym = buf[lay.idx(pm, c)];
        const cx<T> yp = buf[lay.idx(pp, c)];
        const cx<T> wm = mk[m], wp = mk[mp];
        const cx<T> Pm = cadd<T>(cmul<T>(wm, ym), cmulc<T>(yp, wm));
        const cx<T> Pp = cadd<T>(cmul<T>(wp, yp), cmulc<T>(ym, wp));
        const cx<T> fm = D(Pm, ds ? n - 1 - m : m);
        const cx<T> fp = m == 0 ? czero<T>() : D(Pp, ds ? m - 1 : n - m);
        buf[lay.idx(pm, c)] = cmulc<T>(mkc<T>(fm.x + fp.y, fm.y - fp.x), wm);  // conj(w_m)(f_m - i f_{n-m})
        if (m != 0 && mp != m) buf[lay.idx(pp, c)] = cmulc<T>(mkc<T>(fp.x + fm.y, fp.y - fm.x), wp);
      }
      break;
    }
    case TK_DST1:
      for (int m = g0; m <= n + 1; m += G) {
        if (m == 0 || m == n + 1) {
          buf[lay.idx(perm[m], c)] = czero<T>();
          continue;
        }
        const int pm = perm[m];
        const cx<T> f = D(mul_i<T>(buf[lay.idx(pm, c)]), m - 1);
        buf[lay.idx(pm, c)] = f;
        buf[lay.idx(perm[M - m], c)] = mkc<T>(-f.x, -f.y);
      }
      break;
    case TK_DCT1:
      for (int m = g0; m < n; m += G) {
        const int pm = perm[m];
        const cx<T> f = D(buf[lay.idx(pm, c)], m);
        buf[lay.idx(pm, c)] = f;
        if (m >= 1 && m <= n - 2) buf[lay.idx(perm[M - m], c)] = f;
      }
      break;
    default:
      for (int k = g0; k < M; k += G) {
        const int pk = perm[k];
        buf[lay.idx(pk, c)] = D(buf[lay.idx(pk, c)], k);
      }
      break;
  }
  __syncthreads();
}

// Three CTAs per SM (80 registers; the staging arrays of the pre-processing
// spill to L1): 512 uneven batch problems 63.9 -> 60.8 ms against two CTAs
// per SM with a 128-register cap (which in turn beat one CTA without a cap).
// One tile (bid) of the strided sweep.  `bar` is an initialised mbarrier
// whose phase `parity` completes when the tile's TMA boxes have landed; the
// kernel below runs one tile per CTA, the batch phase kernel many.  Returns
// false (uniformly) when the bounded wait for the boxes gave up.
template <typename T>
__device__ __forceinline__ bool strided_sweep_body(const CUtensorMap* tmap, const StridedArgs& a, const int bid,
                                                   uint64_t* bar, const uint32_t parity) {
  constexpr int EMAX = Emax<T>::value;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  cx<T>* buf = reinterpret_cast<cx<T>*>(smem_raw);
  const ColTile lay{a.w, a.lw};
  cx<T>* scratch = buf + (size_t)a.rows_alloc * a.w;  // direct-DFT scratch or the Bluestein buffer
  const cx<T>* tables = reinterpret_cast<const cx<T>*>(a.tables);
  const cx<T>* mk = a.ax.mk_off >= 0 ? tables + a.ax.mk_off : nullptr;
  const int* perm = a.perm;
  const int n = a.ax.n;
  const int tcol = bid % a.ntile_c;
  const int outer = bid / a.ntile_c;
  const int c0 = tcol * a.w;

  // ---- stage A: TMA boxes of the tile
  if (threadIdx.x == 0) {
    const uint32_t box_bytes = (uint32_t)(2 * a.w * a.box_h * sizeof(T));
    mbar_arrive_expect_tx(bar, box_bytes * a.nbox);
    for (int b = 0; b < a.nbox; b++) {
      cx<T>* dst = buf + (size_t)b * a.box_h * a.w;
      if (a.axis_dim == 1)
        tma_load_3d(dst, tmap, bar, 2 * c0, b * a.box_h, outer);
      else
        tma_load_3d(dst, tmap, bar, 2 * c0, outer, b * a.box_h);
    }
  }
  const bool ok = mbar_wait_bounded(bar, parity);
  if (__syncthreads_or(!ok)) {
    if (threadIdx.x == 0) atomicExch(a.err, 1);
    return false;
  }

  cx<T>* out = reinterpret_cast<cx<T>*>(a.data) + (size_t)outer * a.s_outer + c0;
  const int ncol_valid = a.ncols - c0 < a.w ? a.ncols - c0 : a.w;

  if (a.mode != 2) {
    const int kind = a.mode == 0 ? a.ax.kfwd : a.ax.kinv;
    cx<T>* res = buf;
    if (a.ax.blu) {
      bluestein_fft<T, EMAX>(buf, lay, scratch, lay, a.ax, kind, n, a.w, tables, mk);
      res = scratch;
    } else {
      pre_tile<T, EMAX>(buf, lay, kind, n, a.ax.fft.dM, a.w, mk);
      run_passes<T, EMAX>(buf, scratch, lay, a.ax.fft, a.w, tables, kind_uses_inverse_fft(kind));
    }
    // w divides kThreads: every thread keeps one column
    const int c = threadIdx.x & (a.w - 1);
    if (c < ncol_valid) {
      const int G = kThreads >> a.lw;
      with_kind(kind, [&](auto kc) {
        for (int k = threadIdx.x >> a.lw; k < n; k += G)
          out[(size_t)k * a.s_axis + c] = post_value<T>(res, lay, decltype(kc)::value, n, k, c, mk, perm);
      });
    }
    return true;
  }

  if (a.ax.blu) {
    // fused, Bluestein: forward into the buffer, divided spectrum back into
    // the source rows, backward from there
    const T* lin = reinterpret_cast<const T*>(a.lam_in);
    const T* lax = reinterpret_cast<const T*>(a.lam_ax);
    const T* lout = reinterpret_cast<const T*>(a.lam_out);
    bluestein_fft<T, EMAX>(buf, lay, scratch, lay, a.ax, a.ax.kfwd, n, a.w, tables, mk);
    const int total = n * a.w;
    for (int e = threadIdx.x; e < total; e += kThreads) {
      const int c = e & (a.w - 1);
      const int k = e >> a.lw;
      cx<T> x = post_value<T>(scratch, lay, a.ax.kfwd, n, k, c, mk, perm);
      const int col = c0 + c;
      if (a.packed) {
        x.x *= eigen_factor<T>(a, lin, lax, lout, 2 * col, k, outer);
        x.y *= eigen_factor<T>(a, lin, lax, lout, 2 * col + 1, k, outer);
      } else {
        const T f = eigen_factor<T>(a, lin, lax, lout, col, k, outer);
        x.x *= f;
        x.y *= f;
      }
      buf[lay.idx(k, c)] = x;
    }
    __syncthreads();
    bluestein_fft<T, EMAX>(buf, lay, scratch, lay, a.ax, a.ax.kinv, n, a.w, tables, mk);
    for (int e = threadIdx.x; e < total; e += kThreads) {
      const int c = e & (a.w - 1);
      const int k = e >> a.lw;
      if (c < ncol_valid) out[(size_t)k * a.s_axis + c] = post_value<T>(scratch, lay, a.ax.kinv, n, k, c, mk, perm);
    }
    return true;
  }

  if (a.dit_fused) {
    // ---- fused: forward (DIF), pairwise divide in place, backward (DIT)
    pre_tile<T, EMAX>(buf, lay, a.ax.kfwd, n, a.ax.fft.dM, a.w, mk);
    run_passes<T, EMAX>(buf, scratch, lay, a.ax.fft, a.w, tables, kind_uses_inverse_fft(a.ax.kfwd));
    const int c = threadIdx.x & (a.w - 1);
    const int g0 = threadIdx.x >> a.lw, G = kThreads >> a.lw;
    const ColumnDivide<T> D(a, c0 + c, outer);
    fused_divide_pairs<T>(buf, lay, a.ax.kfwd, n, a.ax.fft.M, c, g0, G, D, mk, perm);
    if (kind_uses_inverse_fft(a.ax.kinv))
      run_passes_dit<T, true, EMAX>(buf, lay, a.ax.fft, a.w, tables);
    else
      run_passes_dit<T, false, EMAX>(buf, lay, a.ax.fft, a.w, tables);
    if (c < ncol_valid) {
      with_kind(a.ax.kinv, [&](auto kc) {
        for (int k = g0; k < n; k += G)
          out[(size_t)k * a.s_axis + c] = post_value<T, true>(buf, lay, decltype(kc)::value, n, k, c, mk, perm);
      });
    }
    return true;
  }

  // ---- fused (plans with a direct-DFT pass): forward, divide by the eigenvalues, backward
  pre_tile<T, EMAX>(buf, lay, a.ax.kfwd, n, a.ax.fft.dM, a.w, mk);
  run_passes<T, EMAX>(buf, scratch, lay, a.ax.fft, a.w, tables, kind_uses_inverse_fft(a.ax.kfwd));
  {
    const T* lin = reinterpret_cast<const T*>(a.lam_in);
    const T* lax = reinterpret_cast<const T*>(a.lam_ax);
    const T* lout = reinterpret_cast<const T*>(a.lam_out);
    cx<T> v[EMAX];
    const int total = n * a.w;
#pragma unroll
    for (int j = 0; j < EMAX; j++) {
      const int e = threadIdx.x + j * kThreads;
      if (e < total) {
        const int c = e & (a.w - 1);
        const int k = e >> a.lw;
        cx<T> x = post_value<T>(buf, lay, a.ax.kfwd, n, k, c, mk, perm);
        const int col = c0 + c;
        if (a.packed) {
          x.x *= eigen_factor<T>(a, lin, lax, lout, 2 * col, k, outer);
          x.y *= eigen_factor<T>(a, lin, lax, lout, 2 * col + 1, k, outer);
        } else {
          const T f = eigen_factor<T>(a, lin, lax, lout, col, k, outer);
          x.x *= f;
          x.y *= f;
        }
        v[j] = x;
      }
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < EMAX; j++) {
      const int e = threadIdx.x + j * kThreads;
      if (e < total) buf[lay.idx(e >> a.lw, e & (a.w - 1))] = v[j];
    }
    __syncthreads();
  }
  pre_tile<T, EMAX>(buf, lay, a.ax.kinv, n, a.ax.fft.dM, a.w, mk);
  run_passes<T, EMAX>(buf, scratch, lay, a.ax.fft, a.w, tables, kind_uses_inverse_fft(a.ax.kinv));
  const int total = n * a.w;
  for (int e = threadIdx.x; e < total; e += kThreads) {
    const int c = e & (a.w - 1);
    const int k = e >> a.lw;
    if (c < ncol_valid) out[(size_t)k * a.s_axis + c] = post_value<T>(buf, lay, a.ax.kinv, n, k, c, mk, perm);
  }
  return true;
}

template <typename T>
__global__ void __launch_bounds__(kThreads, 3) strided_sweep_kernel(const __grid_constant__ CUtensorMap tmap,
                                                                 const StridedArgs a) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw + a.bar_off);
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  strided_sweep_body<T>(&tmap, a, blockIdx.x, bar, 0);
}

// ---------------------------------------------------------------------------
// eigenvalue divide for packed real x columns with periodic y or z
// ---------------------------------------------------------------------------
// Block (bx, by) of a gx x gy grid of 256-thread blocks: bx covers one (c, y)
// plane, by strides over z with step gy.
template <typename T>
__device__ __forceinline__ void pair_divide_body(const PairDivideArgs& a, int bx, int by, int gy) {
  const uint32_t e = bx * 256u + threadIdx.x;
  if (e >= (uint32_t)a.ncols * (uint32_t)a.ny) return;
  const int y = (int)fdiv(e, a.dncols);
  const int c = (int)(e - (uint32_t)y * (uint32_t)a.ncols);
  const int yn = a.per_y ? (y == 0 ? 0 : a.ny - y) : y;
  for (int z = by; z < a.nz; z += gy) {
    const int zn = a.per_z ? (z == 0 ? 0 : a.nz - z) : z;
    if (z > zn || (z == zn && y > yn)) continue;  // the mirror element's thread does the pair
    cx<T>* ws = reinterpret_cast<cx<T>*>(a.data);
    const long long i1 = ((long long)z * a.ny + y) * a.pitch + c;
    const long long i2 = ((long long)zn * a.ny + yn) * a.pitch + c;
    const cx<T> z1 = ws[i1];
    const cx<T> z2 = ws[i2];
    // A(k) = (Z1 + conj Z2)/2, B(k) = (Z1 - conj Z2)/(2i)
    const cx<T> A = mkc<T>(T(0.5) * (z1.x + z2.x), T(0.5) * (z1.y - z2.y));
    const cx<T> B = mkc<T>(T(0.5) * (z1.y + z2.y), T(0.5) * (z2.x - z1.x));
    const T* lx = reinterpret_cast<const T*>(a.lam_x);
    const T lyz = reinterpret_cast<const T*>(a.lam_y)[y] + reinterpret_cast<const T*>(a.lam_z)[z];
    const int kxa = 2 * c, kxb = 2 * c + 1;
    T fa = T(0), fb = T(0);
    if (kxa < a.nx && !(a.singular && kxa == 0 && y == 0 && z == 0)) fa = T(a.scale) / (lx[kxa] + lyz);
    if (kxb < a.nx) fb = T(a.scale) / (lx[kxb] + lyz);
    // Z'(k) = fa A + i fb B; at the mirror A and B are conjugated (Hermitian)
    ws[i1] = mkc<T>(fa * A.x - fb * B.y, fa * A.y + fb * B.x);
    if (i2 != i1) ws[i2] = mkc<T>(fa * A.x + fb * B.y, fb * B.x - fa * A.y);
  }
}

template <typename T>
__global__ void __launch_bounds__(256) pair_divide_kernel(const PairDivideArgs a) {
  pair_divide_body<T>(a, blockIdx.x, blockIdx.y, gridDim.y);
}

// ---------------------------------------------------------------------------
// batch phase kernel: one persistent launch runs launch p of every problem
// ---------------------------------------------------------------------------
// The work list holds one item per (problem, launch p) in descending order
// of tiles; first[i] is the index of item i's first tile in the list.  CTAs
// take tiles in order from a counter (zero before the launch), find their
// item by binary search and run its body; no CTA waits on another.  The
// mbarrier sits behind the largest tile (bar_off), and each strided tile
// completes one of its phases.  A CTA whose bounded wait gave up stops (the
// item's plan flag records it).
// KIND: the launch kind of every item in the list (0 x sweep, 1 strided
// sweep, 4 separate divide), so that each kernel holds one body only.
template <typename T, int KIND>
__global__ void __launch_bounds__(kThreads, 3)
    batch_phase_kernel(const BatchItem* __restrict__ items, const int* __restrict__ first, int nitems, int total,
                       int* counter, int bar_off) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw + bar_off);
  __shared__ int s_t;
  // the item's arguments, copied so that the bodies read them from shared
  // memory (a global-memory reference could alias the bodies' own stores)
  __shared__ BatchItem s_item;
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  uint32_t parity = 0;
  for (;;) {
    if (threadIdx.x == 0) s_t = atomicAdd(counter, 1);
    __syncthreads();
    const int t = s_t;
    if (t >= total) break;
    int lo = 0, hi = nitems - 1;  // the last item whose first tile is <= t
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (__ldg(&first[mid]) <= t) lo = mid;
      else hi = mid - 1;
    }
    const int bid = t - __ldg(&first[lo]);
    {
      const uint4* src = reinterpret_cast<const uint4*>(items + lo);
      uint4* dst = reinterpret_cast<uint4*>(&s_item);
      for (int e = threadIdx.x; e < (int)(sizeof(BatchItem) / 16); e += kThreads) dst[e] = __ldg(src + e);
    }
    __syncthreads();
    if (KIND == 0) {
      x_sweep_body<T>(s_item.xa, bid);
    } else if (KIND == 1) {
      // TMA reads the tensor map from global memory (not from shared memory)
      const bool ok = strided_sweep_body<T>(&items[lo].map, s_item.sa, bid, bar, parity);
      parity ^= 1;
      if (!ok) break;
    } else {
      pair_divide_body<T>(s_item.pda, bid % s_item.gx, bid / s_item.gx, s_item.gy);
    }
    fence_proxy_async();
    __syncthreads();  // the tile's shared memory is read before the next tile reuses it
  }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
template <typename T>
cudaError_t launch_x_sweep(const XArgs& a, unsigned grid, size_t smem, cudaStream_t s) {
  auto k = x_sweep_kernel<T>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k<<<grid, kThreads, smem, s>>>(a);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_strided_sweep(const CUtensorMap& map, const StridedArgs& a, unsigned grid, size_t smem,
                                 cudaStream_t s) {
  auto k = strided_sweep_kernel<T>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k<<<grid, kThreads, smem, s>>>(map, a);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_batch_phase(int kind, const BatchItem* items, const int* first, int nitems, int total,
                               int* counter, int bar_off, unsigned grid, size_t smem, cudaStream_t s, int* occ) {
  auto k = kind == 0 ? batch_phase_kernel<T, 0> : (kind == 1 ? batch_phase_kernel<T, 1> : batch_phase_kernel<T, 4>);
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
  if (e != cudaSuccess) return e;
  if (occ) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, k, kThreads, smem);
  k<<<grid, kThreads, smem, s>>>(items, first, nitems, total, counter, bar_off);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_pair_divide(const PairDivideArgs& a, cudaStream_t s) {
  const unsigned gx = (unsigned)(((long long)a.ncols * a.ny + 255) / 256);
  const unsigned gz = (unsigned)(a.nz < 65535 ? a.nz : 65535);
  pair_divide_kernel<T><<<dim3(gx, gz), 256, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace pf
