// Device-side FFT engine for the sweep kernels (sm_103a).
//
// A CTA holds a tile of complex lines in shared memory and transforms every
// line in place with mixed-radix decimation-in-frequency passes (natural
// order in, digit-reversed order out; see dif_pass).  Radices 2, 3, 4, 5,
// 7, 8, 16 and 32 are unrolled register butterflies; any other prime runs as
// direct DFT butterflies through a scratch tile.
//
// The pre- and post-processing gathers turn the FFT into the real transforms
// of Table 1 (see internal.h for the mapping of each kind).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace pf {

// ---------------------------------------------------------------------------
// complex arithmetic
// ---------------------------------------------------------------------------
template <typename T> struct CxOf;
template <> struct CxOf<float> { using type = float2; };
template <> struct CxOf<double> { using type = double2; };
template <typename T> using cx = typename CxOf<T>::type;

template <typename T> __device__ __forceinline__ cx<T> mkc(T r, T i) { cx<T> z; z.x = r; z.y = i; return z; }
template <typename T> __device__ __forceinline__ cx<T> cadd(cx<T> a, cx<T> b) { return mkc<T>(a.x + b.x, a.y + b.y); }
template <typename T> __device__ __forceinline__ cx<T> csub(cx<T> a, cx<T> b) { return mkc<T>(a.x - b.x, a.y - b.y); }
template <typename T> __device__ __forceinline__ cx<T> cmul(cx<T> a, cx<T> b) {
  return mkc<T>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * conj(b)
template <typename T> __device__ __forceinline__ cx<T> cmulc(cx<T> a, cx<T> b) {
  return mkc<T>(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
template <typename T> __device__ __forceinline__ cx<T> cscale(cx<T> a, T s) { return mkc<T>(a.x * s, a.y * s); }
template <typename T> __device__ __forceinline__ cx<T> cconj(cx<T> a) { return mkc<T>(a.x, -a.y); }
template <typename T> __device__ __forceinline__ cx<T> mul_i(cx<T> a) { return mkc<T>(-a.y, a.x); }     // i*a
template <typename T> __device__ __forceinline__ cx<T> mul_mi(cx<T> a) { return mkc<T>(a.y, -a.x); }    // -i*a
template <typename T> __device__ __forceinline__ cx<T> czero() { return mkc<T>(T(0), T(0)); }

// ---------------------------------------------------------------------------
// unit-circle constants for the unrolled radices (correctly rounded decimals)
// ---------------------------------------------------------------------------
// cos(2 pi m / 32) for m = 0..8 (first quadrant)
__host__ __device__ constexpr double q32(int m) {
  return m == 0 ? 1.0 : m == 1 ? 0.9807852804032304 : m == 2 ? 0.9238795325112867
       : m == 3 ? 0.8314696123025452 : m == 4 ? 0.7071067811865476 : m == 5 ? 0.5555702330196022
       : m == 6 ? 0.3826834323650898 : m == 7 ? 0.19509032201612828 : 0.0;
}
__host__ __device__ constexpr int mod_pos(int a, int n) { return ((a % n) + n) % n; }
// cos(2 pi m / 32), any m
__host__ __device__ constexpr double cos32(int m) {
  return mod_pos(m, 32) <= 8 ? q32(mod_pos(m, 32))
       : mod_pos(m, 32) <= 16 ? -q32(16 - mod_pos(m, 32))
       : mod_pos(m, 32) <= 24 ? -q32(mod_pos(m, 32) - 16)
       : q32(32 - mod_pos(m, 32));
}
__host__ __device__ constexpr double sin32(int m) { return cos32(m - 8); }
// cos / sin(2 pi m / N) for odd N in {3, 5, 7}
__host__ __device__ constexpr double cos_odd(int N, int m) {
  return N == 3 ? (mod_pos(m, 3) == 0 ? 1.0 : -0.5)
       : N == 5 ? (mod_pos(m, 5) == 0 ? 1.0 : (mod_pos(m, 5) == 1 || mod_pos(m, 5) == 4) ? 0.30901699437494745 : -0.8090169943749475)
       : (mod_pos(m, 7) == 0 ? 1.0 : (mod_pos(m, 7) == 1 || mod_pos(m, 7) == 6) ? 0.6234898018587335
          : (mod_pos(m, 7) == 2 || mod_pos(m, 7) == 5) ? -0.2225209339563144 : -0.9009688679024191);
}
__host__ __device__ constexpr double sin_odd(int N, int m) {
  return N == 3 ? (mod_pos(m, 3) == 0 ? 0.0 : mod_pos(m, 3) == 1 ? 0.8660254037844386 : -0.8660254037844386)
       : N == 5 ? (mod_pos(m, 5) == 0 ? 0.0 : mod_pos(m, 5) == 1 ? 0.9510565162951535 : mod_pos(m, 5) == 2 ? 0.5877852522924731
                   : mod_pos(m, 5) == 3 ? -0.5877852522924731 : -0.9510565162951535)
       : (mod_pos(m, 7) == 0 ? 0.0 : mod_pos(m, 7) == 1 ? 0.7818314824680298 : mod_pos(m, 7) == 2 ? 0.9749279121818236
          : mod_pos(m, 7) == 3 ? 0.4338837391175581 : mod_pos(m, 7) == 4 ? -0.4338837391175581
          : mod_pos(m, 7) == 5 ? -0.9749279121818236 : -0.7818314824680298);
}

// a * exp(-+ 2 pi i m / N) for N dividing 32 (sign: forward '-', INV '+').
// Called with compile-time m after unrolling, so the branches fold.
template <typename T, int N, bool INV>
__device__ __forceinline__ cx<T> tw_pow2(cx<T> a, int m) {
  const int r = mod_pos(m, N);
  if (r == 0) return a;
  if (2 * r == N) return mkc<T>(-a.x, -a.y);
  if (4 * r == N) return INV ? mul_i<T>(a) : mul_mi<T>(a);
  if (4 * r == 3 * N) return INV ? mul_mi<T>(a) : mul_i<T>(a);
  const T c = T(cos32(r * (32 / N)));
  const T s = INV ? T(sin32(r * (32 / N))) : T(-sin32(r * (32 / N)));
  return mkc<T>(a.x * c - a.y * s, a.x * s + a.y * c);
}

// ---------------------------------------------------------------------------
// radix-R DFTs in registers (in place, natural order)
// ---------------------------------------------------------------------------
template <typename T, int R, bool INV> struct Dft;

template <typename T, bool INV> struct Dft<T, 1, INV> {
  static __device__ __forceinline__ void run(cx<T>*) {}
};
template <typename T, bool INV> struct Dft<T, 2, INV> {
  static __device__ __forceinline__ void run(cx<T>* u) {
    cx<T> a = cadd<T>(u[0], u[1]), b = csub<T>(u[0], u[1]);
    u[0] = a; u[1] = b;
  }
};
template <typename T, bool INV> struct Dft<T, 4, INV> {
  static __device__ __forceinline__ void run(cx<T>* u) {
    cx<T> s02 = cadd<T>(u[0], u[2]), d02 = csub<T>(u[0], u[2]);
    cx<T> s13 = cadd<T>(u[1], u[3]), d13 = csub<T>(u[1], u[3]);
    cx<T> r13 = INV ? mul_i<T>(d13) : mul_mi<T>(d13);
    u[0] = cadd<T>(s02, s13);
    u[2] = csub<T>(s02, s13);
    u[1] = cadd<T>(d02, r13);
    u[3] = csub<T>(d02, r13);
  }
};
// odd prime radix: y_s = u0 + sum_q (u_q + u_{R-q}) cos(2 pi q s/R) -/+ i (u_q - u_{R-q}) sin(2 pi q s/R)
template <typename T, int R, bool INV> struct DftOdd {
  static __device__ __forceinline__ void run(cx<T>* u) {
    constexpr int H = (R - 1) / 2;
    cx<T> sp[H], sm[H];
#pragma unroll
    for (int q = 1; q <= H; q++) { sp[q - 1] = cadd<T>(u[q], u[R - q]); sm[q - 1] = csub<T>(u[q], u[R - q]); }
    cx<T> y0 = u[0];
#pragma unroll
    for (int q = 0; q < H; q++) y0 = cadd<T>(y0, sp[q]);
    cx<T> out[R];
    out[0] = y0;
#pragma unroll
    for (int s = 1; s <= H; s++) {
      cx<T> a = u[0], b = czero<T>();
#pragma unroll
      for (int q = 1; q <= H; q++) {
        const T c = T(cos_odd(R, q * s)), sn = T(sin_odd(R, q * s));
        a = mkc<T>(a.x + c * sp[q - 1].x, a.y + c * sp[q - 1].y);
        b = mkc<T>(b.x + sn * sm[q - 1].x, b.y + sn * sm[q - 1].y);
      }
      // forward: y_s = a - i b, y_{R-s} = a + i b
      cx<T> ib = mul_i<T>(b);
      out[s] = INV ? cadd<T>(a, ib) : csub<T>(a, ib);
      out[R - s] = INV ? csub<T>(a, ib) : cadd<T>(a, ib);
    }
#pragma unroll
    for (int s = 0; s < R; s++) u[s] = out[s];
  }
};
template <typename T, bool INV> struct Dft<T, 3, INV> : DftOdd<T, 3, INV> {};
template <typename T, bool INV> struct Dft<T, 5, INV> : DftOdd<T, 5, INV> {};
template <typename T, bool INV> struct Dft<T, 7, INV> : DftOdd<T, 7, INV> {};

// N = A*B by one Cooley-Tukey step: input n = B*n1 + n2, output k = k1 + A*k2.
template <typename T, int A, int B, bool INV>
__device__ __forceinline__ void dft_ct(cx<T>* u) {
  constexpr int N = A * B;
  cx<T> t[N];
#pragma unroll
  for (int n2 = 0; n2 < B; n2++) {
    cx<T> a[A];
#pragma unroll
    for (int n1 = 0; n1 < A; n1++) a[n1] = u[B * n1 + n2];
    Dft<T, A, INV>::run(a);
#pragma unroll
    for (int k1 = 0; k1 < A; k1++) t[k1 * B + n2] = tw_pow2<T, N, INV>(a[k1], n2 * k1);
  }
#pragma unroll
  for (int k1 = 0; k1 < A; k1++) {
    cx<T> b[B];
#pragma unroll
    for (int n2 = 0; n2 < B; n2++) b[n2] = t[k1 * B + n2];
    Dft<T, B, INV>::run(b);
#pragma unroll
    for (int k2 = 0; k2 < B; k2++) u[k1 + A * k2] = b[k2];
  }
}
template <typename T, bool INV> struct Dft<T, 8, INV> {
  static __device__ __forceinline__ void run(cx<T>* u) { dft_ct<T, 2, 4, INV>(u); }
};
template <typename T, bool INV> struct Dft<T, 16, INV> {
  static __device__ __forceinline__ void run(cx<T>* u) { dft_ct<T, 4, 4, INV>(u); }
};
template <typename T, bool INV> struct Dft<T, 32, INV> {
  static __device__ __forceinline__ void run(cx<T>* u) { dft_ct<T, 4, 8, INV>(u); }
};

// ---------------------------------------------------------------------------
// tile layouts
// ---------------------------------------------------------------------------
// Column tile of a strided sweep: element (m, c) at m*w + c (TMA box order).
// Consecutive threads take consecutive columns, so every smem access of a
// warp covers whole rows.
struct ColTile {
  int w, lw;
  __device__ __forceinline__ int idx(int m, int c) const { return m * w + c; }
  // split a flat index over (lines of length len) x (w columns)
  __device__ __forceinline__ void split(int b, const FastDiv& /*len*/, int& i, int& c) const {
    c = b & (w - 1);
    i = b >> lw;
  }
};
// Row tile of the contiguous sweep: element (m, line) at line*ld + m + (m >> sh),
// one padding element after every 2^sh (one 128-byte bank sweep of complex
// values).  Without it the digit-reversed gathers of the post-processing and
// the butterflies of the last passes, whose threads step by a power of two,
// meet in one bank; ld >= len + (len >> sh).
struct RowTile {
  int ld, sh;
  __device__ __forceinline__ int idx(int m, int c) const { return c * ld + m + (m >> sh); }
  __device__ __forceinline__ void split(int b, const FastDiv& len, int& i, int& c) const {
    c = (int)fdiv((uint32_t)b, len);
    i = b - c * (int)len.d;
  }
};

// ---------------------------------------------------------------------------
// in-place decimation-in-frequency passes
// ---------------------------------------------------------------------------
// Pass i of radix R works on blocks of L = M/(R_1...R_{i-1}) points.  The
// butterfly (block, j), j < L/R, reads the R points block*L + j + q*(L/R),
// takes their radix-R DFT, multiplies output s by exp(-2 pi i j s / L) and
// writes it back to block*L + j + s*(L/R).  Each butterfly owns its points,
// so passes need one barrier each and no staging.  After the last pass the
// DFT output k = s_1 + R_1 (s_2 + R_2 (s_3 + ...)) sits at position
// sum_i s_i L_i/R_i (digit reversal); the post-processing gathers read it
// through the `perm` table.
template <typename T, int R, bool INV, class LAY>
__device__ __noinline__ void dif_pass(cx<T>* __restrict__ buf, const LAY lay, int M, int ncol, const FastDiv dnbl,
                                      const FastDiv dLr, const cx<T>* __restrict__ tw) {
  const int Lr = (int)dLr.d;
  const int L = Lr * R;
  const int nb = (M / R) * ncol;
  for (int b = threadIdx.x; b < nb; b += kThreads) {
    int t, c;
    lay.split(b, dnbl, t, c);
    const int blk = (int)fdiv((uint32_t)t, dLr);
    const int j = t - blk * Lr;
    const int base = blk * L + j;
    cx<T> u[R];
#pragma unroll
    for (int q = 0; q < R; q++) u[q] = buf[lay.idx(base + q * Lr, c)];
    Dft<T, R, INV>::run(u);
    if (j != 0) {
#pragma unroll
      for (int s = 1; s < R; s++) {
        const cx<T> w = tw[(s - 1) * Lr + j];
        u[s] = INV ? cmulc<T>(u[s], w) : cmul<T>(u[s], w);
      }
    }
#pragma unroll
    for (int s = 0; s < R; s++) buf[lay.idx(base + s * Lr, c)] = u[s];
  }
  __syncthreads();
}

// Direct DFT butterflies for radices without an unrolled kernel (odd primes
// > 7), in the symmetric form: with p_q = u_q + u_{R-q}, m_q = u_q - u_{R-q}
// (q = 1..H, H = (R-1)/2), a_s = u_0 + sum_q p_q cos(2 pi q s/R) and
// b_s = sum_q m_q sin(2 pi q s/R), the outputs are y_s = a_s -+ i b_s and
// y_{R-s} = a_s +- i b_s, y_0 = u_0 + sum_q p_q.  A work item is one
// butterfly and one output pair (s, R-s) (group 0: y_0), so each input pair
// is read once per two outputs.  Results go to `scratch`, and the tile is
// copied back afterwards.  roots[m] = exp(-2 pi i m/R).
template <typename T, bool INV, class LAY>
__device__ __noinline__ void dif_pass_generic(cx<T>* __restrict__ buf, cx<T>* __restrict__ scratch, const LAY lay,
                                              const FastDiv dM, int ncol, int R, const FastDiv dL, const FastDiv dLr,
                                              const cx<T>* __restrict__ tw, const cx<T>* __restrict__ roots) {
  const int Lr = (int)dLr.d;
  const int L = (int)dL.d;
  const int M = (int)dM.d;
  const int H = (R - 1) >> 1;
  const int items = (M / R) * (H + 1);  // per column
  const FastDiv dG = make_fastdiv((uint32_t)(H + 1));
  const FastDiv dI = make_fastdiv((uint32_t)items);
  const int total = items * ncol;
  for (int e = threadIdx.x; e < total; e += kThreads) {
    int it, c;
    lay.split(e, dI, it, c);
    const int t = (int)fdiv((uint32_t)it, dG);  // butterfly
    const int g = it - t * (H + 1);             // output pair
    const int blk = (int)fdiv((uint32_t)t, dLr);
    const int j = t - blk * Lr;
    const int base = blk * L + j;
    const cx<T> u0 = buf[lay.idx(base, c)];
    if (g == 0) {
      cx<T> y = u0;
      for (int q = 1; q < R; q++) y = cadd<T>(y, buf[lay.idx(base + q * Lr, c)]);
      scratch[lay.idx(base, c)] = y;
      continue;
    }
    cx<T> a = u0, b = czero<T>();
    int qs = 0;  // (q*g) mod R
    for (int q = 1; q <= H; q++) {
      qs += g;
      if (qs >= R) qs -= R;
      const cx<T> x1 = buf[lay.idx(base + q * Lr, c)];
      const cx<T> x2 = buf[lay.idx(base + (R - q) * Lr, c)];
      const cx<T> r = roots[qs];  // (cos, -sin)
      a.x += r.x * (x1.x + x2.x);
      a.y += r.x * (x1.y + x2.y);
      b.x -= r.y * (x1.x - x2.x);
      b.y -= r.y * (x1.y - x2.y);
    }
    const cx<T> ib = mul_i<T>(b);
    cx<T> y1 = INV ? cadd<T>(a, ib) : csub<T>(a, ib);  // output g
    cx<T> y2 = INV ? csub<T>(a, ib) : cadd<T>(a, ib);  // output R - g
    if (j != 0) {
      const cx<T> w1 = tw[(g - 1) * Lr + j];
      const cx<T> w2 = tw[(R - g - 1) * Lr + j];
      y1 = INV ? cmulc<T>(y1, w1) : cmul<T>(y1, w1);
      y2 = INV ? cmulc<T>(y2, w2) : cmul<T>(y2, w2);
    }
    scratch[lay.idx(base + g * Lr, c)] = y1;
    scratch[lay.idx(base + (R - g) * Lr, c)] = y2;
  }
  __syncthreads();
  const int tot2 = M * ncol;
  for (int e = threadIdx.x; e < tot2; e += kThreads) {
    int pos, c;
    lay.split(e, dM, pos, c);
    buf[lay.idx(pos, c)] = scratch[lay.idx(pos, c)];
  }
  __syncthreads();
}

// Decimation-in-time pass (the transpose of dif_pass): butterfly (block, j)
// multiplies input q by exp(-+2 pi i j q / L), takes the radix-R DFT and
// writes output s back to block*L + j + s*(L/R).  Run in the reverse order
// of the DIF passes, DIT takes the DIF output arrangement to natural order.
template <typename T, int R, bool INV, class LAY>
__device__ __noinline__ void dit_pass(cx<T>* __restrict__ buf, const LAY lay, int M, int ncol, const FastDiv dnbl,
                                      const FastDiv dLr, const cx<T>* __restrict__ tw) {
  const int Lr = (int)dLr.d;
  const int L = Lr * R;
  const int nb = (M / R) * ncol;
  for (int b = threadIdx.x; b < nb; b += kThreads) {
    int t, c;
    lay.split(b, dnbl, t, c);
    const int blk = (int)fdiv((uint32_t)t, dLr);
    const int j = t - blk * Lr;
    const int base = blk * L + j;
    cx<T> u[R];
#pragma unroll
    for (int q = 0; q < R; q++) u[q] = buf[lay.idx(base + q * Lr, c)];
    if (j != 0) {
#pragma unroll
      for (int q = 1; q < R; q++) {
        const cx<T> w = tw[(q - 1) * Lr + j];
        u[q] = INV ? cmulc<T>(u[q], w) : cmul<T>(u[q], w);
      }
    }
    Dft<T, R, INV>::run(u);
#pragma unroll
    for (int s = 0; s < R; s++) buf[lay.idx(base + s * Lr, c)] = u[s];
  }
  __syncthreads();
}

// DIT passes of a plan whose radices are all unrolled (the Bluestein
// convolution and the fused divide of the strided sweep): digit-reversed
// input, natural-order output.
template <typename T, bool INV, int EMAX, class LAY>
__device__ __forceinline__ void run_passes_dit(cx<T>* buf, const LAY lay, const FftDesc& f, int ncol,
                                               const cx<T>* __restrict__ tables) {
  for (int ps = f.npass - 1; ps >= 0; ps--) {
    const int R = f.radix[ps];
    const FastDiv dNb = f.dNb[ps], dLr = f.dLr[ps];
    const cx<T>* tw = tables + f.tw_off[ps];
    switch (R) {
      case 2: dit_pass<T, 2, INV>(buf, lay, f.M, ncol, dNb, dLr, tw); break;
      case 3: dit_pass<T, 3, INV>(buf, lay, f.M, ncol, dNb, dLr, tw); break;
      case 4: dit_pass<T, 4, INV>(buf, lay, f.M, ncol, dNb, dLr, tw); break;
      case 5: dit_pass<T, 5, INV>(buf, lay, f.M, ncol, dNb, dLr, tw); break;
      case 7: dit_pass<T, 7, INV>(buf, lay, f.M, ncol, dNb, dLr, tw); break;
      case 8: dit_pass<T, 8, INV>(buf, lay, f.M, ncol, dNb, dLr, tw); break;
      case 16: dit_pass<T, 16, INV>(buf, lay, f.M, ncol, dNb, dLr, tw); break;
      default:
        if constexpr (EMAX >= 32) dit_pass<T, 32, INV>(buf, lay, f.M, ncol, dNb, dLr, tw);
        break;
    }
  }
}

template <typename T, bool INV, int EMAX, class LAY>
__device__ __forceinline__ void run_passes_dir(cx<T>* buf, cx<T>* scratch, const LAY lay, const FftDesc& f, int ncol,
                                               const cx<T>* __restrict__ tables) {
  for (int ps = 0; ps < f.npass; ps++) {
    const int R = f.radix[ps];
    const FastDiv dNb = f.dNb[ps], dLr = f.dLr[ps];
    const cx<T>* tw = tables + f.tw_off[ps];
    switch (R) {
      case 2: dif_pass<T, 2, INV>(buf, lay, f.M, ncol, dNb, dLr, tw); break;
      case 3: dif_pass<T, 3, INV>(buf, lay, f.M, ncol, dNb, dLr, tw); break;
      case 4: dif_pass<T, 4, INV>(buf, lay, f.M, ncol, dNb, dLr, tw); break;
      case 5: dif_pass<T, 5, INV>(buf, lay, f.M, ncol, dNb, dLr, tw); break;
      case 7: dif_pass<T, 7, INV>(buf, lay, f.M, ncol, dNb, dLr, tw); break;
      case 8: dif_pass<T, 8, INV>(buf, lay, f.M, ncol, dNb, dLr, tw); break;
      case 16: dif_pass<T, 16, INV>(buf, lay, f.M, ncol, dNb, dLr, tw); break;
      case 32:
        if constexpr (EMAX >= 32) { dif_pass<T, 32, INV>(buf, lay, f.M, ncol, dNb, dLr, tw); break; }
        // fall through to the direct DFT when 32 complex values exceed the register budget
      default:
        dif_pass_generic<T, INV>(buf, scratch, lay, f.dM, ncol, R, f.dL[ps], dLr, tw, tables + f.gen_off[ps]);
        break;
    }
  }
}

template <typename T, int EMAX, class LAY>
__device__ __forceinline__ void run_passes(cx<T>* buf, cx<T>* scratch, const LAY lay, const FftDesc& f, int ncol,
                                           const cx<T>* tables, bool inverse) {
  if (inverse)
    run_passes_dir<T, true, EMAX>(buf, scratch, lay, f, ncol, tables);
  else
    run_passes_dir<T, false, EMAX>(buf, scratch, lay, f, ncol, tables);
}

// ---------------------------------------------------------------------------
// pre- and post-processing gathers (Table 1 transforms from one FFT)
// ---------------------------------------------------------------------------
// FFT input position m of the transform `kind` applied to the source line
// held in rows 0..n-1 of `buf` (column c).  mk[k] = exp(-i pi k/(2n)).
template <typename T, class LAY>
__device__ __forceinline__ cx<T> pre_value(const cx<T>* buf, const LAY& lay, int kind, int n, int M, int m, int c,
                                           const cx<T>* __restrict__ mk) {
  switch (kind) {
    case TK_DCT2:
    case TK_DST2: {
      // v_m = x_{2m} (m < ceil(n/2)), v_m = x_{2n-1-2m} otherwise
      const int src = (2 * m < n) ? 2 * m : 2 * n - 1 - 2 * m;
      cx<T> v = buf[lay.idx(src, c)];
      if (kind == TK_DST2 && (src & 1)) v = mkc<T>(-v.x, -v.y);  // DST-II(x)_k = DCT-II((-1)^j x_j)_{n-1-k}
      return v;
    }
    case TK_DST1: {  // odd extension of length 2(n+1)
      if (m == 0 || m == n + 1) return czero<T>();
      if (m <= n) return buf[lay.idx(m - 1, c)];
      const cx<T> v = buf[lay.idx(M - 1 - m, c)];
      return mkc<T>(-v.x, -v.y);
    }
    case TK_DCT1:  // even extension of length 2(n-1)
      return buf[lay.idx(m < n ? m : M - m, c)];
    case TK_DCT3:
    case TK_DST3: {
      // DCT-III: V_m = conj(w_m) (f_m - i f_{n-m}), f_n = 0
      // DST-III(f)_k = (-1)^k DCT-III(h)_k with h_j = f_{n-1-j}
      cx<T> a, b;
      if (kind == TK_DCT3) {
        a = buf[lay.idx(m, c)];
        b = (m == 0) ? czero<T>() : buf[lay.idx(n - m, c)];
      } else {
        a = buf[lay.idx(n - 1 - m, c)];
        b = (m == 0) ? czero<T>() : buf[lay.idx(m - 1, c)];
      }
      const cx<T> t = mkc<T>(a.x + b.y, a.y - b.x);  // a - i b
      return cmulc<T>(t, mk[m]);
    }
    default:
      return buf[lay.idx(m, c)];
  }
}

// Output k of the transform `kind` from the FFT output held in `buf`; FFT
// output index i sits at position perm[i] (digit reversal of the DIF
// passes), or at i itself when NAT (after DIT passes).
template <typename T, bool NAT = false, class LAY>
__device__ __forceinline__ cx<T> post_value(const cx<T>* buf, const LAY& lay, int kind, int n, int k, int c,
                                            const cx<T>* __restrict__ mk, const int* __restrict__ perm_tab) {
  auto perm = [&](int i) { return NAT ? i : perm_tab[i]; };
  switch (kind) {
    case TK_DCT2:
    case TK_DST2: {
      // X_k = w_k Y_k + conj(w_k) Y_{(n-k) mod n};  DST-II reads DCT-II output n-1-k
      const int kk = (kind == TK_DCT2) ? k : n - 1 - k;
      const cx<T> w = mk[kk];
      const cx<T> y1 = buf[lay.idx(perm(kk), c)];
      const cx<T> y2 = buf[lay.idx(perm(kk == 0 ? 0 : n - kk), c)];
      return cadd<T>(cmul<T>(w, y1), cmulc<T>(y2, w));
    }
    case TK_DST1:
      return mul_i<T>(buf[lay.idx(perm(k + 1), c)]);
    case TK_DCT3:
    case TK_DST3: {
      // outputs 2j and 2j+1 are FFT outputs j and n-1-j
      const int pos = (k & 1) ? n - 1 - (k >> 1) : (k >> 1);
      cx<T> v = buf[lay.idx(perm(pos), c)];
      if (kind == TK_DST3 && (k & 1)) v = mkc<T>(-v.x, -v.y);
      return v;
    }
    default:  // DFT, IDFT, DCT1, NULL
      return buf[lay.idx(perm(k), c)];
  }
}

// Calls f(KindC<kind>{}) so that the transform kind is a compile-time
// constant inside the element loops (no per-element indirect branch).
template <int K> struct KindC { static constexpr int value = K; };
template <class F>
__device__ __forceinline__ void with_kind(int kind, F&& f) {
  switch (kind) {
    case TK_DFT: f(KindC<TK_DFT>{}); break;
    case TK_IDFT: f(KindC<TK_IDFT>{}); break;
    case TK_DCT2: f(KindC<TK_DCT2>{}); break;
    case TK_DCT3: f(KindC<TK_DCT3>{}); break;
    case TK_DST2: f(KindC<TK_DST2>{}); break;
    case TK_DST3: f(KindC<TK_DST3>{}); break;
    case TK_DST1: f(KindC<TK_DST1>{}); break;
    case TK_DCT1: f(KindC<TK_DCT1>{}); break;
    default: f(KindC<TK_NULL>{}); break;
  }
}

inline __device__ bool kind_needs_pre(int kind) {
  return !(kind == TK_DFT || kind == TK_IDFT || kind == TK_NULL);
}

// In-place pre-processing of a whole tile: rows 0..n-1 (source) -> 0..M-1.
template <typename T, int EMAX, class LAY>
__device__ __forceinline__ void pre_tile(cx<T>* buf, const LAY lay, int kind, int n, const FastDiv dM, int ncol,
                                         const cx<T>* __restrict__ mk) {
  if (!kind_needs_pre(kind)) return;
  with_kind(kind, [&](auto kc) {
    constexpr int K = decltype(kc)::value;
    if constexpr (K != TK_DFT && K != TK_IDFT && K != TK_NULL) {
      cx<T> v[EMAX];
      const int M = (int)dM.d;
      const int total = M * ncol;
#pragma unroll
      for (int j = 0; j < EMAX; j++) {
        const int e = threadIdx.x + j * kThreads;
        if (e < total) {
          int m, c;
          lay.split(e, dM, m, c);
          v[j] = pre_value<T>(buf, lay, K, n, M, m, c, mk);
        }
      }
      __syncthreads();
#pragma unroll
      for (int j = 0; j < EMAX; j++) {
        const int e = threadIdx.x + j * kThreads;
        if (e < total) {
          int m, c;
          lay.split(e, dM, m, c);
          buf[lay.idx(m, c)] = v[j];
        }
      }
      __syncthreads();
    }
  });
}

// ---------------------------------------------------------------------------
// Bluestein (chirp-z) FFT of length M through a length-L convolution
// ---------------------------------------------------------------------------
// X_k = conj(c_k) sum_j (x_j conj(c_j)) c_{k-j},  c_m = exp(i pi m^2 / M)
// (Bluestein 1970): the sum is a circular convolution of length L >= 2M-1,
// done as DIF(L), a pointwise product with the precomputed kernel spectrum,
// and an inverse DIT(L).  The FFT input x_j is the pre-processing value of
// the transform `kind` gathered from the source lines in `src`; the result
// X_k (natural order, k < M) is left in `dst` rows 0..M-1 for post_value
// with an identity permutation.  The inverse direction conjugates input and
// output.  No staging: src and dst are different smem regions.
template <typename T, int EMAX, class LS, class LD>
__device__ __forceinline__ void bluestein_fft(const cx<T>* src, const LS ls, cx<T>* dst, const LD ld,
                                              const AxisDesc& ax, int kind, int n, int ncol,
                                              const cx<T>* __restrict__ tables, const cx<T>* __restrict__ mk) {
  const int M = ax.blu_M;
  const int L = ax.fft.M;
  const bool inv = kind_uses_inverse_fft(kind);
  const cx<T>* chirp = tables + ax.chirp_off;
  const cx<T>* bhat = tables + ax.bhat_off;
  const int total = L * ncol;
  for (int e = threadIdx.x; e < total; e += kThreads) {
    int j, c;
    ld.split(e, ax.fft.dM, j, c);
    cx<T> v = czero<T>();
    if (j < M) {
      v = pre_value<T>(src, ls, kind, n, M, j, c, mk);
      if (inv) v = cconj<T>(v);
      v = cmulc<T>(v, chirp[j]);
    }
    dst[ld.idx(j, c)] = v;
  }
  __syncthreads();
  run_passes_dir<T, false, EMAX>(dst, dst, ld, ax.fft, ncol, tables);
  for (int e = threadIdx.x; e < total; e += kThreads) {
    int p, c;
    ld.split(e, ax.fft.dM, p, c);
    dst[ld.idx(p, c)] = cmul<T>(dst[ld.idx(p, c)], bhat[p]);
  }
  __syncthreads();
  run_passes_dit<T, true, EMAX>(dst, ld, ax.fft, ncol, tables);
  const int tm = M * ncol;
  for (int e = threadIdx.x; e < tm; e += kThreads) {
    int k, c;
    ld.split(e, ax.dblu_M, k, c);
    cx<T> x = cmulc<T>(dst[ld.idx(k, c)], chirp[k]);
    dst[ld.idx(k, c)] = inv ? cconj<T>(x) : x;
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// mbarrier / TMA (cp.async.bulk.tensor) wrappers
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Wait for phase `parity` of the barrier for at most ~2 s of wall time.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = globaltimer_ns();
  for (uint32_t it = 0; it < (1u << 30); ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 255u) == 255u && globaltimer_ns() - t0 > 2000000000ull) return false;
  }
  return false;
}
// Asynchronous element copy global -> shared (cp.async, 4 or 8 bytes); a
// copy with valid == false reads nothing and writes zeros.
template <int BYTES>
__device__ __forceinline__ void cp_async_elem(void* dst, const void* src, bool valid) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;" ::"r"(smem_u32(dst)), "l"(src), "n"(BYTES),
               "r"(valid ? BYTES : 0)
               : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Untiled bulk copy global -> shared of `bytes` (a multiple of 16; both
// addresses 16-byte aligned), completing on the mbarrier's transaction count.
__device__ __forceinline__ void bulk_load_1d(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
// Untiled bulk copy shared -> global of `bytes` (a multiple of 16; both
// addresses 16-byte aligned), tracked by the bulk-group counters.
__device__ __forceinline__ void bulk_store_1d(void* dst, const void* src, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(smem_u32(src)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_commit_group() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// wait until the shared-memory sources of this thread's bulk copies have been read
__device__ __forceinline__ void bulk_wait_group_read0() {
  asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar, int c0, int c1, int c2) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(c0), "r"(c1), "r"(c2)
      : "memory");
}

// Tiled tensor store shared -> global of one box at coordinates (c0, c1, c2)
// (c0 a multiple of 16 bytes, no coordinate negative); elements outside the
// tensor are not written.  Tracked by the bulk-group counters.
__device__ __forceinline__ void tma_store_3d(const CUtensorMap* map, const void* src, int c0, int c1, int c2) {
  asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.tile.bulk_group [%0, {%2, %3, %4}], [%1];" ::"l"(
                   reinterpret_cast<uint64_t>(map)),
               "r"(smem_u32(src)), "r"(c0), "r"(c1), "r"(c2)
               : "memory");
}

}  // namespace pf
