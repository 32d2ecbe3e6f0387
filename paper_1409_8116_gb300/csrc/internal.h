// Internal descriptors shared by the host planner and the sweep kernels.
//
// Vocabulary (Sec. 2 of the paper): a "sweep" applies the 1D transform of
// Table 2 chosen by one axis's boundary condition to every grid line along
// that axis.  Each transform is computed by one complex FFT of length M per
// line plus a gather before it (pre-processing) and a gather after it
// (post-processing):
//   DFT / IDFT          M = n       (Eqs. DFT / IDFT, unnormalised here)
//   DCT-II / DCT-III    M = n       (even-odd reordering, Makhoul 1980)
//   DST-II / DST-III    M = n       (DCT-II/III with index reversal and signs)
//   DST-I               M = 2(n+1)  (odd extension)
//   DCT-I               M = 2(n-1)  (even extension)
// All transform maps are real matrices applied to complex data, so each
// line may carry two independent real lines in its real and imaginary parts.
#pragma once

#include <cuda.h>

#include <stdint.h>

namespace pf {

enum TKind : int {
  TK_NULL = 0,  // length-1 identity (the absent axes of 1D problems)
  TK_DFT = 1,   // forward DFT, exp(-2 pi i k j / n)
  TK_IDFT = 2,  // backward DFT, exp(+2 pi i k j / n)
  TK_DCT2 = 3,
  TK_DCT3 = 4,
  TK_DST2 = 5,
  TK_DST3 = 6,
  TK_DST1 = 7,
  TK_DCT1 = 8
};

// FFT direction used by each kind: true = exp(+...), the inverse FFT.
inline __host__ __device__ bool kind_uses_inverse_fft(int k) {
  return k == TK_IDFT || k == TK_DCT3 || k == TK_DST3;
}

constexpr int kMaxPass = 12;
constexpr int kThreads = 256;          // threads per CTA of every sweep kernel

// Unsigned 32-bit division by a run-time invariant d >= 1 as one multiply-high,
// a subtract, an add and two shifts (Granlund & Montgomery, "Division by
// invariant integers using multiplication", 1994, Fig. 4.1): with
// l = ceil(log2 d) and m = floor(2^32 (2^l - d) / d) + 1,
// n / d = (t + ((n - t) >> min(l,1))) >> max(l-1,0), t = mulhi(m, n),
// exact for every 32-bit n.  The sweep kernels use it for the tile index
// splits that a hardware-less integer division would otherwise dominate.
struct FastDiv {
  uint32_t d, m;
  int s1, s2;
};
inline __host__ __device__ FastDiv make_fastdiv(uint32_t d) {
  int l = 0;
  while ((1ull << l) < d) l++;
  const uint64_t m = ((1ull << 32) * ((1ull << l) - d)) / d + 1;  // < 2^32 because 2^l < 2d
  return FastDiv{d, (uint32_t)m, l < 1 ? l : 1, l > 1 ? l - 1 : 0};
}
__host__ __device__ __forceinline__ uint32_t fdiv(uint32_t n, const FastDiv& f) {
#ifdef __CUDA_ARCH__
  const uint32_t t = __umulhi(n, f.m);
#else
  const uint32_t t = (uint32_t)(((uint64_t)n * f.m) >> 32);
#endif
  return (t + ((n - t) >> f.s1)) >> f.s2;
}

struct FftDesc {
  int M;                  // FFT length
  int npass;
  int radix[kMaxPass];    // radix of each DIF pass
  int p[kMaxPass];        // block length L of the pass (M / product of the earlier radices)
  int tw_off[kMaxPass];   // offset (complex entries) of the pass twiddles exp(-2 pi i j s/L)
  int gen_off[kMaxPass];  // offset of the radix-R unit roots for generic radices, -1 otherwise
  FastDiv dM;             // divisions by M and, per pass, by M/R (butterflies per line),
  FastDiv dNb[kMaxPass];  // L/R (butterfly offset) and L
  FastDiv dLr[kMaxPass];
  FastDiv dL[kMaxPass];
};

struct AxisDesc {
  int n;                  // grid points on the axis
  int kfwd, kinv;         // TKind of the forward and backward transforms
  int mk_off;             // offset of the Makhoul twiddles exp(-i pi k/(2n)), k < n; -1 if unused
  FftDesc fft;
  // Bluestein (chirp-z) form of the length-M FFT, used when M has a large
  // prime factor: a circular convolution of power-of-two length L >= 2M-1.
  int blu;                // 1: use it (fft describes the length-L passes then)
  int blu_M;              // the DFT length M
  FastDiv dblu_M;
  int chirp_off;          // c_m = exp(+i pi m^2 / M), m < M
  int bhat_off;           // DFT_L of the chirp kernel / L, in DIF output order
};

// Contiguous-axis (x) sweep.  Rows of the field are processed in pairs: row a
// in the real part and row b in the imaginary part of one complex line.
struct XArgs {
  AxisDesc ax;
  const void* tables;     // complex table base of the axis
  const int* perm;        // FFT output i -> smem position (digit reversal)
  int mode;               // 0: g -> workspace (forward), 1: workspace -> phi (backward)
  int r2c;                // 1: periodic x (half-spectrum R2C / C2R); 0: real transform
  int nx;
  int lines;              // line pairs per CTA
  int ld;                 // smem line stride in complex elements
  long long nrows;        // ny * nz
  long long ws_ld;        // workspace row stride: complex elements (r2c) or reals (real)
  const void* g;
  void* phi;
  void* ws;
  int* err;
  int ny;                 // rows per z plane (row r = y + ny*z)
  FastDiv dnx, dnh, dny;  // divisions by nx, nx/2+1 and ny
  long long g_sy, g_sz;   // element strides of g between y rows and z planes
  long long phi_sy, phi_sz;
};

// Strided-axis (y or z) sweep on the complex workspace [nz][ny][pitch].
// A CTA owns a tile of `w` consecutive columns times the whole axis at one
// outer index; the tile arrives by TMA boxes of `box_h` axis rows.
struct StridedArgs {
  AxisDesc ax;
  const void* tables;
  const int* perm;
  int mode;               // 0 forward, 1 backward, 2 forward + eigen divide + backward
  int axis_dim;           // tensor-map dimension of the swept axis: 1 (y) or 2 (z)
  int w, lw;              // tile columns (power of two) and log2(w)
  int ncols;              // valid complex columns
  int ntile_c;            // ceil(ncols / w)
  int nouter;             // extent of the third dimension
  int box_h, nbox;        // TMA box rows and boxes per tile
  int rows_alloc;         // smem rows of the tile (>= M and >= nbox*box_h)
  int bar_off;            // byte offset of the mbarrier in dynamic smem
  long long s_axis;       // complex-element stride along the axis
  long long s_outer;      // complex-element stride along the outer dimension
  void* data;             // workspace base
  // fused divide (mode 2): factor = scale / (lam_in[kx] + lam_ax[k] + lam_out[o])
  const void* lam_in;     // x eigenvalues, indexed by kx = 0..nx-1
  const void* lam_ax;     // swept-axis eigenvalues
  const void* lam_out;    // outer-axis eigenvalues
  double scale;           // product of the Table 2 normalisations
  int singular;           // every axis P/NR/NS: zero the all-zero mode
  int packed;             // 1: column c carries kx = 2c (real part) and 2c+1 (imag part)
  int dit_fused;          // mode 2 with unrolled radices only: backward FFT as DIT passes
  int nx;                 // number of x points (valid kx < nx when packed)
  int* err;
};

// Eigenvalue divide over the whole spectrum when x is not periodic but y or
// z is: every complex workspace element carries two real x columns
// (kx = 2c real part, 2c + 1 imaginary part) whose y/z DFTs are mixed.  The
// element at k = (c, ky, kz) and its mirror -k (negated along periodic axes)
// give A(k) = (Z(k) + conj Z(-k))/2 and B(k) = (Z(k) - conj Z(-k))/(2i),
// the spectra of the two columns, which are divided separately.
struct PairDivideArgs {
  void* data;             // workspace [nz][ny][pitch] complex
  long long pitch;
  int ncols, nx, ny, nz;
  FastDiv dncols;
  int per_y, per_z;       // axis is periodic (mirror index (n - k) mod n)
  const void* lam_x;      // kx = 0..nx-1
  const void* lam_y;
  const void* lam_z;
  double scale;
  int singular;
};

// One launch of one problem in a batch phase (batch_phase_kernel): the
// launch's arguments, its tensor map (strided sweeps; TMA reads it from
// global memory, hence the 64-byte alignment) and, for the separate divide,
// its grid.
struct __align__(64) BatchItem {
  CUtensorMap map;
  XArgs xa;
  StridedArgs sa;
  PairDivideArgs pda;
  int kind;               // 0 x sweep, 1 strided sweep, 4 separate divide
  int gx, gy;             // separate divide: its grid of 256-thread blocks
};

}  // namespace pf
