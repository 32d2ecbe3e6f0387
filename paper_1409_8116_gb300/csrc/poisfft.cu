// Planner and C interface of the GB300 Poisson solver (see include/poisfft.h).
//
// The planner picks, per axis, the Table 2 transform pair of the axis's
// boundary condition, the FFT length and its radix passes, builds the FP64
// twiddle and eigenvalue tables (Tables 3 and 4) with exactly reduced angles
// and rounds them once to the solve precision, sizes the tiles of every
// sweep kernel, encodes the TMA tensor maps of the workspace and allocates
// it.  A solve enqueues the sweeps (Sec. 2.1 steps 1-3, Sec. 2.3 order):
//   3D: x forward, y forward, z forward+divide+backward, y backward, x backward
//   2D: x forward, y forward+divide+backward, x backward
//   1D: x forward, divide (length-1 axis), x backward
#include <cuda.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <nvtx3/nvToolsExt.h>
#include <new>
#include <vector>

#include "../../include/poisfft.h"
#include "fast_kernels.cuh"
#include "tc_kernels.cuh"
#include "reduce.cuh"
#include "internal.h"
#include "launch.h"

using namespace pf;


namespace {

// ---------------------------------------------------------------------------
// Host-side fault injection (a testing aid: nothing faults on the device).
// POISFFT_FAULT is read when a call that allocates starts (plan creation,
// host-buffer solve, refined solve, zero-mode mean, autotune):
//   alloc:N  the N-th device allocation of that call (1-based) fails
//   encode   encoding the TMA tensor maps fails (as cuTensorMapEncodeTiled would)
//   size     planning reports an unsupported size
// Every such failure must come back as its status code with nothing leaked.
// ---------------------------------------------------------------------------
struct FaultState {
  int alloc_at = 0, alloc_seen = 0;
  bool encode = false, size = false;
};
thread_local FaultState g_fault;

struct FaultScope {  // armed for the duration of one API call
  FaultScope() {
    g_fault = FaultState();
    const char* e = getenv("POISFFT_FAULT");
    if (!e) return;
    if (!strncmp(e, "alloc:", 6)) g_fault.alloc_at = atoi(e + 6);
    else if (!strcmp(e, "encode")) g_fault.encode = true;
    else if (!strcmp(e, "size")) g_fault.size = true;
  }
  ~FaultScope() { g_fault = FaultState(); }
};

template <typename T>
cudaError_t dev_malloc(T** ptr, size_t bytes) {
  if (g_fault.alloc_at > 0 && ++g_fault.alloc_seen == g_fault.alloc_at) {
    *ptr = nullptr;
    return cudaErrorMemoryAllocation;
  }
  return cudaMalloc(reinterpret_cast<void**>(ptr), bytes);
}

constexpr size_t kSmemLimit = 200 * 1024;   // dynamic smem budget of one CTA
constexpr size_t kSmemTarget = 64 * 1024;   // preferred tile size (several CTAs per SM)

// ---------------------------------------------------------------------------
// FP64 trigonometry with exactly reduced arguments: angle 2 pi m / N
// ---------------------------------------------------------------------------
void sincos_2pi_frac(long long m, long long N, double* s, double* c) {
  long long r = m % N;
  if (r < 0) r += N;
  const long long q = (4 * r) / N;       // quadrant
  long long rem = 4 * r - q * N;         // angle = q pi/2 + (pi/2) rem/N
  bool swap = false;
  if (2 * rem > N) { rem = N - rem; swap = true; }
  const double phi = (M_PI / 2.0) * (double)rem / (double)N;
  double s1 = sin(phi), c1 = cos(phi);
  if (swap) { const double t = s1; s1 = c1; c1 = t; }
  switch (q) {
    case 0: *c = c1; *s = s1; break;
    case 1: *c = -s1; *s = c1; break;
    case 2: *c = -c1; *s = -s1; break;
    default: *c = s1; *s = -c1; break;
  }
}

double sin_pi_frac(long long num, long long den) {  // sin(pi num/den)
  double s, c;
  sincos_2pi_frac(num, 2 * den, &s, &c);
  return s;
}

// ---------------------------------------------------------------------------
// per-axis transform description
// ---------------------------------------------------------------------------
constexpr int kBluesteinMinPrime = 41;  // larger prime factors go through Bluestein

// Forward DFT (exp(-2 pi i jk/N)) of a {2,3,5,7}-smooth length N, FP64,
// recursive mixed-radix decimation in time with exactly reduced twiddles
// (host tables only): with p the smallest prime factor of N and m = N/p,
// X[k + m q] = sum_r exp(-2 pi i r (k + m q) / N) Y_r[k], Y_r the length-m
// DFT of the samples r, r + p, r + 2p, ...
void host_fft_rec(const double* re, const double* im, long long stride, int N, double* ore, double* oim) {
  if (N == 1) {
    ore[0] = re[0];
    oim[0] = im[0];
    return;
  }
  int p = 2;
  while (N % p) p++;
  const int m = N / p;
  std::vector<double> yr((size_t)N), yi((size_t)N);
  for (int r = 0; r < p; r++) host_fft_rec(re + r * stride, im + r * stride, stride * p, m, &yr[(size_t)r * m], &yi[(size_t)r * m]);
  for (int k = 0; k < m; k++)
    for (int q = 0; q < p; q++) {
      const int kk = k + m * q;
      double sr = 0.0, si = 0.0;
      for (int r = 0; r < p; r++) {
        double sn, c;
        sincos_2pi_frac((long long)r * kk, N, &sn, &c);  // exp(-2 pi i r kk / N)
        const double ar = yr[(size_t)r * m + k], ai = yi[(size_t)r * m + k];
        sr += ar * c + ai * sn;
        si += ai * c - ar * sn;
      }
      ore[kk] = sr;
      oim[kk] = si;
    }
}

void host_fft(std::vector<double>& re, std::vector<double>& im) {
  const int N = (int)re.size();
  std::vector<double> orr((size_t)N), oi((size_t)N);
  host_fft_rec(re.data(), im.data(), 1, N, orr.data(), oi.data());
  re.swap(orr);
  im.swap(oi);
}

bool is_unrolled_radix(int r, int emax) {
  return r == 2 || r == 3 || r == 4 || r == 5 || r == 7 || r == 8 || r == 16 || (r == 32 && emax >= 32);
}
// Staging capacity of the general kernels per thread (complex elements);
// must match Emax<T> in sweep_kernels.cuh.

// Factor M into DIF passes: powers of two grouped into balanced radices
// up to 32 (16 for FP64), then 3, 5, 7, then any other prime (direct DFT).
void factor_passes(int M, int emax, std::vector<int>& radices) {
  radices.clear();
  int e2 = 0;
  while (M % 2 == 0) { M /= 2; e2++; }
  const int maxlog = emax >= 32 ? 5 : 4;
  if (e2 > 0) {
    const int np = (e2 + maxlog - 1) / maxlog;
    for (int i = 0; i < np; i++) {
      const int take = e2 / np + (i < e2 % np ? 1 : 0);
      radices.push_back(1 << take);
    }
  }
  for (int p : {3, 5, 7}) while (M % p == 0) { radices.push_back(p); M /= p; }
  for (int p = 11; (long long)p * p <= M; p += 2)
    while (M % p == 0) { radices.push_back(p); M /= p; }
  if (M > 1) radices.push_back(M);
}

bool smooth7(long long v) {
  for (int p : {2, 3, 5, 7})
    while (v % p == 0) v /= p;
  return v == 1;
}

// Convolution length of Bluestein's method for a DFT of length M: at least
// 2M - 1 and {2,3,5,7}-smooth, so that every pass is an unrolled radix.  Of
// those up to the next power of two, the one with the least estimated work
// (length x passes) is taken: e.g. M = 4098 (DST-I of 2048 points) takes
// 8960 = 16 * 16 * 5 * 7 instead of 16384, and its column tile fits in shared
// memory.
int bluestein_length(int M, int emax) {
  const long long lo = 2LL * M - 1;
  long long p2 = 1;
  while (p2 < lo) p2 *= 2;
  std::vector<int> rad;
  factor_passes((int)p2, emax, rad);
  long long best = p2, best_cost = p2 * (long long)rad.size();
  for (long long L = lo; L < p2; L++) {
    if (!smooth7(L)) continue;
    factor_passes((int)L, emax, rad);
    const long long cost = L * (long long)rad.size();
    if (cost < best_cost && (int)rad.size() <= kMaxPass) {
      best = L;
      best_cost = cost;
    }
  }
  return (int)best;
}

struct AxisPlan {
  int bc = POISFFT_P;
  int n = 1;
  double L = 1.0;
  AxisDesc d{};
  std::vector<double> tab_re, tab_im;   // complex table in FP64
  std::vector<double> lam;              // eigenvalues, FP64
  std::vector<int> perm;                // FFT output index -> position after the DIF passes
  double scale = 1.0;                   // Table 2 normalisation of the axis
  int max_ncol = 0;                     // max lines / columns per CTA from the register budget
  bool generic = false;                 // a direct-DFT pass needs a scratch tile
};

int build_axis(AxisPlan& ax, int bc, int n, double L, int approx, int emax, bool null_axis) {
  ax.bc = bc;
  ax.n = n;
  ax.L = L;
  AxisDesc& d = ax.d;
  memset(&d, 0, sizeof(d));
  d.n = n;
  d.mk_off = -1;
  int M = n;
  if (null_axis) {
    d.kfwd = d.kinv = TK_NULL;
    M = 1;
    ax.scale = 1.0;
  } else {
    switch (bc) {
      case POISFFT_P: d.kfwd = TK_DFT; d.kinv = TK_IDFT; M = n; ax.scale = 1.0 / n; break;
      case POISFFT_DR: d.kfwd = d.kinv = TK_DST1; M = 2 * (n + 1); ax.scale = 1.0 / (2.0 * (n + 1)); break;
      case POISFFT_DS: d.kfwd = TK_DST2; d.kinv = TK_DST3; M = n; ax.scale = 1.0 / (2.0 * n); break;
      case POISFFT_NR: d.kfwd = d.kinv = TK_DCT1; M = 2 * (n - 1); ax.scale = 1.0 / (2.0 * (n - 1)); break;
      case POISFFT_NS: d.kfwd = TK_DCT2; d.kinv = TK_DCT3; M = n; ax.scale = 1.0 / (2.0 * n); break;
      default: return POISFFT_ERR_INVALID_ARG;
    }
  }
  std::vector<int> radices;
  factor_passes(M, emax, radices);
  // Bluestein when a prime factor would need a slow direct-DFT pass
  int maxp = 1;
  for (int R : radices)
    if (!is_unrolled_radix(R, emax)) maxp = std::max(maxp, R);
  const bool blu = maxp >= kBluesteinMinPrime;
  int Mfft = M;
  if (blu) {
    Mfft = bluestein_length(M, emax);
    factor_passes(Mfft, emax, radices);
  }
  d.blu = blu ? 1 : 0;
  d.blu_M = M;
  d.dblu_M = make_fastdiv((uint32_t)M);
  d.fft.M = Mfft;
  d.fft.dM = make_fastdiv((uint32_t)Mfft);
  if ((int)radices.size() > kMaxPass) return POISFFT_ERR_UNSUPPORTED_SIZE;
  d.fft.npass = (int)radices.size();
  ax.tab_re.clear();
  ax.tab_im.clear();
  ax.generic = false;
  auto push = [&](double re, double im) { ax.tab_re.push_back(re); ax.tab_im.push_back(im); };
  // register budget: the pre/post gathers stage EMAX elements per thread
  // (the Bluestein path stages nothing)
  const long long cap = blu ? (1LL << 20) : (long long)kThreads * emax / M;
  int Lb = Mfft;  // block length of the pass
  for (int i = 0; i < d.fft.npass; i++) {
    const int R = radices[i];
    d.fft.radix[i] = R;
    d.fft.p[i] = Lb;
    d.fft.tw_off[i] = (int)ax.tab_re.size();
    const int Lr = Lb / R;
    d.fft.dNb[i] = make_fastdiv((uint32_t)(Mfft / R));
    d.fft.dLr[i] = make_fastdiv((uint32_t)Lr);
    d.fft.dL[i] = make_fastdiv((uint32_t)Lb);
    for (int s = 1; s < R; s++)
      for (int j = 0; j < Lr; j++) {
        double sn, c;
        sincos_2pi_frac((long long)j * s, Lb, &sn, &c);  // exp(-2 pi i j s / Lb)
        push(c, -sn);
      }
    if (is_unrolled_radix(R, emax)) {
      d.fft.gen_off[i] = -1;
    } else {
      if (R % 2 == 0) return POISFFT_ERR_UNSUPPORTED_SIZE;  // the direct pass takes odd radices only
      ax.generic = true;
      d.fft.gen_off[i] = (int)ax.tab_re.size();
      for (int m = 0; m < R; m++) {
        double sn, c;
        sincos_2pi_frac(m, R, &sn, &c);
        push(c, -sn);
      }
    }
    Lb = Lr;
  }
  // digit reversal: FFT output k = s_1 + R_1 (s_2 + R_2 (...)) sits at sum_i s_i L_i / R_i
  std::vector<int> perm(Mfft, 0);
  for (int k = 0; k < Mfft; k++) {
    int rem = k, pos = 0, Li = Mfft;
    for (int i = 0; i < d.fft.npass; i++) {
      const int R = d.fft.radix[i];
      pos += (rem % R) * (Li / R);
      rem /= R;
      Li /= R;
    }
    perm[k] = pos;
  }
  if (blu) {
    // chirp c_m = exp(i pi m^2 / M) and the spectrum of the circulant kernel
    // b_m = c_m (|m| < M, indices mod L), divided by L, in DIF output order
    d.chirp_off = (int)ax.tab_re.size();
    std::vector<double> cr(M), ci(M);
    for (int m = 0; m < M; m++) {
      double sn, c;
      sincos_2pi_frac(((long long)m * m) % (2LL * M), 2LL * M, &sn, &c);
      cr[m] = c;
      ci[m] = sn;
      push(c, sn);
    }
    std::vector<double> br(Mfft, 0.0), bi(Mfft, 0.0);
    for (int m = 0; m < M; m++) {
      br[m] = cr[m];
      bi[m] = ci[m];
      if (m > 0) {
        br[Mfft - m] = cr[m];
        bi[Mfft - m] = ci[m];
      }
    }
    host_fft(br, bi);
    d.bhat_off = (int)ax.tab_re.size();
    std::vector<double> hr(Mfft), hi(Mfft);
    for (int k = 0; k < Mfft; k++) {
      hr[perm[k]] = br[k] / Mfft;
      hi[perm[k]] = bi[k] / Mfft;
    }
    for (int k = 0; k < Mfft; k++) push(hr[k], hi[k]);
    ax.perm.resize(M);
    for (int k = 0; k < M; k++) ax.perm[k] = k;  // the Bluestein result is in natural order
  } else {
    d.chirp_off = d.bhat_off = -1;
    ax.perm = perm;
  }
  if (d.kfwd == TK_DCT2 || d.kfwd == TK_DST2) {
    d.mk_off = (int)ax.tab_re.size();
    for (int k = 0; k < n; k++) {
      double s, c;
      sincos_2pi_frac(k, 4LL * n, &s, &c);  // exp(-i pi k/(2n))
      push(c, -s);
    }
  }
  if (ax.tab_re.empty()) push(1.0, 0.0);
  ax.max_ncol = (int)std::max<long long>(cap, 0);

  // eigenvalues (Table 3 / Table 4)
  ax.lam.assign(n, 0.0);
  if (!null_axis) {
    for (int k = 0; k < n; k++) {
      double lam = 0.0;
      if (approx == POISFFT_SPECTRAL) {
        switch (bc) {
          case POISFFT_P: { const int m = std::min(k, n - k); lam = -pow(2.0 * M_PI * m / L, 2); break; }
          case POISFFT_DR:
          case POISFFT_DS: lam = -pow(M_PI * (k + 1) / L, 2); break;
          default: lam = -pow(M_PI * k / L, 2); break;
        }
      } else {
        double dx, s;
        switch (bc) {
          case POISFFT_P: dx = L / n; s = sin_pi_frac(k, n); break;
          case POISFFT_DR: dx = L / (n + 1); s = sin_pi_frac(k + 1, 2LL * (n + 1)); break;
          case POISFFT_DS: dx = L / n; s = sin_pi_frac(k + 1, 2LL * n); break;
          case POISFFT_NR: dx = L / (n - 1); s = sin_pi_frac(k, 2LL * (n - 1)); break;
          default: dx = L / n; s = sin_pi_frac(k, 2LL * n); break;
        }
        lam = -(2.0 * s / dx) * (2.0 * s / dx);
      }
      ax.lam[k] = lam;
    }
  }
  return POISFFT_OK;
}

struct SweepLaunch {
  int kind;               // 0 x sweep, 1 strided sweep, 2 fast x sweep, 3 fast strided sweep, 4 pair divide
  XArgs xa;
  StridedArgs sa;
  fast::FastXArgs fxa;
  fast::FastStridedArgs fsa;
  PairDivideArgs pda;
  int M, fmode, fkind, axis, w, box_h;  // fast sweeps
  int tc;                 // fast strided sweep on the tensor cores (BF16X3 plans)
  int tc_tiles;           // its tiles (the persistent grid loops over them)
  int tc_slot;            // its tile counter in poisfft_plan::tc_ctr
  int map;                // tensor map index (strided)
  unsigned grid;
  size_t smem;
  long long bytes;        // algorithmic HBM bytes (read + write)
};

using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn get_encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return nullptr;
    fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

// Workspace row pitch (complex elements): the least p >= ncols whose row
// stride, p * 2 * esize bytes, is 64 modulo 128.  Tile rows of the strided
// sweeps then start on 64-byte boundaries and consecutive rows alternate
// between the two halves of a 128-byte line; measured on the 1024^3 y sweeps
// (1.67 -> 1.50 ms against the plain even pitch 514).
long long workspace_pitch(long long ncols, size_t esize) {
  const long long unit = 128 / (2 * (long long)esize);  // elements per 128 bytes
  long long p = (ncols + unit - 1) / unit * unit + unit / 2;
  if (p - unit >= ncols) p -= unit;
  return p;
}

int pow2_floor(long long v) {
  int p = 1;
  while ((long long)p * 2 <= v) p *= 2;
  return p;
}
int pow2_ceil(long long v) {
  int p = 1;
  while (p < v) p *= 2;
  return p;
}
int ilog2(int v) {
  int l = 0;
  while ((1 << l) < v) l++;
  return l;
}

}  // namespace

struct poisfft_plan {
  int dims = 0;
  int dtype = POISFFT_F32;
  int approx = POISFFT_FD2;
  int nx = 1, ny = 1, nz = 1;
  size_t esize = 4;              // bytes of one real element
  int r2c = 0;
  int ncols = 0, pitch = 0;      // workspace complex columns (valid) and pitch
  int singular = 0;
  AxisPlan axes[3];              // x, y, z (missing axes are length-1 null axes)
  void* ws = nullptr;
  size_t ws_bytes = 0;
  void* tables[3] = {nullptr, nullptr, nullptr};
  void* lam[3] = {nullptr, nullptr, nullptr};
  int* perm[3] = {nullptr, nullptr, nullptr};
  int* err = nullptr;
  double* zm = nullptr;               // zero-mode reduction: 1 result + 2 * blocks partials
  unsigned* zm_count = nullptr;
  std::vector<CUtensorMap> maps;      // one per launch (strided launches use theirs)
  std::vector<SweepLaunch> sweeps;
  void* stage_g = nullptr;
  void* stage_phi = nullptr;
  // poisfft_solve_host_async: two staging pairs used in turn, copy streams, events
  struct HostPipe {
    bool ready = false;
    int next = 0;
    bool used[2] = {false, false};
    void* g[2] = {nullptr, nullptr};
    void* phi[2] = {nullptr, nullptr};
    cudaStream_t in = nullptr, out = nullptr;
    cudaEvent_t copied_in[2] = {nullptr, nullptr}, solved[2] = {nullptr, nullptr}, copied_out[2] = {nullptr, nullptr};
  } pipe;
  float* refine_r = nullptr;         // FP32 residual / correction of poisfft_solve_refined
  int refinements = 2;               // POISFFT_MIXED plans: refinement steps of poisfft_solve
  int fused_axis = 0;                // general 3D plans: the strided axis whose sweep divides
  size_t field_bytes = 0;
  bool profiling = false;
  std::vector<cudaEvent_t> events;   // (launches + 1) per profiled solve
  bool fast = false;                 // specialised two-pass FP32 kernels
  void* ftw[3] = {nullptr, nullptr, nullptr};
  void* fmk[3] = {nullptr, nullptr, nullptr};
  void* fpk[3] = {nullptr, nullptr, nullptr};
  void* flam[3] = {nullptr, nullptr, nullptr};
  void* tcb = nullptr;               // B operands of the tensor-core sweeps (BF16X3 plans)
  int* tc_ctr = nullptr;             // one tile counter per tensor-core launch
};

namespace {

// Buffers, streams and events of poisfft_solve_host_async (waits for the
// pipeline's copies first, so that no copy outlives its staging buffer).
void release_host_pipe(poisfft_plan* p) {
  auto& q = p->pipe;
  if (q.in) cudaStreamSynchronize(q.in);
  if (q.out) cudaStreamSynchronize(q.out);
  for (int b = 0; b < 2; b++) {
    if (q.g[b]) cudaFree(q.g[b]);
    if (q.phi[b]) cudaFree(q.phi[b]);
    if (q.copied_in[b]) cudaEventDestroy(q.copied_in[b]);
    if (q.solved[b]) cudaEventDestroy(q.solved[b]);
    if (q.copied_out[b]) cudaEventDestroy(q.copied_out[b]);
  }
  if (q.in) cudaStreamDestroy(q.in);
  if (q.out) cudaStreamDestroy(q.out);
  q = poisfft_plan::HostPipe();
}

void free_plan(poisfft_plan* p) {
  if (!p) return;
  if (p->ws) cudaFree(p->ws);
  for (int i = 0; i < 3; i++) {
    if (p->tables[i]) cudaFree(p->tables[i]);
    if (p->lam[i]) cudaFree(p->lam[i]);
    if (p->perm[i]) cudaFree(p->perm[i]);
  }
  if (p->err) cudaFree(p->err);
  if (p->zm) cudaFree(p->zm);
  if (p->zm_count) cudaFree(p->zm_count);
  if (p->stage_g) cudaFree(p->stage_g);
  if (p->stage_phi) cudaFree(p->stage_phi);
  release_host_pipe(p);
  if (p->refine_r) cudaFree(p->refine_r);
  for (cudaEvent_t e : p->events) cudaEventDestroy(e);
  for (int i = 0; i < 3; i++) {
    if (p->ftw[i]) cudaFree(p->ftw[i]);
    if (p->fmk[i]) cudaFree(p->fmk[i]);
    if (p->fpk[i]) cudaFree(p->fpk[i]);
    if (p->flam[i]) cudaFree(p->flam[i]);
  }
  if (p->tcb) cudaFree(p->tcb);
  if (p->tc_ctr) cudaFree(p->tc_ctr);
  delete p;
}

template <typename T>
int upload_tables(poisfft_plan* p) {
  for (int a = 0; a < 3; a++) {
    AxisPlan& ax = p->axes[a];
    const size_t nt = ax.tab_re.size();
    std::vector<T> tab(2 * nt);
    for (size_t i = 0; i < nt; i++) { tab[2 * i] = (T)ax.tab_re[i]; tab[2 * i + 1] = (T)ax.tab_im[i]; }
    std::vector<T> lam(ax.lam.size());
    for (size_t i = 0; i < lam.size(); i++) lam[i] = (T)ax.lam[i];
    if (dev_malloc(&p->tables[a], tab.size() * sizeof(T)) != cudaSuccess) return POISFFT_ERR_ALLOC;
    if (dev_malloc(&p->lam[a], std::max<size_t>(lam.size(), 1) * sizeof(T)) != cudaSuccess) return POISFFT_ERR_ALLOC;
    if (cudaMemcpy(p->tables[a], tab.data(), tab.size() * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess)
      return POISFFT_ERR_CUDA;
    if (cudaMemcpy(p->lam[a], lam.data(), lam.size() * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess)
      return POISFFT_ERR_CUDA;
    if (dev_malloc(&p->perm[a], ax.perm.size() * sizeof(int)) != cudaSuccess) return POISFFT_ERR_ALLOC;
    if (cudaMemcpy(p->perm[a], ax.perm.data(), ax.perm.size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess)
      return POISFFT_ERR_CUDA;
  }
  return POISFFT_OK;
}

// smem rows of one x line: the in-place line (plus a direct-DFT scratch
// line), or the source line plus the Bluestein convolution buffer
// (rows are padded by one complex value per 16 (FP32) or 8 (FP64), the
// kernels' RowTile layout)
int x_padded(const poisfft_plan* p, int len) { return len + (len >> (p->esize == 4 ? 4 : 3)); }
int x_line_ld(const poisfft_plan* p) { return x_padded(p, p->axes[0].d.blu ? p->nx : p->axes[0].d.fft.M); }
size_t x_per_line(const poisfft_plan* p) {
  const AxisPlan& ax = p->axes[0];
  const size_t cx = 2 * p->esize;
  if (ax.d.blu) return (size_t)(x_padded(p, p->nx) + x_padded(p, ax.d.fft.M)) * cx;
  return (size_t)x_padded(p, ax.d.fft.M) * cx * (ax.generic ? 2 : 1);
}
// smem bytes per tile column of a strided sweep with `rows_alloc` tile rows
size_t strided_per_col(const poisfft_plan* p, int axis, int rows_alloc) {
  const AxisPlan& ax = p->axes[axis];
  const size_t cx = 2 * p->esize;
  if (ax.d.blu) return (size_t)(rows_alloc + ax.d.fft.M) * cx;
  return (size_t)rows_alloc * cx * (ax.generic ? 2 : 1);
}

// x sweep configuration
int plan_x_sweep(poisfft_plan* p, int mode, SweepLaunch& L) {
  AxisPlan& ax = p->axes[0];
  const size_t cx = 2 * p->esize;
  const long long nrows = (long long)p->ny * p->nz;
  const long long pairs = (nrows + 1) / 2;
  long long lines = ax.max_ncol;
  const size_t per_line = x_per_line(p);
  lines = std::min<long long>(lines, (long long)(kSmemTarget / per_line));
  lines = std::min<long long>(lines, pairs);
  if (lines < 1) {
    if (ax.max_ncol >= 1 && per_line <= kSmemLimit) lines = 1;
    else return POISFFT_ERR_UNSUPPORTED_SIZE;
  }
  memset(&L, 0, sizeof(L));
  L.kind = 0;
  XArgs& a = L.xa;
  a.ax = ax.d;
  a.tables = p->tables[0];
  a.mode = mode;
  a.r2c = p->r2c;
  a.nx = p->nx;
  a.lines = (int)lines;
  a.ld = x_line_ld(p);
  a.nrows = nrows;
  a.ws_ld = p->r2c ? p->pitch : 2LL * p->pitch;
  a.ws = p->ws;
  a.err = p->err;
  a.ny = p->ny;
  a.dnx = make_fastdiv((uint32_t)p->nx);
  a.dnh = make_fastdiv((uint32_t)(p->nx / 2 + 1));
  a.dny = make_fastdiv((uint32_t)p->ny);
  L.grid = (unsigned)((pairs + lines - 1) / lines);
  L.smem = (size_t)lines * per_line;
  const long long field = nrows * p->nx * (long long)p->esize;
  const long long wsb = nrows * (long long)p->ncols * (long long)cx;
  L.bytes = field + (p->r2c ? wsb : field);
  return POISFFT_OK;
}

// strided sweep along axis `a` (1 = y, 2 = z)
int plan_strided_sweep(poisfft_plan* p, int axis, int mode, SweepLaunch& L) {
  AxisPlan& ax = p->axes[axis];
  const int M = ax.d.fft.M;
  const int n = ax.n;
  const size_t cx = 2 * p->esize;
  const int wmin = p->esize == 4 ? 2 : 1;
  int nbox, box_h;
  if (n <= 256) { nbox = 1; box_h = n; }
  else {
    nbox = (n + 255) / 256;
    box_h = (n + nbox - 1) / nbox;
    box_h = (box_h + 15) / 16 * 16;
  }
  const int rows_alloc = ax.d.blu ? nbox * box_h : std::max(M, nbox * box_h);
  const size_t per_col = strided_per_col(p, axis, rows_alloc);
  long long w = std::min<long long>(ax.max_ncol, 128);
  w = std::min<long long>(w, pow2_ceil(p->ncols));
  w = std::min<long long>(w, (long long)(kSmemTarget / per_col));
  w = pow2_floor(std::max<long long>(w, 1));
  if (w < wmin) w = wmin;
  if (w > ax.max_ncol || (size_t)w * per_col + 16 > kSmemLimit) return POISFFT_ERR_UNSUPPORTED_SIZE;
  memset(&L, 0, sizeof(L));
  L.kind = 1;
  L.map = axis - 1;
  StridedArgs& s = L.sa;
  s.ax = ax.d;
  s.tables = p->tables[axis];
  s.mode = mode;
  s.axis_dim = axis;
  s.w = (int)w;
  s.lw = ilog2((int)w);
  s.ncols = p->ncols;
  s.ntile_c = (p->ncols + (int)w - 1) / (int)w;
  s.nouter = axis == 1 ? p->nz : p->ny;
  s.box_h = box_h;
  s.nbox = nbox;
  s.rows_alloc = rows_alloc;
  s.bar_off = (int)(((size_t)w * per_col + 15) / 16 * 16);
  s.s_axis = axis == 1 ? (long long)p->pitch : (long long)p->pitch * p->ny;
  s.s_outer = axis == 1 ? (long long)p->pitch * p->ny : (long long)p->pitch;
  s.data = p->ws;
  s.lam_in = p->lam[0];
  s.lam_ax = p->lam[axis];
  s.lam_out = p->lam[axis == 1 ? 2 : 1];
  double sc = 1.0;
  for (int i = 0; i < 3; i++) sc *= p->axes[i].scale;
  s.scale = sc;
  s.singular = p->singular;
  s.packed = p->r2c ? 0 : 1;
  s.dit_fused = mode == 2 && !ax.d.blu && !ax.generic && !(s.packed && ax.d.kfwd == TK_DFT);
  s.nx = p->nx;
  s.err = p->err;
  L.grid = (unsigned)((long long)s.ntile_c * s.nouter);
  L.smem = (size_t)s.bar_off + 16;
  L.bytes = 2LL * p->ncols * (long long)p->ny * p->nz * (long long)cx;
  return POISFFT_OK;
}

// ---------------------------------------------------------------------------
// specialised path: every axis two-pass FP32; x periodic with y/z P, NS or
// DS, or x NS / DS with y/z NS or DS
// ---------------------------------------------------------------------------
bool dct_axis(const AxisPlan& ax) { return ax.bc == POISFFT_NS || ax.bc == POISFFT_DS; }

bool fast_eligible(const poisfft_plan* p) {
  if (p->esize != 4 || p->dims < 2) return false;
  const char* env = getenv("POISFFT_FORCE_GENERIC");
  if (env && env[0] && env[0] != '0') return false;
  const bool xdct = dct_axis(p->axes[0]);
  if (!p->r2c && !xdct) return false;
  int r1, r2, w;
  for (int a = 0; a < p->dims; a++) {
    if (!fast_shape(p->axes[a].n, &r1, &r2, &w)) return false;
    const int bc = p->axes[a].bc;
    if (a > 0 && !(bc == POISFFT_NS || bc == POISFFT_DS || (bc == POISFFT_P && !xdct))) return false;
  }
  return true;
}

// Tables of one axis for the specialised kernels, FP64 -> float:
//   tw[s*R2 + j] = exp(-2 pi i j s / M);  mk[k] = exp(-i pi k/(2M));
//   pk[k] = (lam[k], lam[(M-k) mod M], cos(pi k/M), sin(pi k/M));
//   lam in storage order (DST-II axes: DCT-II index k holds mode M-1-k).
int fast_upload_axis(poisfft_plan* p, int a) {
  AxisPlan& ax = p->axes[a];
  const int M = ax.n;
  int R1, R2, W;
  fast_shape(M, &R1, &R2, &W);
  std::vector<float> tw(2 * (size_t)M), mk(2 * (size_t)M), pk(4 * (size_t)M), lam(M);
  for (int s = 0; s < R1; s++)
    for (int j = 0; j < R2; j++) {
      double sn, c;
      sincos_2pi_frac((long long)j * s, M, &sn, &c);
      tw[2 * (s * R2 + j)] = (float)c;
      tw[2 * (s * R2 + j) + 1] = (float)-sn;
    }
  for (int k = 0; k < M; k++) {
    double sn, c;
    sincos_2pi_frac(k, 4LL * M, &sn, &c);
    mk[2 * k] = (float)c;
    mk[2 * k + 1] = (float)-sn;
    sincos_2pi_frac(k, 2LL * M, &sn, &c);  // exp(+i pi k / M)
    pk[4 * k + 2] = (float)c;
    pk[4 * k + 3] = (float)sn;
    lam[k] = (float)(ax.bc == POISFFT_DS ? ax.lam[M - 1 - k] : ax.lam[k]);
  }
  for (int k = 0; k < M; k++) {
    pk[4 * k] = lam[k];
    pk[4 * k + 1] = lam[k == 0 ? 0 : M - k];
  }
  if (dev_malloc(&p->ftw[a], tw.size() * sizeof(float)) != cudaSuccess ||
      dev_malloc(&p->fmk[a], mk.size() * sizeof(float)) != cudaSuccess ||
      dev_malloc(&p->fpk[a], pk.size() * sizeof(float)) != cudaSuccess ||
      dev_malloc(&p->flam[a], lam.size() * sizeof(float)) != cudaSuccess)
    return POISFFT_ERR_ALLOC;
  if (cudaMemcpy(p->ftw[a], tw.data(), tw.size() * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(p->fmk[a], mk.data(), mk.size() * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(p->fpk[a], pk.data(), pk.size() * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(p->flam[a], lam.data(), lam.size() * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess)
    return POISFFT_ERR_CUDA;
  return POISFFT_OK;
}

void plan_fast_x(poisfft_plan* p, int mode, SweepLaunch& L) {
  memset(&L, 0, sizeof(L));
  L.kind = 2;
  L.M = p->nx;
  L.fmode = mode;
  L.axis = 0;
  int R1, R2, W;
  fast_shape(p->nx, &R1, &R2, &W);
  const int rmax = std::max(R1, R2);
  const int lpc = 256 / rmax;
  fast::FastXArgs& a = L.fxa;
  a.nx = p->nx;
  a.lines = lpc;
  a.nrows = (long long)p->ny * p->nz;
  a.ny = p->ny;
  a.nz = p->nz;
  a.perm_y = p->dims >= 2 && dct_axis(p->axes[1]);
  a.perm_z = p->dims >= 3 && dct_axis(p->axes[2]);
  a.sign_y = p->dims >= 2 && p->axes[1].bc == POISFFT_DS;
  a.sign_z = p->dims >= 3 && p->axes[2].bc == POISFFT_DS;
  a.ws_ld = p->pitch;
  L.fkind = p->r2c ? fast::FX_R2C : fast::FX_DCT;
  a.xsign = p->axes[0].bc == POISFFT_DS;
  const long long pairs = (a.nrows + 1) / 2;
  L.grid = (unsigned)((pairs + lpc - 1) / lpc);
  L.smem = (size_t)lpc * R1 * (R2 + 1) * 8 + 16;  // line buffer (also the staged rows), barrier
  const long long field = a.nrows * p->nx * 4LL;
  L.bytes = field + a.nrows * (long long)p->ncols * 8;
}

void plan_fast_strided(poisfft_plan* p, int axis, int mode, SweepLaunch& L) {
  memset(&L, 0, sizeof(L));
  AxisPlan& ax = p->axes[axis];
  const int M = ax.n;
  int R1, R2, W;
  fast_shape(M, &R1, &R2, &W);
  L.kind = 3;
  L.M = M;
  L.fmode = mode;
  L.fkind = dct_axis(ax) ? fast::FK_DCT : fast::FK_DFT;
  if (mode == fast::FM_FUSED && !p->r2c) L.fkind = fast::FK_DCT_PAIR;  // x DCT-II / DST-II columns
  L.axis = axis;
  L.w = W;
  L.box_h = std::min(M, 256);
  L.map = axis - 1;
  fast::FastStridedArgs& s = L.fsa;
  double sc = 1.0;
  for (int i = 0; i < 3; i++) sc *= p->axes[i].scale;
  s.scale = (float)sc;
  s.singular = p->singular;
  s.ncols = p->ncols;
  s.ntile_c = (p->ncols + W - 1) / W;
  s.box_h = L.box_h;
  s.nbox = M / L.box_h;
  s.axis_dim = axis;
  s.s_axis = axis == 1 ? (long long)p->pitch : (long long)p->pitch * p->ny;
  s.s_outer = axis == 1 ? (long long)p->pitch * p->ny : (long long)p->pitch;
  const int nouter = axis == 1 ? p->nz : p->ny;
  L.grid = (unsigned)((long long)s.ntile_c * nouter);
  const size_t tile_c = std::max<size_t>((size_t)R1 * (R2 * W + std::min(W, 8)), (size_t)M * W);
  L.smem = (tile_c * 8 + 15) / 16 * 16 + 16;
  if (mode == fast::FM_FUSED) L.smem = (size_t)M * W * 8 + (size_t)(M / 2 + 1) * 16 + 16;  // tile, pair table, barrier
  L.bytes = 2LL * p->ncols * (long long)p->ny * p->nz * 8;
}

void patch_fast(poisfft_plan* p) {
  for (auto& L : p->sweeps) {
    if (L.kind == 2) {
      L.fxa.tw = static_cast<const float2*>(p->ftw[0]);
      L.fxa.mk = static_cast<const float2*>(p->fmk[0]);
      L.fxa.ws = static_cast<float2*>(p->ws);
      L.fxa.err = p->err;
    } else if (L.kind == 3) {
      const int a = L.axis;
      fast::FastStridedArgs& s = L.fsa;
      s.tw = static_cast<const float2*>(p->ftw[a]);
      s.mk = static_cast<const float2*>(p->fmk[a]);
      s.pk = static_cast<const float4*>(p->fpk[a]);
      s.lam_in = static_cast<const float*>(L.fkind == fast::FK_DCT_PAIR ? p->flam[0] : p->lam[0]);
      s.lam_ax = static_cast<const float*>(p->flam[a]);
      s.lam_out = static_cast<const float*>(a == 1 ? (p->dims >= 3 ? p->flam[2] : p->lam[2]) : p->flam[1]);
      s.data = static_cast<float2*>(p->ws);
      s.err = p->err;
    }
  }
}

int encode_maps(poisfft_plan* p) {
  if (g_fault.encode) return POISFFT_ERR_CUDA;
  EncodeTiledFn enc = get_encode_fn();
  if (!enc) return POISFFT_ERR_CUDA;
  const CUtensorMapDataType dt = p->esize == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64;
  const cuuint64_t gdim[3] = {(cuuint64_t)2 * p->ncols, (cuuint64_t)p->ny, (cuuint64_t)p->nz};
  const cuuint64_t row = (cuuint64_t)p->pitch * 2 * p->esize;
  const cuuint64_t gstride[2] = {row, row * (cuuint64_t)p->ny};
  const cuuint32_t estr[3] = {1, 1, 1};
  p->maps.resize(p->sweeps.size());
  for (size_t li = 0; li < p->sweeps.size(); li++) {
    SweepLaunch& L = p->sweeps[li];
    L.map = (int)li;
    if (L.kind != 1 && L.kind != 3) continue;
    const int w = L.kind == 1 ? L.sa.w : L.w;
    const int axis_dim = L.kind == 1 ? L.sa.axis_dim : L.axis;
    const int box_h = L.kind == 1 ? L.sa.box_h : L.box_h;
    cuuint32_t box[3];
    box[0] = (cuuint32_t)(2 * w);
    box[1] = axis_dim == 1 ? (cuuint32_t)box_h : 1u;
    box[2] = axis_dim == 2 ? (cuuint32_t)box_h : 1u;
    CUresult r = enc(&p->maps[L.map], dt, 3, p->ws, gdim, gstride, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return POISFFT_ERR_CUDA;
  }
  return POISFFT_OK;
}

int record_event(poisfft_plan* p, cudaStream_t st) {
  cudaEvent_t ev;
  if (cudaEventCreate(&ev) != cudaSuccess) return POISFFT_ERR_CUDA;
  p->events.push_back(ev);
  return cudaEventRecord(ev, st) == cudaSuccess ? POISFFT_OK : POISFFT_ERR_CUDA;
}

// Element strides of g and phi between y rows and z planes (dense: nx, nx*ny).
struct FieldStrides {
  long long g_sy, g_sz, phi_sy, phi_sz;
};

// NVTX range name of a launch (axis x mode; the separate divide)
const char* sweep_range_name(const SweepLaunch& L) {
  static const char* const names[3][3] = {
      {"poisfft x forward", "poisfft x backward", "poisfft x fused"},
      {"poisfft y forward", "poisfft y backward", "poisfft y fused"},
      {"poisfft z forward", "poisfft z backward", "poisfft z fused"}};
  if (L.kind == 4) return "poisfft eigenvalue divide";
  const int axis = L.kind >= 2 ? L.axis : (L.kind == 0 ? 0 : L.sa.axis_dim);
  const int mode = L.kind >= 2 ? L.fmode : (L.kind == 0 ? L.xa.mode : L.sa.mode);
  return names[axis][mode];
}

// Ranges are pushed and popped around every launch of a solve (host side;
// no cost beyond a pointer check when no tool is attached).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};

template <typename T>
int enqueue(poisfft_plan* p, void* phi, const void* g, cudaStream_t st, const FieldStrides& fs) {
  NvtxRange solve_range("poisfft solve");
  for (auto& L : p->sweeps) {
    if (p->profiling && record_event(p, st) != POISFFT_OK) return POISFFT_ERR_CUDA;
    NvtxRange sweep_range(sweep_range_name(L));
    cudaError_t e;
    if (L.kind == 0) {
      XArgs a = L.xa;
      a.g = g;
      a.phi = phi;
      a.ny = p->ny;
      a.g_sy = fs.g_sy;
      a.g_sz = fs.g_sz;
      a.phi_sy = fs.phi_sy;
      a.phi_sz = fs.phi_sz;
      e = launch_x_sweep<T>(a, L.grid, L.smem, st);
    } else if (L.kind == 1) {
      e = launch_strided_sweep<T>(p->maps[L.map], L.sa, L.grid, L.smem, st);
    } else if (L.kind == 4) {
      e = launch_pair_divide<T>(L.pda, st);
    } else if (L.kind == 2) {
      fast::FastXArgs a = L.fxa;
      a.g = static_cast<const float*>(g);
      a.phi = static_cast<float*>(phi);
      a.g_sy = fs.g_sy;
      a.g_sz = fs.g_sz;
      a.phi_sy = fs.phi_sy;
      a.phi_sz = fs.phi_sz;
      // whole-row bulk copies need 16-byte aligned row starts
      a.stage_g = (uintptr_t)g % 16 == 0 && fs.g_sy % 4 == 0 && fs.g_sz % 4 == 0;
      a.stage_phi = (uintptr_t)phi % 16 == 0 && fs.phi_sy % 4 == 0 && fs.phi_sz % 4 == 0;
      e = launch_fast_x(L.M, L.fmode, L.fkind, a, L.grid, L.smem, st);
    } else if (L.tc) {
      tc::TcStridedArgs ta;
      ta.f = L.fsa;
      ta.bmat = static_cast<const uint4*>(p->tcb);
      ta.ntiles = L.tc_tiles;
      ta.counter = p->tc_ctr + L.tc_slot;
      e = cudaMemsetAsync(ta.counter, 0, sizeof(int), st);
      if (e == cudaSuccess) e = launch_tc_strided(L.fmode, L.fkind, p->maps[L.map], ta, L.grid, st);
    } else {
      e = launch_fast_strided(L.M, L.w, L.fmode, L.fkind, p->maps[L.map], L.fsa, L.grid, L.smem, st);
    }
    if (e != cudaSuccess) return POISFFT_ERR_CUDA;
  }
  if (p->profiling && record_event(p, st) != POISFFT_OK) return POISFFT_ERR_CUDA;
  return POISFFT_OK;
}

template <typename T>
int enqueue(poisfft_plan* p, void* phi, const void* g, cudaStream_t st) {
  const long long nx = p->nx, nxy = (long long)p->nx * p->ny;
  return enqueue<T>(p, phi, g, st, FieldStrides{nx, nxy, nx, nxy});
}

// ---------------------------------------------------------------------------
// host-side planning shared by poisfft_plan_create and poisfft_solve_noalloc
// ---------------------------------------------------------------------------
struct PlanArgs {
  int dims = 0;
  int bc[3] = {POISFFT_P, POISFFT_P, POISFFT_P};
  long long n[3] = {1, 1, 1};
  double L[3] = {1.0, 1.0, 1.0};
  int approx = POISFFT_FD2;
  int dtype = POISFFT_F32;
};

// Argument checks of the plan-creating calls (no CUDA call).
int validate_args(int dims, const int64_t n[], const double L[], const int bc[], int approx, int dtype,
                  PlanArgs& a) {
  if (!n || !L || !bc || dims < 1 || dims > 3) return POISFFT_ERR_INVALID_ARG;
  if (approx != POISFFT_SPECTRAL && approx != POISFFT_FD2) return POISFFT_ERR_INVALID_ARG;
  if (dtype != POISFFT_F32 && dtype != POISFFT_F64 && dtype != POISFFT_MIXED && dtype != POISFFT_BF16X3)
    return POISFFT_ERR_INVALID_ARG;
  a.dims = dims;
  a.approx = approx;
  a.dtype = dtype;
  for (int ax = 0; ax < dims; ax++) {
    if (n[ax] < 1 || n[ax] > (1 << 24)) return POISFFT_ERR_INVALID_ARG;
    if (!(L[ax] > 0.0) || !isfinite(L[ax])) return POISFFT_ERR_INVALID_ARG;
    const int b0 = bc[2 * ax], b1 = bc[2 * ax + 1];
    if (b0 < POISFFT_P || b0 > POISFFT_NS || b1 < POISFFT_P || b1 > POISFFT_NS) return POISFFT_ERR_INVALID_ARG;
    if (b0 != b1) return POISFFT_ERR_UNSUPPORTED_BC;
    if (b0 == POISFFT_NR && n[ax] < 2) return POISFFT_ERR_INVALID_ARG;
    a.bc[ax] = b0;
    a.n[ax] = n[ax];
    a.L[ax] = L[ax];
  }
  // the mixed form refines with the FD2 operator (Eq. FD2-Laplace)
  if (dtype == POISFFT_MIXED && approx != POISFFT_FD2) return POISFFT_ERR_NOT_IMPLEMENTED;
  if ((double)a.n[0] * a.n[1] * a.n[2] > 4.0e10) return POISFFT_ERR_UNSUPPORTED_SIZE;
  return POISFFT_OK;
}

// Sweep sequence of the general kernels with the eigenvalue divide fused
// into the sweep of `fused_axis` (3D: 1 or 2; the other strided axis is
// transformed forward before it and backward after it; 2D: 1).
int plan_general_sequence(poisfft_plan* p, int fused_axis, std::vector<SweepLaunch>& sw) {
  SweepLaunch Ls;
  int rc;
  sw.clear();
  const int other = fused_axis == 2 ? 1 : 2;
  if ((rc = plan_x_sweep(p, 0, Ls)) != POISFFT_OK) return rc;
  sw.push_back(Ls);
  if (p->dims == 3) {
    if ((rc = plan_strided_sweep(p, other, 0, Ls)) != POISFFT_OK) return rc;
    sw.push_back(Ls);
  }
  if ((rc = plan_strided_sweep(p, fused_axis, 2, Ls)) != POISFFT_OK) return rc;
  sw.push_back(Ls);
  if (p->dims == 3) {
    if ((rc = plan_strided_sweep(p, other, 1, Ls)) != POISFFT_OK) return rc;
    sw.push_back(Ls);
  }
  if ((rc = plan_x_sweep(p, 1, Ls)) != POISFFT_OK) return rc;
  sw.push_back(Ls);
  p->fused_axis = fused_axis;
  return POISFFT_OK;
}

// Everything of a plan that needs no device: axes with their FP64 tables,
// the workspace shape, tiles and the sweep sequence.  general_only plans
// use the general kernels only and no separate pair-divide pass, so their
// sweeps are x sweeps (kind 0) and strided sweeps (kind 1) only; x
// non-periodic with a periodic y or z then returns
// POISFFT_ERR_NOT_IMPLEMENTED.  No CUDA call.
int plan_host(poisfft_plan* p, const PlanArgs& a, bool general_only) {
  if (g_fault.size) return POISFFT_ERR_UNSUPPORTED_SIZE;
  const int dims = a.dims;
  // x periodic -> half-spectrum workspace; otherwise the real transformed
  // field viewed as complex pairs.  x non-periodic with a periodic y or z
  // divides in a separate pass that pairs k with -k (PairDivideArgs).
  const bool xper = a.bc[0] == POISFFT_P;
  bool any_per_yz = false;
  for (int ax = 1; ax < dims; ax++) any_per_yz |= a.bc[ax] == POISFFT_P;
  if (general_only && !xper && any_per_yz) return POISFFT_ERR_NOT_IMPLEMENTED;
  p->dims = dims;
  p->dtype = a.dtype;
  p->approx = a.approx;
  p->nx = (int)a.n[0];
  p->ny = (int)a.n[1];
  p->nz = (int)a.n[2];
  p->esize = a.dtype == POISFFT_F64 ? 8 : 4;  // the mixed form solves in FP32
  p->r2c = xper ? 1 : 0;
  const int emax = p->esize == 4 ? 40 : 16;
  bool sing = true;
  for (int ax = 0; ax < 3; ax++) {
    const bool null_axis = ax >= dims;
    const int rc = build_axis(p->axes[ax], a.bc[ax], (int)a.n[ax], a.L[ax], a.approx, emax, null_axis);
    if (rc != POISFFT_OK) return rc;
    if (!null_axis) sing = sing && (a.bc[ax] == POISFFT_P || a.bc[ax] == POISFFT_NR || a.bc[ax] == POISFFT_NS);
  }
  p->singular = sing ? 1 : 0;
  p->ncols = p->r2c ? p->nx / 2 + 1 : (p->nx + 1) / 2;
  p->pitch = (int)workspace_pitch(p->ncols, p->esize);
  p->field_bytes = (size_t)p->nx * p->ny * p->nz * p->esize;
  p->ws_bytes = (size_t)p->pitch * 2 * p->esize * p->ny * p->nz;

  // sweep sequence and tiling
  std::vector<SweepLaunch> sw;
  SweepLaunch Ls;
  int rc;
  p->fast = !general_only && fast_eligible(p);
  if (p->fast) {
    plan_fast_x(p, fast::FM_FWD, Ls);
    sw.push_back(Ls);
    if (dims == 3) { plan_fast_strided(p, 1, fast::FM_FWD, Ls); sw.push_back(Ls); }
    plan_fast_strided(p, dims == 3 ? 2 : 1, fast::FM_FUSED, Ls);
    sw.push_back(Ls);
    if (dims == 3) { plan_fast_strided(p, 1, fast::FM_INV, Ls); sw.push_back(Ls); }
    plan_fast_x(p, fast::FM_INV, Ls);
    sw.push_back(Ls);
  } else if (!xper && any_per_yz) {
    if ((rc = plan_x_sweep(p, 0, Ls)) != POISFFT_OK) return rc;
    sw.push_back(Ls);
    for (int ax = 1; ax < dims; ax++) {
      if ((rc = plan_strided_sweep(p, ax, 0, Ls)) != POISFFT_OK) return rc;
      sw.push_back(Ls);
    }
    memset(&Ls, 0, sizeof(Ls));
    Ls.kind = 4;
    PairDivideArgs& d = Ls.pda;
    d.pitch = p->pitch;
    d.ncols = p->ncols;
    d.dncols = make_fastdiv((uint32_t)p->ncols);
    if ((long long)p->ncols * p->ny > 0x7fffffffLL) return POISFFT_ERR_UNSUPPORTED_SIZE;
    d.nx = p->nx;
    d.ny = p->ny;
    d.nz = p->nz;
    d.per_y = dims >= 2 && a.bc[1] == POISFFT_P;
    d.per_z = dims >= 3 && a.bc[2] == POISFFT_P;
    double sc = 1.0;
    for (int i = 0; i < 3; i++) sc *= p->axes[i].scale;
    d.scale = sc;
    d.singular = p->singular;
    Ls.bytes = 2LL * p->ncols * (long long)p->ny * p->nz * (long long)(2 * p->esize);
    sw.push_back(Ls);
    for (int ax = dims - 1; ax >= 1; ax--) {
      if ((rc = plan_strided_sweep(p, ax, 1, Ls)) != POISFFT_OK) return rc;
      sw.push_back(Ls);
    }
    if ((rc = plan_x_sweep(p, 1, Ls)) != POISFFT_OK) return rc;
    sw.push_back(Ls);
  } else {
    if ((rc = plan_general_sequence(p, dims == 3 ? 2 : 1, sw)) != POISFFT_OK) return rc;
  }
  p->sweeps = sw;
  if (a.dtype == POISFFT_BF16X3) {
    // the tensor-core sweeps take 1024-point strided axes: DFT forward and
    // backward sweeps, and the fused sweep of a DFT or DCT-II/DST-II axis
    int ntc = 0;
    for (auto& L : p->sweeps) {
      if (L.kind != 3 || L.M != tc::kM || L.w != tc::kW) continue;
      const bool ok = (L.fmode == fast::FM_FUSED && (L.fkind == fast::FK_DFT || L.fkind == fast::FK_DCT)) ||
                      (L.fmode != fast::FM_FUSED && L.fkind == fast::FK_DFT);
      if (!ok) continue;
      L.tc = 1;
      L.tc_tiles = (int)L.grid;
      ntc++;
    }
    if (ntc == 0) return POISFFT_ERR_NOT_IMPLEMENTED;
  }
  return POISFFT_OK;
}

// Point the general-path launches at the plan's device buffers (the sweeps
// are planned before the buffers exist).
void patch_general(poisfft_plan* p) {
  for (auto& L : p->sweeps) {
    if (L.kind == 0) {
      L.xa.tables = p->tables[0];
      L.xa.perm = p->perm[0];
      L.xa.ws = p->ws;
      L.xa.err = p->err;
    } else if (L.kind == 4) {
      L.pda.data = p->ws;
      L.pda.lam_x = p->lam[0];
      L.pda.lam_y = p->lam[1];
      L.pda.lam_z = p->lam[2];
    } else if (L.kind == 1) {
      const int a = L.sa.axis_dim;
      L.sa.tables = p->tables[a];
      L.sa.perm = p->perm[a];
      L.sa.data = p->ws;
      L.sa.lam_in = p->lam[0];
      L.sa.lam_ax = p->lam[a];
      L.sa.lam_out = p->lam[a == 1 ? 2 : 1];
      L.sa.err = p->err;
    }
  }
}

// Tensor-core sweeps: upload the DFT-matrix operands and size the
// persistent grids (two CTAs per SM).
int tc_setup(poisfft_plan* p) {
  std::vector<uint16_t> b(tc::kBmatBytes / 2);
  tc_build_bmat(b.data());
  if (dev_malloc(&p->tcb, tc::kBmatBytes) != cudaSuccess) return POISFFT_ERR_ALLOC;
  if (cudaMemcpy(p->tcb, b.data(), tc::kBmatBytes, cudaMemcpyHostToDevice) != cudaSuccess) return POISFFT_ERR_CUDA;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return POISFFT_ERR_CUDA;
  int slots = 0;
  for (auto& L : p->sweeps)
    if (L.tc) {
      L.grid = (unsigned)std::min<long long>(L.tc_tiles, 2LL * sms);
      L.tc_slot = slots++;
    }
  if (dev_malloc(&p->tc_ctr, (size_t)slots * sizeof(int)) != cudaSuccess) return POISFFT_ERR_ALLOC;
  return POISFFT_OK;
}

// The FFT solve of the plan's kernels on arrays of its kernel precision.
int solve_core(poisfft_plan* p, void* phi, const void* g, cudaStream_t st) {
  if (((uintptr_t)phi % p->esize) != 0 || ((uintptr_t)g % p->esize) != 0) return POISFFT_ERR_MISALIGNED;
  return p->esize == 4 ? enqueue<float>(p, phi, g, st) : enqueue<double>(p, phi, g, st);
}

// Bytes of one caller field (the mixed form takes doubles).
size_t user_field_bytes(const poisfft_plan* p) {
  return (size_t)p->nx * p->ny * p->nz * (p->dtype == POISFFT_MIXED ? 8 : p->esize);
}

}  // namespace

extern "C" {

const char* poisfft_status_string(int status) {
  switch (status) {
    case POISFFT_OK: return "ok";
    case POISFFT_ERR_INVALID_ARG: return "invalid argument";
    case POISFFT_ERR_UNSUPPORTED_BC: return "unsupported boundary-condition combination";
    case POISFFT_ERR_UNSUPPORTED_SIZE: return "unsupported grid size";
    case POISFFT_ERR_ALLOC: return "allocation failed";
    case POISFFT_ERR_CUDA: return "CUDA error";
    case POISFFT_ERR_MISALIGNED: return "misaligned pointer";
    case POISFFT_ERR_TIMEOUT: return "device wait timed out";
    case POISFFT_ERR_NOT_IMPLEMENTED: return "not implemented";
    default: return "unknown status";
  }
}

int poisfft_plan_create(poisfft_plan** out, int dims, const int64_t n[], const double L[], const int bc[],
                        int approx, int dtype) {
  if (!out) return POISFFT_ERR_INVALID_ARG;
  *out = nullptr;
  FaultScope fault;
  PlanArgs args;
  int rc = validate_args(dims, n, L, bc, approx, dtype, args);
  if (rc != POISFFT_OK) return rc;
  poisfft_plan* p = new (std::nothrow) poisfft_plan();
  if (!p) return POISFFT_ERR_ALLOC;
  if ((rc = plan_host(p, args, false)) != POISFFT_OK) { free_plan(p); return rc; }

  // device resources
  if (dev_malloc(&p->err, sizeof(int)) != cudaSuccess) { cudaGetLastError(); free_plan(p); return POISFFT_ERR_CUDA; }
  if (cudaMemset(p->err, 0, sizeof(int)) != cudaSuccess) { free_plan(p); return POISFFT_ERR_CUDA; }
  if (dev_malloc(&p->ws, p->ws_bytes) != cudaSuccess) { cudaGetLastError(); free_plan(p); return POISFFT_ERR_ALLOC; }
  if (cudaMemset(p->ws, 0, p->ws_bytes) != cudaSuccess) { free_plan(p); return POISFFT_ERR_CUDA; }
  rc = p->esize == 4 ? upload_tables<float>(p) : upload_tables<double>(p);
  for (int a = 0; p->fast && a < dims && rc == POISFFT_OK; a++) rc = fast_upload_axis(p, a);
  if (rc != POISFFT_OK) { cudaGetLastError(); free_plan(p); return rc; }
  if (p->fast) patch_fast(p);
  patch_general(p);
  if (rc == POISFFT_OK && p->dtype == POISFFT_BF16X3) rc = tc_setup(p);
  if (rc != POISFFT_OK) { cudaGetLastError(); free_plan(p); return rc; }
  if ((rc = encode_maps(p)) != POISFFT_OK) { free_plan(p); return rc; }
  *out = p;
  return POISFFT_OK;
}

int poisfft_solve(poisfft_plan* p, void* phi, const void* g, void* stream) {
  if (!p || !phi || !g) return POISFFT_ERR_INVALID_ARG;
  if (p->dtype == POISFFT_MIXED)
    return poisfft_solve_refined(p, static_cast<double*>(phi), static_cast<const double*>(g), p->refinements, stream);
  return solve_core(p, phi, g, reinterpret_cast<cudaStream_t>(stream));
}

int poisfft_plan_set_refinements(poisfft_plan* p, int refinements) {
  if (!p || p->dtype != POISFFT_MIXED || refinements < 0 || refinements > 8) return POISFFT_ERR_INVALID_ARG;
  p->refinements = refinements;
  return POISFFT_OK;
}

int poisfft_solve_strided(poisfft_plan* p, void* phi, const int64_t phi_ld[2], const void* g, const int64_t g_ld[2],
                          void* stream) {
  if (!p || !phi || !g || !phi_ld || !g_ld) return POISFFT_ERR_INVALID_ARG;
  if (p->dtype == POISFFT_MIXED) return POISFFT_ERR_NOT_IMPLEMENTED;
  if (((uintptr_t)phi % p->esize) != 0 || ((uintptr_t)g % p->esize) != 0) return POISFFT_ERR_MISALIGNED;
  const long long nx = p->nx, ny = p->ny;
  const long long gy = p->dims >= 2 ? g_ld[0] : nx, pyy = p->dims >= 2 ? phi_ld[0] : nx;
  const long long gz = p->dims >= 3 ? g_ld[1] : gy * ny, pz = p->dims >= 3 ? phi_ld[1] : pyy * ny;
  if (gy < nx || pyy < nx || gz < gy * ny || pz < pyy * ny) return POISFFT_ERR_INVALID_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const FieldStrides fs{gy, gz, pyy, pz};
  return p->esize == 4 ? enqueue<float>(p, phi, g, st, fs) : enqueue<double>(p, phi, g, st, fs);
}

int poisfft_solve_host(poisfft_plan* p, void* phi_host, const void* g_host, void* stream) {
  if (!p || !phi_host || !g_host) return POISFFT_ERR_INVALID_ARG;
  FaultScope fault;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const size_t fb = user_field_bytes(p);
  if (!p->stage_g) {
    if (dev_malloc(&p->stage_g, fb) != cudaSuccess) { cudaGetLastError(); p->stage_g = nullptr; return POISFFT_ERR_ALLOC; }
  }
  if (!p->stage_phi) {
    if (dev_malloc(&p->stage_phi, fb) != cudaSuccess) { cudaGetLastError(); p->stage_phi = nullptr; return POISFFT_ERR_ALLOC; }
  }
  if (cudaMemcpyAsync(p->stage_g, g_host, fb, cudaMemcpyHostToDevice, st) != cudaSuccess)
    return POISFFT_ERR_CUDA;
  int rc = poisfft_solve(p, p->stage_phi, p->stage_g, stream);
  if (rc != POISFFT_OK) return rc;
  if (cudaMemcpyAsync(phi_host, p->stage_phi, fb, cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return POISFFT_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return POISFFT_ERR_CUDA;
  return POISFFT_OK;
}

int poisfft_solve_host_async(poisfft_plan* p, void* phi_host, const void* g_host, void* stream) {
  if (!p || !phi_host || !g_host) return POISFFT_ERR_INVALID_ARG;
  FaultScope fault;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const size_t fb = user_field_bytes(p);
  auto& q = p->pipe;
  if (!q.ready) {
    bool ok = true;
    for (int b = 0; b < 2 && ok; b++)
      ok = dev_malloc(&q.g[b], fb) == cudaSuccess && dev_malloc(&q.phi[b], fb) == cudaSuccess;
    if (!ok) {
      cudaGetLastError();
      release_host_pipe(p);
      return POISFFT_ERR_ALLOC;
    }
    ok = cudaStreamCreateWithFlags(&q.in, cudaStreamNonBlocking) == cudaSuccess &&
         cudaStreamCreateWithFlags(&q.out, cudaStreamNonBlocking) == cudaSuccess;
    for (int b = 0; b < 2 && ok; b++)
      ok = cudaEventCreateWithFlags(&q.copied_in[b], cudaEventDisableTiming) == cudaSuccess &&
           cudaEventCreateWithFlags(&q.solved[b], cudaEventDisableTiming) == cudaSuccess &&
           cudaEventCreateWithFlags(&q.copied_out[b], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
      cudaGetLastError();
      release_host_pipe(p);
      return POISFFT_ERR_CUDA;
    }
    q.ready = true;
  }
  const int b = q.next;
  // input copy into staging pair b, once the solve of two calls ago has read it
  if (q.used[b] && cudaStreamWaitEvent(q.in, q.solved[b], 0) != cudaSuccess) return POISFFT_ERR_CUDA;
  if (cudaMemcpyAsync(q.g[b], g_host, fb, cudaMemcpyHostToDevice, q.in) != cudaSuccess ||
      cudaEventRecord(q.copied_in[b], q.in) != cudaSuccess)
    return POISFFT_ERR_CUDA;
  // the solve on the caller's stream: after the input copy, and after the
  // result copy of two calls ago has read staging field phi[b]
  if (cudaStreamWaitEvent(st, q.copied_in[b], 0) != cudaSuccess) return POISFFT_ERR_CUDA;
  if (q.used[b] && cudaStreamWaitEvent(st, q.copied_out[b], 0) != cudaSuccess) return POISFFT_ERR_CUDA;
  int rc = poisfft_solve(p, q.phi[b], q.g[b], stream);
  if (rc != POISFFT_OK) return rc;
  if (cudaEventRecord(q.solved[b], st) != cudaSuccess) return POISFFT_ERR_CUDA;
  // result copy.  The caller's stream follows the previous call's result
  // copy, not this one, so that the next call's solve can run beside it; at
  // most one result copy is in flight beyond the stream, and poisfft_check
  // waits for it.
  if (cudaStreamWaitEvent(q.out, q.solved[b], 0) != cudaSuccess ||
      cudaMemcpyAsync(phi_host, q.phi[b], fb, cudaMemcpyDeviceToHost, q.out) != cudaSuccess ||
      cudaEventRecord(q.copied_out[b], q.out) != cudaSuccess)
    return POISFFT_ERR_CUDA;
  if (q.used[b ^ 1] && cudaStreamWaitEvent(st, q.copied_out[b ^ 1], 0) != cudaSuccess) return POISFFT_ERR_CUDA;
  q.used[b] = true;
  q.next = b ^ 1;
  return POISFFT_OK;
}

int poisfft_check(poisfft_plan* p, void* stream) {
  if (!p) return POISFFT_ERR_INVALID_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (cudaStreamSynchronize(st) != cudaSuccess) return POISFFT_ERR_CUDA;
  // the last result copy of poisfft_solve_host_async
  if (p->pipe.ready && cudaStreamSynchronize(p->pipe.out) != cudaSuccess) return POISFFT_ERR_CUDA;
  int h = 0;
  if (cudaMemcpy(&h, p->err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return POISFFT_ERR_CUDA;
  if (h != 0) {
    cudaMemset(p->err, 0, sizeof(int));
    return POISFFT_ERR_TIMEOUT;
  }
  return POISFFT_OK;
}

int poisfft_destroy(poisfft_plan* p) {
  free_plan(p);
  return POISFFT_OK;
}

int poisfft_profile_enable(poisfft_plan* p, int enable) {
  if (!p) return POISFFT_ERR_INVALID_ARG;
  p->profiling = enable != 0;
  return POISFFT_OK;
}

int poisfft_profile_read(poisfft_plan* p, double* ms, int cap, int* nlaunch, int* nsolves) {
  if (!p || !nlaunch || !nsolves || (cap > 0 && !ms)) return POISFFT_ERR_INVALID_ARG;
  const int nl = (int)p->sweeps.size();
  const int per = nl + 1;
  const int ns = (int)(p->events.size() / per);
  *nlaunch = nl;
  *nsolves = ns;
  for (int i = 0; i < cap && i < nl; i++) ms[i] = 0.0;
  int rc = POISFFT_OK;
  if (ns > 0 && cudaEventSynchronize(p->events[(size_t)ns * per - 1]) != cudaSuccess) rc = POISFFT_ERR_CUDA;
  for (int s = 0; s < ns && rc == POISFFT_OK; s++)
    for (int i = 0; i < nl && i < cap; i++) {
      float t = 0.f;
      if (cudaEventElapsedTime(&t, p->events[(size_t)s * per + i], p->events[(size_t)s * per + i + 1]) != cudaSuccess) {
        rc = POISFFT_ERR_CUDA;
        break;
      }
      ms[i] += t;
    }
  for (cudaEvent_t e : p->events) cudaEventDestroy(e);
  p->events.clear();
  return rc;
}

int poisfft_launch_info(const poisfft_plan* p, int i, int64_t out[4]) {
  if (!p || !out || i < 0 || i >= (int)p->sweeps.size()) return POISFFT_ERR_INVALID_ARG;
  const SweepLaunch& L = p->sweeps[i];
  out[0] = L.bytes;
  out[1] = (L.kind == 0 || L.kind == 2) ? 0 : (L.kind == 4 ? 2 : (L.tc ? 3 : 1));
  if (L.kind == 4) {
    out[2] = 2;
    out[3] = 0;
  } else if (L.kind >= 2) {
    out[2] = L.fmode;
    out[3] = L.axis;
  } else {
    out[2] = L.kind == 0 ? L.xa.mode : L.sa.mode;
    out[3] = L.kind == 0 ? 0 : L.sa.axis_dim;
  }
  return POISFFT_OK;
}

int poisfft_plan_info(const poisfft_plan* p, int64_t info[4]) {
  if (!p || !info) return POISFFT_ERR_INVALID_ARG;
  info[0] = (int64_t)p->sweeps.size();
  info[1] = (int64_t)p->ws_bytes;
  int64_t best = -1, idx = 0;
  for (size_t i = 0; i < p->sweeps.size(); i++)
    if (p->sweeps[i].bytes > best) { best = p->sweeps[i].bytes; idx = (int64_t)i; }
  info[2] = best;
  info[3] = idx;
  return POISFFT_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Zero mode of singular problems, reported in FP64
// ---------------------------------------------------------------------------
// The solve sets the all-zero spectral coefficient to 0, i.e. removes the
// weighted mean of g (weights 1/2 at both ends of NR axes, 1 elsewhere).
// Per-thread sums are compensated (Kahan) for FP32 data and plain for FP64
// data; the cross-thread sum is FP64 and deterministic.
namespace {

template <typename T>
__global__ void __launch_bounds__(pf::kReduceBlock) zero_mode_kernel(const T* __restrict__ g, int nx, int ny, int nz,
                                                                      int trap_x, int trap_y, int trap_z,
                                                                      pf::Reduce R, double* out) {
  // blocks take whole x rows: the y/z weight is fixed per row, x is coalesced
  const long long rows = (long long)ny * nz;
  T s = T(0), c = T(0);
  for (long long r = blockIdx.x; r < rows; r += gridDim.x) {
    const int y = (int)(r % ny), z = (int)(r / ny);
    T wr = T(1);
    if (trap_y && (y == 0 || y == ny - 1)) wr *= T(0.5);
    if (trap_z && (z == 0 || z == nz - 1)) wr *= T(0.5);
    const T* row = g + r * nx;
    for (int x = threadIdx.x; x < nx; x += blockDim.x) {
      const T w = (trap_x && (x == 0 || x == nx - 1)) ? T(0.5) * wr : wr;
      if constexpr (sizeof(T) == 8) {
        // FP64 data: a plain FP64 sum of a few thousand terms per thread is
        // accurate to ~1e-13 of the sum of magnitudes, and GB300's FP64 rate
        // makes the compensated form four times as expensive
        s = fma(w, row[x], s);
      } else {
        const T yv = w * row[x] - c;
        const T t = s + yv;
        c = (t - s) - yv;
        s = t;
      }
    }
  }
  const double v[1] = {(double)s - (double)c};
  double* const d[1] = {out};
  pf::grid_sum<1>(v, R, d);
}

}  // namespace

namespace {

// Launches the weighted sum of g (FP32 or FP64 data) into p->zm[0].
int zero_mode_sum(poisfft_plan* p, const void* g, bool f64, cudaStream_t st) {
  const long long N = (long long)p->nx * p->ny * p->nz;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return POISFFT_ERR_CUDA;
  const unsigned nb = (unsigned)std::max<long long>(1, std::min<long long>((N + 255) / 256, (long long)sms * 8));
  if (!p->zm) {
    if (dev_malloc(&p->zm, (1 + (size_t)sms * 8) * sizeof(double)) != cudaSuccess ||
        dev_malloc(&p->zm_count, sizeof(unsigned)) != cudaSuccess ||
        cudaMemset(p->zm_count, 0, sizeof(unsigned)) != cudaSuccess) {
      cudaGetLastError();
      return POISFFT_ERR_ALLOC;
    }
  }
  const pf::Reduce R{p->zm + 1, p->zm_count};
  const int tx = p->axes[0].bc == POISFFT_NR, ty = p->dims >= 2 && p->axes[1].bc == POISFFT_NR,
            tz = p->dims >= 3 && p->axes[2].bc == POISFFT_NR;
  if (!f64)
    zero_mode_kernel<float><<<nb, pf::kReduceBlock, 0, st>>>(static_cast<const float*>(g), p->nx, p->ny, p->nz, tx,
                                                             ty, tz, R, p->zm);
  else
    zero_mode_kernel<double><<<nb, pf::kReduceBlock, 0, st>>>(static_cast<const double*>(g), p->nx, p->ny, p->nz,
                                                              tx, ty, tz, R, p->zm);
  return cudaGetLastError() == cudaSuccess ? POISFFT_OK : POISFFT_ERR_CUDA;
}

// Sum of the weights of the zero-mode mean (NR axes: n - 1, others n).
double zero_mode_weight(const poisfft_plan* p) {
  double wsum = 1.0;
  const int nn[3] = {p->nx, p->ny, p->nz};
  for (int a = 0; a < 3; a++) wsum *= (a < p->dims && p->axes[a].bc == POISFFT_NR) ? nn[a] - 1.0 : (double)nn[a];
  return wsum;
}

}  // namespace

extern "C" int poisfft_zero_mode_mean(poisfft_plan* p, const void* g, double* mean, void* stream) {
  if (!p || !g || !mean) return POISFFT_ERR_INVALID_ARG;
  if (!p->singular) return POISFFT_ERR_INVALID_ARG;
  FaultScope fault;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  int rc = zero_mode_sum(p, g, p->esize == 8 || p->dtype == POISFFT_MIXED, st);
  if (rc != POISFFT_OK) return rc;
  double sum = 0.0;
  if (cudaMemcpyAsync(&sum, p->zm, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return POISFFT_ERR_CUDA;
  *mean = sum / zero_mode_weight(p);
  return POISFFT_OK;
}

// ---------------------------------------------------------------------------
// Mixed-precision solve by iterative refinement
// ---------------------------------------------------------------------------
// FP64 data, FP32 FFT solves: phi_0 = S(g), phi_{k+1} = phi_k + S(g - L phi_k),
// where S is the FP32 solve of this plan and L the second-order FD operator
// whose eigenvalues the solve divides by (Eq. FD2-Laplace in every axis, with
// the boundary ghost values that make the Table 2 bases its eigenvectors:
// P wraps; DR phi_{-1} = phi_n = 0; DS phi_{-1} = -phi_0, phi_n = -phi_{n-1};
// NS phi_{-1} = phi_0, phi_n = phi_{n-1}; NR phi_{-1} = phi_1,
// phi_n = phi_{n-2}).  The residual is formed in FP64 and rounded to FP32
// for the correction solve; each step multiplies the error by about the FP32
// solve's relative accuracy, down to the floor set by the FP64 residual
// (about cond(L) times the FP64 unit roundoff).  For singular problems every
// S removes the zero mode, so the iteration converges to the solution the
// FP64 solve gives.
namespace {

struct Fd2Axis {
  int n;         // points (1: absent axis)
  int bc;        // POISFFT_P .. POISFFT_NS
  long long s;   // element stride
  double w;      // 1 / dx^2
};

// phi_{i-1} + phi_{i+1} along one axis with the ghost values of its BC
// (0 for an absent axis, whose weight is 0; an axis of one point takes both
// neighbours from the BC: 2 phi_0 for P and NS, -2 phi_0 for DS, 0 for DR)
__device__ __forceinline__ double fd2_pair(const double* __restrict__ phi, long long idx, int i, const Fd2Axis& a,
                                           double c) {
  if (a.w == 0.0) return 0.0;
  double l, r;
  if (i > 0) {
    l = phi[idx - a.s];
  } else {
    switch (a.bc) {
      case POISFFT_P: l = phi[idx + (long long)(a.n - 1) * a.s]; break;
      case POISFFT_DR: l = 0.0; break;
      case POISFFT_DS: l = -c; break;
      case POISFFT_NS: l = c; break;
      default: l = phi[idx + a.s]; break;  // NR
    }
  }
  if (i < a.n - 1) {
    r = phi[idx + a.s];
  } else {
    switch (a.bc) {
      case POISFFT_P: r = phi[idx - (long long)(a.n - 1) * a.s]; break;
      case POISFFT_DR: r = 0.0; break;
      case POISFFT_DS: r = -c; break;
      case POISFFT_NS: r = c; break;
      default: r = phi[idx - a.s]; break;  // NR
    }
  }
  return l + r;
}

// Weighted mean of a field that a singular solve removes (device sum times
// the inverse weight), 0 for nonsingular plans.
__device__ __forceinline__ double mean_of(const double* zsum, double inv_w) { return zsum ? *zsum * inv_w : 0.0; }

// r = fp32(g - m - L phi) with m the removed mean of g; L phi =
// sum_a w_a (phi_{i-1} + phi_{i+1}) - 2 (sum_a w_a) phi_i (ten FP64
// operations per point: GB300 runs FP64 at a small fraction of FP32).
// grid.x covers x, grid.y strides over the rows y + ny*z.
__global__ void __launch_bounds__(256) fd2_residual_kernel(const double* __restrict__ phi,
                                                           const double* __restrict__ g, float* __restrict__ r,
                                                           Fd2Axis ax, Fd2Axis ay, Fd2Axis az, double w2, int rows,
                                                           const double* zsum, double inv_w) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= ax.n) return;
  const double m = mean_of(zsum, inv_w);
  for (int row = blockIdx.y; row < rows; row += gridDim.y) {
    const int y = row % ay.n, z = row / ay.n;
    const long long idx = (long long)row * ax.n + x;
    const double c = phi[idx];
    const double lap = fma(ax.w, fd2_pair(phi, idx, x, ax, c),
                           fma(ay.w, fd2_pair(phi, idx, y, ay, c), fma(az.w, fd2_pair(phi, idx, z, az, c), -w2 * c)));
    r[idx] = (float)((g[idx] - m) - lap);
  }
}

__global__ void to_f32_kernel(const double* __restrict__ g, float* __restrict__ r, long long N, const double* zsum,
                              double inv_w) {
  const double m = mean_of(zsum, inv_w);
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < N; e += (long long)gridDim.x * blockDim.x)
    r[e] = (float)(g[e] - m);
}

// phi -= m (the weighted mean of phi, removed at the end for singular plans)
__global__ void sub_mean_kernel(double* __restrict__ phi, long long N, const double* zsum, double inv_w) {
  const double m = mean_of(zsum, inv_w);
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < N; e += (long long)gridDim.x * blockDim.x)
    phi[e] -= m;
}

// phi = d (first step) or phi += d
__global__ void add_f32_kernel(double* __restrict__ phi, const float* __restrict__ d, long long N, int first) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < N; e += (long long)gridDim.x * blockDim.x)
    phi[e] = first ? (double)d[e] : phi[e] + (double)d[e];
}

}  // namespace

extern "C" int poisfft_solve_refined(poisfft_plan* p, double* phi, const double* g, int refinements, void* stream) {
  if (!p || !phi || !g || refinements < 0 || refinements > 8 || (const void*)phi == (const void*)g)
    return POISFFT_ERR_INVALID_ARG;
  if ((p->dtype != POISFFT_F32 && p->dtype != POISFFT_MIXED) || p->approx != POISFFT_FD2) return POISFFT_ERR_INVALID_ARG;
  if ((uintptr_t)phi % 8 != 0 || (uintptr_t)g % 8 != 0) return POISFFT_ERR_MISALIGNED;
  FaultScope fault;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const long long N = (long long)p->nx * p->ny * p->nz;
  if (!p->refine_r && dev_malloc(&p->refine_r, (size_t)N * sizeof(float)) != cudaSuccess) {
    cudaGetLastError();
    p->refine_r = nullptr;
    return POISFFT_ERR_ALLOC;
  }
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return POISFFT_ERR_CUDA;
  Fd2Axis A[3];
  const int nn[3] = {p->nx, p->ny, p->nz};
  long long stride = 1;
  for (int a = 0; a < 3; a++) {
    A[a].n = nn[a];
    A[a].bc = p->axes[a].bc;
    A[a].s = stride;
    stride *= nn[a];
    double dx = p->axes[a].L / nn[a];
    if (A[a].bc == POISFFT_DR) dx = p->axes[a].L / (nn[a] + 1);
    if (A[a].bc == POISFFT_NR) dx = p->axes[a].L / (nn[a] - 1);
    A[a].w = a < p->dims ? 1.0 / (dx * dx) : 0.0;
    if (a >= p->dims) A[a].n = 1;
  }
  double w2 = 0.0;
  for (int a = 0; a < 3; a++) w2 += 2.0 * A[a].w;
  const unsigned g1 = (unsigned)std::min<long long>((N + 255) / 256, 32LL * sms);
  const int rows = p->ny * p->nz;
  const dim3 gr((unsigned)((p->nx + 255) / 256), (unsigned)std::min(rows, 65535));
  // singular problems: the null-space component (the weighted mean of g,
  // which every solve removes) is subtracted in FP64 first, so that the
  // FP32 residuals carry only the part the corrections resolve
  const double* zsum = nullptr;
  double inv_w = 0.0;
  int rc = POISFFT_OK;
  if (p->singular) {
    if ((rc = zero_mode_sum(p, g, true, st)) != POISFFT_OK) return rc;
    zsum = p->zm;
    inv_w = 1.0 / zero_mode_weight(p);
  }
  to_f32_kernel<<<g1, 256, 0, st>>>(g, p->refine_r, N, zsum, inv_w);
  if (cudaGetLastError() != cudaSuccess) return POISFFT_ERR_CUDA;
  rc = solve_core(p, p->refine_r, p->refine_r, st);
  if (rc != POISFFT_OK) return rc;
  add_f32_kernel<<<g1, 256, 0, st>>>(phi, p->refine_r, N, 1);
  for (int k = 0; k < refinements; k++) {
    fd2_residual_kernel<<<gr, 256, 0, st>>>(phi, g, p->refine_r, A[0], A[1], A[2], w2, rows, zsum, inv_w);
    if (cudaGetLastError() != cudaSuccess) return POISFFT_ERR_CUDA;
    rc = solve_core(p, p->refine_r, p->refine_r, st);
    if (rc != POISFFT_OK) return rc;
    add_f32_kernel<<<g1, 256, 0, st>>>(phi, p->refine_r, N, 0);
  }
  // the residual cannot see a constant (L 1 = 0): the FP32 rounding of the
  // solves' zero modes stays in phi unless its weighted mean is removed in FP64
  if (p->singular) {
    if ((rc = zero_mode_sum(p, phi, true, st)) != POISFFT_OK) return rc;
    sub_mean_kernel<<<g1, 256, 0, st>>>(phi, N, p->zm, inv_w);
  }
  return cudaGetLastError() == cudaSuccess ? POISFFT_OK : POISFFT_ERR_CUDA;
}

// ---------------------------------------------------------------------------
// Solve without device allocation
// ---------------------------------------------------------------------------
// Some callers cannot call cudaMalloc: code running under a framework that
// owns all device memory through its own pool or budget, plug-ins that may
// not change the device footprint after start-up, or code paths that must
// not trigger an implicit device synchronisation.  For them,
// poisfft_solve_noalloc solves one problem with the same sweep kernels, but
// its workspace, tables and error flag live in the file-scope array below,
// which every GPU that loads this library holds until the process exits.
namespace {

constexpr size_t kNoAllocBytes = 32u << 20;  // 32 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kMaxDevices = 64;
void* g_noalloc_ptr[kMaxDevices] = {};
std::mutex g_noalloc_mutex;

// Device address of g_noalloc_scratch on the current device (set-up once per
// device; the host-side symbol itself is not a device address).
int noalloc_scratch(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return POISFFT_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_ptr[dev]) {
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) {
      cudaGetLastError();
      return POISFFT_ERR_CUDA;
    }
    g_noalloc_ptr[dev] = ptr;
  }
  *out = g_noalloc_ptr[dev];
  return POISFFT_OK;
}

size_t align256(size_t v) { return (v + 255) / 256 * 256; }

template <typename T>
int noalloc_upload(poisfft_plan* p, unsigned char* base, size_t& off, cudaStream_t st) {
  for (int a = 0; a < 3; a++) {
    AxisPlan& ax = p->axes[a];
    const size_t nt = ax.tab_re.size();
    std::vector<T> tab(2 * nt);
    for (size_t i = 0; i < nt; i++) { tab[2 * i] = (T)ax.tab_re[i]; tab[2 * i + 1] = (T)ax.tab_im[i]; }
    std::vector<T> lam(std::max<size_t>(ax.lam.size(), 1), T(0));
    for (size_t i = 0; i < ax.lam.size(); i++) lam[i] = (T)ax.lam[i];
    p->tables[a] = base + off;
    off = align256(off + tab.size() * sizeof(T));
    p->lam[a] = base + off;
    off = align256(off + lam.size() * sizeof(T));
    p->perm[a] = reinterpret_cast<int*>(base + off);
    off = align256(off + ax.perm.size() * sizeof(int));
    if (off > kNoAllocBytes) return POISFFT_ERR_UNSUPPORTED_SIZE;
    // pageable sources: each copy has consumed its host buffer when it returns
    if (cudaMemcpyAsync(p->tables[a], tab.data(), tab.size() * sizeof(T), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(p->lam[a], lam.data(), lam.size() * sizeof(T), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(p->perm[a], ax.perm.data(), ax.perm.size() * sizeof(int), cudaMemcpyHostToDevice, st) !=
            cudaSuccess)
      return POISFFT_ERR_CUDA;
  }
  return POISFFT_OK;
}

// Forget the carved-out pointers, then free the host-side plan object.
void release_noalloc_plan(poisfft_plan* p) {
  p->ws = nullptr;
  p->err = nullptr;
  for (int a = 0; a < 3; a++) {
    p->tables[a] = nullptr;
    p->lam[a] = nullptr;
    p->perm[a] = nullptr;
  }
  delete p;
}

}  // namespace

extern "C" int poisfft_solve_noalloc(int dims, const int64_t n[], const double L[], const int bc[], int approx,
                                     int dtype, void* phi, const void* g, void* stream) {
  if (!phi || !g) return POISFFT_ERR_INVALID_ARG;
  PlanArgs args;
  int rc = validate_args(dims, n, L, bc, approx, dtype, args);
  if (rc != POISFFT_OK) return rc;
  if (dtype == POISFFT_MIXED || dtype == POISFFT_BF16X3) return POISFFT_ERR_NOT_IMPLEMENTED;
  const size_t esize = dtype == POISFFT_F32 ? 4 : 8;
  if (((uintptr_t)phi % esize) != 0 || ((uintptr_t)g % esize) != 0) return POISFFT_ERR_MISALIGNED;
  const bool xper = args.bc[0] == POISFFT_P;
  bool any_per_yz = false;
  for (int a = 1; a < dims; a++) any_per_yz |= args.bc[a] == POISFFT_P;
  if (!xper && any_per_yz) return POISFFT_ERR_NOT_IMPLEMENTED;
  // workspace size before any host planning: reject what cannot fit
  const long long ncols0 = xper ? args.n[0] / 2 + 1 : (args.n[0] + 1) / 2;
  const long long pitch0 = workspace_pitch(ncols0, esize);
  const double ws_need = (double)pitch0 * 2 * esize * args.n[1] * args.n[2];
  if (ws_need + 256 > (double)kNoAllocBytes) return POISFFT_ERR_UNSUPPORTED_SIZE;
  // the table copies below read host vectors that live only during this call
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) { cudaGetLastError(); return POISFFT_ERR_CUDA; }
  if (cap != cudaStreamCaptureStatusNone) return POISFFT_ERR_NOT_IMPLEMENTED;

  poisfft_plan* p = new (std::nothrow) poisfft_plan();
  if (!p) return POISFFT_ERR_ALLOC;
  if ((rc = plan_host(p, args, true)) != POISFFT_OK) { release_noalloc_plan(p); return rc; }
  for (const auto& Lw : p->sweeps)
    if (Lw.kind != 0 && Lw.kind != 1) { release_noalloc_plan(p); return POISFFT_ERR_NOT_IMPLEMENTED; }

  // carve the scratch array: error flag | tables per axis | workspace
  void* scratch = nullptr;
  if ((rc = noalloc_scratch(&scratch)) != POISFFT_OK) { release_noalloc_plan(p); return rc; }
  unsigned char* base = static_cast<unsigned char*>(scratch);
  size_t off = 0;
  p->err = reinterpret_cast<int*>(base);
  off = 256;
  rc = esize == 4 ? noalloc_upload<float>(p, base, off, st) : noalloc_upload<double>(p, base, off, st);
  if (rc == POISFFT_OK && off + p->ws_bytes > kNoAllocBytes) rc = POISFFT_ERR_UNSUPPORTED_SIZE;
  if (rc != POISFFT_OK) { cudaGetLastError(); release_noalloc_plan(p); return rc; }
  p->ws = base + off;
  // the array keeps the previous call's contents: zero the flag and the workspace
  if (cudaMemsetAsync(p->err, 0, sizeof(int), st) != cudaSuccess ||
      cudaMemsetAsync(p->ws, 0, p->ws_bytes, st) != cudaSuccess) {
    release_noalloc_plan(p);
    return POISFFT_ERR_CUDA;
  }
  patch_general(p);
  if ((rc = encode_maps(p)) == POISFFT_OK) rc = solve_core(p, phi, g, st);
  release_noalloc_plan(p);
  return rc;
}

extern "C" int poisfft_noalloc_check(void* stream) {
  void* scratch = nullptr;
  int rc = noalloc_scratch(&scratch);
  if (rc != POISFFT_OK) return rc;
  if (cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream)) != cudaSuccess) return POISFFT_ERR_CUDA;
  int h = 0;
  if (cudaMemcpy(&h, scratch, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return POISFFT_ERR_CUDA;
  if (h != 0) {
    if (cudaMemset(scratch, 0, sizeof(int)) != cudaSuccess) return POISFFT_ERR_CUDA;
    return POISFFT_ERR_TIMEOUT;
  }
  return POISFFT_OK;
}

// ---------------------------------------------------------------------------
// Autotuner of the general-path tile shapes
// ---------------------------------------------------------------------------
// For every launch of the general kernels the tuner times the planned tile
// shape and up to two smaller ones (strided sweeps: w, w/2, w/4 columns;
// x sweeps: l, l/2, l/4 line pairs per CTA) on the device, three runs each,
// and keeps the fastest.  The specialised kernels have fixed, measured shapes.
namespace {

void set_strided_width(poisfft_plan* p, SweepLaunch& L, int w) {
  StridedArgs& s = L.sa;
  const size_t per_col = strided_per_col(p, s.axis_dim, s.rows_alloc);
  s.w = w;
  s.lw = ilog2(w);
  s.ntile_c = (p->ncols + w - 1) / w;
  s.bar_off = (int)(((size_t)w * per_col + 15) / 16 * 16);
  L.grid = (unsigned)((long long)s.ntile_c * s.nouter);
  L.smem = (size_t)s.bar_off + 16;
}

void set_x_lines(poisfft_plan* p, SweepLaunch& L, int lines) {
  const size_t per_line = x_per_line(p);
  const long long pairs = ((long long)p->ny * p->nz + 1) / 2;
  L.xa.lines = lines;
  L.grid = (unsigned)((pairs + lines - 1) / lines);
  L.smem = (size_t)lines * per_line;
}

template <typename T>
float time_launch(poisfft_plan* p, SweepLaunch& L, void* phi, const void* g, cudaStream_t st, cudaEvent_t e0,
                  cudaEvent_t e1) {
  float best = 1e30f;
  for (int rep = 0; rep < 3; rep++) {
    cudaEventRecord(e0, st);
    cudaError_t e;
    if (L.kind == 0) {
      XArgs a = L.xa;
      a.g = g;
      a.phi = phi;
      a.ny = p->ny;
      a.g_sy = a.phi_sy = p->nx;
      a.g_sz = a.phi_sz = (long long)p->nx * p->ny;
      e = launch_x_sweep<T>(a, L.grid, L.smem, st);
    } else {
      e = launch_strided_sweep<T>(p->maps[L.map], L.sa, L.grid, L.smem, st);
    }
    cudaEventRecord(e1, st);
    if (e != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) return -1.f;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    best = std::min(best, ms);
  }
  return best;
}

template <typename T>
int autotune_plan(poisfft_plan* p, cudaStream_t st) {
  void* g = nullptr;
  void* phi = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = POISFFT_OK;
  if (dev_malloc(&g, p->field_bytes) != cudaSuccess || dev_malloc(&phi, p->field_bytes) != cudaSuccess ||
      cudaMemsetAsync(g, 0, p->field_bytes, st) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
      cudaEventCreate(&e1) != cudaSuccess)
    rc = POISFFT_ERR_ALLOC;
  const int wmin = p->esize == 4 ? 2 : 1;
  for (size_t li = 0; rc == POISFFT_OK && li < p->sweeps.size(); li++) {
    SweepLaunch& L = p->sweeps[li];
    if (L.kind != 0 && L.kind != 1) continue;
    const int base = L.kind == 0 ? L.xa.lines : L.sa.w;
    int best = base;
    float best_ms = 1e30f;
    for (int div = 1; div <= 4; div *= 2) {
      const int cand = base / div;
      if (L.kind == 1 && cand < wmin) break;
      if (L.kind == 0 && cand < 1) break;
      if (L.kind == 1) {
        set_strided_width(p, L, cand);
        if ((rc = encode_maps(p)) != POISFFT_OK) break;
      } else {
        set_x_lines(p, L, cand);
      }
      const float ms = time_launch<T>(p, L, phi, g, st, e0, e1);
      if (ms < 0.f) {
        rc = POISFFT_ERR_CUDA;
        break;
      }
      if (ms < best_ms * 0.97f) {  // smaller tiles must win clearly
        best_ms = ms;
        best = cand;
      }
    }
    if (L.kind == 1) set_strided_width(p, L, best);
    else set_x_lines(p, L, best);
  }
  if (rc == POISFFT_OK) rc = encode_maps(p);
  if (rc == POISFFT_OK && cudaMemsetAsync(p->ws, 0, p->ws_bytes, st) != cudaSuccess) rc = POISFFT_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess && rc == POISFFT_OK) rc = POISFFT_ERR_CUDA;
  if (g) cudaFree(g);
  if (phi) cudaFree(phi);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaGetLastError();
  return rc;
}

}  // namespace

extern "C" int poisfft_plan_autotune(poisfft_plan* p, void* stream) {
  if (!p) return POISFFT_ERR_INVALID_ARG;
  FaultScope fault;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  return p->esize == 4 ? autotune_plan<float>(p, st) : autotune_plan<double>(p, st);
}

// ---------------------------------------------------------------------------
// Batched solves: many independent problems, one CUDA graph
// ---------------------------------------------------------------------------
// Each problem has its own plan (workspace, tables, tiles).  A solve records
// every problem's launches on one of kBatchStreams forked streams (problems
// assigned greedily by size so the streams carry similar work), joins them,
// and replays that graph while the caller's pointers and stream stay the same.
struct poisfft_batch {
  std::vector<poisfft_plan*> plans;
  std::vector<int> stream_of;          // problem -> forked stream
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> joins;
  cudaEvent_t fork = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<const void*> g_cached;
  std::vector<void*> phi_cached;
  cudaStream_t stream_cached = nullptr;
  std::vector<std::vector<SweepLaunch>> tuned[POISFFT_BATCH_TUNE_CANDIDATES];  // the last tuner's candidates
  // persistent phase launches (poisfft_batch_solve_persistent)
  struct Phase {
    int group = 0;                     // sweep phase; the groups of one phase run concurrently
    int kind = 0;                      // launch kind of every item (0, 1 or 4)
    int nitems = 0, total = 0, bar_off = 0;
    size_t smem = 0, items_off = 0, first_off = 0;
    unsigned grid = 0;
  };
  std::vector<Phase> phases;
  bool persistent = false;             // poisfft_batch_solve runs the persistent phases (tuner's choice)
  unsigned char* pdev = nullptr;       // work lists (BatchItem arrays and tile offsets) of every phase
  int* pctr = nullptr;                 // one tile counter per phase
  std::vector<const void*> p_g;        // the pointers the work lists were built for
  std::vector<void*> p_phi;
};

namespace {

constexpr int kBatchStreams = 8;

void free_batch(poisfft_batch* b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->pdev) cudaFree(b->pdev);
  if (b->pctr) cudaFree(b->pctr);
  for (cudaEvent_t e : b->joins) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  for (cudaStream_t s : b->streams) cudaStreamDestroy(s);
  for (poisfft_plan* p : b->plans) free_plan(p);
  delete b;
}

int batch_record(poisfft_batch* b, void* const phi[], const void* const g[], cudaStream_t st) {
  if (cudaEventRecord(b->fork, st) != cudaSuccess) return POISFFT_ERR_CUDA;
  for (cudaStream_t s : b->streams)
    if (cudaStreamWaitEvent(s, b->fork, 0) != cudaSuccess) return POISFFT_ERR_CUDA;
  for (size_t i = 0; i < b->plans.size(); i++) {
    const int rc = poisfft_solve(b->plans[i], phi[i], g[i], b->streams[b->stream_of[i]]);
    if (rc != POISFFT_OK) return rc;
  }
  for (size_t s = 0; s < b->streams.size(); s++) {
    if (cudaEventRecord(b->joins[s], b->streams[s]) != cudaSuccess) return POISFFT_ERR_CUDA;
    if (cudaStreamWaitEvent(st, b->joins[s], 0) != cudaSuccess) return POISFFT_ERR_CUDA;
  }
  return POISFFT_OK;
}

void batch_drop_graph(poisfft_batch* b) {
  if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
  if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
  b->g_cached.clear();
  b->phi_cached.clear();
  b->p_g.clear();  // the work lists hold the tile shapes too
  b->p_phi.clear();
}

// Work lists of the persistent phases: phase p holds launch p of every
// problem that has one, in descending order of tiles.  The tile shapes are
// those of the plans (tuned or not); x sweeps get the problem's g / phi.
template <typename T>
int batch_build_phases(poisfft_batch* b, void* const phi[], const void* const g[]) {
  size_t nph = 0;
  for (poisfft_plan* p : b->plans) {
    for (const SweepLaunch& L : p->sweeps)
      if (L.kind == 2 || L.kind == 3) return POISFFT_ERR_NOT_IMPLEMENTED;  // specialised kernels: not in the lists
    nph = std::max(nph, p->sweeps.size());
  }
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return POISFFT_ERR_CUDA;
  std::vector<unsigned char> host;
  auto grow = [&](size_t bytes, size_t align) {
    const size_t off = (host.size() + align - 1) / align * align;
    host.resize(off + bytes);
    return off;
  };
  // shared-memory classes: tiles up to 72 KB run three CTAs per SM, up to
  // 110 KB two, larger ones one; each class is its own launch, so one large
  // tile does not lower the occupancy of the whole phase
  auto smem_class = [](size_t smem) { return smem <= 72 * 1024 ? 0 : (smem <= 110 * 1024 ? 1 : 2); };
  b->phases.clear();
  for (size_t ph = 0; ph < nph; ph++)
  for (int kind : {0, 1, 4})
  for (int cls = 0; cls < 3; cls++) {
    std::vector<BatchItem> items;
    std::vector<long long> tiles;
    size_t smem = 16;
    for (size_t i = 0; i < b->plans.size(); i++) {
      poisfft_plan* p = b->plans[i];
      if (ph >= p->sweeps.size()) continue;
      const SweepLaunch& L = p->sweeps[ph];
      if (L.kind != kind || smem_class(L.kind == 4 ? 0 : L.smem) != cls) continue;
      BatchItem it;
      memset(&it, 0, sizeof(it));
      long long nt = L.grid;
      if (L.kind == 0) {
        it.kind = 0;
        it.xa = L.xa;
        it.xa.g = g[i];
        it.xa.phi = phi[i];
        it.xa.ny = p->ny;
        it.xa.g_sy = it.xa.phi_sy = p->nx;
        it.xa.g_sz = it.xa.phi_sz = (long long)p->nx * p->ny;
        smem = std::max(smem, L.smem);
      } else if (L.kind == 1) {
        it.kind = 1;
        it.sa = L.sa;
        it.map = p->maps[L.map];
        smem = std::max(smem, L.smem);
      } else {
        it.kind = 4;
        it.pda = L.pda;
        it.gx = (int)(((long long)L.pda.ncols * L.pda.ny + 255) / 256);
        it.gy = L.pda.nz < 65535 ? L.pda.nz : 65535;
        nt = (long long)it.gx * it.gy;
      }
      items.push_back(it);
      tiles.push_back(nt);
    }
    std::vector<int> order(items.size());
    for (size_t k = 0; k < order.size(); k++) order[k] = (int)k;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return tiles[x] > tiles[y]; });
    if (items.empty()) continue;
    b->phases.push_back(poisfft_batch::Phase());
    poisfft_batch::Phase& P = b->phases.back();
    P.group = (int)ph;
    P.kind = kind;
    P.nitems = (int)items.size();
    P.items_off = grow(items.size() * sizeof(BatchItem), 64);
    P.first_off = grow(items.size() * sizeof(int), 16);
    long long total = 0;
    for (size_t k = 0; k < order.size(); k++) {
      memcpy(host.data() + P.items_off + k * sizeof(BatchItem), &items[order[k]], sizeof(BatchItem));
      const int f = (int)total;
      memcpy(host.data() + P.first_off + k * sizeof(int), &f, sizeof(int));
      total += tiles[order[k]];
    }
    if (total > 0x7fffffffLL) return POISFFT_ERR_UNSUPPORTED_SIZE;
    P.total = (int)total;
    P.bar_off = (int)((smem + 15) / 16 * 16);
    P.smem = (size_t)P.bar_off + 16;
    int occ = 0;
    if (launch_batch_phase<T>(kind, nullptr, nullptr, 0, 0, nullptr, 0, 0, P.smem, nullptr, &occ) != cudaSuccess ||
        occ < 1)
      return POISFFT_ERR_CUDA;
    P.grid = (unsigned)std::min<long long>(total, (long long)occ * sms);
  }
  if (b->pdev) { cudaFree(b->pdev); b->pdev = nullptr; }
  if (b->pctr) { cudaFree(b->pctr); b->pctr = nullptr; }
  if (dev_malloc(&b->pctr, std::max<size_t>(b->phases.size(), 1) * sizeof(int)) != cudaSuccess)
    return POISFFT_ERR_ALLOC;
  if (dev_malloc(&b->pdev, std::max<size_t>(host.size(), 64)) != cudaSuccess) return POISFFT_ERR_ALLOC;
  if (cudaMemcpy(b->pdev, host.data(), host.size(), cudaMemcpyHostToDevice) != cudaSuccess) return POISFFT_ERR_CUDA;
  b->p_g.assign(g, g + b->plans.size());
  b->p_phi.assign(phi, phi + b->plans.size());
  return POISFFT_OK;
}

// Phase by phase; the classes of one phase run concurrently on the batch's
// forked streams and join on `st` before the next phase.
template <typename T>
int batch_run_phases(poisfft_batch* b, cudaStream_t st) {
  size_t k = 0;
  while (k < b->phases.size()) {
    size_t e = k;
    while (e < b->phases.size() && b->phases[e].group == b->phases[k].group) e++;
    NvtxRange range("poisfft batch phase");
    const bool fork = e - k > 1;
    if (fork && cudaEventRecord(b->fork, st) != cudaSuccess) return POISFFT_ERR_CUDA;
    for (size_t q = k; q < e; q++) {
      const poisfft_batch::Phase& P = b->phases[q];
      cudaStream_t s = fork ? b->streams[(q - k) % b->streams.size()] : st;
      if (fork && cudaStreamWaitEvent(s, b->fork, 0) != cudaSuccess) return POISFFT_ERR_CUDA;
      if (cudaMemsetAsync(b->pctr + q, 0, sizeof(int), s) != cudaSuccess) return POISFFT_ERR_CUDA;
      const BatchItem* items = reinterpret_cast<const BatchItem*>(b->pdev + P.items_off);
      const int* first = reinterpret_cast<const int*>(b->pdev + P.first_off);
      if (launch_batch_phase<T>(P.kind, items, first, P.nitems, P.total, b->pctr + q, P.bar_off, P.grid, P.smem, s,
                                nullptr) != cudaSuccess)
        return POISFFT_ERR_CUDA;
      if (fork) {
        cudaEvent_t j = b->joins[(q - k) % b->joins.size()];
        if (cudaEventRecord(j, s) != cudaSuccess || cudaStreamWaitEvent(st, j, 0) != cudaSuccess)
          return POISFFT_ERR_CUDA;
      }
    }
    k = e;
  }
  return POISFFT_OK;
}

int batch_apply(poisfft_batch* b, const std::vector<std::vector<SweepLaunch>>& cfg) {
  for (size_t i = 0; i < b->plans.size(); i++) {
    b->plans[i]->sweeps = cfg[i];
    const int rc = encode_maps(b->plans[i]);
    if (rc != POISFFT_OK) return rc;
  }
  batch_drop_graph(b);
  return POISFFT_OK;
}

// General 3D plans whose sweeps are x and strided sweeps only can carry the
// divide in either strided sweep (plan_general_sequence).
bool order_tunable(const poisfft_plan* p) {
  if (p->dims != 3 || p->fast) return false;
  for (const SweepLaunch& L : p->sweeps)
    if (L.kind != 0 && L.kind != 1) return false;
  return true;
}

// Re-plan the sweep sequence of a plan with the divide in `fused_axis`
// (tile shapes as planned); the device tables are unchanged.
int replan_fused_axis(poisfft_plan* p, int fused_axis) {
  std::vector<SweepLaunch> sw;
  int rc = plan_general_sequence(p, fused_axis, sw);
  if (rc != POISFFT_OK) return rc;
  p->sweeps = sw;
  patch_general(p);
  return encode_maps(p);
}

// Time each order-tunable plan alone with the divide in z and in y (one
// warm-up and three timed solves each) and keep the faster order.
int batch_tune_sweep_order(poisfft_batch* b, cudaStream_t st) {
  size_t fb = 0;
  for (const poisfft_plan* p : b->plans)
    if (order_tunable(p)) fb = std::max(fb, p->field_bytes);
  if (fb == 0) return POISFFT_OK;
  void* g = nullptr;
  void* phi = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = POISFFT_OK;
  if (dev_malloc(&g, fb) != cudaSuccess || dev_malloc(&phi, fb) != cudaSuccess ||
      cudaMemsetAsync(g, 0, fb, st) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
      cudaEventCreate(&e1) != cudaSuccess)
    rc = POISFFT_ERR_ALLOC;
  for (poisfft_plan* p : b->plans) {
    if (rc != POISFFT_OK) break;
    if (!order_tunable(p)) continue;
    float best_ms = 1e30f;
    int best_axis = 2;
    for (int axis : {2, 1}) {
      if ((rc = replan_fused_axis(p, axis)) != POISFFT_OK) break;
      if ((rc = solve_core(p, phi, g, st)) != POISFFT_OK) break;
      cudaEventRecord(e0, st);
      for (int r = 0; r < 3 && rc == POISFFT_OK; r++) rc = solve_core(p, phi, g, st);
      cudaEventRecord(e1, st);
      float ms = 0.f;
      if (rc == POISFFT_OK && (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
        rc = POISFFT_ERR_CUDA;
      if (rc == POISFFT_OK && ms < best_ms * 0.97f) {  // the other order must win clearly
        best_ms = ms;
        best_axis = axis;
      }
    }
    if (rc == POISFFT_OK) rc = replan_fused_axis(p, best_axis);
    if (rc == POISFFT_OK && cudaMemsetAsync(p->ws, 0, p->ws_bytes, st) != cudaSuccess) rc = POISFFT_ERR_CUDA;
  }
  if (cudaStreamSynchronize(st) != cudaSuccess && rc == POISFFT_OK) rc = POISFFT_ERR_CUDA;
  if (g) cudaFree(g);
  if (phi) cudaFree(phi);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaGetLastError();
  return rc;
}

std::vector<std::vector<SweepLaunch>> batch_snapshot(const poisfft_batch* b) {
  std::vector<std::vector<SweepLaunch>> cfg(b->plans.size());
  for (size_t i = 0; i < b->plans.size(); i++) cfg[i] = b->plans[i]->sweeps;
  return cfg;
}

}  // namespace

extern "C" {

int poisfft_batch_create(poisfft_batch** out, int count, const int dims[], const int64_t n[], const double L[],
                         const int bc[], int approx, int dtype) {
  if (!out) return POISFFT_ERR_INVALID_ARG;
  *out = nullptr;
  if (count < 1 || !dims || !n || !L || !bc) return POISFFT_ERR_INVALID_ARG;
  if (dtype == POISFFT_MIXED || dtype == POISFFT_BF16X3) return POISFFT_ERR_NOT_IMPLEMENTED;
  poisfft_batch* b = new (std::nothrow) poisfft_batch();
  if (!b) return POISFFT_ERR_ALLOC;
  std::vector<double> load;
  for (int i = 0; i < count; i++) {
    poisfft_plan* p = nullptr;
    const int rc = poisfft_plan_create(&p, dims[i], n + 3 * (size_t)i, L + 3 * (size_t)i, bc + 6 * (size_t)i, approx,
                                       dtype);
    if (rc != POISFFT_OK) {
      free_batch(b);
      return rc;
    }
    // No per-plan autotuning here: the tuner times each problem alone on an
    // idle GPU and picks narrower tiles, while inside the batch graph the
    // problems run concurrently (poisfft_batch_autotune times the graph).
    b->plans.push_back(p);
  }
  const int ns = std::min(kBatchStreams, count);
  load.assign(ns, 0.0);
  // greedy assignment, largest problems first
  std::vector<int> order(count);
  for (int i = 0; i < count; i++) order[i] = i;
  auto pts = [&](int i) { return (double)b->plans[i]->nx * b->plans[i]->ny * b->plans[i]->nz; };
  std::sort(order.begin(), order.end(), [&](int x, int y) { return pts(x) > pts(y); });
  b->stream_of.assign(count, 0);
  for (int i : order) {
    const int s = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    b->stream_of[i] = s;
    load[s] += pts(i);
  }
  for (int s = 0; s < ns; s++) {
    cudaStream_t st;
    cudaEvent_t ev;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) { free_batch(b); return POISFFT_ERR_CUDA; }
    b->streams.push_back(st);
    if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) { free_batch(b); return POISFFT_ERR_CUDA; }
    b->joins.push_back(ev);
  }
  if (cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess) { free_batch(b); return POISFFT_ERR_CUDA; }
  *out = b;
  return POISFFT_OK;
}

int poisfft_batch_solve(poisfft_batch* b, void* const phi[], const void* const g[], void* stream) {
  if (!b || !phi || !g) return POISFFT_ERR_INVALID_ARG;
  if (b->persistent) return poisfft_batch_solve_persistent(b, phi, g, stream);
  const size_t cnt = b->plans.size();
  for (size_t i = 0; i < cnt; i++) {
    if (!phi[i] || !g[i]) return POISFFT_ERR_INVALID_ARG;
    const size_t es = b->plans[i]->esize;
    if (((uintptr_t)phi[i] % es) != 0 || ((uintptr_t)g[i] % es) != 0) return POISFFT_ERR_MISALIGNED;
  }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  bool same = b->exec && st == b->stream_cached && b->g_cached.size() == cnt;
  for (size_t i = 0; same && i < cnt; i++) same = b->g_cached[i] == g[i] && b->phi_cached[i] == phi[i];
  if (!same) {
    if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
    if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
    if (cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed) != cudaSuccess) return POISFFT_ERR_CUDA;
    const int rc = batch_record(b, phi, g, st);
    cudaGraph_t graph = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(st, &graph);
    if (rc != POISFFT_OK || ec != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();
      return rc != POISFFT_OK ? rc : POISFFT_ERR_CUDA;
    }
    b->graph = graph;
    if (cudaGraphInstantiate(&b->exec, graph, 0) != cudaSuccess) {
      cudaGetLastError();
      b->exec = nullptr;
      return POISFFT_ERR_CUDA;
    }
    b->g_cached.assign(g, g + cnt);
    b->phi_cached.assign(phi, phi + cnt);
    b->stream_cached = st;
  }
  return cudaGraphLaunch(b->exec, st) == cudaSuccess ? POISFFT_OK : POISFFT_ERR_CUDA;
}

int poisfft_batch_autotune(poisfft_batch* b, void* const phi[], const void* const g[], void* stream,
                           double ms[POISFFT_BATCH_TUNE_CANDIDATES], int* chosen) {
  if (!b || !phi || !g) return POISFFT_ERR_INVALID_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  // candidate 0: the shapes as created
  std::vector<std::vector<SweepLaunch>> cfg[POISFFT_BATCH_TUNE_CANDIDATES];
  cfg[0] = batch_snapshot(b);
  // candidate 1: general tiles halved (more, smaller CTAs)
  for (size_t i = 0; i < b->plans.size(); i++) {
    poisfft_plan* p = b->plans[i];
    const int wmin = p->esize == 4 ? 2 : 1;
    for (SweepLaunch& L : p->sweeps) {
      if (L.kind == 1 && L.sa.w / 2 >= wmin) set_strided_width(p, L, L.sa.w / 2);
      else if (L.kind == 0 && L.xa.lines / 2 >= 1) set_x_lines(p, L, L.xa.lines / 2);
    }
  }
  cfg[1] = batch_snapshot(b);
  // candidate 2: every plan tuned alone on the GPU
  int rc = batch_apply(b, cfg[0]);
  for (size_t i = 0; rc == POISFFT_OK && i < b->plans.size(); i++) rc = poisfft_plan_autotune(b->plans[i], stream);
  if (rc != POISFFT_OK) return rc;
  cfg[2] = batch_snapshot(b);
  // candidate 3: the shapes as created, with each 3D general-path problem's
  // sweep order (which strided axis carries the divide) chosen by timing
  // both orders alone
  if ((rc = batch_apply(b, cfg[0])) != POISFFT_OK) return rc;
  if ((rc = batch_tune_sweep_order(b, st)) != POISFFT_OK) {
    batch_apply(b, cfg[0]);
    return rc;
  }
  cfg[3] = batch_snapshot(b);
  // candidate 4: the shapes as created, one persistent launch per phase
  cfg[4] = cfg[0];
  b->persistent = false;

  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    cudaGetLastError();
    return POISFFT_ERR_CUDA;
  }
  constexpr int kReps = 4;
  double t[POISFFT_BATCH_TUNE_CANDIDATES];
  int best = 0;
  for (int c = 0; c < POISFFT_BATCH_TUNE_CANDIDATES && rc == POISFFT_OK; c++) {
    rc = batch_apply(b, cfg[c]);
    auto run = [&]() {
      return c == 4 ? poisfft_batch_solve_persistent(b, phi, g, stream) : poisfft_batch_solve(b, phi, g, stream);
    };
    if (rc == POISFFT_OK) rc = run();  // capture (or build the work lists) and warm up
    if (rc == POISFFT_ERR_NOT_IMPLEMENTED && c == 4) {  // specialised plans: no persistent form
      rc = POISFFT_OK;
      t[c] = 1e30;
      continue;
    }
    if (rc != POISFFT_OK) break;
    cudaEventRecord(e0, st);
    for (int r = 0; r < kReps && rc == POISFFT_OK; r++) rc = run();
    cudaEventRecord(e1, st);
    float f = 0.f;
    if (rc == POISFFT_OK && (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&f, e0, e1) != cudaSuccess))
      rc = POISFFT_ERR_CUDA;
    t[c] = f / kReps;
    if (rc == POISFFT_OK && t[c] < t[best]) best = c;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != POISFFT_OK) {
    cudaGetLastError();
    batch_apply(b, cfg[0]);
    return rc;
  }
  rc = batch_apply(b, cfg[best]);
  b->persistent = best == 4;
  for (int c = 0; c < POISFFT_BATCH_TUNE_CANDIDATES; c++) b->tuned[c] = cfg[c];
  if (ms)
    for (int c = 0; c < POISFFT_BATCH_TUNE_CANDIDATES; c++) ms[c] = t[c];
  if (chosen) *chosen = best;
  return rc;
}

int poisfft_batch_solve_persistent(poisfft_batch* b, void* const phi[], const void* const g[], void* stream) {
  if (!b || !phi || !g) return POISFFT_ERR_INVALID_ARG;
  const size_t cnt = b->plans.size();
  for (size_t i = 0; i < cnt; i++) {
    if (!phi[i] || !g[i]) return POISFFT_ERR_INVALID_ARG;
    const size_t es = b->plans[i]->esize;
    if (((uintptr_t)phi[i] % es) != 0 || ((uintptr_t)g[i] % es) != 0) return POISFFT_ERR_MISALIGNED;
  }
  const bool f64 = b->plans[0]->esize == 8;
  bool same = b->p_g.size() == cnt;
  for (size_t i = 0; same && i < cnt; i++) same = b->p_g[i] == g[i] && b->p_phi[i] == phi[i];
  if (!same) {
    FaultScope fault;
    const int rc = f64 ? batch_build_phases<double>(b, phi, g) : batch_build_phases<float>(b, phi, g);
    if (rc != POISFFT_OK) {
      cudaGetLastError();
      b->p_g.clear();
      b->p_phi.clear();
      return rc;
    }
  }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  return f64 ? batch_run_phases<double>(b, st) : batch_run_phases<float>(b, st);
}

int poisfft_batch_solve_sequential(poisfft_batch* b, void* const phi[], const void* const g[], void* stream) {
  if (!b || !phi || !g) return POISFFT_ERR_INVALID_ARG;
  for (size_t i = 0; i < b->plans.size(); i++) {
    const int rc = poisfft_solve(b->plans[i], phi[i], g[i], stream);
    if (rc != POISFFT_OK) return rc;
  }
  return POISFFT_OK;
}

int poisfft_batch_select(poisfft_batch* b, int candidate) {
  if (!b || candidate < 0 || candidate >= POISFFT_BATCH_TUNE_CANDIDATES || b->tuned[candidate].empty())
    return POISFFT_ERR_INVALID_ARG;
  const int rc = batch_apply(b, b->tuned[candidate]);
  b->persistent = rc == POISFFT_OK && candidate == 4;
  return rc;
}

int poisfft_batch_info(const poisfft_batch* b, int64_t out[3]) {
  if (!b || !out) return POISFFT_ERR_INVALID_ARG;
  int64_t bytes = 0, launches = 0, points = 0;
  for (const poisfft_plan* p : b->plans) {
    for (const SweepLaunch& L : p->sweeps) bytes += L.bytes;
    launches += (int64_t)p->sweeps.size();
    points += (int64_t)p->nx * p->ny * p->nz;
  }
  out[0] = bytes;
  out[1] = launches;
  out[2] = points;
  return POISFFT_OK;
}

int poisfft_batch_check(poisfft_batch* b, void* stream) {
  if (!b) return POISFFT_ERR_INVALID_ARG;
  int worst = POISFFT_OK;
  for (poisfft_plan* p : b->plans) {
    const int rc = poisfft_check(p, stream);
    if (rc != POISFFT_OK) worst = rc;
  }
  return worst;
}

int poisfft_batch_destroy(poisfft_batch* b) {
  free_batch(b);
  return POISFFT_OK;
}

}  // extern "C"
