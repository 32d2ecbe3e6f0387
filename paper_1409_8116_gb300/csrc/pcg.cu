// FFT-preconditioned conjugate gradients for div(a grad phi) = g.
//
// Sec. 1 of the paper notes that the fast direct solve on a regular grid can
// precondition problems with non-constant coefficients.  Discretisation
// (cell centred, second order; reduces to the Table 4 staggered-Dirichlet
// stencil times a for constant a):
//   (A phi)_i = sum_d [ a_{i+1/2}(phi_{i+e} - phi_i) - a_{i-1/2}(phi_i - phi_{i-e}) ] / dx_d^2
// with harmonic-mean faces 2 a_i a_j / (a_i + a_j); a boundary face takes the
// cell's own a and the ghost value -phi_i (phi = 0 on the wall).
//
// The face coefficients over dx^2 are computed once (FP64, and rounded to
// FP32 for the single-precision operator), so no iteration divides.  CG runs
// on K = -A (symmetric positive definite) with the flexible (Polak-Ribiere)
// beta; the preconditioner z = -(1/a_ref) L_h^{-1} r is the library's FP32
// Poisson solve with staggered Dirichlet on every face.
//
// Two precisions:
//  * POISFFT_PCG_F64: vectors, operator and inner products in FP64 (the
//    iteration of the FP64 reference, step for step).
//  * POISFFT_PCG_MIXED: the iteration in FP32 (vectors, operator; inner
//    products accumulated in FP64 across threads) on the correction e of the
//    FP64 solution, with reliable updates (Sleijpen & van der Vorst, 1996):
//    whenever the FP32 residual has dropped by kReliableDelta since the last
//    update, or meets the tolerance, the correction is added to phi in FP64,
//    the true residual -g - K phi is recomputed in FP64 and replaces the
//    FP32 one.  Convergence is decided on that true residual only.
//
// The scalars of the iteration stay on the device: each inner product is
// reduced deterministically inside the kernel that produces its operands,
// and the step lengths are read from device memory by the kernels that use
// them.  The host enqueues iteration k before it reads the convergence flag
// of iteration k-1, and kernels after convergence return at once.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <new>

#include "../../include/poisfft.h"
#include "reduce.cuh"

namespace {

using pf::Reduce;
using pf::grid_sum;
constexpr int kBlock = pf::kReduceBlock;
constexpr int kBlocksPerSM = 8;
// FP32 residual reduction between two FP64 residual replacements; FP32
// recursion keeps ~6 significant digits, so three decades are safe.
constexpr double kReliableDelta = 1e-3;

struct Grid {
  int nx, ny, nz;
  unsigned N;
  double idx2, idy2, idz2;   // 1/dx^2 per axis
  float fidx2, fidy2, fidz2;
};

template <typename T> __device__ __forceinline__ T inv_dx2(const Grid& G, int d);
template <> __device__ __forceinline__ double inv_dx2<double>(const Grid& G, int d) {
  return d == 0 ? G.idx2 : (d == 1 ? G.idy2 : G.idz2);
}
template <> __device__ __forceinline__ float inv_dx2<float>(const Grid& G, int d) {
  return d == 0 ? G.fidx2 : (d == 1 ? G.fidy2 : G.fidz2);
}

// Coefficient over dx^2 of the lower face of every cell along each axis.
template <typename T> struct Faces {
  const T* c[3];
};

__device__ __forceinline__ double harm(double ai, double aj) { return 2.0 * ai * aj / (ai + aj); }

__device__ __forceinline__ void cell_xyz(const Grid& G, unsigned i, int& x, int& y, int& z) {
  const unsigned r = i / (unsigned)G.nx;
  x = (int)(i - r * (unsigned)G.nx);
  z = (int)(r / (unsigned)G.ny);
  y = (int)(r - (unsigned)z * (unsigned)G.ny);
}

// (K v)_i = -(A v)_i.  The upper wall face takes the cell's own a.
template <typename T>
__device__ __forceinline__ T k_apply(const T* __restrict__ v, const Faces<T>& F, const float* __restrict__ a,
                                     const Grid& G, unsigned i, int x, int y, int z, T vi) {
  const unsigned st[3] = {1u, (unsigned)G.nx, (unsigned)G.nx * (unsigned)G.ny};
  const int pos[3] = {x, y, z};
  const int len[3] = {G.nx, G.ny, G.nz};
  T acc = T(0);
#pragma unroll
  for (int d = 0; d < 3; d++) {
    const T fl = F.c[d][i];
    const T vl = pos[d] > 0 ? v[i - st[d]] : -vi;
    const bool up = pos[d] < len[d] - 1;
    const T fh = up ? F.c[d][i + st[d]] : T(a[i]) * inv_dx2<T>(G, d);
    const T vh = up ? v[i + st[d]] : -vi;
    acc += fh * (vh - vi) - fl * (vi - vl);
  }
  return -acc;
}

#define GRID_STRIDE(i, N) for (unsigned i = blockIdx.x * kBlock + threadIdx.x; i < (N); i += gridDim.x * kBlock)

__device__ __forceinline__ bool gated(const int* flag) { return flag && *(volatile const int*)flag; }

__global__ void __launch_bounds__(kBlock) faces_kernel(const float* __restrict__ a, Grid G, double* c0, double* c1,
                                                       double* c2, float* f0, float* f1, float* f2) {
  double* c[3] = {c0, c1, c2};
  float* f[3] = {f0, f1, f2};
  const unsigned st[3] = {1u, (unsigned)G.nx, (unsigned)G.nx * (unsigned)G.ny};
  const double id2[3] = {G.idx2, G.idy2, G.idz2};
  GRID_STRIDE(i, G.N) {
    int x, y, z;
    cell_xyz(G, i, x, y, z);
    const int pos[3] = {x, y, z};
    const double ai = a[i];
    for (int d = 0; d < 3; d++) {
      const double v = (pos[d] > 0 ? harm(ai, (double)a[i - st[d]]) : ai) * id2[d];
      c[d][i] = v;
      f[d][i] = (float)v;
    }
  }
}

// Scalars of the iteration.  Iteration k stores its inner products in slot
// k % 2 and reads rz of slot (k - 1) % 2.
struct Scalars {
  double pq[2], rr[2], rz[2], rdz[2];
  double gg, bnorm, rel;
  double rrt;      // true residual norm^2 of the last FP64 evaluation
  double rr_rel;   // residual norm^2 at the last reliable update
  int done, it, reliable, n_true;
};

// q = K p; dot = p.q (per-thread partials in T, across threads in FP64)
template <typename T>
__global__ void __launch_bounds__(kBlock) apply_kernel(const T* __restrict__ p, Faces<T> F,
                                                       const float* __restrict__ a, Grid G, T* __restrict__ q,
                                                       Reduce R, double* dot, const int* done) {
  if (gated(done)) return;
  T part = T(0);
  GRID_STRIDE(i, G.N) {
    int x, y, z;
    cell_xyz(G, i, x, y, z);
    const T pi = p[i];
    const T qi = k_apply<T>(p, F, a, G, i, x, y, z, pi);
    q[i] = qi;
    part += pi * qi;
  }
  if (dot) {
    const double v[1] = {(double)part};
    double* const d[1] = {dot};
    grid_sum<1>(v, R, d);
  }
}

// ---- FP64 iteration --------------------------------------------------------

// r = -g - K phi; r32 = float(r); rrt = r.r; gg = g.g
__global__ void __launch_bounds__(kBlock) f64_init_kernel(const double* __restrict__ phi,
                                                          const double* __restrict__ g, Faces<double> F,
                                                          const float* __restrict__ a, Grid G,
                                                          double* __restrict__ r, float* __restrict__ r32,
                                                          Scalars* S, Reduce R) {
  double v = 0.0, w = 0.0;
  GRID_STRIDE(i, G.N) {
    int x, y, z;
    cell_xyz(G, i, x, y, z);
    const double gi = g[i];
    const double ri = -gi - k_apply<double>(phi, F, a, G, i, x, y, z, phi[i]);
    r[i] = ri;
    r32[i] = (float)ri;
    v += ri * ri;
    w += gi * gi;
  }
  const double vw[2] = {v, w};
  double* const d[2] = {&S->rrt, &S->gg};
  grid_sum<2>(vw, R, d);
}

// Initial test: bnorm = |g|; done when g = 0 or the initial guess already
// meets the tolerance.
__global__ void init_check_kernel(Scalars* S, double tol) {
  S->bnorm = sqrt(S->gg);
  S->rel = S->bnorm > 0.0 ? sqrt(S->rrt) / S->bnorm : 0.0;
  S->rr_rel = S->rrt;
  S->it = 0;
  S->n_true = 1;
  S->done = (S->bnorm == 0.0 || S->rel <= tol) ? 1 : 0;
}

// alpha = rz_{k-1} / (p.q); x += alpha p; r -= alpha q; rr = r.r; r32 = float(r)
__global__ void __launch_bounds__(kBlock) f64_update_kernel(double* __restrict__ x, double* __restrict__ r,
                                                            const double* __restrict__ p,
                                                            const double* __restrict__ q, float* __restrict__ r32,
                                                            Scalars* S, Reduce R, int s, int sp, unsigned N) {
  if (gated(&S->done)) return;
  const double alpha = S->rz[sp] / S->pq[s];
  double v = 0.0;
  GRID_STRIDE(i, N) {
    x[i] += alpha * p[i];
    const double ri = r[i] - alpha * q[i];
    r[i] = ri;
    r32[i] = (float)ri;
    v += ri * ri;
  }
  const double vv[1] = {v};
  double* const d[1] = {&S->rr[s]};
  grid_sum<1>(vv, R, d);
}

// Convergence test of iteration k on the recursive residual (one thread).
__global__ void f64_check_kernel(Scalars* S, int s, int k, double tol) {
  if (S->done) return;
  S->rel = sqrt(S->rr[s]) / S->bnorm;
  S->it = k;
  if (S->rel <= tol) S->done = 1;
}

// z_new = scale * z32; rz = r.z_new; rdz = r.(z_new - z_old); z = z_new.
// first: z_old is taken as 0 (z is not read).
__global__ void __launch_bounds__(kBlock) f64_precond_kernel(const float* __restrict__ z32,
                                                             const double* __restrict__ r, double* __restrict__ z,
                                                             double scale, Scalars* S, Reduce R, int s, int first,
                                                             unsigned N) {
  if (gated(&S->done)) return;
  double v = 0.0, w = 0.0;
  GRID_STRIDE(i, N) {
    const double zn = scale * (double)z32[i];
    const double ri = r[i];
    v += ri * zn;
    w += ri * (first ? zn : zn - z[i]);
    z[i] = zn;
  }
  const double vw[2] = {v, w};
  double* const d[2] = {&S->rz[s], &S->rdz[s]};
  grid_sum<2>(vw, R, d);
}

// p = z + beta p with beta = rdz_k / rz_{k-1}; first: p = z.
__global__ void __launch_bounds__(kBlock) f64_dir_kernel(double* __restrict__ p, const double* __restrict__ z,
                                                         Scalars* S, int s, int sp, int first, unsigned N) {
  if (gated(&S->done)) return;
  const double beta = first ? 0.0 : S->rdz[s] / S->rz[sp];
  GRID_STRIDE(i, N) p[i] = first ? z[i] : z[i] + beta * p[i];
}

// ---- mixed iteration: FP32 correction, FP64 solution and true residual ----

// r = float(-g - K phi) (FP64 operator); rrt = |r|^2 in FP64; gg = g.g when
// with_gg.  Runs only when *gate is set (reliable update) unless gate is null.
__global__ void __launch_bounds__(kBlock) mx_resid_kernel(const double* __restrict__ phi,
                                                          const double* __restrict__ g, Faces<double> F,
                                                          const float* __restrict__ a, Grid G,
                                                          float* __restrict__ r, Scalars* S, Reduce R,
                                                          const int* gate, int with_gg) {
  if (gated(&S->done) || (gate && !*(volatile const int*)gate)) return;
  double v = 0.0, w = 0.0;
  GRID_STRIDE(i, G.N) {
    int x, y, z;
    cell_xyz(G, i, x, y, z);
    const double gi = g[i];
    const double ri = -gi - k_apply<double>(phi, F, a, G, i, x, y, z, phi[i]);
    r[i] = (float)ri;
    v += ri * ri;
    w += gi * gi;
  }
  if (with_gg) {
    const double vw[2] = {v, w};
    double* const d[2] = {&S->rrt, &S->gg};
    grid_sum<2>(vw, R, d);
  } else {
    const double vv[1] = {v};
    double* const d[1] = {&S->rrt};
    grid_sum<1>(vv, R, d);
  }
}

// phi += e; e = 0 (when *gate is set, or always when gate is null)
__global__ void __launch_bounds__(kBlock) mx_axpy_kernel(double* __restrict__ phi, float* __restrict__ e,
                                                         const int* done, const int* gate, unsigned N) {
  if (gated(done) || (gate && !*(volatile const int*)gate)) return;
  GRID_STRIDE(i, N) {
    phi[i] += (double)e[i];
    e[i] = 0.f;
  }
}

// alpha = rz_{k-1} / (p.q); e += alpha p; r -= alpha q; rr = r.r
__global__ void __launch_bounds__(kBlock) mx_update_kernel(float* __restrict__ e, float* __restrict__ r,
                                                           const float* __restrict__ p, const float* __restrict__ q,
                                                           Scalars* S, Reduce R, int s, int sp, unsigned N) {
  if (gated(&S->done)) return;
  const float alpha = (float)(S->rz[sp] / S->pq[s]);
  float v = 0.f;
  GRID_STRIDE(i, N) {
    e[i] += alpha * p[i];
    const float ri = r[i] - alpha * q[i];
    r[i] = ri;
    v += ri * ri;
  }
  const double vv[1] = {(double)v};
  double* const d[1] = {&S->rr[s]};
  grid_sum<1>(vv, R, d);
}

// Iteration k: ask for a reliable update when the FP32 residual has dropped by
// delta since the last one or meets the tolerance (one thread).
__global__ void mx_check_kernel(Scalars* S, int s, int k, double tol, double delta) {
  if (S->done) return;
  const double rr = S->rr[s];
  S->it = k;
  S->rel = sqrt(rr) / S->bnorm;
  S->reliable = (S->rel <= tol || rr <= delta * delta * S->rr_rel) ? 1 : 0;
}

// After a reliable update: the true residual replaces the recursive one and
// decides convergence (one thread).
__global__ void mx_check2_kernel(Scalars* S, double tol) {
  if (S->done || !S->reliable) return;
  S->rr_rel = S->rrt;
  S->rel = sqrt(S->rrt) / S->bnorm;
  S->n_true++;
  S->reliable = 0;
  if (S->rel <= tol) S->done = 1;
}

// Final true residual when the iteration stopped at maxit (one thread).
__global__ void mx_final_kernel(Scalars* S) {
  if (S->done) return;
  S->rel = S->bnorm > 0.0 ? sqrt(S->rrt) / S->bnorm : 0.0;
  S->n_true++;
}

// rz = scale r.zA; rdz = scale r.(zA - zB) with zA the preconditioner's raw
// output for the current r and zB the previous one (first: zB taken as 0).
__global__ void __launch_bounds__(kBlock) mx_precond_kernel(const float* __restrict__ r,
                                                            const float* __restrict__ zA,
                                                            const float* __restrict__ zB, double scale, Scalars* S,
                                                            Reduce R, int s, int first, unsigned N) {
  if (gated(&S->done)) return;
  float v = 0.f, w = 0.f;
  GRID_STRIDE(i, N) {
    const float ri = r[i], za = zA[i];
    v += ri * za;
    w += ri * (first ? za : za - zB[i]);
  }
  const double vw[2] = {scale * (double)v, scale * (double)w};
  double* const d[2] = {&S->rz[s], &S->rdz[s]};
  grid_sum<2>(vw, R, d);
}

// p = scale zA + beta p with beta = rdz_k / rz_{k-1}; first: p = scale zA.
__global__ void __launch_bounds__(kBlock) mx_dir_kernel(float* __restrict__ p, const float* __restrict__ zA,
                                                        float scale, Scalars* S, int s, int sp, int first,
                                                        unsigned N) {
  if (gated(&S->done)) return;
  const float beta = first ? 0.f : (float)(S->rdz[s] / S->rz[sp]);
  GRID_STRIDE(i, N) p[i] = first ? scale * zA[i] : scale * zA[i] + beta * p[i];
}

// ---- mixed iteration, four cells per thread (nx a multiple of 4) ----------
// The same arithmetic as the kernels above on 128-bit loads: every thread
// keeps four cells' loads in flight, which the scalar forms cannot (they
// stall on memory latency at a third to a half of the DRAM bandwidth).

__device__ __forceinline__ float4 ld4(const float* p, unsigned i4) { return reinterpret_cast<const float4*>(p)[i4]; }
__device__ __forceinline__ void st4(float* p, unsigned i4, float4 v) { reinterpret_cast<float4*>(p)[i4] = v; }
__device__ __forceinline__ float get(const float4& v, int k) { return k == 0 ? v.x : (k == 1 ? v.y : (k == 2 ? v.z : v.w)); }

// q = K p for cells 4 i4 .. 4 i4 + 3 (one x row segment); dot += p.q
__global__ void __launch_bounds__(kBlock) apply4_kernel(const float* __restrict__ p, Faces<float> F,
                                                        const float* __restrict__ a, Grid G, float* __restrict__ q,
                                                        Reduce R, double* dot, const int* done) {
  if (gated(done)) return;
  const unsigned N4 = G.N / 4, sy4 = (unsigned)G.nx / 4, sz4 = sy4 * (unsigned)G.ny;
  float part = 0.f;
  GRID_STRIDE(i4, N4) {
    const unsigned i = 4 * i4;
    int x, y, z;
    cell_xyz(G, i, x, y, z);
    const float4 pc = ld4(p, i4);
    const float pv[4] = {pc.x, pc.y, pc.z, pc.w};
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    // x faces: lower faces of the four cells, and the one above the last
    const float4 fx = ld4(F.c[0], i4);
    const bool has_l = x > 0, has_r = x + 4 < G.nx;
    const float pl = has_l ? p[i - 1] : 0.f;
    const float pr = has_r ? p[i + 4] : 0.f;
    const float fr = has_r ? F.c[0][i + 4] : a[i + 3] * G.fidx2;
    {
      const float fl[5] = {fx.x, fx.y, fx.z, fx.w, fr};
#pragma unroll
      for (int k = 0; k < 4; k++) {
        const float vl = k > 0 ? pv[k - 1] : (has_l ? pl : -pv[0]);
        const float vh = k < 3 ? pv[k + 1] : (has_r ? pr : -pv[3]);
        acc[k] += fl[k + 1] * (vh - pv[k]) - fl[k] * (pv[k] - vl);
      }
    }
    // y and z faces: whole float4 rows of the neighbouring lines
#pragma unroll
    for (int d = 1; d < 3; d++) {
      const unsigned st = d == 1 ? sy4 : sz4;
      const bool lo = (d == 1 ? y : z) > 0;
      const bool hi = (d == 1 ? y < G.ny - 1 : z < G.nz - 1);
      const float4 fl = ld4(F.c[d], i4);
      const float4 plo = lo ? ld4(p, i4 - st) : pc;
      const float4 phi = hi ? ld4(p, i4 + st) : pc;
      float4 fh;
      if (hi) {
        fh = ld4(F.c[d], i4 + st);
      } else {
        const float4 av = ld4(a, i4);
        const float s2 = d == 1 ? G.fidy2 : G.fidz2;
        fh = make_float4(av.x * s2, av.y * s2, av.z * s2, av.w * s2);
      }
#pragma unroll
      for (int k = 0; k < 4; k++) {
        const float vk = pv[k];
        const float vl = lo ? get(plo, k) : -vk;
        const float vh = hi ? get(phi, k) : -vk;
        acc[k] += get(fh, k) * (vh - vk) - get(fl, k) * (vk - vl);
      }
    }
    const float4 qv = make_float4(-acc[0], -acc[1], -acc[2], -acc[3]);
    st4(q, i4, qv);
    part += pc.x * qv.x + pc.y * qv.y + pc.z * qv.z + pc.w * qv.w;
  }
  if (dot) {
    const double v[1] = {(double)part};
    double* const d[1] = {dot};
    grid_sum<1>(v, R, d);
  }
}

__global__ void __launch_bounds__(kBlock) mx_update4_kernel(float* __restrict__ e, float* __restrict__ r,
                                                            const float* __restrict__ p,
                                                            const float* __restrict__ q, Scalars* S, Reduce R, int s,
                                                            int sp, unsigned N4) {
  if (gated(&S->done)) return;
  const float alpha = (float)(S->rz[sp] / S->pq[s]);
  float v = 0.f;
  GRID_STRIDE(i4, N4) {
    const float4 ev = ld4(e, i4), rv = ld4(r, i4), pv = ld4(p, i4), qv = ld4(q, i4);
    const float4 en = make_float4(ev.x + alpha * pv.x, ev.y + alpha * pv.y, ev.z + alpha * pv.z, ev.w + alpha * pv.w);
    const float4 rn = make_float4(rv.x - alpha * qv.x, rv.y - alpha * qv.y, rv.z - alpha * qv.z, rv.w - alpha * qv.w);
    st4(e, i4, en);
    st4(r, i4, rn);
    v += rn.x * rn.x + rn.y * rn.y + rn.z * rn.z + rn.w * rn.w;
  }
  const double vv[1] = {(double)v};
  double* const d[1] = {&S->rr[s]};
  grid_sum<1>(vv, R, d);
}

__global__ void __launch_bounds__(kBlock) mx_precond4_kernel(const float* __restrict__ r,
                                                             const float* __restrict__ zA,
                                                             const float* __restrict__ zB, double scale, Scalars* S,
                                                             Reduce R, int s, int first, unsigned N4) {
  if (gated(&S->done)) return;
  float v = 0.f, w = 0.f;
  GRID_STRIDE(i4, N4) {
    const float4 rv = ld4(r, i4), za = ld4(zA, i4);
    v += rv.x * za.x + rv.y * za.y + rv.z * za.z + rv.w * za.w;
    if (first) {
      w += rv.x * za.x + rv.y * za.y + rv.z * za.z + rv.w * za.w;
    } else {
      const float4 zb = ld4(zB, i4);
      w += rv.x * (za.x - zb.x) + rv.y * (za.y - zb.y) + rv.z * (za.z - zb.z) + rv.w * (za.w - zb.w);
    }
  }
  const double vw[2] = {scale * (double)v, scale * (double)w};
  double* const d[2] = {&S->rz[s], &S->rdz[s]};
  grid_sum<2>(vw, R, d);
}

__global__ void __launch_bounds__(kBlock) mx_dir4_kernel(float* __restrict__ p, const float* __restrict__ zA,
                                                         float scale, Scalars* S, int s, int sp, int first,
                                                         unsigned N4) {
  if (gated(&S->done)) return;
  const float beta = first ? 0.f : (float)(S->rdz[s] / S->rz[sp]);
  GRID_STRIDE(i4, N4) {
    const float4 za = ld4(zA, i4);
    const float4 pv = first ? make_float4(0.f, 0.f, 0.f, 0.f) : ld4(p, i4);
    st4(p, i4, make_float4(scale * za.x + beta * pv.x, scale * za.y + beta * pv.y, scale * za.z + beta * pv.z,
                           scale * za.w + beta * pv.w));
  }
}

// ---- features of the learned initial guess --------------------------------

// Sums that set the feature scales: r.r, z.z, sum log a, sum (log a)^2
__global__ void __launch_bounds__(kBlock) feat_stats_kernel(const float* __restrict__ r, const float* __restrict__ z,
                                                            const float* __restrict__ a, unsigned N, double* fs,
                                                            Reduce R) {
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  GRID_STRIDE(i, N) {
    const double ri = r[i], zi = z[i], la = logf(a[i]);
    v[0] += ri * ri;
    v[1] += zi * zi;
    v[2] += la;
    v[3] += la * la;
  }
  double* const d[4] = {&fs[0], &fs[1], &fs[2], &fs[3]};
  grid_sum<4>(v, R, d);
}

struct FeatScale {
  float inv_rms_r, inv_rms_z, mean_la, inv_sd_la;
};

__device__ __forceinline__ FeatScale feat_scale(const double* fs, unsigned N) {
  FeatScale s;
  const double rr = fs[0] / N, zz = fs[1] / N, mu = fs[2] / N;
  const double var = fmax(fs[3] / N - mu * mu, 0.0);
  s.inv_rms_r = rr > 0.0 ? (float)(1.0 / sqrt(rr)) : 0.f;
  s.inv_rms_z = zz > 0.0 ? (float)(1.0 / sqrt(zz)) : 0.f;
  s.mean_la = (float)mu;
  s.inv_sd_la = var > 0.0 ? (float)(1.0 / sqrt(var)) : 1.f;
  return s;
}

// feats = [r / rms(r), (log a - mean) / std, z / rms(z)]
__global__ void __launch_bounds__(kBlock) feat_write_kernel(const float* __restrict__ r, const float* __restrict__ z,
                                                            const float* __restrict__ a, const double* fs, unsigned N,
                                                            float* __restrict__ feats) {
  const FeatScale sc = feat_scale(fs, N);
  GRID_STRIDE(i, N) {
    feats[i] = r[i] * sc.inv_rms_r;
    feats[(size_t)N + i] = (logf(a[i]) - sc.mean_la) * sc.inv_sd_la;
    feats[2 * (size_t)N + i] = z[i] * sc.inv_rms_z;
  }
}

// target = (phi - phi0) / rms(phi0), phi0 = z / a_ref
__global__ void __launch_bounds__(kBlock) target_kernel(const double* __restrict__ phi, const float* __restrict__ z,
                                                        double inv_aref, const double* fs, unsigned N,
                                                        float* __restrict__ t) {
  const double rz = sqrt(fs[1] / N);
  const double s = rz > 0.0 ? 1.0 / (rz * inv_aref) : 0.0;
  GRID_STRIDE(i, N) t[i] = (float)((phi[i] - (double)z[i] * inv_aref) * s);
}

// phi (=|+=) phi0 + rms(phi0) y
__global__ void __launch_bounds__(kBlock) guess_kernel(double* __restrict__ phi, const float* __restrict__ z,
                                                       const float* __restrict__ y, double inv_aref, const double* fs,
                                                       unsigned N, int add) {
  const double rp = sqrt(fs[1] / N) * inv_aref;
  GRID_STRIDE(i, N) {
    const double v = (double)z[i] * inv_aref + rp * (double)y[i];
    phi[i] = add ? phi[i] + v : v;
  }
}

__global__ void __launch_bounds__(kBlock) to_f32_kernel(const double* __restrict__ x, float* __restrict__ y,
                                                        unsigned N) {
  GRID_STRIDE(i, N) y[i] = (float)x[i];
}

// r = float(g - A phi) = float(g + K phi) with the FP64 operator
__global__ void __launch_bounds__(kBlock) residual_kernel(const double* __restrict__ phi,
                                                          const double* __restrict__ g, Faces<double> F,
                                                          const float* __restrict__ a, Grid G, float* __restrict__ r) {
  GRID_STRIDE(i, G.N) {
    int x, y, z;
    cell_xyz(G, i, x, y, z);
    r[i] = (float)(g[i] + k_apply<double>(phi, F, a, G, i, x, y, z, phi[i]));
  }
}

}  // namespace

struct poisfft_pcg {
  Grid G{};
  unsigned N = 0;
  unsigned nb = 0;              // blocks of the grid-stride kernels
  double a_ref = 1.0;
  float* a = nullptr;
  double* c64[3] = {nullptr, nullptr, nullptr};
  float* c32[3] = {nullptr, nullptr, nullptr};
  // FP64 iteration
  double *r = nullptr, *p = nullptr, *q = nullptr, *z = nullptr;
  float *r32 = nullptr, *z32 = nullptr;
  // mixed iteration (r32 doubles as its residual)
  float *e = nullptr, *p32 = nullptr, *q32 = nullptr, *zb32 = nullptr;
  Scalars* S = nullptr;         // device
  double* part = nullptr;       // 4 * nb partial sums
  unsigned* count = nullptr;    // last-block counter
  Scalars* hS = nullptr;        // pinned host copies, two slots
  cudaEvent_t ev[2] = {nullptr, nullptr};
  poisfft_plan* plan = nullptr;
  int64_t stats[4] = {0, 0, 0, 0};
  // learned initial guess (allocated on first use)
  float *feats = nullptr, *ybuf = nullptr;
  double* fs = nullptr;         // feature sums
};

namespace {

void free_pcg(poisfft_pcg* s) {
  if (!s) return;
  void* bufs[] = {s->a, s->c64[0], s->c64[1], s->c64[2], s->c32[0], s->c32[1], s->c32[2], s->r, s->p, s->q,
                  s->z, s->r32, s->z32, s->e, s->p32, s->q32, s->zb32, s->S, s->part, s->count,
                  s->feats, s->ybuf, s->fs};
  for (void* b : bufs) cudaFree(b);
  if (s->hS) cudaFreeHost(s->hS);
  for (cudaEvent_t e : s->ev)
    if (e) cudaEventDestroy(e);
  if (s->plan) poisfft_destroy(s->plan);
  delete s;
}

template <typename T> Faces<T> faces_of(const poisfft_pcg* s);
template <> Faces<double> faces_of<double>(const poisfft_pcg* s) { return Faces<double>{{s->c64[0], s->c64[1], s->c64[2]}}; }
template <> Faces<float> faces_of<float>(const poisfft_pcg* s) { return Faces<float>{{s->c32[0], s->c32[1], s->c32[2]}}; }

// Copy a, compute the face coefficients and a_ref (<= 0: the mean of a).
int load_coefficient(poisfft_pcg* s, const float* a, double a_ref) {
  const size_t N = s->N;
  if (cudaMemcpy(s->a, a, N * sizeof(float), cudaMemcpyDefault) != cudaSuccess) return POISFFT_ERR_CUDA;
  faces_kernel<<<s->nb, kBlock>>>(s->a, s->G, s->c64[0], s->c64[1], s->c64[2], s->c32[0], s->c32[1], s->c32[2]);
  if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) return POISFFT_ERR_CUDA;
  if (a_ref > 0.0) {
    s->a_ref = a_ref;
    return POISFFT_OK;
  }
  float* h = new (std::nothrow) float[N];  // mean of a: host reduction once, FP64
  if (!h) return POISFFT_ERR_ALLOC;
  if (cudaMemcpy(h, s->a, N * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess) {
    delete[] h;
    return POISFFT_ERR_CUDA;
  }
  double sum = 0.0;
  for (size_t i = 0; i < N; i++) sum += h[i];
  delete[] h;
  s->a_ref = sum / (double)N;
  return POISFFT_OK;
}

// Features of right-hand side g into s->feats; leaves z = L^{-1} g in s->z32
// and the sums in s->fs.  `r_is_set`: s->r32 already holds the right-hand side.
int learned_features(poisfft_pcg* s, const double* g, int r_is_set, cudaStream_t st) {
  if (!s->feats) {
    if (cudaMalloc(&s->feats, 3 * (size_t)s->N * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&s->ybuf, (size_t)s->N * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&s->fs, 4 * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      return POISFFT_ERR_ALLOC;
    }
  }
  if (!r_is_set) to_f32_kernel<<<s->nb, kBlock, 0, st>>>(g, s->r32, s->N);
  int rc = poisfft_solve(s->plan, s->z32, s->r32, st);
  if (rc != POISFFT_OK) return rc;
  feat_stats_kernel<<<s->nb, kBlock, 0, st>>>(s->r32, s->z32, s->a, s->N, s->fs, Reduce{s->part, s->count});
  feat_write_kernel<<<s->nb, kBlock, 0, st>>>(s->r32, s->z32, s->a, s->fs, s->N, s->feats);
  return cudaGetLastError() == cudaSuccess ? POISFFT_OK : POISFFT_ERR_CUDA;
}

int publish(poisfft_pcg* s, int k, cudaStream_t st) {
  if (cudaMemcpyAsync(&s->hS[k & 1], s->S, sizeof(Scalars), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaEventRecord(s->ev[k & 1], st) != cudaSuccess)
    return POISFFT_ERR_CUDA;
  return POISFFT_OK;
}

int finish(poisfft_pcg* s, cudaStream_t st, int* iters, double* relres, int mode, int64_t precond) {
  if (cudaStreamSynchronize(st) != cudaSuccess) return POISFFT_ERR_CUDA;
  if (cudaMemcpy(&s->hS[0], s->S, sizeof(Scalars), cudaMemcpyDeviceToHost) != cudaSuccess) return POISFFT_ERR_CUDA;
  if (iters) *iters = s->hS[0].it;
  if (relres) *relres = s->hS[0].rel;
  s->stats[0] = s->hS[0].it;
  s->stats[1] = s->hS[0].n_true;
  s->stats[2] = precond;
  s->stats[3] = mode;
  return POISFFT_OK;
}

int solve_f64(poisfft_pcg* s, double* phi, const double* g, double tol, int maxit, int* iters, double* relres,
              void* stream) {
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const unsigned N = s->N, nb = s->nb;
  const double scale = -1.0 / s->a_ref;
  const Reduce R{s->part, s->count};
  const Faces<double> F = faces_of<double>(s);
  int64_t precond = 0;
  auto precondition = [&](int slot, int first, int sp) -> int {
    int rc = poisfft_solve(s->plan, s->z32, s->r32, stream);
    if (rc != POISFFT_OK) return rc;
    precond++;
    f64_precond_kernel<<<nb, kBlock, 0, st>>>(s->z32, s->r, s->z, scale, s->S, R, slot, first, N);
    f64_dir_kernel<<<nb, kBlock, 0, st>>>(s->p, s->z, s->S, slot, sp, first, N);
    return cudaGetLastError() == cudaSuccess ? POISFFT_OK : POISFFT_ERR_CUDA;
  };
  if (cudaMemsetAsync(s->S, 0, sizeof(Scalars), st) != cudaSuccess) return POISFFT_ERR_CUDA;
  f64_init_kernel<<<nb, kBlock, 0, st>>>(phi, g, F, s->a, s->G, s->r, s->r32, s->S, R);
  init_check_kernel<<<1, 1, 0, st>>>(s->S, tol);
  if (cudaGetLastError() != cudaSuccess) return POISFFT_ERR_CUDA;
  int rc = POISFFT_OK;
  if (maxit > 0 && (rc = precondition(0, 1, 1)) != POISFFT_OK) return rc;
  if ((rc = publish(s, 0, st)) != POISFFT_OK) return rc;
  for (int k = 1; k <= maxit; k++) {
    const int sl = k & 1, sp = sl ^ 1;
    apply_kernel<double><<<nb, kBlock, 0, st>>>(s->p, F, s->a, s->G, s->q, R, &s->S->pq[sl], &s->S->done);
    f64_update_kernel<<<nb, kBlock, 0, st>>>(phi, s->r, s->p, s->q, s->r32, s->S, R, sl, sp, N);
    f64_check_kernel<<<1, 1, 0, st>>>(s->S, sl, k, tol);
    if (cudaGetLastError() != cudaSuccess) return POISFFT_ERR_CUDA;
    if ((rc = publish(s, k, st)) != POISFFT_OK) return rc;
    if (k < maxit && (rc = precondition(sl, 0, sp)) != POISFFT_OK) return rc;
    if (cudaEventSynchronize(s->ev[(k - 1) & 1]) != cudaSuccess) return POISFFT_ERR_CUDA;
    if (s->hS[(k - 1) & 1].done) break;
  }
  return finish(s, st, iters, relres, POISFFT_PCG_F64, precond);
}

int solve_mixed(poisfft_pcg* s, double* phi, const double* g, double tol, int maxit, int* iters, double* relres,
                void* stream) {
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const unsigned N = s->N, nb = s->nb;
  const double scale = -1.0 / s->a_ref;
  const Reduce R{s->part, s->count};
  const Faces<double> F64 = faces_of<double>(s);
  const Faces<float> F32 = faces_of<float>(s);
  int* done = &s->S->done;
  int* rel_flag = &s->S->reliable;
  const bool vec4 = s->G.nx % 4 == 0;  // 128-bit rows (device buffers are 256-byte aligned)
  float* zA = s->z32;   // preconditioner output for the current residual
  float* zB = s->zb32;  // ... for the previous one
  int64_t precond = 0;
  auto precondition = [&](int slot, int first, int sp) -> int {
    int rc = poisfft_solve(s->plan, zA, s->r32, stream);
    if (rc != POISFFT_OK) return rc;
    precond++;
    if (vec4) {
      mx_precond4_kernel<<<nb, kBlock, 0, st>>>(s->r32, zA, zB, scale, s->S, R, slot, first, N / 4);
      mx_dir4_kernel<<<nb, kBlock, 0, st>>>(s->p32, zA, (float)scale, s->S, slot, sp, first, N / 4);
    } else {
      mx_precond_kernel<<<nb, kBlock, 0, st>>>(s->r32, zA, zB, scale, s->S, R, slot, first, N);
      mx_dir_kernel<<<nb, kBlock, 0, st>>>(s->p32, zA, (float)scale, s->S, slot, sp, first, N);
    }
    std::swap(zA, zB);
    return cudaGetLastError() == cudaSuccess ? POISFFT_OK : POISFFT_ERR_CUDA;
  };
  if (cudaMemsetAsync(s->S, 0, sizeof(Scalars), st) != cudaSuccess ||
      cudaMemsetAsync(s->e, 0, (size_t)N * sizeof(float), st) != cudaSuccess)
    return POISFFT_ERR_CUDA;
  mx_resid_kernel<<<nb, kBlock, 0, st>>>(phi, g, F64, s->a, s->G, s->r32, s->S, R, nullptr, 1);
  init_check_kernel<<<1, 1, 0, st>>>(s->S, tol);
  if (cudaGetLastError() != cudaSuccess) return POISFFT_ERR_CUDA;
  int rc = POISFFT_OK;
  if (maxit > 0 && (rc = precondition(0, 1, 1)) != POISFFT_OK) return rc;
  if ((rc = publish(s, 0, st)) != POISFFT_OK) return rc;
  for (int k = 1; k <= maxit; k++) {
    const int sl = k & 1, sp = sl ^ 1;
    if (vec4) {
      apply4_kernel<<<nb, kBlock, 0, st>>>(s->p32, F32, s->a, s->G, s->q32, R, &s->S->pq[sl], done);
      mx_update4_kernel<<<nb, kBlock, 0, st>>>(s->e, s->r32, s->p32, s->q32, s->S, R, sl, sp, N / 4);
    } else {
      apply_kernel<float><<<nb, kBlock, 0, st>>>(s->p32, F32, s->a, s->G, s->q32, R, &s->S->pq[sl], done);
      mx_update_kernel<<<nb, kBlock, 0, st>>>(s->e, s->r32, s->p32, s->q32, s->S, R, sl, sp, N);
    }
    mx_check_kernel<<<1, 1, 0, st>>>(s->S, sl, k, tol, kReliableDelta);
    mx_axpy_kernel<<<nb, kBlock, 0, st>>>(phi, s->e, done, rel_flag, N);
    mx_resid_kernel<<<nb, kBlock, 0, st>>>(phi, g, F64, s->a, s->G, s->r32, s->S, R, rel_flag, 0);
    mx_check2_kernel<<<1, 1, 0, st>>>(s->S, tol);
    if (cudaGetLastError() != cudaSuccess) return POISFFT_ERR_CUDA;
    if ((rc = publish(s, k, st)) != POISFFT_OK) return rc;
    if (k < maxit && (rc = precondition(sl, 0, sp)) != POISFFT_OK) return rc;
    if (cudaEventSynchronize(s->ev[(k - 1) & 1]) != cudaSuccess) return POISFFT_ERR_CUDA;
    if (s->hS[(k - 1) & 1].done) break;
  }
  // stopped at maxit: fold the correction in and take the true residual
  mx_axpy_kernel<<<nb, kBlock, 0, st>>>(phi, s->e, done, nullptr, N);
  mx_resid_kernel<<<nb, kBlock, 0, st>>>(phi, g, F64, s->a, s->G, s->r32, s->S, R, nullptr, 0);
  mx_final_kernel<<<1, 1, 0, st>>>(s->S);
  if (cudaGetLastError() != cudaSuccess) return POISFFT_ERR_CUDA;
  return finish(s, st, iters, relres, POISFFT_PCG_MIXED, precond);
}

}  // namespace

namespace {
// device arrays must be aligned to their element size (a misaligned pointer
// would fault in the kernels, so it is refused here)
template <typename T> bool aligned(const T* p) { return p == nullptr || (uintptr_t)p % sizeof(T) == 0; }
}  // namespace

extern "C" {

int poisfft_pcg_create(poisfft_pcg** out, const int64_t n[3], const double L[3], const float* a, double a_ref) {
  if (!out) return POISFFT_ERR_INVALID_ARG;
  *out = nullptr;
  if (!n || !L || !a) return POISFFT_ERR_INVALID_ARG;
  for (int d = 0; d < 3; d++)
    if (n[d] < 1 || n[d] > (1 << 20) || !(L[d] > 0.0) || !isfinite(L[d])) return POISFFT_ERR_INVALID_ARG;
  if ((double)n[0] * n[1] * n[2] >= 2147483648.0) return POISFFT_ERR_UNSUPPORTED_SIZE;
  poisfft_pcg* s = new (std::nothrow) poisfft_pcg();
  if (!s) return POISFFT_ERR_ALLOC;
  s->G.nx = (int)n[0];
  s->G.ny = (int)n[1];
  s->G.nz = (int)n[2];
  s->N = (unsigned)(n[0] * n[1] * n[2]);
  s->G.N = s->N;
  s->G.idx2 = (n[0] / L[0]) * (n[0] / L[0]);
  s->G.idy2 = (n[1] / L[1]) * (n[1] / L[1]);
  s->G.idz2 = (n[2] / L[2]) * (n[2] / L[2]);
  s->G.fidx2 = (float)s->G.idx2;
  s->G.fidy2 = (float)s->G.idy2;
  s->G.fidz2 = (float)s->G.idz2;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    delete s;
    return POISFFT_ERR_CUDA;
  }
  s->nb = (unsigned)std::min<long long>(((long long)s->N + kBlock - 1) / kBlock, (long long)sms * kBlocksPerSM);
  const int bc[6] = {POISFFT_DS, POISFFT_DS, POISFFT_DS, POISFFT_DS, POISFFT_DS, POISFFT_DS};
  int rc = poisfft_plan_create(&s->plan, 3, n, L, bc, POISFFT_FD2, POISFFT_F32);
  if (rc != POISFFT_OK) {
    free_pcg(s);
    return rc;
  }
  const size_t N = s->N;
  bool ok = cudaMalloc(&s->a, N * sizeof(float)) == cudaSuccess;
  for (int d = 0; d < 3; d++) {
    ok = ok && cudaMalloc(&s->c64[d], N * sizeof(double)) == cudaSuccess;
    ok = ok && cudaMalloc(&s->c32[d], N * sizeof(float)) == cudaSuccess;
  }
  double** d64[] = {&s->r, &s->p, &s->q, &s->z};
  for (double** b : d64) ok = ok && cudaMalloc(b, N * sizeof(double)) == cudaSuccess;
  float** d32[] = {&s->r32, &s->z32, &s->e, &s->p32, &s->q32, &s->zb32};
  for (float** b : d32) ok = ok && cudaMalloc(b, N * sizeof(float)) == cudaSuccess;
  ok = ok && cudaMalloc(&s->S, sizeof(Scalars)) == cudaSuccess &&
       cudaMalloc(&s->part, 4 * sizeof(double) * s->nb) == cudaSuccess &&
       cudaMalloc(&s->count, sizeof(unsigned)) == cudaSuccess &&
       cudaMallocHost(&s->hS, 2 * sizeof(Scalars)) == cudaSuccess &&
       cudaEventCreateWithFlags(&s->ev[0], cudaEventDisableTiming) == cudaSuccess &&
       cudaEventCreateWithFlags(&s->ev[1], cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    free_pcg(s);
    return POISFFT_ERR_ALLOC;
  }
  if (cudaMemset(s->count, 0, sizeof(unsigned)) != cudaSuccess) {
    free_pcg(s);
    return POISFFT_ERR_CUDA;
  }
  if ((rc = load_coefficient(s, a, a_ref)) != POISFFT_OK) {
    free_pcg(s);
    return rc;
  }
  *out = s;
  return POISFFT_OK;
}

int poisfft_pcg_apply(poisfft_pcg* s, double* out, const double* in, void* stream) {
  if (!s || !out || !in) return POISFFT_ERR_INVALID_ARG;
  if (!aligned(out) || !aligned(in)) return POISFFT_ERR_MISALIGNED;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  apply_kernel<double><<<s->nb, kBlock, 0, st>>>(in, faces_of<double>(s), s->a, s->G, out,
                                                 Reduce{s->part, s->count}, nullptr, nullptr);
  return cudaGetLastError() == cudaSuccess ? POISFFT_OK : POISFFT_ERR_CUDA;
}

int poisfft_pcg_solve(poisfft_pcg* s, double* phi, const double* g, double tol, int maxit, int precision, int* iters,
                      double* relres, void* stream) {
  if (!s || !phi || !g || maxit < 0 || !(tol >= 0.0)) return POISFFT_ERR_INVALID_ARG;
  if (!aligned(phi) || !aligned(g)) return POISFFT_ERR_MISALIGNED;
  if (precision == POISFFT_PCG_F64) return solve_f64(s, phi, g, tol, maxit, iters, relres, stream);
  if (precision == POISFFT_PCG_MIXED) return solve_mixed(s, phi, g, tol, maxit, iters, relres, stream);
  return POISFFT_ERR_INVALID_ARG;
}

int poisfft_pcg_stats(const poisfft_pcg* s, int64_t out[4]) {
  if (!s || !out) return POISFFT_ERR_INVALID_ARG;
  for (int i = 0; i < 4; i++) out[i] = s->stats[i];
  return POISFFT_OK;
}

int poisfft_pcg_set_coefficient(poisfft_pcg* s, const float* a, double a_ref) {
  if (!s || !a) return POISFFT_ERR_INVALID_ARG;
  return load_coefficient(s, a, a_ref);
}

int poisfft_pcg_features(poisfft_pcg* s, const double* g, const double* phi, float* feats, float* target,
                         void* stream) {
  if (!s || !g || !feats) return POISFFT_ERR_INVALID_ARG;
  if (!aligned(g) || !aligned(phi) || !aligned(feats) || !aligned(target)) return POISFFT_ERR_MISALIGNED;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  int rc = learned_features(s, g, 0, st);
  if (rc != POISFFT_OK) return rc;
  if (cudaMemcpyAsync(feats, s->feats, 3 * (size_t)s->N * sizeof(float), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return POISFFT_ERR_CUDA;
  if (phi && target) target_kernel<<<s->nb, kBlock, 0, st>>>(phi, s->z32, 1.0 / s->a_ref, s->fs, s->N, target);
  return cudaGetLastError() == cudaSuccess ? POISFFT_OK : POISFFT_ERR_CUDA;
}

int poisfft_pcg_learned_guess(poisfft_pcg* s, poisfft_sno* sno, double* phi, const double* g, int corrections,
                              void* stream) {
  if (!s || !sno || !phi || !g || corrections < 0) return POISFFT_ERR_INVALID_ARG;
  if (!aligned(phi) || !aligned(g)) return POISFFT_ERR_MISALIGNED;
  int64_t info[8];
  if (poisfft_sno_info(sno, info) != POISFFT_OK) return POISFFT_ERR_INVALID_ARG;
  if (info[0] != s->G.nx || info[1] != s->G.ny || info[2] != s->G.nz || info[3] != 1) return POISFFT_ERR_INVALID_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const double inv_aref = 1.0 / s->a_ref;
  for (int c = 0; c <= corrections; c++) {
    if (c > 0) residual_kernel<<<s->nb, kBlock, 0, st>>>(phi, g, faces_of<double>(s), s->a, s->G, s->r32);
    int rc = learned_features(s, g, c > 0, st);
    if (rc != POISFFT_OK) return rc;
    if ((rc = poisfft_sno_forward(sno, s->ybuf, s->feats, stream)) != POISFFT_OK) return rc;
    guess_kernel<<<s->nb, kBlock, 0, st>>>(phi, s->z32, s->ybuf, inv_aref, s->fs, s->N, c > 0);
  }
  return cudaGetLastError() == cudaSuccess ? POISFFT_OK : POISFFT_ERR_CUDA;
}

int poisfft_pcg_destroy(poisfft_pcg* s) {
  free_pcg(s);
  return POISFFT_OK;
}

}  // extern "C"
