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
// Flexible (Polak-Ribiere) PCG on K = -A (symmetric positive definite):
// vectors, the operator and all inner products in FP64; the preconditioner
// z = -(1/a_ref) L_h^{-1} r is the library's FP32 Poisson solve (staggered
// Dirichlet on every face).  Each inner product is fused into the kernel
// that produces its operands (block reduction, one FP64 atomic per block).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <new>

#include "../../include/poisfft.h"

namespace {

constexpr int kBlock = 256;

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Deterministic grid-wide sums of K values per thread.  Each block writes its
// K partial sums to part[k * gridDim.x + block]; the last block to finish
// (counted with one atomic) adds the partials in a fixed order and stores the
// totals to dst[k], then resets the counter.  The result does not depend on
// the order in which blocks run, so repeated solves are bitwise identical.
struct Reduce {
  double* part;     // K * gridDim.x doubles
  unsigned* count;  // zero between kernels
};

template <int K>
__device__ __forceinline__ void grid_sum(const double (&v)[K], Reduce R, double* const (&dst)[K]) {
  __shared__ double sh[K][kBlock / 32];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < K; k++) {
    const double w = warp_sum(v[k]);
    if (lane == 0) sh[k][warp] = w;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < K; k++) {
      double t = 0.0;
      for (int w = 0; w < kBlock / 32; w++) t += sh[k][w];
      R.part[(size_t)k * gridDim.x + blockIdx.x] = t;
    }
    __threadfence();
    last = atomicAdd(R.count, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
#pragma unroll
  for (int k = 0; k < K; k++) {
    double t = 0.0;
    for (unsigned b = threadIdx.x; b < gridDim.x; b += kBlock) t += __ldcg(&R.part[(size_t)k * gridDim.x + b]);
    t = warp_sum(t);
    __syncthreads();
    if (lane == 0) sh[k][warp] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
      double u = 0.0;
      for (int w = 0; w < kBlock / 32; w++) u += sh[k][w];
      *dst[k] = u;
    }
  }
  if (threadIdx.x == 0) *R.count = 0u;
}

struct Grid {
  int nx, ny, nz;
  double idx2, idy2, idz2;  // 1/dx^2 per axis
};

// Scalars of the iteration, kept on the device so that no step waits for the
// host.  Iteration k stores its inner products in slot k % 2 and reads rz of
// slot (k - 1) % 2.
struct Scalars {
  double pq[2], rr[2], rz[2], rdz[2];
  double gg, bnorm, rel;
  int done, it;
};

__device__ __forceinline__ double harm(double ai, double aj) { return 2.0 * ai * aj / (ai + aj); }

// q = K p = -(A p); optional dot += p.q.  Gated: returns at once when the
// iteration has converged.
__global__ void __launch_bounds__(kBlock) vc_apply_kernel(const double* __restrict__ p, const float* __restrict__ a,
                                                          double* __restrict__ q, double* dot, Reduce R,
                                                          const int* done, Grid G) {
  if (done && *(volatile const int*)done) return;
  const long long N = (long long)G.nx * G.ny * G.nz;
  const long long i = (long long)blockIdx.x * kBlock + threadIdx.x;
  double contrib = 0.0;
  if (i < N) {
    const int x = (int)(i % G.nx);
    const long long r = i / G.nx;
    const int y = (int)(r % G.ny);
    const int z = (int)(r / G.ny);
    const double pi = p[i];
    const double ai = a[i];
    double acc = 0.0;
    const long long sy = G.nx, sz = (long long)G.nx * G.ny;
    {
      const double fl = x > 0 ? harm(ai, a[i - 1]) : ai;
      const double pl = x > 0 ? p[i - 1] : -pi;
      const double fh = x < G.nx - 1 ? harm(ai, a[i + 1]) : ai;
      const double ph = x < G.nx - 1 ? p[i + 1] : -pi;
      acc += (fh * (ph - pi) - fl * (pi - pl)) * G.idx2;
    }
    {
      const double fl = y > 0 ? harm(ai, a[i - sy]) : ai;
      const double pl = y > 0 ? p[i - sy] : -pi;
      const double fh = y < G.ny - 1 ? harm(ai, a[i + sy]) : ai;
      const double ph = y < G.ny - 1 ? p[i + sy] : -pi;
      acc += (fh * (ph - pi) - fl * (pi - pl)) * G.idy2;
    }
    {
      const double fl = z > 0 ? harm(ai, a[i - sz]) : ai;
      const double pl = z > 0 ? p[i - sz] : -pi;
      const double fh = z < G.nz - 1 ? harm(ai, a[i + sz]) : ai;
      const double ph = z < G.nz - 1 ? p[i + sz] : -pi;
      acc += (fh * (ph - pi) - fl * (pi - pl)) * G.idz2;
    }
    q[i] = -acc;
    contrib = pi * -acc;
  }
  if (dot) {
    const double v[1] = {contrib};
    double* const d[1] = {dot};
    grid_sum<1>(v, R, d);
  }
}

// r = -g - q (b - K x0 with b = -g); rr += r.r; gg += g.g; r32 = float(r)
__global__ void __launch_bounds__(kBlock) pcg_init_kernel(const double* __restrict__ g, const double* __restrict__ q,
                                                          double* __restrict__ r, float* __restrict__ r32,
                                                          Scalars* S, Reduce R, long long N) {
  const long long i = (long long)blockIdx.x * kBlock + threadIdx.x;
  double v = 0.0, w = 0.0;
  if (i < N) {
    const double ri = -g[i] - q[i];
    r[i] = ri;
    r32[i] = (float)ri;
    v = ri * ri;
    w = g[i] * g[i];
  }
  const double vw[2] = {v, w};
  double* const d[2] = {&S->rr[0], &S->gg};
  grid_sum<2>(vw, R, d);
}

// Initial test: bnorm = |g|; done when g = 0 or the initial guess already
// meets the tolerance.
__global__ void pcg_init_check_kernel(Scalars* S, double tol) {
  S->bnorm = sqrt(S->gg);
  S->rel = S->bnorm > 0.0 ? sqrt(S->rr[0]) / S->bnorm : 0.0;
  S->it = 0;
  S->done = (S->bnorm == 0.0 || S->rel <= tol) ? 1 : 0;
}

// alpha = rz_{k-1} / (p.q); x += alpha p; r -= alpha q; rr += r.r; r32 = float(r)
__global__ void __launch_bounds__(kBlock) pcg_update_kernel(double* __restrict__ x, double* __restrict__ r,
                                                            const double* __restrict__ p,
                                                            const double* __restrict__ q, float* __restrict__ r32,
                                                            Scalars* S, Reduce R, int s, int sp, long long N) {
  if (*(volatile const int*)&S->done) return;
  const double alpha = S->rz[sp] / S->pq[s];
  const long long i = (long long)blockIdx.x * kBlock + threadIdx.x;
  double v = 0.0;
  if (i < N) {
    x[i] += alpha * p[i];
    const double ri = r[i] - alpha * q[i];
    r[i] = ri;
    r32[i] = (float)ri;
    v = ri * ri;
  }
  const double vv[1] = {v};
  double* const d[1] = {&S->rr[s]};
  grid_sum<1>(vv, R, d);
}

// Convergence test of iteration k (one thread).
__global__ void pcg_check_kernel(Scalars* S, int s, int k, double tol) {
  if (S->done) return;
  S->rel = sqrt(S->rr[s]) / S->bnorm;
  S->it = k;
  if (S->rel <= tol) S->done = 1;
}

// z_new = scale * z32; rz += r.z_new; rdz += r.(z_new - z_old); z = z_new.
// first: z_old is taken as 0 (z is not read).
__global__ void __launch_bounds__(kBlock) pcg_precond_kernel(const float* __restrict__ z32,
                                                             const double* __restrict__ r, double* __restrict__ z,
                                                             double scale, Scalars* S, Reduce R, int s,
                                                             int first, long long N) {
  if (*(volatile const int*)&S->done) return;
  const long long i = (long long)blockIdx.x * kBlock + threadIdx.x;
  double v = 0.0, w = 0.0;
  if (i < N) {
    const double zn = scale * (double)z32[i];
    const double ri = r[i];
    v = ri * zn;
    w = ri * (first ? zn : zn - z[i]);
    z[i] = zn;
  }
  const double vw[2] = {v, w};
  double* const d[2] = {&S->rz[s], &S->rdz[s]};
  grid_sum<2>(vw, R, d);
}

// p = z + beta p with beta = rdz_k / rz_{k-1} (Polak-Ribiere); first: p = z.
__global__ void __launch_bounds__(kBlock) pcg_dir_kernel(double* __restrict__ p, const double* __restrict__ z,
                                                         Scalars* S, int s, int sp, int first, long long N) {
  if (*(volatile const int*)&S->done) return;
  const double beta = first ? 0.0 : S->rdz[s] / S->rz[sp];
  const long long i = (long long)blockIdx.x * kBlock + threadIdx.x;
  if (i < N) p[i] = first ? z[i] : z[i] + beta * p[i];
}

}  // namespace

struct poisfft_pcg {
  Grid G{};
  long long N = 0;
  double a_ref = 1.0;
  float* a = nullptr;
  double *r = nullptr, *p = nullptr, *q = nullptr, *z = nullptr;
  float *r32 = nullptr, *z32 = nullptr;
  Scalars* S = nullptr;         // device
  double* part = nullptr;       // 2 * blocks partial sums
  unsigned* count = nullptr;    // last-block counter
  Scalars* hS = nullptr;        // pinned host copies, two slots
  cudaEvent_t ev[2] = {nullptr, nullptr};
  poisfft_plan* plan = nullptr;
};

namespace {

void free_pcg(poisfft_pcg* s) {
  if (!s) return;
  cudaFree(s->a);
  cudaFree(s->r);
  cudaFree(s->p);
  cudaFree(s->q);
  cudaFree(s->z);
  cudaFree(s->r32);
  cudaFree(s->z32);
  cudaFree(s->S);
  cudaFree(s->part);
  cudaFree(s->count);
  if (s->hS) cudaFreeHost(s->hS);
  for (cudaEvent_t e : s->ev)
    if (e) cudaEventDestroy(e);
  if (s->plan) poisfft_destroy(s->plan);
  delete s;
}

unsigned blocks(long long N) { return (unsigned)((N + kBlock - 1) / kBlock); }

}  // namespace

extern "C" {

int poisfft_pcg_create(poisfft_pcg** out, const int64_t n[3], const double L[3], const float* a, double a_ref) {
  if (!out) return POISFFT_ERR_INVALID_ARG;
  *out = nullptr;
  if (!n || !L || !a) return POISFFT_ERR_INVALID_ARG;
  for (int d = 0; d < 3; d++)
    if (n[d] < 1 || n[d] > (1 << 20) || !(L[d] > 0.0)) return POISFFT_ERR_INVALID_ARG;
  poisfft_pcg* s = new (std::nothrow) poisfft_pcg();
  if (!s) return POISFFT_ERR_ALLOC;
  s->G.nx = (int)n[0];
  s->G.ny = (int)n[1];
  s->G.nz = (int)n[2];
  s->G.idx2 = (n[0] / L[0]) * (n[0] / L[0]);
  s->G.idy2 = (n[1] / L[1]) * (n[1] / L[1]);
  s->G.idz2 = (n[2] / L[2]) * (n[2] / L[2]);
  s->N = n[0] * n[1] * n[2];
  const int bc[6] = {POISFFT_DS, POISFFT_DS, POISFFT_DS, POISFFT_DS, POISFFT_DS, POISFFT_DS};
  int rc = poisfft_plan_create(&s->plan, 3, n, L, bc, POISFFT_FD2, POISFFT_F32);
  if (rc != POISFFT_OK) {
    free_pcg(s);
    return rc;
  }
  const size_t N = (size_t)s->N;
  if (cudaMalloc(&s->a, N * sizeof(float)) != cudaSuccess || cudaMalloc(&s->r, N * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&s->p, N * sizeof(double)) != cudaSuccess || cudaMalloc(&s->q, N * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&s->z, N * sizeof(double)) != cudaSuccess || cudaMalloc(&s->r32, N * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&s->z32, N * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&s->S, sizeof(Scalars)) != cudaSuccess ||
      cudaMalloc(&s->part, 2 * sizeof(double) * blocks(s->N)) != cudaSuccess ||
      cudaMalloc(&s->count, sizeof(unsigned)) != cudaSuccess ||
      cudaMallocHost(&s->hS, 2 * sizeof(Scalars)) != cudaSuccess ||
      cudaEventCreateWithFlags(&s->ev[0], cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&s->ev[1], cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    free_pcg(s);
    return POISFFT_ERR_ALLOC;
  }
  if (cudaMemcpy(s->a, a, N * sizeof(float), cudaMemcpyDefault) != cudaSuccess) {
    free_pcg(s);
    return POISFFT_ERR_CUDA;
  }
  if (cudaMemset(s->count, 0, sizeof(unsigned)) != cudaSuccess) {
    free_pcg(s);
    return POISFFT_ERR_CUDA;
  }
  if (a_ref > 0.0) {
    s->a_ref = a_ref;
  } else {  // mean of a (host reduction once, FP64)
    float* h = new (std::nothrow) float[N];
    if (!h) {
      free_pcg(s);
      return POISFFT_ERR_ALLOC;
    }
    cudaMemcpy(h, s->a, N * sizeof(float), cudaMemcpyDeviceToHost);
    double sum = 0.0;
    for (size_t i = 0; i < N; i++) sum += h[i];
    delete[] h;
    s->a_ref = sum / (double)N;
  }
  *out = s;
  return POISFFT_OK;
}

int poisfft_pcg_apply(poisfft_pcg* s, double* out, const double* in, void* stream) {
  if (!s || !out || !in) return POISFFT_ERR_INVALID_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  vc_apply_kernel<<<blocks(s->N), kBlock, 0, st>>>(in, s->a, out, nullptr, Reduce{s->part, s->count}, nullptr,
                                                   s->G);
  return cudaGetLastError() == cudaSuccess ? POISFFT_OK : POISFFT_ERR_CUDA;
}

int poisfft_pcg_solve(poisfft_pcg* s, double* phi, const double* g, double tol, int maxit, int* iters,
                      double* relres, void* stream) {
  if (!s || !phi || !g || maxit < 0 || !(tol >= 0.0)) return POISFFT_ERR_INVALID_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const long long N = s->N;
  const unsigned nb = blocks(N);
  const double scale = -1.0 / s->a_ref;
  int* done = &s->S->done;
  const Reduce R{s->part, s->count};
  // Iteration k's kernels are enqueued before the host looks at iteration
  // k-1's test, so the device never idles on the host; kernels after the
  // converged iteration return at once (only one preconditioner solve is
  // spent).
  auto precondition = [&](int slot, int first, int sp) -> int {
    int rc = poisfft_solve(s->plan, s->z32, s->r32, stream);
    if (rc != POISFFT_OK) return rc;
    pcg_precond_kernel<<<nb, kBlock, 0, st>>>(s->z32, s->r, s->z, scale, s->S, R, slot, first, N);
    pcg_dir_kernel<<<nb, kBlock, 0, st>>>(s->p, s->z, s->S, slot, sp, first, N);
    return cudaGetLastError() == cudaSuccess ? POISFFT_OK : POISFFT_ERR_CUDA;
  };
  auto publish = [&](int k) -> int {
    if (cudaMemcpyAsync(&s->hS[k & 1], s->S, sizeof(Scalars), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaEventRecord(s->ev[k & 1], st) != cudaSuccess)
      return POISFFT_ERR_CUDA;
    return POISFFT_OK;
  };
  if (cudaMemsetAsync(s->S, 0, sizeof(Scalars), st) != cudaSuccess) return POISFFT_ERR_CUDA;
  vc_apply_kernel<<<nb, kBlock, 0, st>>>(phi, s->a, s->q, nullptr, R, nullptr, s->G);
  pcg_init_kernel<<<nb, kBlock, 0, st>>>(g, s->q, s->r, s->r32, s->S, R, N);
  pcg_init_check_kernel<<<1, 1, 0, st>>>(s->S, tol);
  if (cudaGetLastError() != cudaSuccess) return POISFFT_ERR_CUDA;
  int rc = POISFFT_OK;
  if (maxit > 0) {
    rc = precondition(0, 1, 1);
    if (rc != POISFFT_OK) return rc;
  }
  if ((rc = publish(0)) != POISFFT_OK) return rc;
  for (int k = 1; k <= maxit; k++) {
    const int sl = k & 1, sp = sl ^ 1;
    vc_apply_kernel<<<nb, kBlock, 0, st>>>(s->p, s->a, s->q, &s->S->pq[sl], R, done, s->G);
    pcg_update_kernel<<<nb, kBlock, 0, st>>>(phi, s->r, s->p, s->q, s->r32, s->S, R, sl, sp, N);
    pcg_check_kernel<<<1, 1, 0, st>>>(s->S, sl, k, tol);
    if (cudaGetLastError() != cudaSuccess) return POISFFT_ERR_CUDA;
    if ((rc = publish(k)) != POISFFT_OK) return rc;
    if (k < maxit && (rc = precondition(sl, 0, sp)) != POISFFT_OK) return rc;
    // test of the previous iteration (already finished or about to)
    if (cudaEventSynchronize(s->ev[(k - 1) & 1]) != cudaSuccess) return POISFFT_ERR_CUDA;
    if (s->hS[(k - 1) & 1].done) break;
  }
  if (cudaStreamSynchronize(st) != cudaSuccess) return POISFFT_ERR_CUDA;
  if (cudaMemcpy(&s->hS[0], s->S, sizeof(Scalars), cudaMemcpyDeviceToHost) != cudaSuccess) return POISFFT_ERR_CUDA;
  if (iters) *iters = s->hS[0].it;
  if (relres) *relres = s->hS[0].rel;
  return POISFFT_OK;
}

int poisfft_pcg_destroy(poisfft_pcg* s) {
  free_pcg(s);
  return POISFFT_OK;
}

}  // extern "C"
