/*
 * poisfft.h -- C interface of the GB300 (sm_103a) fast Poisson solver.
 *
 * Solves the discrete Poisson equation lap(phi) = g (Eq. poisson-continuous,
 * Sec. 1) on a uniform 1-, 2- or 3-D grid by the three-step algorithm of
 * Sec. 2.1: forward transform along every axis chosen by that axis's
 * boundary condition (Table 2), division by the Laplacian eigenvalues
 * (Table 3 pseudo-spectral or Table 4 second-order finite differences,
 * summed over axes as in Sec. 2.3), and the backward transforms (Table 2).
 * The paper's library exposes the same three calls: initialise the solver,
 * compute, finalise (Sec. 3).
 *
 * Array layout everywhere: x fastest.  Element (i, j, k) of an nx*ny*nz
 * field is at offset i + nx*(j + ny*k), i.e. a C array [nz][ny][nx].
 *
 * Every call returns a status code: POISFFT_OK (0) or a negative error.
 * No call aborts the process.
 */
#ifndef POISFFT_H
#define POISFFT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Boundary conditions of one face (Sec. 2.1 grids, Table 2 rows).
 *   POISFFT_P   periodic, regular grid x_j = j L/n                (DFT / IDFT)
 *   POISFFT_DR  Dirichlet, regular grid x_j = (j+1) L/(n+1)       (DST-I)
 *   POISFFT_DS  Dirichlet, staggered grid x_j = (j+1/2) L/n       (DST-II / DST-III)
 *   POISFFT_NR  Neumann, regular grid x_j = j L/(n-1)             (DCT-I)
 *   POISFFT_NS  Neumann, staggered grid x_j = (j+1/2) L/n         (DCT-II / DCT-III) */
typedef enum { POISFFT_P = 0, POISFFT_DR = 1, POISFFT_DS = 2, POISFFT_NR = 3, POISFFT_NS = 4 } poisfft_bc;

/* Eigenvalue set: Table 3 (pseudo-spectral) or Table 4 (2nd-order FD). */
typedef enum { POISFFT_SPECTRAL = 0, POISFFT_FD2 = 1 } poisfft_approx;

/* Storage and arithmetic type of phi and g.  The paper's library offers single
 * and double precision solver objects (Sec. 3).  F32: float arrays, FP32
 * arithmetic with tables rounded once from FP64.  F64: double arrays and
 * arithmetic.  MIXED: double arrays; the transforms run in FP32 (the F32
 * kernels) and the result is refined with residuals of the FD2 operator
 * (Eq. FD2-Laplace) formed in FP64, so the answer reaches the F64 solve's
 * accuracy class at a fraction of its cost (see poisfft_solve_refined, which
 * a MIXED plan's poisfft_solve runs).  MIXED needs approx POISFFT_FD2.
 * BF16X3: float arrays; the radix-32 DFT blocks of 1024-point strided (y,
 * z) axes run on the tensor cores (tcgen05) as GEMMs with operands split
 * into two bfloat16 parts each and three products accumulated in FP32
 * (hi*hi + lo*hi + hi*lo); everything else as F32.  About 2^-17 relative
 * error per GEMM pass instead of 2^-24; plans need a strided axis of 1024
 * points with the specialised FP32 kernels (otherwise
 * POISFFT_ERR_NOT_IMPLEMENTED).  The forward and backward sweeps of a
 * periodic axis and the fused divide sweep of a periodic, Neumann- or
 * Dirichlet-staggered axis use it. */
typedef enum { POISFFT_F32 = 0, POISFFT_F64 = 1, POISFFT_MIXED = 2, POISFFT_BF16X3 = 3 } poisfft_dtype;

/* Status codes. */
enum {
  POISFFT_OK = 0,
  POISFFT_ERR_INVALID_ARG = -1,     /* null pointer, dims outside 1..3, n < 1, L <= 0, bad enum */
  POISFFT_ERR_UNSUPPORTED_BC = -2,  /* the two faces of an axis differ, or periodic paired with non-periodic */
  POISFFT_ERR_UNSUPPORTED_SIZE = -3,/* an axis length the kernels cannot tile (reported, never truncated) */
  POISFFT_ERR_ALLOC = -4,           /* device or host allocation failed; nothing is leaked */
  POISFFT_ERR_CUDA = -5,            /* a CUDA runtime/driver call failed (no device, launch error, ...) */
  POISFFT_ERR_MISALIGNED = -6,      /* phi or g not aligned to the element size */
  POISFFT_ERR_TIMEOUT = -7,         /* a bounded device wait gave up (error flag set by a kernel) */
  POISFFT_ERR_NOT_IMPLEMENTED = -8  /* valid arguments outside what this entry point implements */
};

typedef struct poisfft_plan poisfft_plan;  /* opaque; owned by the library */

/* Create a solver for one grid.
 *   out    : receives the plan (set to NULL on error).
 *   dims   : 1, 2 or 3 (Sec. 3: 1, 2 and 3 dimensions).
 *   n      : n[0..dims-1] = points along x, y, z.  n >= 1; NR needs n >= 2.
 *   L      : L[0..dims-1] = domain lengths; dx per axis follows the grid of
 *            the axis's BC (L/n for P and staggered, L/(n+1) DR, L/(n-1) NR).
 *   bc     : bc[2*a] and bc[2*a+1] = the two faces of axis a (low, high).
 *            Both faces must be equal (the transforms of Table 2 are defined
 *            per axis); every per-axis combination is accepted.
 *   approx : poisfft_approx.   dtype : poisfft_dtype; MIXED with approx
 *            SPECTRAL returns POISFFT_ERR_NOT_IMPLEMENTED.
 * Allocates the device workspace (about one field of the plan's dtype plus
 * padding; one FP32 field for MIXED) and FP64-derived tables on the current
 * CUDA device.  All argument checks happen before any CUDA call, so
 * argument errors are reported even without a GPU.
 * FP32 plans of 2 or 3 dimensions with every length in {64, 128, 256, 512,
 * 1024} use specialised two-pass kernels when x is periodic and y/z are
 * periodic or staggered (Dirichlet or Neumann), or when x, y and z are all
 * staggered; all others use the general mixed-radix kernels.  Setting the environment variable POISFFT_FORCE_GENERIC=1 at plan
 * creation selects the general kernels for every plan (testing aid). */
int poisfft_plan_create(poisfft_plan** out, int dims, const int64_t n[], const double L[],
                        const int bc[], int approx, int dtype);

/* Solve lap(phi) = g on the plan's grid (Sec. 2.1 algorithm).
 *   phi, g : device pointers to dense x-fastest arrays of n[0]*n[1]*n[2]
 *            elements of the plan's dtype, aligned to the element size.
 *            g is only read.  phi == g (in place) is allowed; any other
 *            overlap is not.
 *   stream : a cudaStream_t (NULL = legacy default stream).
 * Asynchronous: returns after enqueueing the kernels on `stream`.  A plan
 * owns one workspace, so one plan must not run on two streams at once.
 * For singular problems (every axis P, NR or NS) the component of g in the
 * null space is removed (the all-zero spectral coefficient is set to 0), so
 * phi has zero mean (trapezoid-weighted along NR axes).
 * MIXED plans: phi and g are arrays of doubles (8-byte aligned) and must be
 * distinct; the call is poisfft_solve_refined(plan, phi, g, k, stream) with
 * k = 2 refinements unless poisfft_plan_set_refinements chose another k. */
int poisfft_solve(poisfft_plan* plan, void* phi, const void* g, void* stream);

/* Refinement steps (0..8) that poisfft_solve runs on a MIXED plan.  Each step
 * costs one FP32 solve plus an FP64 residual; 1 step gives about 5e-11 and 2
 * steps about 4e-14 relative error on a 1024^3 FD2 problem.  Returns
 * POISFFT_ERR_INVALID_ARG for other plans or k out of range. */
int poisfft_plan_set_refinements(poisfft_plan* plan, int refinements);

/* The same solve on arrays that are part of larger arrays, e.g. fields with
 * ghost cells (Sec. 3: the right-hand side and the solution can be a subset
 * of a larger array).  phi and g point at element (0,0,0) of the grid;
 * element (i,j,k) is at offset i + j*ld[0] + k*ld[1] (ld in elements).
 *   ld[0] >= n[0] (y rows), ld[1] >= ld[0]*n[1] (z planes); entries for
 *   axes the plan does not have are ignored.
 * Elements outside the grid (ghost cells) are neither read nor written.
 * phi == g with equal strides is allowed.  POISFFT_ERR_INVALID_ARG for
 * strides that would overlap rows or planes; POISFFT_ERR_NOT_IMPLEMENTED for
 * MIXED plans. */
int poisfft_solve_strided(poisfft_plan* plan, void* phi, const int64_t phi_ld[2], const void* g, const int64_t g_ld[2],
                          void* stream);

/* The same solve from and to HOST memory: copies g to the device, solves,
 * copies phi back, all on `stream`, then synchronises the stream.  Pinned
 * host buffers give full copy bandwidth; pageable ones work too.  Device
 * staging buffers (two fields) are allocated on first use and kept by the
 * plan until poisfft_destroy. */
int poisfft_solve_host(poisfft_plan* plan, void* phi_host, const void* g_host, void* stream);

/* The host-buffer solve without waiting, for many right-hand sides in a row.
 * Enqueues the copy of g_host to the device (on an internal copy stream),
 * the solve (on `stream`) and the copy of the result to phi_host (on a
 * second internal copy stream), and returns.  The plan uses two staging
 * pairs in turn, so one call's result copy runs while the next call's input
 * copy and solve proceed, and the two directions of the CPU-GPU link work at
 * once.  `stream` is made to wait for the PREVIOUS call's result copy, so
 * synchronising it completes every call but the last; poisfft_check(plan,
 * stream) waits for the last result copy as well.  No host buffer of a call
 * may be touched until poisfft_check has returned; pinned host buffers are
 * needed for the copies to overlap.  Staging (four fields) is allocated on
 * the first call and kept until poisfft_destroy.  Same status codes as
 * poisfft_solve; POISFFT_ERR_ALLOC if staging cannot be allocated.  The
 * paper has no counterpart (Sec. 3 describes one solve call on caller-owned
 * arrays). */
int poisfft_solve_host_async(poisfft_plan* plan, void* phi_host, const void* g_host, void* stream);

/* Read and clear the plan's device error flag (bounded waits in the kernels
 * set it instead of hanging).  Synchronises `stream` and the result copies of
 * poisfft_solve_host_async.  Returns POISFFT_OK, POISFFT_ERR_TIMEOUT or
 * POISFFT_ERR_CUDA. */
int poisfft_check(poisfft_plan* plan, void* stream);

/* Release the plan's device memory and tables.  NULL is a no-op.  The caller
 * must make sure no solve on the plan is still running. */
int poisfft_destroy(poisfft_plan* plan);

/* Static description of a status code (never NULL). */
const char* poisfft_status_string(int status);

/* Plan introspection for benchmarks and tests (host only, no CUDA calls).
 *   info[0] = number of kernel launches per solve
 *   info[1] = workspace bytes
 *   info[2] = bytes of the dominant (largest-traffic) sweep's algorithmic
 *             HBM traffic per launch: read + write of its tile data
 *   info[3] = index (0-based, launch order) of that sweep
 * Returns POISFFT_OK or POISFFT_ERR_INVALID_ARG. */
int poisfft_plan_info(const poisfft_plan* plan, int64_t info[4]);

/* Solve one problem without allocating device memory.  The paper has no
 * counterpart; this entry point exists for callers that cannot call
 * cudaMalloc -- code inside a framework that owns all device memory through
 * its own pool or budget, plug-ins whose device footprint is fixed after
 * start-up, or paths that must avoid the implicit synchronisation of an
 * allocation.  It runs the same sweep kernels as poisfft_solve (arguments as
 * in poisfft_plan_create plus phi, g, stream as in poisfft_solve) but keeps
 * workspace, tables and error flag in one file-scope device array of
 * 32 MiB that every GPU loading this library holds until the process exits.
 *   - Sizes whose workspace and tables exceed 32 MiB return
 *     POISFFT_ERR_UNSUPPORTED_SIZE before any CUDA call (FP32: up to about
 *     200^3 or 2048^2 with a periodic x axis).
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current; make that first call
 *     before any stream capture.
 *   - All calls share the array and it keeps the last call's contents; each
 *     call clears what must start at zero.  Calls that overlap on the GPU
 *     (other streams, other host threads) race on the array: serialise them.
 *   - Tables are copied from pageable host memory, so the call waits for
 *     the work already queued on `stream` before it returns.  Those copies
 *     read host memory that does not outlive the call, so while `stream`
 *     is being captured the call returns POISFFT_ERR_NOT_IMPLEMENTED and
 *     enqueues nothing.
 * x non-periodic together with a periodic y or z, and dtypes MIXED and BF16X3, return
 * POISFFT_ERR_NOT_IMPLEMENTED here (poisfft_solve handles them).
 * Returns the status codes of poisfft_plan_create / poisfft_solve.  A
 * bounded device wait that gives up does not make the stream fail: it sets
 * the error flag in the shared array, which poisfft_noalloc_check reads. */
int poisfft_solve_noalloc(int dims, const int64_t n[], const double L[], const int bc[], int approx, int dtype,
                          void* phi, const void* g, void* stream);

/* Error flag of poisfft_solve_noalloc on the current device (no paper
 * counterpart).  Synchronises `stream`, reads the flag word at the start of
 * the shared array and clears it.  Every poisfft_solve_noalloc call clears
 * the flag when it starts, so check after each call whose result matters.
 * Returns POISFFT_OK, POISFFT_ERR_TIMEOUT (a kernel's bounded wait gave up:
 * phi is not valid) or POISFFT_ERR_CUDA.  Allocates nothing. */
int poisfft_noalloc_check(void* stream);

/* Mixed-precision solve by iterative refinement (FP64 data, FP32 FFT
 * solves).  `plan` is an FP32 plan with approx POISFFT_FD2; g and phi are
 * distinct device arrays of doubles in the plan's dense layout (8-byte
 * aligned).  phi_0 = S(g) and phi_{k+1} = phi_k + S(g - L phi_k) for
 * `refinements` steps (0..8), where S is the plan's FP32 solve (Sec. 2.1
 * algorithm, Table 4 eigenvalues) and L the second-order FD operator of
 * Eq. FD2-Laplace on every axis with the boundary ghost values whose
 * eigenvectors are the Table 2 bases (P wraps; DR phi_-1 = phi_n = 0; DS
 * phi_-1 = -phi_0, phi_n = -phi_n-1; NS phi_-1 = phi_0, phi_n = phi_n-1; NR
 * phi_-1 = phi_1, phi_n = phi_n-2).  L phi is evaluated in FP64 and the
 * residual rounded to FP32 for S.  Each step multiplies the relative error
 * by about the FP32 solve's (~1e-6) until the FP64 residual's floor, about
 * cond(L) x 1.1e-16.  Singular problems converge to the zero-mode-free
 * solution of the FP64 solve.  `plan` may also be a MIXED plan.  Allocates
 * one FP32 field on first use (kept by the plan); asynchronous on `stream`.
 * Returns POISFFT_OK, INVALID_ARG (FP64 or spectral plan, phi == g,
 * refinements out of range), MISALIGNED, ALLOC or CUDA. */
int poisfft_solve_refined(poisfft_plan* plan, double* phi, const double* g, int refinements, void* stream);

/* Tune the tile shapes of the plan's general-path launches on the device
 * (strided sweeps: w, w/2, w/4 columns per tile; x sweeps: l, l/2, l/4 line
 * pairs per CTA; three timed runs each, the fastest kept).  Allocates two
 * temporary fields, synchronises `stream`, leaves the workspace zeroed.
 * Plans on the specialised kernels keep their fixed shapes.  No paper
 * counterpart.  Returns POISFFT_OK, ALLOC or CUDA. */
int poisfft_plan_autotune(poisfft_plan* plan, void* stream);

/* ---- Batched solves (many independent problems; no paper counterpart) ----
 * poisfft_batch_create: one plan per problem i with dims[i], n[3i..3i+2],
 *   L[3i..3i+2], bc[6i..6i+5] (entries beyond dims[i] ignored), a shared
 *   approx and dtype (F32 or F64; MIXED and BF16X3 return NOT_IMPLEMENTED), with the
 *   default tile shapes (poisfft_batch_autotune tunes them in the batch's
 *   own setting).  Fails with the first failing plan's status.
 * poisfft_batch_solve: solves every problem (phi[i], g[i] as in
 *   poisfft_solve) on `stream` (persistently when the tuner chose that).  The problems' launches run on forked
 *   streams inside one CUDA graph, captured on the first call and replayed
 *   while the pointers and the stream are unchanged (re-captured otherwise).
 *   Capture happens on `stream`, so `stream` must not be the legacy default
 *   stream (use a created stream).
 * poisfft_batch_solve_sequential: the same problems one after another on
 *   `stream` without a graph (the plain form, for comparison).
 * poisfft_batch_autotune: tuning in the batch's own setting.  Times the
 *   whole batch (one capture or work-list build, then 4 solves on `stream`)
 *   under each of POISFFT_BATCH_TUNE_CANDIDATES configurations: 0 = the
 *   tile shapes as created, 1 = every strided tile and x line block halved,
 *   2 = every plan's tiles tuned alone (poisfft_plan_autotune), 3 = the
 *   shapes as created with each 3D general-path problem's sweep order (the
 *   strided axis whose sweep carries the divide: z or y) chosen by timing
 *   both alone, 4 = the shapes as created run as persistent phase launches
 *   (poisfft_batch_solve_persistent; skipped, at 1e30 ms, for batches with
 *   specialised plans); keeps the fastest, and poisfft_batch_solve then
 *   runs it.  phi and g as in poisfft_batch_solve (phi is overwritten with
 *   solutions).  ms (may be NULL) receives the milliseconds per batch solve
 *   of each candidate, chosen (may be NULL) the kept one.
 *   Synchronises `stream`; the next poisfft_batch_solve re-captures the
 *   graph.  Returns POISFFT_OK, INVALID_ARG, ALLOC or CUDA (on failure the
 *   shapes as created are restored).
 * poisfft_batch_check: poisfft_check over all plans (synchronises).
 * poisfft_batch_destroy: frees the plans, streams and graph. */
typedef struct poisfft_batch poisfft_batch;
int poisfft_batch_create(poisfft_batch** out, int count, const int dims[], const int64_t n[], const double L[],
                         const int bc[], int approx, int dtype);
int poisfft_batch_solve(poisfft_batch* batch, void* const phi[], const void* const g[], void* stream);
int poisfft_batch_solve_sequential(poisfft_batch* batch, void* const phi[], const void* const g[], void* stream);
/* poisfft_batch_solve_persistent: the same solves as poisfft_batch_solve as
 * one persistent launch per sweep phase: phase p runs launch p of every
 * problem (x sweeps, strided sweeps, separate divides) from a device work
 * list of (problem, tile) items, largest problems first; CTAs take tiles
 * from an atomic counter and never wait on one another.  The work lists are
 * built and uploaded on the first call and again whenever phi / g change
 * (synchronously; later calls only enqueue a 4-byte memset and one launch
 * per phase on `stream`).  Plans on the specialised FP32 kernels
 * (power-of-two lengths 64..1024 with fitting BCs) are not in the lists:
 * POISFFT_ERR_NOT_IMPLEMENTED.  Returns POISFFT_OK, INVALID_ARG,
 * MISALIGNED, ALLOC or CUDA. */
int poisfft_batch_solve_persistent(poisfft_batch* batch, void* const phi[], const void* const g[], void* stream);
#define POISFFT_BATCH_TUNE_CANDIDATES 5
int poisfft_batch_autotune(poisfft_batch* batch, void* const phi[], const void* const g[], void* stream,
                           double ms[POISFFT_BATCH_TUNE_CANDIDATES], int* chosen);
int poisfft_batch_check(poisfft_batch* batch, void* stream);
/* poisfft_batch_info (host only): out[0] = algorithmic HBM bytes of one
 * batch solve (reads + writes of every launch's data, summed over the
 * problems), out[1] = kernel launches per batch solve, out[2] = grid points
 * of all problems.  Returns POISFFT_OK or POISFFT_ERR_INVALID_ARG. */
int poisfft_batch_info(const poisfft_batch* batch, int64_t out[3]);
/* poisfft_batch_select: apply candidate configuration `candidate` (0..
 * POISFFT_BATCH_TUNE_CANDIDATES-1) of the last poisfft_batch_autotune call,
 * e.g. to time the plain form with every plan tuned alone.  The next
 * poisfft_batch_solve re-captures the graph.  POISFFT_ERR_INVALID_ARG when
 * no tuning has run or the candidate is out of range. */
int poisfft_batch_select(poisfft_batch* batch, int candidate);
int poisfft_batch_destroy(poisfft_batch* batch);

/* ---- FFT-preconditioned CG for div(a grad phi) = g (Sec. 1: the fast solve
 * as a preconditioner for non-constant coefficients) ----
 * Grid: n[3] cells on [0,L0]x[0,L1]x[0,L2], x fastest, cell-centred, phi = 0
 * on every wall (staggered Dirichlet).  Operator: second-order fluxes with
 * harmonic-mean face coefficients 2 a_i a_j / (a_i + a_j); a wall face uses
 * the cell's a and the ghost value -phi.  For constant a it is a times the
 * Table 4 staggered-Dirichlet FD2 Laplacian.  The paper gives no
 * discretisation; this is the library's reading.
 * poisfft_pcg_create: a = cell coefficients (n0*n1*n2 floats, host or device,
 *   copied); a_ref > 0 is the preconditioner's constant coefficient, a_ref
 *   <= 0 selects the mean of a.  The preconditioner is an FP32
 *   poisfft_solve with staggered Dirichlet on every face.  At most 2^31 - 1
 *   cells (POISFFT_ERR_UNSUPPORTED_SIZE).  Synchronises the device once.
 * poisfft_pcg_solve: phi (device doubles) holds the initial guess on entry
 *   and the solution on return; g (device doubles) the right-hand side.
 *   Iterates until ||g - A phi|| <= tol ||g|| or maxit iterations; *iters
 *   and *relres (either may be NULL) report the iterations and the relative
 *   residual reached.  precision:
 *     POISFFT_PCG_F64    flexible (Polak-Ribiere) PCG with FP64 vectors,
 *                        operator and inner products;
 *     POISFFT_PCG_MIXED  the same iteration in FP32 on a correction of phi,
 *                        with reliable updates: phi and the true residual are
 *                        refreshed in FP64 whenever the FP32 residual has
 *                        dropped 1000-fold, and convergence is decided on the
 *                        FP64 residual only (relres is that residual).
 *   Blocks the calling thread: the convergence flag is read on the host one
 *   iteration behind the device.  One solve at a time per object.
 * poisfft_pcg_stats: out[0] iterations, out[1] FP64 (true) residual
 *   evaluations, out[2] preconditioner solves, out[3] precision of the last
 *   poisfft_pcg_solve.
 * poisfft_pcg_apply: out = -(A in) (device doubles), the operator alone.
 * Device arrays must be aligned to their element size
 * (POISFFT_ERR_MISALIGNED otherwise). */
typedef enum { POISFFT_PCG_F64 = 0, POISFFT_PCG_MIXED = 1 } poisfft_pcg_precision;
typedef struct poisfft_pcg poisfft_pcg;
int poisfft_pcg_create(poisfft_pcg** out, const int64_t n[3], const double L[3], const float* a, double a_ref);
int poisfft_pcg_solve(poisfft_pcg* pcg, double* phi, const double* g, double tol, int maxit, int precision,
                      int* iters, double* relres, void* stream);
int poisfft_pcg_stats(const poisfft_pcg* pcg, int64_t out[4]);
int poisfft_pcg_apply(poisfft_pcg* pcg, double* out, const double* in, void* stream);
int poisfft_pcg_destroy(poisfft_pcg* pcg);
/* poisfft_pcg_set_coefficient: replace a (same grid; host or device floats)
 *   and a_ref (<= 0: mean of a); recomputes the face coefficients.
 *   Synchronises the device. */
int poisfft_pcg_set_coefficient(poisfft_pcg* pcg, const float* a, double a_ref);

/* ---- Learned initial guess for the PCG (no paper counterpart: the
 * network is this library's addition on top of the Sec. 1 preconditioner) ----
 * A spectral neural operator in the truncated sine basis of the walls:
 *   v_0 = P f + p;  layer l < L: pre = W_l v_l + b_l + S_inv(R_l . S(v_l)),
 *   v_{l+1} = gelu(pre) (identity for the last layer);  y = Q v_L + q,
 * with S[m,j] = (2/n) sin(pi (m+1)(2j+1) / 2n) (K modes per axis),
 * S_inv[j,m] = sin(pi (m+1)(2j+1) / 2n) and R_l one C x C matrix per mode.
 * Features f of a right-hand side r (3 per cell): r / rms(r),
 * (log a - mean) / std(log a), z / rms(z) with z = L_h^{-1} r (the FD2
 * Poisson solve with staggered Dirichlet walls).  phi0 = z / a_ref solves the
 * problem for the constant coefficient a_ref; the network's output y gives
 * phi0 + rms(phi0) y.
 * Parameters: one FP32 vector, in the order P (C x 3), p (C), per layer W
 * (C x C), b (C), R (K^3 x C x C, mode (mz K + my) K + mx), then Q (C), q;
 * the kernels use it rounded to bfloat16, with FP32 activations and sums.
 * Arrays: activations and features [B][C or 3][n2][n1][n0], x fastest; y and
 * targets [B][n2][n1][n0]; all device memory.
 * poisfft_sno_num_params: parameter count, or -1 outside C <= 32, K <= 16,
 *   L <= 8.
 * poisfft_sno_create: grid n[3] (each >= modes), batch B; train = 1 keeps
 *   the activations for poisfft_sno_backward and the optimiser state.
 *   Parameters start at zero.
 * poisfft_sno_set_params / _get_params: FP32 vector (host or device);
 *   set_params also resets the optimiser state.  Synchronise the device.
 * poisfft_sno_forward: y = network(feats) on `stream`.
 * poisfft_sno_backward: grad = d(sum dy . y)/d(theta) for the activations
 *   of the last forward (train objects only); grad is overwritten.
 * poisfft_sno_loss: L = sum (y - t)^2 / sum t^2 over the batch (to *loss,
 *   host, when non-NULL: synchronises `stream`) and dy = dL/dy (when dy is
 *   non-NULL).
 * poisfft_sno_adam: one Adam step (bias-corrected, step >= 1) on the FP32
 *   parameters, then the bfloat16 copy is refreshed.
 * poisfft_sno_info: out = {n0, n1, n2, B, C, K, L, train}.
 * poisfft_pcg_features: the features of right-hand side g (device doubles)
 *   for the PCG's coefficient into feats (3 N floats); when phi and target
 *   are non-NULL also the training target (phi - phi0) / rms(phi0) (N floats).
 * poisfft_pcg_learned_guess: phi (device doubles, overwritten) = phi0 +
 *   rms(phi0) y for g, then `corrections` times: r = g - A phi (FP64),
 *   phi += the same construction for r.  The network must have batch 1 and
 *   the PCG's grid.  Synchronises nothing; pass phi to poisfft_pcg_solve.
 * Device arrays must be aligned to their element size
 * (POISFFT_ERR_MISALIGNED otherwise). */
typedef struct poisfft_sno poisfft_sno;
int64_t poisfft_sno_num_params(int channels, int modes, int layers);
int poisfft_sno_create(poisfft_sno** out, const int64_t n[3], int batch, int channels, int modes, int layers,
                       int train);
int poisfft_sno_set_params(poisfft_sno* sno, const float* theta);
int poisfft_sno_get_params(const poisfft_sno* sno, float* theta);
int poisfft_sno_forward(poisfft_sno* sno, float* y, const float* feats, void* stream);
int poisfft_sno_backward(poisfft_sno* sno, float* grad, const float* dy, const float* feats, void* stream);
int poisfft_sno_loss(poisfft_sno* sno, const float* y, const float* t, float* dy, double* loss, void* stream);
int poisfft_sno_adam(poisfft_sno* sno, const float* grad, double lr, double beta1, double beta2, double eps, int step,
                     void* stream);
int poisfft_sno_info(const poisfft_sno* sno, int64_t out[8]);
int poisfft_sno_destroy(poisfft_sno* sno);
int poisfft_pcg_features(poisfft_pcg* pcg, const double* g, const double* phi, float* feats, float* target,
                         void* stream);
int poisfft_pcg_learned_guess(poisfft_pcg* pcg, poisfft_sno* sno, double* phi, const double* g, int corrections,
                              void* stream);

/* Zero mode of a singular problem (every axis P, NR or NS), which the solve
 * removes from g (the paper does not discuss it; the reading: the all-zero
 * spectral coefficient is set to 0).  *mean = sum w g / sum w with w = 1/2
 * at both ends of NR axes (the k = 0 row of the Table 2 forward
 * transforms) and 1 elsewhere, summed with compensation per thread and in
 * FP64 across threads.  g: device array of the plan's dtype, dense.
 * POISFFT_ERR_INVALID_ARG for a plan that is not singular.  Synchronises
 * `stream`. */
int poisfft_zero_mode_mean(poisfft_plan* plan, const void* g, double* mean, void* stream);

/* Per-launch timing for benchmarks (no paper counterpart; measurement aid).
 * When enabled, every solve records a CUDA event on its stream before each
 * kernel launch and after the last one.  Host cost: one event record per
 * launch.  Returns POISFFT_OK or POISFFT_ERR_INVALID_ARG. */
int poisfft_profile_enable(poisfft_plan* plan, int enable);

/* Synchronise the recorded events and return, per launch position i of a
 * solve, the summed device milliseconds over all profiled solves since the
 * last call: ms[i] for i < min(cap, *nlaunch).  *nsolves = number of
 * profiled solves.  Clears the record.  POISFFT_ERR_CUDA on event errors. */
int poisfft_profile_read(poisfft_plan* plan, double* ms, int cap, int* nlaunch, int* nsolves);

/* Description of launch position i of a solve (host only).
 *   out[0] = algorithmic HBM bytes of the launch (reads + writes of its data)
 *   out[1] = kernel: 0 contiguous (x) sweep, 1 strided (y/z) sweep,
 *            2 separate eigenvalue divide (x non-periodic with periodic y/z),
 *            3 strided sweep on the tensor cores (BF16X3 plans)
 *   out[2] = mode: 0 forward, 1 backward, 2 forward + divide + backward
 *   out[3] = axis: 0 x, 1 y, 2 z
 * Returns POISFFT_OK or POISFFT_ERR_INVALID_ARG (i out of range). */
int poisfft_launch_info(const poisfft_plan* plan, int i, int64_t out[4]);

#ifdef __cplusplus
}
#endif

#endif /* POISFFT_H */
