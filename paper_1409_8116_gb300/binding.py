"""Thin ctypes binding of libpoisfft.so (argument marshalling only).

Every call goes through the C interface declared in include/poisfft.h; all
arithmetic of the solve runs in the library's CUDA kernels.  PyTorch is used
only by callers that want device tensors and streams; the functions here take
raw pointers (ints) or torch tensors and pass their addresses.

If the shared library is missing the import of this module fails loudly --
there is no CPU fallback.
"""

from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpoisfft.so")

P, DR, DS, NR, NS = 0, 1, 2, 3, 4
PCG_F64, PCG_MIXED = 0, 1
SPECTRAL, FD2 = 0, 1
F32, F64, MIXED, BF16X3 = 0, 1, 2, 3

OK = 0
ERR_INVALID_ARG = -1
ERR_UNSUPPORTED_BC = -2
ERR_UNSUPPORTED_SIZE = -3
ERR_ALLOC = -4
ERR_CUDA = -5
ERR_MISALIGNED = -6
ERR_TIMEOUT = -7
ERR_NOT_IMPLEMENTED = -8

EXPORTED = [
    "poisfft_plan_create",
    "poisfft_solve",
    "poisfft_solve_host",
    "poisfft_solve_host_async",
    "poisfft_check",
    "poisfft_destroy",
    "poisfft_status_string",
    "poisfft_plan_info",
    "poisfft_profile_enable",
    "poisfft_profile_read",
    "poisfft_launch_info",
    "poisfft_solve_noalloc",
    "poisfft_noalloc_check",
    "poisfft_plan_set_refinements",
    "poisfft_solve_strided",
    "poisfft_plan_autotune",
    "poisfft_batch_create",
    "poisfft_batch_solve",
    "poisfft_batch_solve_sequential",
    "poisfft_batch_solve_persistent",
    "poisfft_batch_autotune",
    "poisfft_batch_check",
    "poisfft_batch_info",
    "poisfft_batch_select",
    "poisfft_batch_destroy",
    "poisfft_pcg_create",
    "poisfft_pcg_solve",
    "poisfft_pcg_apply",
    "poisfft_pcg_stats",
    "poisfft_pcg_destroy",
    "poisfft_pcg_set_coefficient",
    "poisfft_pcg_features",
    "poisfft_pcg_learned_guess",
    "poisfft_sno_num_params",
    "poisfft_sno_create",
    "poisfft_sno_set_params",
    "poisfft_sno_get_params",
    "poisfft_sno_forward",
    "poisfft_sno_backward",
    "poisfft_sno_loss",
    "poisfft_sno_adam",
    "poisfft_sno_info",
    "poisfft_sno_destroy",
    "poisfft_zero_mode_mean",
    "poisfft_solve_refined",
]


class PoisFFTError(RuntimeError):
    def __init__(self, status, where=""):
        self.status = status
        super().__init__(f"{where}: {status_string(status)} ({status})")


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"{LIB_PATH} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(LIB_PATH)
    i64p = ctypes.POINTER(ctypes.c_int64)
    lib.poisfft_plan_create.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, i64p,
                                        ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int),
                                        ctypes.c_int, ctypes.c_int]
    lib.poisfft_plan_create.restype = ctypes.c_int
    lib.poisfft_solve.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    lib.poisfft_solve.restype = ctypes.c_int
    lib.poisfft_solve_host.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    lib.poisfft_solve_host.restype = ctypes.c_int
    lib.poisfft_solve_host_async.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    lib.poisfft_solve_host_async.restype = ctypes.c_int
    lib.poisfft_check.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    lib.poisfft_check.restype = ctypes.c_int
    lib.poisfft_destroy.argtypes = [ctypes.c_void_p]
    lib.poisfft_destroy.restype = ctypes.c_int
    lib.poisfft_status_string.argtypes = [ctypes.c_int]
    lib.poisfft_status_string.restype = ctypes.c_char_p
    lib.poisfft_plan_info.argtypes = [ctypes.c_void_p, i64p]
    lib.poisfft_plan_info.restype = ctypes.c_int
    lib.poisfft_profile_enable.argtypes = [ctypes.c_void_p, ctypes.c_int]
    lib.poisfft_profile_enable.restype = ctypes.c_int
    lib.poisfft_profile_read.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int,
                                         ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
    lib.poisfft_profile_read.restype = ctypes.c_int
    lib.poisfft_launch_info.argtypes = [ctypes.c_void_p, ctypes.c_int, i64p]
    lib.poisfft_launch_info.restype = ctypes.c_int
    lib.poisfft_solve_noalloc.argtypes = [ctypes.c_int, i64p, ctypes.POINTER(ctypes.c_double),
                                          ctypes.POINTER(ctypes.c_int), ctypes.c_int, ctypes.c_int,
                                          ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    lib.poisfft_solve_noalloc.restype = ctypes.c_int
    lib.poisfft_noalloc_check.argtypes = [ctypes.c_void_p]
    lib.poisfft_noalloc_check.restype = ctypes.c_int
    lib.poisfft_plan_set_refinements.argtypes = [ctypes.c_void_p, ctypes.c_int]
    lib.poisfft_plan_set_refinements.restype = ctypes.c_int
    lib.poisfft_solve_strided.argtypes = [ctypes.c_void_p, ctypes.c_void_p, i64p, ctypes.c_void_p, i64p,
                                          ctypes.c_void_p]
    lib.poisfft_solve_strided.restype = ctypes.c_int
    lib.poisfft_plan_autotune.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    lib.poisfft_plan_autotune.restype = ctypes.c_int
    vpp = ctypes.POINTER(ctypes.c_void_p)
    lib.poisfft_batch_create.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                         i64p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int),
                                         ctypes.c_int, ctypes.c_int]
    lib.poisfft_batch_create.restype = ctypes.c_int
    lib.poisfft_batch_info.argtypes = [ctypes.c_void_p, i64p]
    lib.poisfft_batch_info.restype = ctypes.c_int
    lib.poisfft_batch_select.argtypes = [ctypes.c_void_p, ctypes.c_int]
    lib.poisfft_batch_select.restype = ctypes.c_int
    for nm in ("poisfft_batch_solve", "poisfft_batch_solve_sequential", "poisfft_batch_solve_persistent"):
        getattr(lib, nm).argtypes = [ctypes.c_void_p, vpp, vpp, ctypes.c_void_p]
        getattr(lib, nm).restype = ctypes.c_int
    lib.poisfft_solve_refined.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                          ctypes.c_void_p]
    lib.poisfft_solve_refined.restype = ctypes.c_int
    lib.poisfft_batch_autotune.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                           ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)]
    lib.poisfft_batch_autotune.restype = ctypes.c_int
    lib.poisfft_batch_check.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    lib.poisfft_batch_check.restype = ctypes.c_int
    lib.poisfft_batch_destroy.argtypes = [ctypes.c_void_p]
    lib.poisfft_batch_destroy.restype = ctypes.c_int
    lib.poisfft_pcg_create.argtypes = [ctypes.POINTER(ctypes.c_void_p), i64p, ctypes.POINTER(ctypes.c_double),
                                       ctypes.c_void_p, ctypes.c_double]
    lib.poisfft_pcg_create.restype = ctypes.c_int
    lib.poisfft_pcg_solve.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double,
                                      ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                      ctypes.POINTER(ctypes.c_double), ctypes.c_void_p]
    lib.poisfft_pcg_stats.argtypes = [ctypes.c_void_p, i64p]
    lib.poisfft_pcg_stats.restype = ctypes.c_int
    lib.poisfft_pcg_solve.restype = ctypes.c_int
    lib.poisfft_pcg_apply.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    lib.poisfft_pcg_apply.restype = ctypes.c_int
    lib.poisfft_pcg_destroy.argtypes = [ctypes.c_void_p]
    lib.poisfft_pcg_destroy.restype = ctypes.c_int
    vp, ci, cd = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    lib.poisfft_pcg_set_coefficient.argtypes = [vp, vp, cd]
    lib.poisfft_pcg_features.argtypes = [vp, vp, vp, vp, vp, vp]
    lib.poisfft_pcg_learned_guess.argtypes = [vp, vp, vp, vp, ci, vp]
    lib.poisfft_sno_num_params.argtypes = [ci, ci, ci]
    lib.poisfft_sno_num_params.restype = ctypes.c_int64
    lib.poisfft_sno_create.argtypes = [ctypes.POINTER(vp), i64p, ci, ci, ci, ci, ci]
    lib.poisfft_sno_set_params.argtypes = [vp, vp]
    lib.poisfft_sno_get_params.argtypes = [vp, vp]
    lib.poisfft_sno_forward.argtypes = [vp, vp, vp, vp]
    lib.poisfft_sno_backward.argtypes = [vp, vp, vp, vp, vp]
    lib.poisfft_sno_loss.argtypes = [vp, vp, vp, vp, ctypes.POINTER(cd), vp]
    lib.poisfft_sno_adam.argtypes = [vp, vp, cd, cd, cd, cd, ci, vp]
    lib.poisfft_sno_info.argtypes = [vp, i64p]
    lib.poisfft_sno_destroy.argtypes = [vp]
    lib.poisfft_zero_mode_mean.argtypes = [vp, vp, ctypes.POINTER(cd), vp]
    lib.poisfft_zero_mode_mean.restype = ci
    for name in ("poisfft_pcg_set_coefficient", "poisfft_pcg_features", "poisfft_pcg_learned_guess",
                 "poisfft_sno_create", "poisfft_sno_set_params", "poisfft_sno_get_params", "poisfft_sno_forward",
                 "poisfft_sno_backward", "poisfft_sno_loss", "poisfft_sno_adam", "poisfft_sno_info",
                 "poisfft_sno_destroy"):
        getattr(lib, name).restype = ci
    return lib


lib = _load()


def status_string(status: int) -> str:
    return lib.poisfft_status_string(int(status)).decode()


def plan_create(n, L, bc, approx, dtype):
    """Create a plan.  n, L: per-axis sequences (x first).  bc: per-axis codes
    (one per axis, used for both faces) or 2*dims face codes."""
    dims = len(n)
    if len(bc) == dims:
        faces = [b for b in bc for _ in (0, 1)]
    else:
        faces = list(bc)
    plan = ctypes.c_void_p()
    n_arr = (ctypes.c_int64 * max(dims, 1))(*[int(v) for v in n])
    L_arr = (ctypes.c_double * max(dims, 1))(*[float(v) for v in L])
    bc_arr = (ctypes.c_int * max(len(faces), 1))(*[int(v) for v in faces])
    rc = lib.poisfft_plan_create(ctypes.byref(plan), dims, n_arr, L_arr, bc_arr, int(approx), int(dtype))
    return rc, plan


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        return x.ctypes.data
    raise TypeError(f"cannot take the address of {type(x)}")


def _stream(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def solve(plan, phi, g, stream=None):
    return lib.poisfft_solve(plan, _ptr(phi), _ptr(g), _stream(stream))


def solve_host(plan, phi, g, stream=None):
    return lib.poisfft_solve_host(plan, _ptr(phi), _ptr(g), _stream(stream))


def solve_host_async(plan, phi, g, stream=None):
    return lib.poisfft_solve_host_async(plan, _ptr(phi), _ptr(g), _stream(stream))


def solve_noalloc(n, L, bc, approx, dtype, phi, g, stream=None):
    """poisfft_solve_noalloc: one solve with no device allocation (workspace in
    the library's fixed 32 MiB device array).  Returns the status code."""
    dims = len(n)
    faces = [b for b in bc for _ in (0, 1)] if len(bc) == dims else list(bc)
    n_arr = (ctypes.c_int64 * dims)(*[int(v) for v in n])
    L_arr = (ctypes.c_double * dims)(*[float(v) for v in L])
    bc_arr = (ctypes.c_int * len(faces))(*[int(v) for v in faces])
    return lib.poisfft_solve_noalloc(dims, n_arr, L_arr, bc_arr, int(approx), int(dtype), _ptr(phi), _ptr(g),
                                     _stream(stream))


def noalloc_check(stream=None):
    """poisfft_noalloc_check: synchronise `stream`, read and clear the error
    flag of poisfft_solve_noalloc.  Returns the status code."""
    return lib.poisfft_noalloc_check(_stream(stream))


def check(plan, stream=None):
    return lib.poisfft_check(plan, _stream(stream))


def destroy(plan):
    return lib.poisfft_destroy(plan)


def plan_info(plan):
    info = (ctypes.c_int64 * 4)()
    rc = lib.poisfft_plan_info(plan, info)
    return rc, list(info)


class Plan:
    """RAII wrapper: Plan(n, L, bc, approx, dtype); .solve(phi, g, stream)."""

    def __init__(self, n, L, bc, approx=FD2, dtype=F32):
        rc, p = plan_create(n, L, bc, approx, dtype)
        if rc != OK:
            raise PoisFFTError(rc, "poisfft_plan_create")
        self._p = p
        self.n = tuple(int(v) for v in n)
        self.dtype = dtype

    @property
    def handle(self):
        return self._p

    def solve(self, phi, g, stream=None):
        rc = solve(self._p, phi, g, stream)
        if rc != OK:
            raise PoisFFTError(rc, "poisfft_solve")

    def set_refinements(self, refinements):
        """Refinement steps of poisfft_solve on a MIXED plan."""
        rc = lib.poisfft_plan_set_refinements(self._p, int(refinements))
        if rc != OK:
            raise PoisFFTError(rc, "poisfft_plan_set_refinements")

    def solve_refined(self, phi, g, refinements=2, stream=None):
        """Mixed-precision solve of an FP32 FD2 plan: float64 g in, float64
        phi out (phi and g distinct), FP32 FFT solves refined with FP64
        residuals."""
        rc = lib.poisfft_solve_refined(self._p, _ptr(phi), _ptr(g), int(refinements), _stream(stream))
        if rc != OK:
            raise PoisFFTError(rc, "poisfft_solve_refined")

    def solve_strided(self, phi, phi_ld, g, g_ld, stream=None):
        """phi, g: addresses (or tensors) of element (0,0,0); *_ld = (row, plane)
        strides in elements of the enclosing arrays."""
        pl = (ctypes.c_int64 * 2)(*[int(v) for v in phi_ld])
        gl = (ctypes.c_int64 * 2)(*[int(v) for v in g_ld])
        rc = lib.poisfft_solve_strided(self._p, _ptr(phi), pl, _ptr(g), gl, _stream(stream))
        if rc != OK:
            raise PoisFFTError(rc, "poisfft_solve_strided")

    def solve_host(self, phi, g, stream=None):
        rc = solve_host(self._p, phi, g, stream)
        if rc != OK:
            raise PoisFFTError(rc, "poisfft_solve_host")

    def solve_host_async(self, phi, g, stream=None):
        rc = solve_host_async(self._p, phi, g, stream)
        if rc != OK:
            raise PoisFFTError(rc, "poisfft_solve_host_async")

    def check(self, stream=None):
        return check(self._p, stream)

    def info(self):
        rc, info = plan_info(self._p)
        if rc != OK:
            raise PoisFFTError(rc, "poisfft_plan_info")
        return dict(launches=info[0], workspace_bytes=info[1], dominant_bytes=info[2], dominant_index=info[3])

    def zero_mode_mean(self, g, stream=None):
        """Weighted mean of g that the solve of a singular problem removes (FP64)."""
        m = ctypes.c_double()
        rc = lib.poisfft_zero_mode_mean(self._p, _ptr(g), ctypes.byref(m), _stream(stream))
        if rc != OK:
            raise PoisFFTError(rc, "poisfft_zero_mode_mean")
        return m.value

    def launches(self):
        """Per launch position: dict(bytes, kernel, mode, axis)."""
        out = []
        for i in range(self.info()["launches"]):
            v = (ctypes.c_int64 * 4)()
            rc = lib.poisfft_launch_info(self._p, i, v)
            if rc != OK:
                raise PoisFFTError(rc, "poisfft_launch_info")
            out.append(dict(bytes=v[0], kernel=("x_sweep", "strided_sweep", "pair_divide", "tc_strided_sweep")[v[1]],
                            mode=("forward", "backward", "fused")[v[2]], axis="xyz"[v[3]]))
        return out

    def autotune(self, stream=None):
        rc = lib.poisfft_plan_autotune(self._p, _stream(stream))
        if rc != OK:
            raise PoisFFTError(rc, "poisfft_plan_autotune")

    def profile(self, enable=True):
        rc = lib.poisfft_profile_enable(self._p, 1 if enable else 0)
        if rc != OK:
            raise PoisFFTError(rc, "poisfft_profile_enable")

    def profile_read(self):
        """(summed ms per launch position, number of profiled solves)."""
        cap = 16
        ms = (ctypes.c_double * cap)()
        nl, ns = ctypes.c_int(), ctypes.c_int()
        rc = lib.poisfft_profile_read(self._p, ms, cap, ctypes.byref(nl), ctypes.byref(ns))
        if rc != OK:
            raise PoisFFTError(rc, "poisfft_profile_read")
        return [ms[i] for i in range(min(cap, nl.value))], ns.value

    def close(self):
        if self._p:
            destroy(self._p)
            self._p = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Batch:
    """Many independent problems solved through one CUDA graph.

    problems: sequence of (n, L, bc) with per-problem dims = len(n)."""

    def __init__(self, problems, approx=FD2, dtype=F32):
        cnt = len(problems)
        dims = (ctypes.c_int * cnt)()
        n = (ctypes.c_int64 * (3 * cnt))()
        L = (ctypes.c_double * (3 * cnt))()
        bc = (ctypes.c_int * (6 * cnt))()
        for i, (nn, LL, bb) in enumerate(problems):
            d = len(nn)
            dims[i] = d
            for a in range(3):
                n[3 * i + a] = int(nn[a]) if a < d else 1
                L[3 * i + a] = float(LL[a]) if a < d else 1.0
                bc[6 * i + 2 * a] = bc[6 * i + 2 * a + 1] = int(bb[a]) if a < d else 0
        h = ctypes.c_void_p()
        rc = lib.poisfft_batch_create(ctypes.byref(h), cnt, dims, n, L, bc, int(approx), int(dtype))
        if rc != OK:
            raise PoisFFTError(rc, "poisfft_batch_create")
        self._b = h
        self.count = cnt

    def _ptrs(self, xs):
        arr = (ctypes.c_void_p * self.count)(*[_ptr(x) for x in xs])
        return arr

    def solve(self, phis, gs, stream=None):
        rc = lib.poisfft_batch_solve(self._b, self._ptrs(phis), self._ptrs(gs), _stream(stream))
        if rc != OK:
            raise PoisFFTError(rc, "poisfft_batch_solve")

    def solve_sequential(self, phis, gs, stream=None):
        rc = lib.poisfft_batch_solve_sequential(self._b, self._ptrs(phis), self._ptrs(gs), _stream(stream))
        if rc != OK:
            raise PoisFFTError(rc, "poisfft_batch_solve_sequential")

    TUNE_CANDIDATES = ("as created", "tiles halved", "each plan tuned alone", "sweep order tuned per problem",
                       "persistent phase launches")

    def solve_persistent(self, phis, gs, stream=None):
        """One persistent launch per sweep phase over all problems."""
        rc = lib.poisfft_batch_solve_persistent(self._b, self._ptrs(phis), self._ptrs(gs), _stream(stream))
        if rc != OK:
            raise PoisFFTError(rc, "poisfft_batch_solve_persistent")

    def autotune(self, phis, gs, stream=None):
        """Times the batch graph under each tile configuration and keeps the
        fastest (phis are overwritten).  Returns (chosen index, ms per replay
        of every candidate)."""
        ms = (ctypes.c_double * len(self.TUNE_CANDIDATES))()
        chosen = ctypes.c_int()
        rc = lib.poisfft_batch_autotune(self._b, self._ptrs(phis), self._ptrs(gs), _stream(stream), ms,
                                        ctypes.byref(chosen))
        if rc != OK:
            raise PoisFFTError(rc, "poisfft_batch_autotune")
        return chosen.value, list(ms)

    def select(self, candidate):
        """Apply one of the last autotune's candidate configurations."""
        rc = lib.poisfft_batch_select(self._b, int(candidate))
        if rc != OK:
            raise PoisFFTError(rc, "poisfft_batch_select")

    def info(self):
        """dict(bytes, launches, points) of one batch solve."""
        out = (ctypes.c_int64 * 3)()
        rc = lib.poisfft_batch_info(self._b, out)
        if rc != OK:
            raise PoisFFTError(rc, "poisfft_batch_info")
        return dict(bytes=out[0], launches=out[1], points=out[2])

    def check(self, stream=None):
        return lib.poisfft_batch_check(self._b, _stream(stream))

    def close(self):
        if self._b:
            lib.poisfft_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class PCG:
    """FFT-preconditioned CG for div(a grad phi) = g (staggered Dirichlet walls).

    n, L: cells and lengths (x first); a: float32 cell coefficients (tensor or
    address, n[2] x n[1] x n[0] x-fastest); a_ref <= 0 uses the mean of a."""

    def __init__(self, n, L, a, a_ref=0.0):
        h = ctypes.c_void_p()
        n_arr = (ctypes.c_int64 * 3)(*[int(v) for v in n])
        L_arr = (ctypes.c_double * 3)(*[float(v) for v in L])
        rc = lib.poisfft_pcg_create(ctypes.byref(h), n_arr, L_arr, _ptr(a), float(a_ref))
        if rc != OK:
            raise PoisFFTError(rc, "poisfft_pcg_create")
        self._h = h

    def solve(self, phi, g, tol=1e-8, maxit=500, stream=None, precision=None):
        """phi: initial guess in, solution out (float64 device).  precision:
        PCG_MIXED (default) or PCG_F64.  Returns (iterations, relres)."""
        it = ctypes.c_int()
        rel = ctypes.c_double()
        prec = PCG_MIXED if precision is None else int(precision)
        rc = lib.poisfft_pcg_solve(self._h, _ptr(phi), _ptr(g), float(tol), int(maxit), prec, ctypes.byref(it),
                                   ctypes.byref(rel), _stream(stream))
        if rc != OK:
            raise PoisFFTError(rc, "poisfft_pcg_solve")
        return it.value, rel.value

    def set_coefficient(self, a, a_ref=0.0):
        """Replace the cell coefficients (same grid); a_ref <= 0: mean of a."""
        rc = lib.poisfft_pcg_set_coefficient(self._h, _ptr(a), float(a_ref))
        if rc != OK:
            raise PoisFFTError(rc, "poisfft_pcg_set_coefficient")

    def features(self, g, feats, phi=None, target=None, stream=None):
        """Network features of right-hand side g into feats (3 N float32);
        with phi and target also the training target (N float32)."""
        rc = lib.poisfft_pcg_features(self._h, _ptr(g), _ptr(phi), _ptr(feats), _ptr(target), _stream(stream))
        if rc != OK:
            raise PoisFFTError(rc, "poisfft_pcg_features")

    def learned_guess(self, sno, phi, g, corrections=1, stream=None):
        """phi = the network's initial guess for g (plus `corrections` residual corrections)."""
        rc = lib.poisfft_pcg_learned_guess(self._h, sno._h, _ptr(phi), _ptr(g), int(corrections), _stream(stream))
        if rc != OK:
            raise PoisFFTError(rc, "poisfft_pcg_learned_guess")

    def stats(self):
        """Last solve: dict(iterations, true_residuals, preconditioner_solves, precision)."""
        v = (ctypes.c_int64 * 4)()
        rc = lib.poisfft_pcg_stats(self._h, v)
        if rc != OK:
            raise PoisFFTError(rc, "poisfft_pcg_stats")
        return dict(iterations=v[0], true_residuals=v[1], preconditioner_solves=v[2], precision=v[3])

    def apply(self, out, x, stream=None):
        """out = -(A x)."""
        rc = lib.poisfft_pcg_apply(self._h, _ptr(out), _ptr(x), _stream(stream))
        if rc != OK:
            raise PoisFFTError(rc, "poisfft_pcg_apply")

    def close(self):
        if self._h:
            lib.poisfft_pcg_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def sno_num_params(channels, modes, layers):
    return int(lib.poisfft_sno_num_params(int(channels), int(modes), int(layers)))


class SNO:
    """Spectral neural operator (truncated sine basis) for the learned PCG guess.

    n: grid (x first); batch; channels C; modes K per axis; layers L; train:
    keep activations for backward and the Adam state."""

    def __init__(self, n, batch=1, channels=16, modes=12, layers=4, train=False):
        h = ctypes.c_void_p()
        n_arr = (ctypes.c_int64 * 3)(*[int(v) for v in n])
        rc = lib.poisfft_sno_create(ctypes.byref(h), n_arr, int(batch), int(channels), int(modes), int(layers),
                                    1 if train else 0)
        if rc != OK:
            raise PoisFFTError(rc, "poisfft_sno_create")
        self._h = h
        self.n, self.batch, self.channels, self.modes, self.layers = tuple(n), batch, channels, modes, layers
        self.num_params = sno_num_params(channels, modes, layers)

    def _check(self, rc, what):
        if rc != OK:
            raise PoisFFTError(rc, what)

    def set_params(self, theta):
        self._check(lib.poisfft_sno_set_params(self._h, _ptr(theta)), "poisfft_sno_set_params")

    def get_params(self, theta):
        self._check(lib.poisfft_sno_get_params(self._h, _ptr(theta)), "poisfft_sno_get_params")

    def forward(self, y, feats, stream=None):
        self._check(lib.poisfft_sno_forward(self._h, _ptr(y), _ptr(feats), _stream(stream)), "poisfft_sno_forward")

    def backward(self, grad, dy, feats, stream=None):
        self._check(lib.poisfft_sno_backward(self._h, _ptr(grad), _ptr(dy), _ptr(feats), _stream(stream)),
                    "poisfft_sno_backward")

    def loss(self, y, t, dy=None, stream=None, read=True):
        """Relative squared error (returned when read) and its gradient into dy."""
        val = ctypes.c_double()
        self._check(lib.poisfft_sno_loss(self._h, _ptr(y), _ptr(t), _ptr(dy), ctypes.byref(val) if read else None,
                                         _stream(stream)), "poisfft_sno_loss")
        return val.value if read else None

    def adam(self, grad, lr, step, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
        self._check(lib.poisfft_sno_adam(self._h, _ptr(grad), float(lr), float(beta1), float(beta2), float(eps),
                                         int(step), _stream(stream)), "poisfft_sno_adam")

    def close(self):
        if self._h:
            lib.poisfft_sno_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
