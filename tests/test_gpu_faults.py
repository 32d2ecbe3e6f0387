"""Failure detection without a GPU fault: host-side injection
(POISFFT_FAULT) makes each device allocation of a plan creation fail in
turn, or the tensor-map encoding, or the size check.  Every call must
return its status code, leak no device memory, and leave the library able
to create and run the same plan afterwards.  Also the bounded device
waits: a plan whose error flag was never set reports OK."""

import os

import numpy as np
import pytest

import workloads as W
from oracle import poisson as O
from tests._lib import ensure_built

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ensure_built()
    from paper_1409_8116_gb300 import binding
    return binding


def _free():
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


PLANS = [
    ((64, 64, 128), (W.P, W.DS, W.NS), "F32"),      # specialised kernels
    ((30, 28, 45), (W.DR, W.NR, W.P), "F32"),       # general kernels, pair divide
    ((64, 64, 1024), (W.P, W.P, W.NS), "BF16X3"),   # tensor-core sweep
    ((24, 20), (W.NS, W.P), "MIXED"),
]


@pytest.mark.parametrize("n,bcs,dt", PLANS, ids=lambda v: str(v))
def test_every_allocation_failure_is_reported_and_leaks_nothing(pb, n, bcs, dt, monkeypatch):
    dtype = getattr(pb, dt)
    Ls = (1.0,) * len(n)
    with pb.Plan(n, Ls, bcs, pb.FD2, dtype):  # warm the context and the kernels' attributes
        pass
    base = _free()
    seen_ok = False
    for k in range(1, 64):
        monkeypatch.setenv("POISFFT_FAULT", f"alloc:{k}")
        rc, plan = pb.plan_create(n, Ls, bcs, pb.FD2, dtype)
        monkeypatch.delenv("POISFFT_FAULT")
        if rc == pb.OK:  # fewer than k allocations: the plan was made
            pb.destroy(plan)
            seen_ok = True
            break
        assert rc in (pb.ERR_ALLOC, pb.ERR_CUDA), (k, rc)
        assert not plan.value
        assert _free() == base, f"allocation failure {k} leaked device memory"
    assert seen_ok
    for fault, want in (("encode", pb.ERR_CUDA), ("size", pb.ERR_UNSUPPORTED_SIZE)):
        monkeypatch.setenv("POISFFT_FAULT", fault)
        rc, plan = pb.plan_create(n, Ls, bcs, pb.FD2, dtype)
        monkeypatch.delenv("POISFFT_FAULT")
        assert rc == want and not plan.value
        assert _free() == base
    # the library still works: the same plan solves correctly
    shape = tuple(reversed(n))
    npdt = np.float64 if dt == "MIXED" else np.float32
    g = W.normal(shape, 3, dtype=npdt)
    ref = O.solve(g.astype(np.float64), bcs, Ls, O.FD2, method="fft")
    gd = torch.from_numpy(g).cuda()
    phi = torch.empty_like(gd)
    with pb.Plan(n, Ls, bcs, pb.FD2, dtype) as plan:
        plan.solve(phi, gd, torch.cuda.current_stream())
        assert plan.check() == pb.OK
    tol = {"F32": 1e-5, "BF16X3": 1e-4, "MIXED": 1e-10}[dt]
    assert O.rel_max_error(phi.cpu().numpy(), ref) < tol


def test_lazy_allocations_fail_cleanly(pb, monkeypatch):
    """The host-buffer solve's staging buffers and the refined solve's
    FP32 field are allocated on first use: a failure there is reported and
    the next call succeeds."""
    n, bcs, Ls = (32, 24, 16), (W.P, W.DS, W.NS), (1.0, 1.0, 1.0)
    g = W.normal((16, 24, 32), 5, dtype=np.float32)
    ref = O.solve(g.astype(np.float64), bcs, Ls, O.FD2, method="fft")
    with pb.Plan(n, Ls, bcs, pb.FD2, pb.F32) as plan:
        ph = np.zeros_like(g)
        monkeypatch.setenv("POISFFT_FAULT", "alloc:2")
        assert pb.solve_host(plan.handle, ph, g) == pb.ERR_ALLOC
        monkeypatch.delenv("POISFFT_FAULT")
        plan.solve_host(ph, g)
        assert O.rel_max_error(ph, ref) < 1e-5
        g64 = torch.from_numpy(g.astype(np.float64)).cuda()
        p64 = torch.empty_like(g64)
        monkeypatch.setenv("POISFFT_FAULT", "alloc:1")
        with pytest.raises(pb.PoisFFTError) as e:
            plan.solve_refined(p64, g64, 1)
        assert e.value.status == pb.ERR_ALLOC
        monkeypatch.delenv("POISFFT_FAULT")
        plan.solve_refined(p64, g64, 1)
        torch.cuda.synchronize()
        assert O.rel_max_error(p64.cpu().numpy(), ref) < 1e-9
        assert plan.check() == pb.OK
