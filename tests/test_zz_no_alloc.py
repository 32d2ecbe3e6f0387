"""poisfft_solve_noalloc: the solve for callers that cannot allocate device
memory (frameworks that own the device memory through their own pool,
plug-ins with a fixed footprint).  Every call reuses the same fixed device
array, so each result is checked, call after call, against the FP64 CPU
oracle on the same input, and against the plan-based poisfft_solve; the
error flag that poisfft_noalloc_check reads must be clear after each call.
This file is collected last on purpose."""

import numpy as np
import pytest

import workloads as W
from oracle import poisson as O
from tests._lib import ensure_built

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

CASES = [
    # (n physical, bcs, approx, dtype, tol)
    ((40, 36, 30), (W.P, W.DS, W.NS), W.FD2, "f32", 1e-5),
    ((33, 17, 12), (W.DR, W.NR, W.DS), W.SPECTRAL, "f64", 1e-12),
    ((96, 70), (W.P, W.NR), W.FD2, "f32", 1e-5),
    ((50,), (W.NS,), W.FD2, "f64", 1e-12),
]


@pytest.fixture(scope="module")
def pb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ensure_built()
    from paper_1409_8116_gb300 import binding
    return binding


@pytest.mark.parametrize("n,bcs,approx,dtype,tol", CASES)
def test_noalloc_matches_oracle_twice(pb, n, bcs, approx, dtype, tol):
    Ls = tuple(1.0 + 0.1 * a for a in range(len(n)))
    pdt = pb.F32 if dtype == "f32" else pb.F64
    tdt = torch.float32 if dtype == "f32" else torch.float64
    stream = torch.cuda.current_stream()
    with pb.Plan(n, Ls, bcs, approx, pdt) as plan:
        for call in range(2):
            g64 = W.normal(tuple(reversed(n)), 40 + call, dtype=np.float64)
            g = torch.from_numpy(g64).to("cuda", tdt)
            # the oracle sees exactly the values the GPU reads
            oracle = O.solve(g.cpu().numpy().astype(np.float64), bcs, Ls, approx)
            out = torch.full_like(g, float("nan"))
            rc = pb.solve_noalloc(n, Ls, bcs, approx, pdt, out, g, stream)
            assert rc == pb.OK, pb.status_string(rc)
            assert pb.noalloc_check(stream) == pb.OK
            err = O.rel_max_error(out.cpu().numpy(), oracle)
            assert err < tol, f"call {call}: rel err {err:.3e} vs the FP64 oracle"
            ref = torch.empty_like(g)
            plan.solve(ref, g, stream)
            torch.cuda.synchronize()
            err2 = O.rel_max_error(out.cpu().numpy(), ref.cpu().numpy())
            assert err2 < tol, f"call {call}: rel err {err2:.3e} vs poisfft_solve"


def test_noalloc_rejects_oversized_grid(pb):
    g = torch.zeros(1, device="cuda")
    rc = pb.solve_noalloc((512, 512, 512), (1, 1, 1), (W.P, W.P, W.NS), W.FD2, pb.F32, g, g, None)
    assert rc == pb.ERR_UNSUPPORTED_SIZE


def test_noalloc_refuses_stream_capture(pb):
    """Its table copies read host memory that does not outlive the call, so
    a capturing stream gets NOT_IMPLEMENTED and nothing is recorded."""
    n = (16, 12)
    g = torch.zeros(n[1], n[0], device="cuda")
    phi = torch.zeros_like(g)
    s = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    torch.cuda.synchronize()
    with torch.cuda.graph(graph, stream=s):
        phi.mul_(1.0)  # keeps the captured graph non-empty
        rc = pb.solve_noalloc(n, (1, 1), (W.P, W.NS), W.FD2, pb.F32, phi, g, s)
    assert rc == pb.ERR_NOT_IMPLEMENTED
    assert pb.noalloc_check(None) == pb.OK
