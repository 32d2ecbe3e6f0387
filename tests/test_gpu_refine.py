"""Mixed-precision solve by iterative refinement (poisfft_solve_refined):
FP64 data, FP32 FFT solves corrected with FP64 residuals of the FD2
operator, compared with the FP64 oracle.

Bound: each step multiplies the error by about the FP32 solve's relative
accuracy (~1e-6), down to the floor of the FP64 residual, about
cond(L) x 1.1e-16 with cond(L) ~ (2 n_max / pi)^2 (times the ratio of the
largest to smallest 1/dx^2); for n_max <= 128 that is ~1e-12, and the
tests allow 1e-10 after two refinements.  The FP32 solve alone (0 steps)
stays within the FP32 path's 1e-5."""

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


CASES = [
    ((24, 20, 18), (W.P, W.DS, W.NS)),       # general kernels, nonsingular
    ((11, 13, 17), (W.DR, W.NR, W.DS)),      # direct-DFT primes, DST-I / DCT-I axes
    ((21, 27, 45), (W.P, W.P, W.NS)),        # singular (zero mode removed)
    ((16, 12, 10), (W.NR, W.NR, W.NR)),      # singular with trapezoid-weighted mean
    ((64, 64, 128), (W.P, W.DS, W.NS)),      # specialised kernels
    ((64, 128, 64), (W.NS, W.DS, W.NS)),     # specialised kernels, x DCT
    ((40, 300), (W.DR, W.P)),                # 2D
    ((97,), (W.NS,)),                        # 1D singular
    ((16, 12, 1), (W.P, W.DS, W.NS)),        # z of one point (residual takes both neighbours from the BC)
]


@pytest.mark.parametrize("n,bcs", CASES, ids=lambda v: str(v))
def test_refinement_reaches_fp64_accuracy(pb, n, bcs):
    shape = tuple(reversed(n))
    Ls = tuple(1.0 + 0.25 * a for a in range(len(n)))
    g = W.normal(shape, 21, dtype=np.float64)
    ref = O.solve(g, bcs, Ls, O.FD2, method="fft")
    gd = torch.from_numpy(g).cuda()
    errs = []
    with pb.Plan(n, Ls, bcs, pb.FD2, pb.F32) as plan:
        for k in (0, 1, 2):
            phi = torch.full_like(gd, float("nan"))
            plan.solve_refined(phi, gd, refinements=k)
            torch.cuda.synchronize()
            assert plan.check() == pb.OK
            errs.append(O.rel_max_error(phi.cpu().numpy(), ref))
    assert errs[0] < 1e-5, errs
    assert errs[1] < 1e-3 * errs[0] or errs[1] < 1e-10, errs
    assert errs[2] < 1e-10, errs


def test_refinement_argument_checks(pb):
    n, bcs, Ls = (8, 8, 8), (W.P, W.P, W.P), (1.0, 1.0, 1.0)
    g = torch.zeros((8, 8, 8), dtype=torch.float64, device="cuda")
    phi = torch.zeros_like(g)
    with pb.Plan(n, Ls, bcs, pb.FD2, pb.F64) as plan:      # FP64 plan: refuse
        with pytest.raises(pb.PoisFFTError):
            plan.solve_refined(phi, g)
    with pb.Plan(n, Ls, bcs, pb.SPECTRAL, pb.F32) as plan:  # no local operator: refuse
        with pytest.raises(pb.PoisFFTError):
            plan.solve_refined(phi, g)
    with pb.Plan(n, Ls, bcs, pb.FD2, pb.F32) as plan:
        with pytest.raises(pb.PoisFFTError):
            plan.solve_refined(g, g)                         # phi == g
        with pytest.raises(pb.PoisFFTError):
            plan.solve_refined(phi, g, refinements=9)
        plan.solve_refined(phi, g, refinements=1)            # zero source: zero solution
        torch.cuda.synchronize()
        assert float(phi.abs().max()) == 0.0


@pytest.mark.parametrize("n,bcs", [((24, 20, 18), (W.P, W.DS, W.NS)), ((64, 64, 128), (W.P, W.P, W.NS)),
                                   ((16, 12, 10), (W.NR, W.NR, W.NR))], ids=lambda v: str(v))
def test_mixed_dtype_plan_through_poisfft_solve(pb, n, bcs):
    """A POISFFT_MIXED plan (Sec. 3: one solver object per precision) takes
    float64 arrays through the plain poisfft_solve: FP32 transforms refined
    with FP64 FD2 residuals, two steps by default, one after
    poisfft_plan_set_refinements(1)."""
    shape = tuple(reversed(n))
    Ls = (1.0, 1.5, 2.0)
    g = W.normal(shape, 23, dtype=np.float64)
    ref = O.solve(g, bcs, Ls, O.FD2, method="fft")
    gd = torch.from_numpy(g).cuda()
    with pb.Plan(n, Ls, bcs, pb.FD2, pb.MIXED) as plan:
        phi = torch.full_like(gd, float("nan"))
        plan.solve(phi, gd, torch.cuda.current_stream())
        torch.cuda.synchronize()
        assert plan.check() == pb.OK
        err2 = O.rel_max_error(phi.cpu().numpy(), ref)
        plan.set_refinements(0)
        phi0 = torch.full_like(gd, float("nan"))
        plan.solve(phi0, gd, torch.cuda.current_stream())
        torch.cuda.synchronize()
        err0 = O.rel_max_error(phi0.cpu().numpy(), ref)
        # host buffers of doubles through the same plan
        ph = np.full(shape, np.nan)
        plan.set_refinements(2)
        plan.solve_host(ph, g)
        errh = O.rel_max_error(ph, ref)
        with pytest.raises(pb.PoisFFTError):
            plan.solve(gd, gd)                                # in place is refused
        with pytest.raises(pb.PoisFFTError):
            plan.set_refinements(9)
    assert err0 < 1e-5 and err2 < 1e-10 and errh < 1e-10, (err0, err2, errh)
