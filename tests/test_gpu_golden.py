"""The CUDA solve through the C interface against the hand-derived exact
solutions of tests/golden/ (FD2 and pseudo-spectral, every BC, 1-3D):
normwise max relative error below 1e-12 in FP64 and 1e-5 in FP32."""

import numpy as np
import pytest

from oracle import poisson as O
from tests._golden import load_cases
from tests._lib import ensure_built

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

CASES = load_cases()
TOL = {"f64": 1e-12, "f32": 1e-5}


@pytest.fixture(scope="module")
def pb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ensure_built()
    from paper_1409_8116_gb300 import binding
    return binding


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("case", CASES, ids=[c["name"] for c in CASES])
def test_cuda_solve_matches_exact_solution(pb, case, dtype):
    tdt = torch.float64 if dtype == "f64" else torch.float32
    with pb.Plan(case["n"], case["Ls"], case["bcs"], case["approx"], pb.F64 if dtype == "f64" else pb.F32) as plan:
        gd = torch.from_numpy(np.ascontiguousarray(case["g"])).to(device="cuda", dtype=tdt)
        phi = torch.empty_like(gd)
        stream = torch.cuda.current_stream()
        plan.solve(phi, gd, stream)
        assert plan.check(stream) == pb.OK
        out = phi.cpu().numpy().astype(np.float64)
    err = O.rel_max_error(out, case["phi"])
    assert err < TOL[dtype], f"{case['name']} {dtype}: rel err {err:.3e}"
