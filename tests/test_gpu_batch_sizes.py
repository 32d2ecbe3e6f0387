"""Parity at the batched workload's own sizes (Sec. 3: problems of any size
in 1-3 dimensions; Table 2: every BC row): 2D lines up to 2048 points and 3D
axes up to 256 points, every BC on the contiguous (x) and the strided axes,
including DST-I / DCT-I axes whose 2(n +- 1)-point extension needs
Bluestein's method or a direct-DFT prime pass.  Each solve is compared
element by element with the FP64 oracle (its scipy.fft realisation, pinned
to the dense definition by the CPU tests); tolerances 1e-5 (FP32) and 1e-12
(FP64) normwise, as for every other parity test."""

import numpy as np
import pytest

import workloads as W
from oracle import poisson as O
from tests._lib import ensure_built

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

BCS = (W.P, W.DR, W.DS, W.NR, W.NS)
TOL = {"f32": 1e-5, "f64": 1e-12}


@pytest.fixture(scope="module")
def pb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ensure_built()
    from paper_1409_8116_gb300 import binding
    return binding


def _solve_and_compare(pb, n, bcs, dtype, seed):
    shape = tuple(reversed(n))
    npdt = np.float32 if dtype == "f32" else np.float64
    g = W.normal(shape, seed, dtype=npdt)
    Ls = tuple(1.0 for _ in n)
    ref = O.solve(g.astype(np.float64), bcs, Ls, O.FD2, method="fft")
    with pb.Plan(n, Ls, bcs, pb.FD2, pb.F32 if dtype == "f32" else pb.F64) as plan:
        gd = torch.from_numpy(g).cuda()
        phi = torch.full_like(gd, float("nan"))
        plan.solve(phi, gd, torch.cuda.current_stream())
        torch.cuda.synchronize()
        assert plan.check() == pb.OK
        return O.rel_max_error(phi.cpu().numpy(), ref)


# the largest 2D lengths of the workload: 2048 and the 7-smooth 2016, 2000
@pytest.mark.parametrize("bc", BCS, ids=["P", "DR", "DS", "NR", "NS"])
@pytest.mark.parametrize("axis", [0, 1], ids=["x", "y"])
@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_2048_point_lines_every_bc(pb, bc, axis, dtype):
    other = BCS[(bc + 2) % 5]
    n = [72, 72]
    n[axis] = 2048
    bcs = [other, other]
    bcs[axis] = bc
    err = _solve_and_compare(pb, tuple(n), tuple(bcs), dtype, 100 + 10 * bc + axis)
    assert err < TOL[dtype], (n, bcs, err)


@pytest.mark.parametrize("n", [(2016, 2000), (2000, 2048), (2048, 2048)])
@pytest.mark.parametrize("bcs", [(W.DR, W.NR), (W.NR, W.DS), (W.NS, W.DR), (W.P, W.P)])
def test_largest_2d_problems(pb, n, bcs):
    err = _solve_and_compare(pb, n, bcs, "f32", 7)
    assert err < TOL["f32"], (n, bcs, err)


# 3D: 256 points per axis with the same BC on every axis, and mixtures that
# put each BC on each axis once
@pytest.mark.parametrize("bcs", [(b, b, b) for b in BCS] + [(W.DR, W.NR, W.NS), (W.NS, W.DR, W.NR),
                                                             (W.NR, W.NS, W.DR), (W.P, W.DR, W.NR)])
def test_256_cubed_every_bc(pb, bcs):
    err = _solve_and_compare(pb, (256, 256, 256), bcs, "f32", 11)
    assert err < TOL["f32"], (bcs, err)


@pytest.mark.parametrize("bcs", [(W.DR, W.NR, W.DS), (W.NR, W.DR, W.P)])
def test_256_cubed_fp64(pb, bcs):
    err = _solve_and_compare(pb, (256, 240, 250), bcs, "f64", 12)
    assert err < TOL["f64"], (bcs, err)


def test_batch_drawn_from_the_workload_ranges(pb):
    """48 problems drawn from the workload's own ranges (2D n in [64, 2048],
    3D n in [32, 256], 7-smooth, all five BCs), solved through one CUDA
    graph; every problem against the oracle."""
    probs = W.batch_problems(48, 2024)
    assert {b for p in probs for b in p["bcs"]} == set(BCS)
    assert max(max(p["n"]) for p in probs if p["dims"] == 2) > 1000
    gs = [W.normal(tuple(reversed(p["n"])), p["gseed"], dtype=np.float32) for p in probs]
    stream = torch.cuda.Stream()
    with pb.Batch([(p["n"], p["Ls"], p["bcs"]) for p in probs], pb.FD2, pb.F32) as batch:
        gd = [torch.from_numpy(g).cuda() for g in gs]
        phis = [torch.full_like(x, float("nan")) for x in gd]
        torch.cuda.synchronize()
        batch.solve(phis, gd, stream)
        stream.synchronize()
        assert batch.check(stream) == pb.OK
        worst = 0.0
        for p, g, phi in zip(probs, gs, phis):
            ref = O.solve(g.astype(np.float64), p["bcs"], p["Ls"], O.FD2, method="fft")
            err = O.rel_max_error(phi.cpu().numpy(), ref)
            assert err < TOL["f32"], (p, err)
            worst = max(worst, err)
