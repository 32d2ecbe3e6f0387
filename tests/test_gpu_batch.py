"""Batched solves: independent 2D/3D problems of uneven sizes with per-axis
BCs drawn from all five kinds, solved through one CUDA graph; every problem
is compared with the FP64 oracle.  Also the per-plan and the batch tile
autotuners."""

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


def _batch(count, seed):
    return W.batch_problems(count, seed, n2d=(8, 300), n3d=(4, 48))


def _inputs(probs, dtype):
    gs, refs = [], []
    for p in probs:
        g = W.normal(tuple(reversed(p["n"])), p["gseed"], dtype=dtype)
        gs.append(g)
        refs.append(O.solve(g.astype(np.float64), p["bcs"], p["Ls"], O.FD2))
    return gs, refs


@pytest.mark.parametrize("dtype,tol", [("f32", 1e-5), ("f64", 1e-12)])
def test_batch_graph_matches_oracle_per_problem(pb, dtype, tol):
    probs = _batch(48, 7)
    kinds = {b for p in probs for b in p["bcs"]}
    assert kinds == {0, 1, 2, 3, 4} and {p["dims"] for p in probs} == {2, 3}
    npdt = np.float32 if dtype == "f32" else np.float64
    gs, refs = _inputs(probs, npdt)
    stream = torch.cuda.Stream()
    with pb.Batch([(p["n"], p["Ls"], p["bcs"]) for p in probs], pb.FD2,
                  pb.F32 if dtype == "f32" else pb.F64) as batch:
        gd = [torch.from_numpy(g).cuda() for g in gs]
        phis = [torch.full_like(x, float("nan")) for x in gd]
        torch.cuda.synchronize()
        batch.solve(phis, gd, stream)
        stream.synchronize()
        assert batch.check(stream) == pb.OK
        for phi, ref, p in zip(phis, refs, probs):
            assert O.rel_max_error(phi.cpu().numpy(), ref) < tol, p
        # replay with new contents behind the same pointers
        for x in gd:
            x.mul_(-2.0)
        batch.solve(phis, gd, stream)
        stream.synchronize()
        for phi, ref in zip(phis, refs):
            assert O.rel_max_error(phi.cpu().numpy(), -2.0 * ref) < tol
        # new output pointers: the graph is re-captured
        phis2 = [torch.zeros_like(x) for x in gd]
        batch.solve(phis2, gd, stream)
        stream.synchronize()
        for phi, ref in zip(phis2, refs):
            assert O.rel_max_error(phi.cpu().numpy(), -2.0 * ref) < tol
        # the plain form (one problem after another, no graph) agrees
        phis3 = [torch.zeros_like(x) for x in gd]
        batch.solve_sequential(phis3, gd, stream)
        stream.synchronize()
        for a, b in zip(phis2, phis3):
            assert torch.equal(a, b)


def test_autotuned_plan_matches_oracle(pb):
    for n, bcs in [((45, 300, 27), (W.DR, W.P, W.NS)), ((300, 40, 30), (W.P, W.DS, W.NR)), ((77, 91), (W.NR, W.P))]:
        shape = tuple(reversed(n))
        g = W.normal(shape, 3, dtype=np.float32)
        Ls = tuple(1.0 for _ in n)
        ref = O.solve(g.astype(np.float64), bcs, Ls, O.FD2)
        with pb.Plan(n, Ls, bcs, pb.FD2, pb.F32) as plan:
            plan.autotune()
            gd = torch.from_numpy(g).cuda()
            phi = torch.empty_like(gd)
            plan.solve(phi, gd, torch.cuda.current_stream())
            assert plan.check() == pb.OK
            assert O.rel_max_error(phi.cpu().numpy(), ref) < 1e-5


def test_batch_autotune_keeps_results(pb):
    """Each tile configuration the batch tuner tries gives the oracle's
    answer, and the kept one still does after the graph is re-captured."""
    probs = _batch(24, 11)
    gs, refs = _inputs(probs, np.float32)
    stream = torch.cuda.Stream()
    with pb.Batch([(p["n"], p["Ls"], p["bcs"]) for p in probs], pb.FD2, pb.F32) as batch:
        gd = [torch.from_numpy(g).cuda() for g in gs]
        phis = [torch.full_like(x, float("nan")) for x in gd]
        torch.cuda.synchronize()
        chosen, ms = batch.autotune(phis, gd, stream)
        assert chosen in range(len(pb.Batch.TUNE_CANDIDATES)) and len(ms) == len(pb.Batch.TUNE_CANDIDATES)
        assert all(t > 0 for t in ms) and ms[chosen] == min(ms)
        # the tuner's last replays leave the last candidate's solutions in phis
        for phi, ref in zip(phis, refs):
            assert O.rel_max_error(phi.cpu().numpy(), ref) < 1e-5
        for x in phis:
            x.fill_(float("nan"))
        batch.solve(phis, gd, stream)
        stream.synchronize()
        assert batch.check(stream) == pb.OK
        for phi, ref, p in zip(phis, refs, probs):
            assert O.rel_max_error(phi.cpu().numpy(), ref) < 1e-5, p
        # every candidate (tile shapes, per-problem sweep order, persistent
        # phase launches) solves every problem
        for cand in range(len(pb.Batch.TUNE_CANDIDATES)):
            batch.select(cand)
            for x in phis:
                x.fill_(float("nan"))
            batch.solve(phis, gd, stream)
            stream.synchronize()
            assert batch.check(stream) == pb.OK
            for phi, ref, p in zip(phis, refs, probs):
                assert O.rel_max_error(phi.cpu().numpy(), ref) < 1e-5, (cand, p)


@pytest.mark.parametrize("dtype,tol", [("f32", 1e-5), ("f64", 1e-12)])
def test_persistent_phase_launches_match_oracle(pb, dtype, tol):
    """One persistent launch per sweep phase over a (problem, tile) work
    list gives every problem the oracle's solution; new contents behind the
    same pointers reuse the lists, new pointers rebuild them."""
    probs = _batch(40, 13)
    npdt = np.float32 if dtype == "f32" else np.float64
    gs, refs = _inputs(probs, npdt)
    stream = torch.cuda.Stream()
    with pb.Batch([(p["n"], p["Ls"], p["bcs"]) for p in probs], pb.FD2,
                  pb.F32 if dtype == "f32" else pb.F64) as batch:
        gd = [torch.from_numpy(g).cuda() for g in gs]
        phis = [torch.full_like(x, float("nan")) for x in gd]
        torch.cuda.synchronize()
        batch.solve_persistent(phis, gd, stream)
        stream.synchronize()
        assert batch.check(stream) == pb.OK
        for phi, ref, p in zip(phis, refs, probs):
            assert O.rel_max_error(phi.cpu().numpy(), ref) < tol, p
        for x in gd:
            x.mul_(3.0)
        batch.solve_persistent(phis, gd, stream)
        stream.synchronize()
        for phi, ref in zip(phis, refs):
            assert O.rel_max_error(phi.cpu().numpy(), 3.0 * ref) < tol
        phis2 = [torch.zeros_like(x) for x in gd]
        batch.solve_persistent(phis2, gd, stream)
        stream.synchronize()
        phis3 = [torch.zeros_like(x) for x in gd]
        batch.solve(phis3, gd, stream)  # the graph form: identical kernels per tile
        stream.synchronize()
        for a, b in zip(phis2, phis3):
            assert torch.equal(a, b)


def test_persistent_refuses_specialised_plans(pb):
    with pb.Batch([((64, 64, 64), (1.0, 1.0, 1.0), (W.P, W.P, W.NS))], pb.FD2, pb.F32) as batch:
        g = torch.zeros((64, 64, 64), device="cuda")
        with pytest.raises(pb.PoisFFTError) as e:
            batch.solve_persistent([torch.empty_like(g)], [g], torch.cuda.Stream())
        assert e.value.status == pb.ERR_NOT_IMPLEMENTED
