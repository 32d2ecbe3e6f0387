"""GPU parity: the CUDA solve through the C interface against the FP64 oracle.

Same seeded inputs on both sides; normwise max relative error
||phi_gpu - phi_oracle||_inf / ||phi_oracle||_inf below 1e-12 for FP64 and
1e-5 for FP32 (the tolerances stated for the solve).  Shapes span several
tiles of every sweep kernel with ragged tails, odd and prime lengths, axes
longer than one TMA box (256 rows), length-1 and length-2 axes, and every
boundary-condition combination the library implements.
"""

import itertools

import numpy as np
import pytest

import workloads as W
from oracle import poisson as O
from tests._lib import ensure_built

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-5}
BCS = [W.P, W.DR, W.DS, W.NR, W.NS]


@pytest.fixture(scope="module")
def pb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ensure_built()
    from paper_1409_8116_gb300 import binding
    return binding


def gpu_solve(pb, g, bcs, Ls, approx, dtype, inplace=False):
    """Solve through poisfft_solve on device buffers; returns numpy phi."""
    nphys = tuple(reversed(g.shape))
    tdt = torch.float64 if dtype == "f64" else torch.float32
    with pb.Plan(nphys, Ls, bcs, approx, pb.F64 if dtype == "f64" else pb.F32) as plan:
        gd = torch.from_numpy(np.ascontiguousarray(g)).to(device="cuda", dtype=tdt)
        phi = gd if inplace else torch.empty_like(gd)
        stream = torch.cuda.current_stream()
        plan.solve(phi, gd, stream)
        assert plan.check(stream) == pb.OK
        return phi.cpu().numpy().astype(np.float64)


def supported(bcs):
    return True


def check(pb, shape, bcs, approx, dtype, seed=0, Ls=None, method="dense", inplace=False):
    d = len(shape)
    Ls = Ls or tuple(1.0 + 0.25 * a for a in range(d))
    npdt = np.float64 if dtype == "f64" else np.float32
    g = W.normal(shape, seed, dtype=npdt)
    ref = O.solve(g.astype(np.float64), bcs, Ls, approx, method=method)
    out = gpu_solve(pb, g, bcs, Ls, approx, dtype, inplace=inplace)
    err = O.rel_max_error(out, ref)
    assert err < TOL[dtype], f"shape {shape} bcs {bcs} approx {approx} {dtype}: rel err {err:.3e}"
    return err


# ---------------------------------------------------------------------------
# the paper's workloads
# ---------------------------------------------------------------------------

def test_periodic_spectral_32cubed_f64(pb):
    """32^3 periodic, pseudo-spectral, FP64 on [0, 2 pi)^3, U[-1,1] mean-free."""
    spec = W.WORKLOADS["p3_spectral_32_f64"]
    g = W.make_input(spec)
    ref = O.solve(g, spec["bcs"], spec["Ls"], spec["approx"])
    out = gpu_solve(pb, g, spec["bcs"], spec["Ls"], spec["approx"], "f64")
    assert O.rel_max_error(out, ref) < 1e-12
    assert abs(out.mean()) < 1e-12 * np.abs(out).max()


def test_mixed_fd2_256cubed_f32(pb):
    """256^3, x periodic / y staggered Dirichlet / z staggered Neumann, FD2,
    FP32, N(0,1) mean-free; oracle through its library-FFT realisation."""
    spec = W.WORKLOADS["mixed_fd2_256_f32"]
    g = W.make_input(spec)
    ref = O.solve(g.astype(np.float64), spec["bcs"], spec["Ls"], spec["approx"], method="fft")
    out = gpu_solve(pb, g, spec["bcs"], spec["Ls"], spec["approx"], "f32")
    assert O.rel_max_error(out, ref) < 1e-5


# ---------------------------------------------------------------------------
# all 125 BC combinations, 3D, both precisions and approximations (x not
# periodic with a periodic y or z goes through the separate pair divide)
# ---------------------------------------------------------------------------

COMBOS3 = [c for c in itertools.product(BCS, repeat=3) if supported(c)]


@pytest.mark.parametrize("bcs", COMBOS3, ids=lambda b: "".join(O.BC_NAMES[x] for x in b))
def test_all_bc_combinations_3d_f64(pb, bcs):
    check(pb, (11, 14, 18), bcs, W.FD2, "f64", seed=1)


@pytest.mark.parametrize("bcs", COMBOS3, ids=lambda b: "".join(O.BC_NAMES[x] for x in b))
def test_all_bc_combinations_3d_f32_spectral(pb, bcs):
    check(pb, (9, 12, 20), bcs, W.SPECTRAL, "f32", seed=2)


# ---------------------------------------------------------------------------
# tiling: several tiles, ragged tails, long strided axes, odd / prime sizes
# ---------------------------------------------------------------------------

SHAPES = [
    (30, 40, 300),     # x: many line pairs; strided tiles: 2 column tiles, ragged
    (12, 300, 20),     # y axis longer than one TMA box
    (520, 10, 12),     # z axis of 3 TMA boxes
    (21, 27, 45),      # odd sizes (radix 3, 5)
    (11, 13, 17),      # primes (direct-DFT radices)
    (7, 49, 35),       # radix 7
    (64, 64, 64),
    (1, 5, 8),         # length-1 z axis
    (2, 2, 2),
]


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "x".join(map(str, s)))
@pytest.mark.parametrize("bcs", [(W.P, W.DS, W.NS), (W.P, W.P, W.NS), (W.P, W.P, W.P), (W.DR, W.NR, W.DS),
                                 (W.NS, W.NS, W.NS), (W.P, W.DR, W.NR)],
                         ids=lambda b: "".join(O.BC_NAMES[x] for x in b))
def test_tiling_f32(pb, shape, bcs):
    if min(shape) < 2 and W.NR in bcs:
        pytest.skip("NR needs n >= 2")
    check(pb, shape, bcs, W.FD2, "f32", seed=3)


@pytest.mark.parametrize("shape", [(30, 40, 300), (12, 300, 20), (21, 27, 45), (11, 13, 17)],
                         ids=lambda s: "x".join(map(str, s)))
def test_tiling_f64(pb, shape):
    for bcs in [(W.P, W.DS, W.NS), (W.DR, W.NR, W.DS)]:
        check(pb, shape, bcs, W.FD2, "f64", seed=4)


# ---------------------------------------------------------------------------
# 1D and 2D
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("n", [1, 2, 3, 16, 97, 256, 1000, 1024])
@pytest.mark.parametrize("bc", BCS, ids=lambda b: O.BC_NAMES[b])
def test_1d(pb, n, bc):
    if bc == W.NR and n < 2:
        pytest.skip("NR needs n >= 2")
    for dtype in ("f64", "f32"):
        check(pb, (n,), (bc,), W.FD2, dtype, seed=5)
        check(pb, (n,), (bc,), W.SPECTRAL, dtype, seed=6)


COMBOS2 = [c for c in itertools.product(BCS, repeat=2) if supported(c)]


@pytest.mark.parametrize("bcs", COMBOS2, ids=lambda b: "".join(O.BC_NAMES[x] for x in b))
def test_2d(pb, bcs):
    for shape in [(40, 300), (33, 17), (256, 64)]:
        check(pb, shape, bcs, W.FD2, "f32", seed=7)
        check(pb, shape, bcs, W.SPECTRAL, "f64", seed=8)


# ---------------------------------------------------------------------------
# API behaviour
# ---------------------------------------------------------------------------

def test_in_place(pb):
    check(pb, (20, 24, 48), (W.P, W.DS, W.NS), W.FD2, "f32", inplace=True)
    check(pb, (20, 24, 48), (W.DR, W.NR, W.NS), W.FD2, "f64", inplace=True)


def test_repeated_solves_reuse_plan(pb):
    shape = (16, 24, 32)
    g = W.normal(shape, 9, dtype=np.float32)
    bcs, Ls = (W.P, W.P, W.NS), (1.0, 1.0, 1.0)
    ref = O.solve(g.astype(np.float64), bcs, Ls, W.FD2)
    with pb.Plan((32, 24, 16), Ls, bcs, pb.FD2, pb.F32) as plan:
        gd = torch.from_numpy(g).cuda()
        phi = torch.empty_like(gd)
        for _ in range(3):
            phi.fill_(float("nan"))
            plan.solve(phi, gd, torch.cuda.current_stream())
            assert O.rel_max_error(phi.cpu().numpy(), ref) < 1e-5


def test_solve_host_async_pipeline(pb):
    """poisfft_solve_host_async: several right-hand sides in a row, each
    checked against the FP64 oracle after one synchronisation; the two
    staging pairs alternate, so consecutive calls overlap their copies."""
    shape = (20, 24, 32)
    bcs, Ls = (W.P, W.P, W.NS), (1.0, 1.0, 1.0)
    gs = [W.normal(shape, 30 + i, dtype=np.float32) for i in range(5)]
    refs = [O.solve(g.astype(np.float64), bcs, Ls, W.FD2) for g in gs]
    with pb.Plan((32, 24, 20), Ls, bcs, pb.FD2, pb.F32) as plan:
        stream = torch.cuda.Stream()
        ghs = [torch.from_numpy(g).pin_memory() for g in gs]
        phs = [torch.empty_like(gh).pin_memory() for gh in ghs]
        for _ in range(2):  # the second round reuses the staging pairs
            for gh, ph in zip(ghs, phs):
                ph.fill_(float("nan"))
            for gh, ph in zip(ghs, phs):
                plan.solve_host_async(ph, gh, stream)
            assert plan.check(stream) == pb.OK
            for ph, ref in zip(phs, refs):
                assert O.rel_max_error(ph.numpy(), ref) < 1e-5


def test_solve_host_buffers(pb):
    shape = (18, 22, 40)
    g = W.normal(shape, 10, dtype=np.float32)
    bcs, Ls = (W.P, W.DS, W.NS), (1.0, 1.0, 1.0)
    ref = O.solve(g.astype(np.float64), bcs, Ls, W.FD2)
    with pb.Plan((40, 22, 18), Ls, bcs, pb.FD2, pb.F32) as plan:
        gh = torch.from_numpy(g).pin_memory()
        ph = torch.empty_like(gh).pin_memory()
        plan.solve_host(ph, gh, torch.cuda.current_stream())
        assert O.rel_max_error(ph.numpy(), ref) < 1e-5
        # pageable numpy buffers work too (staged copies)
        out = np.empty_like(g)
        plan.solve_host(out, g)
        assert O.rel_max_error(out, ref) < 1e-5
        # bit-identical to the solve on device buffers
        gd = gh.cuda()
        pd = torch.empty_like(gd)
        plan.solve(pd, gd, torch.cuda.current_stream())
        torch.cuda.synchronize()
        assert torch.equal(pd.cpu(), ph)


def test_nonzero_mean_rhs_singular(pb):
    """Singular problem with an incompatible g: the null-space component is
    removed, phi matches the oracle and has zero (weighted) mean."""
    shape = (10, 12, 16)
    g = W.normal(shape, 11, dtype=np.float64) + 3.0
    bcs, Ls = (W.P, W.NR, W.NS), (1.0, 1.0, 1.0)
    ref = O.solve(g, bcs, Ls, W.FD2)
    out = gpu_solve(pb, g, bcs, Ls, W.FD2, "f64")
    assert O.rel_max_error(out, ref) < 1e-12
    assert abs(O.weighted_mean(out, bcs)) < 1e-12 * np.abs(out).max()


def test_misaligned_pointer_rejected(pb):
    with pb.Plan((8, 8, 8), (1, 1, 1), (W.P, W.P, W.P), pb.FD2, pb.F32) as plan:
        buf = torch.zeros(8 * 8 * 8 + 1, device="cuda")
        rc = pb.solve(plan.handle, buf.data_ptr() + 2, buf.data_ptr(), None)
        assert rc == pb.ERR_MISALIGNED


# ---------------------------------------------------------------------------
# specialised two-pass kernels (x periodic with y/z in {P, NS, DS}, or x, y,
# z all in {NS, DS}; lengths 64...1024) and the generic kernels on the same
# shapes
# ---------------------------------------------------------------------------

FAST3 = [(64, 64, 64), (128, 64, 256), (1024, 64, 64), (512, 256, 64), (64, 128, 1024), (256, 1024, 64)]
FAST_BCS = [(W.P, W.P, W.P), (W.P, W.P, W.NS), (W.P, W.DS, W.NS), (W.P, W.NS, W.DS), (W.P, W.DS, W.P),
            (W.P, W.NS, W.NS)]


@pytest.mark.parametrize("n", FAST3, ids=lambda s: "x".join(map(str, s)))
@pytest.mark.parametrize("bcs", FAST_BCS, ids=lambda b: "".join(O.BC_NAMES[x] for x in b))
def test_fast_path_3d(pb, n, bcs):
    shape = tuple(reversed(n))
    method = "dense" if np.prod(n) <= 1 << 20 else "fft"
    check(pb, shape, bcs, W.FD2, "f32", seed=12, method=method)


@pytest.mark.parametrize("n,bcs", [((1024, 512), (W.P, W.NS)), ((64, 1024), (W.P, W.DS)),
                                   ((256, 256), (W.P, W.P)), ((128, 64), (W.P, W.NS))])
def test_fast_path_2d(pb, n, bcs):
    check(pb, tuple(reversed(n)), bcs, W.SPECTRAL, "f32", seed=13, method="fft")


# x Neumann / Dirichlet staggered (DCT-II / DST-II x sweep by Makhoul's
# reordering, two x columns per complex workspace column) with y, z NS / DS
FAST3_X = [(64, 64, 64), (256, 128, 64), (128, 64, 512), (1024, 64, 64)]
FAST_X_BCS = list(itertools.product([W.NS, W.DS], repeat=3))


@pytest.mark.parametrize("n", FAST3_X, ids=lambda s: "x".join(map(str, s)))
@pytest.mark.parametrize("bcs", FAST_X_BCS, ids=lambda b: "".join(O.BC_NAMES[x] for x in b))
def test_fast_path_3d_x_cosine_sine(pb, n, bcs):
    shape = tuple(reversed(n))
    method = "dense" if np.prod(n) <= 1 << 20 else "fft"
    check(pb, shape, bcs, W.FD2, "f32", seed=15, method=method)


@pytest.mark.parametrize("n,bcs,approx", [((256, 512), (W.NS, W.DS), W.SPECTRAL), ((1024, 64), (W.DS, W.NS), W.FD2),
                                          ((64, 64), (W.NS, W.NS), W.FD2), ((512, 128), (W.DS, W.DS), W.SPECTRAL),
                                          ((64, 1024), (W.NS, W.DS), W.FD2)])
def test_fast_path_2d_x_cosine_sine(pb, n, bcs, approx):
    check(pb, tuple(reversed(n)), bcs, approx, "f32", seed=16, method="fft")


@pytest.mark.parametrize("bcs", [(W.P, W.DS, W.NS), (W.NS, W.DS, W.NS), (W.DS, W.DS, W.DS)],
                         ids=lambda b: "".join(O.BC_NAMES[x] for x in b))
def test_fast_and_generic_kernels_agree(pb, monkeypatch, bcs):
    shape = (128, 64, 256)
    Ls = (1.0, 1.0, 1.0)
    g = W.normal(shape, 14, dtype=np.float32)
    fast = gpu_solve(pb, g, bcs, Ls, W.FD2, "f32")
    monkeypatch.setenv("POISFFT_FORCE_GENERIC", "1")
    generic = gpu_solve(pb, g, bcs, Ls, W.FD2, "f32")
    ref = O.solve(g.astype(np.float64), bcs, Ls, W.FD2, method="fft")
    assert O.rel_max_error(fast, ref) < 1e-5
    assert O.rel_max_error(generic, ref) < 1e-5
    assert O.rel_max_error(fast, generic) < 2e-5


@pytest.mark.parametrize("bcs", [(W.NS, W.P, W.DS), (W.DR, W.NR, W.P), (W.DS, W.P, W.P), (W.NR, W.P, W.NS)],
                         ids=lambda b: "".join(O.BC_NAMES[x] for x in b))
def test_pair_divide_tiling(pb, bcs):
    """x non-periodic, y or z periodic: several tiles, odd x (padding column),
    long strided axes; singular problems keep zero weighted mean."""
    for shape in [(20, 300, 33), (520, 12, 17), (9, 16, 64)]:
        if W.NR in bcs and min(shape) < 2:
            continue
        check(pb, shape, bcs, W.FD2, "f32", seed=15)
        check(pb, shape, bcs, W.SPECTRAL, "f64", seed=16)


# ---------------------------------------------------------------------------
# Bluestein: FFT lengths with a prime factor >= 41 (prime n, or 2(n+1), 2(n-1)
# of the DST-I / DCT-I extensions) on every axis
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("n,bcs", [
    ((101,), (W.P,)), ((88,), (W.DR,)), ((84,), (W.NR,)), ((97,), (W.DS,)), ((113,), (W.NS,)),
    ((88, 101, 84), (W.DR, W.P, W.NR)),       # x extension 2*89, y prime, z extension 2*83
    ((101, 60, 113), (W.P, W.DS, W.NS)),       # x prime (R2C), z prime
    ((40, 88, 43), (W.NS, W.DR, W.P)),         # pair divide with Bluestein y and z
], ids=lambda v: str(v))
@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_bluestein_lengths(pb, n, bcs, dtype):
    check(pb, tuple(reversed(n)), bcs, W.FD2, dtype, seed=17)


def test_bluestein_large_2d_batch_case(pb):
    """A batch problem that dominated the direct-DFT timings: y = DST-I with
    n = 1800 (extension 2 * 1801)."""
    check(pb, (1800, 1792), (W.DS, W.DR), W.FD2, "f32", seed=18, method="fft")


@pytest.mark.parametrize("n,bcs", [((64, 48, 40), (W.P, W.P, W.NS)), ((33, 20, 17), (W.NR, W.P, W.NS)),
                                   ((17, 9, 12), (W.NR, W.NR, W.NR)), ((256, 128), (W.NS, W.NR))])
@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_zero_mode_mean_fp64(pb, n, bcs, dtype):
    shape = tuple(reversed(n))
    npdt = np.float32 if dtype == "f32" else np.float64
    g = (W.normal(shape, 41) + 0.375).astype(npdt)
    ref = O.weighted_mean(g.astype(np.float64), bcs)
    with pb.Plan(n, tuple(1.0 for _ in n), bcs, W.FD2, pb.F32 if dtype == "f32" else pb.F64) as plan:
        got = plan.zero_mode_mean(torch.from_numpy(g).cuda())
    assert abs(got - ref) <= (1e-12 if dtype == "f64" else 1e-7) * np.max(np.abs(g))


def test_zero_mode_mean_rejects_nonsingular(pb):
    with pb.Plan((16, 8, 8), (1.0, 1.0, 1.0), (W.P, W.DS, W.NS), W.FD2, pb.F32) as plan:
        with pytest.raises(pb.PoisFFTError):
            plan.zero_mode_mean(torch.zeros(16 * 8 * 8, device="cuda"))
