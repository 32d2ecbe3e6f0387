"""POISFFT_BF16X3: the radix-32 DFT blocks of 1024-point strided axes as
tensor-core GEMMs (tcgen05, split-BF16 operands, FP32 accumulation), the
mixed-precision form of the Sec. 2.1 algorithm (transforms of Table 2,
eigenvalues of Table 4 summed as in Sec. 2.3), against the FP64 oracle.

Stated bound 1e-4 (normwise max relative error): each operand of a GEMM
pass is held to 16 significant bits (hi + lo bfloat16, about 2^-17
relative), the dropped lo*lo product is below 2^-16, so one pass is
accurate to about 2^-16 of its inputs' magnitude; a solve runs at most
eight such passes (y forward, z forward and backward, y backward, two
each), 8 x 2^-16 = 1.2e-4.  The FP32 path stays within 1e-5."""

import numpy as np
import pytest

import workloads as W
from oracle import poisson as O
from tests._lib import ensure_built

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

TOL_TC = 1e-4


@pytest.fixture(scope="module")
def pb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ensure_built()
    from paper_1409_8116_gb300 import binding
    return binding


CASES = [
    ((64, 64, 1024), (W.P, W.P, W.P), "tc_strided_sweep:fused:z"),      # fused DFT
    ((64, 64, 1024), (W.P, W.P, W.NS), "tc_strided_sweep:fused:z"),     # fused DCT-II / DCT-III, singular
    ((64, 64, 1024), (W.P, W.DS, W.DS), "tc_strided_sweep:fused:z"),    # fused DST-II / DST-III
    ((64, 1024, 64), (W.P, W.P, W.P), "tc_strided_sweep:forward:y"),    # y forward and backward
    ((64, 1024, 1024), (W.P, W.P, W.NS), "tc_strided_sweep:backward:y"),  # the benchmark's BCs
    ((128, 1024, 256), (W.P, W.P, W.DS), "tc_strided_sweep:forward:y"),
    ((1024, 16, 1024), (W.NS, W.NS, W.NS), None),                        # x DCT: z pairs columns -> FP32
]


@pytest.mark.parametrize("n,bcs,expect", CASES, ids=lambda v: str(v))
def test_bf16x3_matches_oracle(pb, n, bcs, expect):
    shape = tuple(reversed(n))
    Ls = (1.0, 1.0, 1.0)
    g = W.normal(shape, 31, dtype=np.float32)
    ref = O.solve(g.astype(np.float64), bcs, Ls, O.FD2, method="fft")
    if expect is None:
        with pytest.raises(pb.PoisFFTError) as e:
            pb.Plan(n, Ls, bcs, pb.FD2, pb.BF16X3)
        assert e.value.status == pb.ERR_NOT_IMPLEMENTED
        return
    gd = torch.from_numpy(g).cuda()
    with pb.Plan(n, Ls, bcs, pb.FD2, pb.BF16X3) as plan:
        kinds = [f"{l['kernel']}:{l['mode']}:{l['axis']}" for l in plan.launches()]
        assert expect in kinds, kinds
        for call in range(2):  # the persistent kernels leave nothing behind
            phi = torch.full_like(gd, float("nan"))
            plan.solve(phi, gd, torch.cuda.current_stream())
            torch.cuda.synchronize()
            assert plan.check() == pb.OK
            err = O.rel_max_error(phi.cpu().numpy(), ref)
            assert err < TOL_TC, (call, err)
    # the same solve in FP32 stays at the FP32 bound
    with pb.Plan(n, Ls, bcs, pb.FD2, pb.F32) as plan:
        phi = torch.full_like(gd, float("nan"))
        plan.solve(phi, gd, torch.cuda.current_stream())
        torch.cuda.synchronize()
        assert O.rel_max_error(phi.cpu().numpy(), ref) < 1e-5


def test_bf16x3_manufactured_mode_at_1024(pb):
    """A manufactured DCT-II x DFT source on the full-depth axis: the exact
    discrete solution is the source divided by its Table 4 eigenvalue."""
    n = (64, 64, 1024)
    Ls = (1.0, 1.0, 1.0)
    x = (np.arange(n[0]) + 0.0) / n[0]
    y = np.arange(n[1]) / n[1]
    z = (np.arange(n[2]) + 0.5) / n[2]
    kx, ky, kz = 3, 5, 77
    g = (np.cos(2 * np.pi * kx * x)[None, None, :] * np.cos(2 * np.pi * ky * y)[None, :, None]
         * np.cos(np.pi * kz * z)[:, None, None])
    lam = sum(-(2 * np.sin(np.pi * k / m) * m) ** 2 for k, m in ((kx, n[0]), (ky, n[1])))
    lam += -(2 * np.sin(np.pi * kz / (2 * n[2])) * n[2]) ** 2
    exact = g / lam
    gd = torch.from_numpy(g.astype(np.float32)).cuda()
    with pb.Plan(n, Ls, (W.P, W.P, W.NS), pb.FD2, pb.BF16X3) as plan:
        phi = torch.empty_like(gd)
        plan.solve(phi, gd, torch.cuda.current_stream())
        torch.cuda.synchronize()
        assert plan.check() == pb.OK
    assert O.rel_max_error(phi.cpu().numpy(), exact) < TOL_TC
