"""Parity at the full size of the 1024^3 workload (P, P, NS; FD2; FP32),
in the launch configuration the benchmark times.

The right-hand side is a sum of three products of Table 1 basis functions
(periodic cosines in x and y, staggered-Neumann cosines in z), whose exact
discrete solution is the same sum with every mode divided by its Table 4
eigenvalue sum.  The GPU solution is compared with that closed form on
200 000 sampled cells and on whole lines along each axis."""

import numpy as np
import pytest

from tests._lib import ensure_built

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

N = 1024
MODES = [(3, 5, 7, 1.0), (100, 17, 250, 0.5), (511, 1, 1023, 0.25)]   # (kx, ky, kz, amplitude)


@pytest.fixture(scope="module")
def pb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ensure_built()
    from paper_1409_8116_gb300 import binding
    return binding


def _bases(k, kind):
    j = np.arange(N, dtype=np.float64)
    if kind == "P":
        return np.cos(2 * np.pi * k * j / N), -4.0 * N * N * np.sin(np.pi * k / N) ** 2
    return np.cos(np.pi * k * (j + 0.5) / N), -4.0 * N * N * np.sin(np.pi * k / (2 * N)) ** 2


def test_1024_cubed_manufactured_modes(pb):
    terms = []
    for kx, ky, kz, amp in MODES:
        bx, lx = _bases(kx, "P")
        by, ly = _bases(ky, "P")
        bz, lz = _bases(kz, "NS")
        terms.append((amp, bx, by, bz, lx + ly + lz))
    g = np.zeros((N, N, N), dtype=np.float32)
    for amp, bx, by, bz, _ in terms:
        g += (amp * bz[:, None, None] * by[None, :, None] * bx[None, None, :]).astype(np.float32)

    def exact(z, y, x):
        return sum(amp * bz[z] * by[y] * bx[x] / lam for amp, bx, by, bz, lam in terms)

    with pb.Plan((N, N, N), (1.0, 1.0, 1.0), (pb.P, pb.P, pb.NS), pb.FD2, pb.F32) as plan:
        gd = torch.from_numpy(g).cuda()
        del g
        phi = torch.empty_like(gd)
        plan.solve(phi, gd, torch.cuda.current_stream())
        assert plan.check() == pb.OK
        del gd
        r = np.random.default_rng(0)
        idx = r.integers(0, N, size=(200000, 3))
        flat = torch.from_numpy(idx[:, 0] * N * N + idx[:, 1] * N + idx[:, 2]).cuda()
        got = phi.view(-1)[flat].cpu().numpy().astype(np.float64)
        ref = exact(idx[:, 0], idx[:, 1], idx[:, 2])
        scale = sum(abs(amp / lam) for amp, *_, lam in terms)
        assert np.max(np.abs(got - ref)) <= 1e-5 * scale
        # whole lines along x, y and z
        for (z, y) in [(0, 0), (511, 1023), (1023, 7)]:
            line = phi[z, y, :].cpu().numpy().astype(np.float64)
            assert np.max(np.abs(line - exact(z, y, np.arange(N)))) <= 1e-5 * scale
        line = phi[300, :, 17].cpu().numpy().astype(np.float64)
        assert np.max(np.abs(line - exact(300, np.arange(N), 17))) <= 1e-5 * scale
        line = phi[:, 600, 1000].cpu().numpy().astype(np.float64)
        assert np.max(np.abs(line - exact(np.arange(N), 600, 1000))) <= 1e-5 * scale
