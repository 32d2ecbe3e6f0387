"""Solves on parts of larger arrays, and the projection step of Sec. 5.

* poisfft_solve_strided: g and phi are the interiors of arrays with ghost
  layers (Sec. 3).  Ghost cells hold NaN sentinels: if any were read the
  solution would be NaN, and they must be unchanged afterwards.
* The projection method of Sec. 5 (Eq. projection-Poisson): a random
  staggered (MAC-grid) velocity u*, periodic in x and y with walls in z, is
  corrected by the gradient of phi where lap(phi) = div(u*) (FD2, staggered
  Neumann in z, as in the paper's model); the corrected field must be
  discretely divergence-free.
"""

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


@pytest.mark.parametrize("n,bcs,dtype,tol", [
    ((64, 64, 64), (W.P, W.P, W.NS), "f32", 1e-5),          # specialised kernels
    ((256, 64, 128), (W.P, W.DS, W.NS), "f32", 1e-5),       # specialised kernels
    # 1024-point x lines: dense rows of g are staged by bulk copies, these
    # ghost-cell rows start off a 16-byte boundary and take the direct loads
    ((1024, 64, 64), (W.P, W.P, W.NS), "f32", 1e-5),
    ((33, 20, 17), (W.DR, W.NR, W.P), "f64", 1e-12),        # general kernels + pair divide
    ((45, 27, 21), (W.P, W.DS, W.NR), "f64", 1e-12),        # general kernels
    ((50, 40), (W.P, W.NS), "f32", 1e-5),
])
def test_strided_ghost_cell_arrays(pb, n, bcs, dtype, tol):
    d = len(n)
    shape = tuple(reversed(n))
    ghost = (2, 3, 5)[:d]
    big = tuple(s + 2 * gh for s, gh in zip(shape, reversed(ghost)))
    npdt = np.float32 if dtype == "f32" else np.float64
    tdt = torch.float32 if dtype == "f32" else torch.float64
    g = W.normal(shape, 21, dtype=npdt)
    Ls = tuple(1.0 + 0.2 * a for a in range(d))
    ref = O.solve(g.astype(np.float64), bcs, Ls, W.FD2, method="fft" if np.prod(n) > 1 << 18 else "dense")
    inner = tuple(slice(gh, gh + s) for gh, s in zip(reversed(ghost), shape))
    G = np.full(big, np.nan, dtype=npdt)
    G[inner] = g
    Gd = torch.from_numpy(G).cuda()
    Pd = torch.full(big, 7.25, dtype=tdt, device="cuda")
    es = Gd.element_size()
    strides = [Gd.stride(k) for k in range(d)]          # numpy order: (z, y, x)
    off = sum(gh * st for gh, st in zip(reversed(ghost), strides))
    ld = list(reversed(strides[:-1])) + [0] * (3 - d)   # (y-row stride, z-plane stride)
    with pb.Plan(n, Ls, bcs, pb.FD2, pb.F32 if dtype == "f32" else pb.F64) as plan:
        plan.solve_strided(Pd.data_ptr() + off * es, ld[:2], Gd.data_ptr() + off * es, ld[:2],
                           torch.cuda.current_stream())
        assert plan.check() == pb.OK
        P = Pd.cpu().numpy()
    assert O.rel_max_error(P[inner], ref) < tol
    mask = np.ones(big, bool)
    mask[inner] = False
    assert np.all(P[mask] == npdt(7.25))                # ghost cells untouched


def test_strided_rejects_overlapping_rows(pb):
    with pb.Plan((16, 8, 4), (1, 1, 1), (W.P, W.P, W.P), pb.FD2, pb.F32) as plan:
        buf = torch.zeros(16 * 8 * 4, device="cuda")
        with pytest.raises(pb.PoisFFTError):
            plan.solve_strided(buf, (15, 16 * 8), buf, (16, 16 * 8))
        with pytest.raises(pb.PoisFFTError):
            plan.solve_strided(buf, (16, 16 * 7), buf, (16, 16 * 8))


def _mac_div(u, v, w, dx, dy, dz):
    # u[z, y, i] on the face left of cell i (periodic x), v[z, j, x] left of
    # cell j (periodic y), w[k, y, x] below cell k, k = 0..nz (w = 0 at walls)
    return ((np.roll(u, -1, axis=2) - u) / dx + (np.roll(v, -1, axis=1) - v) / dy + (w[1:] - w[:-1]) / dz)


@pytest.mark.parametrize("dtype,tol", [("f64", 1e-10), ("f32", 2e-4)])
def test_projection_step_makes_velocity_divergence_free(pb, dtype, tol):
    nx, ny, nz = 64, 48, 40
    L = (2.0, 1.5, 1.0)
    dx, dy, dz = L[0] / nx, L[1] / ny, L[2] / nz
    r = np.random.default_rng(31)
    u = r.standard_normal((nz, ny, nx))
    v = r.standard_normal((nz, ny, nx))
    w = r.standard_normal((nz + 1, ny, nx))
    w[0] = w[-1] = 0.0                                  # no flow through the walls
    div = _mac_div(u, v, w, dx, dy, dz)
    npdt = np.float32 if dtype == "f32" else np.float64
    with pb.Plan((nx, ny, nz), L, (W.P, W.P, W.NS), pb.FD2, pb.F32 if dtype == "f32" else pb.F64) as plan:
        dd = torch.from_numpy(div.astype(npdt)).cuda()
        phi = torch.empty_like(dd)
        plan.solve(phi, dd, torch.cuda.current_stream())
        torch.cuda.synchronize()
        p = phi.cpu().numpy().astype(np.float64)
    u2 = u - (p - np.roll(p, 1, axis=2)) / dx
    v2 = v - (p - np.roll(p, 1, axis=1)) / dy
    w2 = w.copy()
    w2[1:-1] -= (p[1:] - p[:-1]) / dz
    div2 = _mac_div(u2, v2, w2, dx, dy, dz)
    assert np.max(np.abs(div2)) < tol * np.max(np.abs(div))
