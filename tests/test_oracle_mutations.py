"""Plant plausible mistakes in the oracle and check that its pins catch them.

Each mutation replaces one oracle function with a subtly wrong version (a
dropped term, a wrong sign or index, a transposed operand, a wrong scale or
grid spacing).  The compact pin battery below (library transforms, inverse
pairs, stencil eigenpairs, FD residual, spectral closed form) must fail for
every one of them, and pass for the unmodified oracle.
"""

import math

import numpy as np
import pytest
import scipy.fft as sf

from oracle import poisson as O

BCS = [O.P, O.DR, O.DS, O.NR, O.NS]


def _pins_hold():
    n = 7
    eye = np.eye(n)
    lib = {
        O.DR: sf.dst(eye, type=1, axis=0), O.DS: sf.dst(eye, type=2, axis=0),
        O.NR: sf.dct(eye, type=1, axis=0), O.NS: sf.dct(eye, type=2, axis=0),
        O.P: np.fft.fft(eye, axis=0) / n,
    }
    for bc in BCS:
        if not np.allclose(O.forward_matrix(bc, n), lib[bc], atol=1e-12):
            return False
        if not np.allclose(O.backward_matrix(bc, n) @ O.forward_matrix(bc, n), eye, atol=1e-12):
            return False
        lam = O.eigenvalues(bc, n, 1.3, O.FD2)
        basis = O.backward_matrix(bc, n)
        for k in range(n):
            v = basis[:, k].real
            if not np.allclose(O.laplacian_fd2(v, [bc], [1.3]), lam[k] * v, atol=1e-10):
                return False
    r = np.random.default_rng(0)
    for bcs in [(O.P, O.DS, O.NS), (O.NR, O.DR, O.P), (O.NS, O.NS, O.NR)]:
        ns = (6, 5, 4)
        Ls = (1.0, 0.8, 1.1)
        g = r.standard_normal((4, 5, 6))
        phi = O.solve(g, bcs, Ls, O.FD2)
        res = O.laplacian_fd2(phi, bcs, Ls) - O.project_range(g, bcs)
        if np.max(np.abs(res)) > 1e-9 * np.max(np.abs(g)):
            return False
    # FD2 converges at second order to the continuous eigenfunction solution
    for bc in BCS:
        errs = []
        for n in (16, 32):
            x = {O.P: np.arange(n) / n, O.DR: (np.arange(n) + 1) / (n + 1),
                 O.NR: np.arange(n) / (n - 1)}.get(bc, (np.arange(n) + 0.5) / n)
            f = np.cos(2 * np.pi * x) if bc == O.P else (np.sin(np.pi * x) if bc in (O.DR, O.DS) else np.cos(np.pi * x))
            lam = -(2 * np.pi) ** 2 if bc == O.P else -np.pi ** 2
            errs.append(np.max(np.abs(O.solve(lam * f, [bc], [1.0], O.FD2) - f)))
        if not (0.2 < errs[1] / errs[0] < 0.3):
            return False
    # spectral: periodic closed form with the highest resolved wavenumbers
    n, L = 8, 2.0
    x = np.arange(n) * L / n
    for m in (1, 3):
        phi = np.cos(2 * np.pi * m * x / L)
        g = -(2 * np.pi * m / L) ** 2 * phi
        if not np.allclose(O.solve(g, [O.P], [L], O.SPECTRAL), phi, atol=1e-12):
            return False
    return True


def test_unmodified_oracle_passes_pin_battery():
    assert _pins_hold()


def _mut_dst3_full_weight(n):
    k = np.arange(n)[:, None]
    j = np.arange(n)[None, :]
    return 2.0 * O.sinpi((j + 1) * (2 * k + 1), 2 * n)          # last column not halved


def _mut_dct2_transposed(n):
    k = np.arange(n)[:, None]
    j = np.arange(n)[None, :]
    return (2.0 * O.cospi((2 * j + 1) * k, 2 * n)).T


def _mut_dft_plus_sign(n):
    k = np.arange(n)[:, None]
    j = np.arange(n)[None, :]
    s, c = O._sincos_pi_frac(2 * k * j, n)
    return (c + 1j * s) / n


def _mut_dst1_index(n):
    k = np.arange(n)[:, None]
    j = np.arange(n)[None, :]
    return 2.0 * O.sinpi((j + 1) * (k + 1), n + 2)              # n+1 -> n+2


_orig_eig = O.eigenvalues
_orig_dx = O.grid_spacing


def _mut_eig_ds_half_angle(bc, n, L, approx):
    if approx == O.FD2 and bc == O.DS:
        k = np.arange(n)
        return -(2.0 * O.sinpi(k + 1, n) / (L / n)) ** 2         # pi(k+1)/(2n) -> pi(k+1)/n
    return _orig_eig(bc, n, L, approx)


def _mut_eig_periodic_no_alias(bc, n, L, approx):
    if approx == O.SPECTRAL and bc == O.P:
        return -(2.0 * math.pi * np.arange(n) / L) ** 2           # k instead of min(k, n-k)
    return _orig_eig(bc, n, L, approx)


def _mut_dx_nr(bc, n, L):
    return L / n if bc == O.NR else _orig_dx(bc, n, L)            # L/(n-1) -> L/n


def _mut_eig_nr_wrong_offset(bc, n, L, approx):
    if approx == O.FD2 and bc == O.NR:
        k = np.arange(n)
        return -(2.0 * O.sinpi(k, 2 * n) / (L / (n - 1))) ** 2   # 2(n-1) -> 2n
    return _orig_eig(bc, n, L, approx)


MUTATIONS = [
    ("dst3_matrix", _mut_dst3_full_weight),
    ("dct2_matrix", _mut_dct2_transposed),
    ("dft_matrix", _mut_dft_plus_sign),
    ("dst1_matrix", _mut_dst1_index),
    ("eigenvalues", _mut_eig_ds_half_angle),
    ("eigenvalues", _mut_eig_periodic_no_alias),
    ("grid_spacing", _mut_dx_nr),
    ("eigenvalues", _mut_eig_nr_wrong_offset),
]


@pytest.mark.parametrize("name,fn", MUTATIONS, ids=[f"{n}:{f.__name__}" for n, f in MUTATIONS])
def test_planted_mistake_is_caught(monkeypatch, name, fn):
    monkeypatch.setattr(O, name, fn)
    assert not _pins_hold()


def test_planted_missing_zero_mode_fix_is_caught(monkeypatch):
    orig = O.is_singular
    monkeypatch.setattr(O, "is_singular", lambda bcs: False if all(b == O.P for b in bcs) else orig(bcs))
    g = np.random.default_rng(1).standard_normal((4, 5, 6))
    with np.errstate(divide="ignore", invalid="ignore"):
        phi = O.solve(g, (O.P, O.P, O.P), (1.0, 1.0, 1.0), O.FD2)
    assert not np.all(np.isfinite(phi)) or abs(phi.mean()) > 1e-6
