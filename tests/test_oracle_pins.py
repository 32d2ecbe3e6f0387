"""Pins of the FP64 oracle to things other than itself (CPU only).

Each check ties the oracle to an independent source of truth:
  * a library (scipy.fft / numpy.fft, whose unnormalised transforms are the
    Table 1 definitions) for every 1D matrix;
  * the Table 2 inverse pairs (backward o forward = identity);
  * the finite-difference stencil of Eq. (FD2-Laplace) applied directly, for
    the Table 4 eigenvalues and for whole solves (residual test);
  * dense LU (LAPACK) on grids up to 8^3;
  * closed-form continuous solutions for the pseudo-spectral tables;
  * manufactured single/multi-mode sources (phi = g / lambda);
  * zero-mean invariants of the singular problems and the imaginary residue
    of the periodic path.
"""

import itertools
import math

import numpy as np
import pytest
import scipy.fft as sf

from oracle import poisson as O

BCS = [O.P, O.DR, O.DS, O.NR, O.NS]
SIZES = [1, 2, 3, 4, 5, 7, 8, 9, 12, 16, 17]


def _valid(bc, n):
    return not (bc == O.NR and n < 2)


# --------------------------------------------------------------------------
# exactly reduced trigonometry
# --------------------------------------------------------------------------

def test_sincospi_matches_libm_and_exact_points():
    for d in [1, 2, 3, 7, 64, 1000, 1024]:
        m = np.arange(-5 * d, 5 * d + 1)
        s, c = O._sincos_pi_frac(m, d)
        np.testing.assert_allclose(s, np.sin(np.pi * m / d), atol=4e-15)
        np.testing.assert_allclose(c, np.cos(np.pi * m / d), atol=4e-15)
        # exact zeros and ones at multiples of pi/2
        half = (2 * m) % d == 0
        q = ((2 * m) // d) % 4
        assert np.all(s[half & (q % 2 == 0)] == 0.0)
        assert np.all(c[half & (q % 2 == 1)] == 0.0)
        assert np.all(np.abs(s[half & (q % 2 == 1)]) == 1.0)


# --------------------------------------------------------------------------
# Table 1 <-> library
# --------------------------------------------------------------------------

@pytest.mark.parametrize("n", SIZES)
def test_table1_matrices_equal_library_transforms(n):
    eye = np.eye(n)
    pairs = [
        (O.dst1_matrix, lambda x: sf.dst(x, type=1, axis=0)),
        (O.dst2_matrix, lambda x: sf.dst(x, type=2, axis=0)),
        (O.dst3_matrix, lambda x: sf.dst(x, type=3, axis=0)),
        (O.dct2_matrix, lambda x: sf.dct(x, type=2, axis=0)),
        (O.dct3_matrix, lambda x: sf.dct(x, type=3, axis=0)),
        (O.dft_matrix, lambda x: np.fft.fft(x, axis=0) / n),
        (O.idft_matrix, lambda x: np.fft.ifft(x, axis=0) * n),
    ]
    if n >= 2:
        pairs.append((O.dct1_matrix, lambda x: sf.dct(x, type=1, axis=0)))
    for mat, lib in pairs:
        np.testing.assert_allclose(mat(n), lib(eye), atol=1e-13 * max(1, n), rtol=0,
                                   err_msg=mat.__name__)


@pytest.mark.parametrize("bc", BCS)
@pytest.mark.parametrize("n", SIZES + [31, 32, 33, 64])
def test_table2_backward_inverts_forward(bc, n):
    if not _valid(bc, n):
        pytest.skip("NR needs n >= 2")
    ident = O.backward_matrix(bc, n) @ O.forward_matrix(bc, n)
    np.testing.assert_allclose(ident, np.eye(n), atol=5e-14 * n, rtol=0)


def test_transform_pair_scales_of_table2():
    """DST-I o DST-I = 2(n+1) I, DCT-I o DCT-I = 2(n-1) I, DST-III o DST-II =
    2n I, DCT-III o DCT-II = 2n I (the unscaled Table 1 matrices)."""
    for n in [2, 3, 5, 8, 13]:
        np.testing.assert_allclose(O.dst1_matrix(n) @ O.dst1_matrix(n), 2 * (n + 1) * np.eye(n), atol=1e-12)
        np.testing.assert_allclose(O.dct1_matrix(n) @ O.dct1_matrix(n), 2 * (n - 1) * np.eye(n), atol=1e-12)
        np.testing.assert_allclose(O.dst3_matrix(n) @ O.dst2_matrix(n), 2 * n * np.eye(n), atol=1e-12)
        np.testing.assert_allclose(O.dct3_matrix(n) @ O.dct2_matrix(n), 2 * n * np.eye(n), atol=1e-12)


# --------------------------------------------------------------------------
# Table 4 eigenpairs <-> the stencil of Eq. (FD2-Laplace)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("bc", BCS)
@pytest.mark.parametrize("n", [2, 3, 4, 5, 8, 11, 16])
def test_fd2_eigenpairs_match_stencil(bc, n):
    L = 1.7
    lam = O.eigenvalues(bc, n, L, O.FD2)
    basis = O.backward_matrix(bc, n)          # column k = eigenvector k on the grid
    for k in range(n):
        v = basis[:, k]
        if bc == O.P:
            # the stencil is real: check the real and imaginary parts
            for part in (v.real, v.imag):
                lv = O.laplacian_fd2(part, [bc], [L])
                np.testing.assert_allclose(lv, lam[k] * part, atol=1e-12 * max(1.0, abs(lam[k])))
        else:
            lv = O.laplacian_fd2(v, [bc], [L])
            np.testing.assert_allclose(lv, lam[k] * v, atol=1e-12 * max(1.0, abs(lam[k])))


@pytest.mark.parametrize("bc", BCS)
def test_spectral_table_is_fd2_limit(bc):
    """Table 3 is the dx -> 0 limit of Table 4 for fixed wavenumber."""
    L = 2.5
    n = 8192
    fd = O.eigenvalues(bc, n, L, O.FD2)[:6]
    sp = O.eigenvalues(bc, n, L, O.SPECTRAL)[:6]
    nz = sp != 0
    np.testing.assert_allclose(fd[nz] / sp[nz], 1.0, rtol=1e-5)
    assert np.all(fd[~nz] == 0)


def test_spectral_periodic_aliasing_reading():
    """min(k, n-k): mode k and n-k carry the same eigenvalue."""
    for n in [7, 8, 32]:
        lam = O.eigenvalues(O.P, n, 1.0, O.SPECTRAL)
        np.testing.assert_allclose(lam[1:], lam[1:][::-1], rtol=1e-15)
        assert lam[n // 2] == -(2 * math.pi * (n // 2)) ** 2


# --------------------------------------------------------------------------
# pseudo-spectral solves of continuous closed forms
# --------------------------------------------------------------------------

def _grid(bc, n, L):
    j = np.arange(n)
    if bc == O.P:
        return j * L / n
    if bc == O.DR:
        return (j + 1) * L / (n + 1)
    if bc == O.NR:
        return j * L / (n - 1)
    return (j + 0.5) * L / n


@pytest.mark.parametrize("bcs", [(O.P, O.P, O.P), (O.DS, O.DR, O.P), (O.NS, O.NR, O.DS), (O.NR, O.NS, O.NR)])
def test_spectral_recovers_band_limited_continuous_solution(bcs):
    """phi = prod_a f_a(x_a) with f a low eigenfunction of d2/dx2 under the
    axis BC; g = lap(phi) in closed form; the pseudo-spectral solve must
    return phi on the grid exactly (up to rounding)."""
    ns = (12, 10, 9)
    Ls = (2.0, 1.3, 3.1)
    modes = (2, 3, 1)
    facs, eig = [], 0.0
    for a in range(3):
        x = _grid(bcs[a], ns[a], Ls[a])
        m = modes[a]
        if bcs[a] == O.P:
            f, lam = np.cos(2 * np.pi * m * x / Ls[a] + 0.3), -(2 * np.pi * m / Ls[a]) ** 2
        elif bcs[a] in (O.DR, O.DS):
            f, lam = np.sin(np.pi * m * x / Ls[a]), -(np.pi * m / Ls[a]) ** 2
        else:
            f, lam = np.cos(np.pi * m * x / Ls[a]), -(np.pi * m / Ls[a]) ** 2
        facs.append(f)
        eig += lam
    phi = facs[2][:, None, None] * facs[1][None, :, None] * facs[0][None, None, :]
    g = eig * phi
    out = O.solve(g, bcs, Ls, O.SPECTRAL)
    assert O.rel_max_error(out, phi) < 1e-12


# --------------------------------------------------------------------------
# manufactured single / multi-mode sources
# --------------------------------------------------------------------------

def _mode(bc, n, k):
    """Eigenvector k of the axis, written from the Table 1 kernels with
    plain numpy trig (independent of the oracle's reduced trig)."""
    j = np.arange(n)
    if bc == O.P:
        return np.cos(2 * np.pi * k * j / n)
    if bc == O.DR:
        return np.sin(np.pi * (j + 1) * (k + 1) / (n + 1))
    if bc == O.DS:
        return np.sin(np.pi * (j + 0.5) * (k + 1) / n)
    if bc == O.NR:
        return np.cos(np.pi * j * k / (n - 1))
    return np.cos(np.pi * (j + 0.5) * k / n)


@pytest.mark.parametrize("approx", [O.SPECTRAL, O.FD2])
def test_manufactured_multimode_sources(approx):
    r = np.random.default_rng(11)
    ns = (9, 8, 6)
    Ls = (1.0, 2.0, 0.7)
    for bcs in itertools.product(BCS, repeat=3):
        g = np.zeros((ns[2], ns[1], ns[0]))
        phi = np.zeros_like(g)
        for _ in range(3):
            ks = [int(r.integers(0, ns[a])) for a in range(3)]
            if O.is_singular(bcs) and all(k == 0 for k in ks):
                continue
            amp = r.standard_normal()
            v = [_mode(bcs[a], ns[a], ks[a]) for a in range(3)]
            mode = amp * v[2][:, None, None] * v[1][None, :, None] * v[0][None, None, :]
            lam = sum(O.eigenvalues(bcs[a], ns[a], Ls[a], approx)[ks[a]] for a in range(3))
            g += mode
            phi += mode / lam
        out = O.solve(g, bcs, Ls, approx)
        assert O.rel_max_error(out, phi) < 1e-12, bcs


# --------------------------------------------------------------------------
# FD residual, zero-mean invariant, imaginary residue
# --------------------------------------------------------------------------

def _norm_L(bcs, ns, Ls):
    return sum(4.0 / O.grid_spacing(bcs[a], ns[a], Ls[a]) ** 2 for a in range(len(bcs)))


@pytest.mark.parametrize("dims", [1, 2, 3])
def test_fd2_residual_all_bc_combinations(dims):
    r = np.random.default_rng(5 + dims)
    ns_all = (13, 10, 7)
    Ls_all = (1.0, 1.5, 0.8)
    ns, Ls = ns_all[:dims], Ls_all[:dims]
    shape = tuple(reversed(ns))
    for bcs in itertools.product(BCS, repeat=dims):
        g = r.standard_normal(shape)
        phi, imag = O.solve(g, bcs, Ls, O.FD2, return_imag=True)
        res = O.laplacian_fd2(phi, bcs, Ls) - O.project_range(g, bcs)
        tol = 1e-12 * _norm_L(bcs, ns, Ls) * np.max(np.abs(phi))
        assert np.max(np.abs(res)) < tol, bcs
        if O.is_singular(bcs):
            assert abs(O.weighted_mean(phi, bcs)) < 1e-13 * np.max(np.abs(phi)), bcs
        assert imag <= 1e-13 * np.max(np.abs(phi)), bcs


def test_fd2_residual_config_shapes():
    """The two FD2 workload BC sets, on 64-point grids."""
    for bcs in [(O.P, O.DS, O.NS), (O.P, O.P, O.NS)]:
        ns = (64, 48, 40)
        shape = tuple(reversed(ns))
        g = np.random.default_rng(3).standard_normal(shape)
        Ls = tuple(n / 256.0 for n in ns)
        phi = O.solve(g, bcs, Ls, O.FD2)
        res = O.laplacian_fd2(phi, bcs, Ls) - O.project_range(g, bcs)
        assert np.max(np.abs(res)) < 1e-12 * _norm_L(bcs, ns, Ls) * np.max(np.abs(phi))


# --------------------------------------------------------------------------
# dense LU brute force
# --------------------------------------------------------------------------

def _dense_operator(shape, bcs, Ls):
    N = int(np.prod(shape))
    A = np.zeros((N, N))
    for i in range(N):
        e = np.zeros(N)
        e[i] = 1.0
        A[:, i] = O.laplacian_fd2(e.reshape(shape), bcs, Ls).ravel()
    return A


@pytest.mark.parametrize("bcs", [(O.P, O.P, O.P), (O.P, O.DS, O.NS), (O.P, O.P, O.NS), (O.DR, O.DS, O.NR),
                                 (O.NR, O.NR, O.NR), (O.NS, O.NR, O.P), (O.DR, O.DR, O.DR), (O.NS, O.NS, O.NS)])
def test_dense_lu_bruteforce(bcs):
    ns = (8, 6, 5)
    Ls = (1.0, 0.9, 1.4)
    shape = tuple(reversed(ns))
    g = np.random.default_rng(17).standard_normal(shape)
    A = _dense_operator(shape, bcs, Ls)
    N = A.shape[0]
    if O.is_singular(bcs):
        w = O.null_weights(shape, bcs).ravel()
        B = np.zeros((N + 1, N + 1))
        B[:N, :N] = A
        B[:N, N] = 1.0
        B[N, :N] = w
        rhs = np.concatenate([g.ravel(), [0.0]])
        x = np.linalg.solve(B, rhs)[:N]
    else:
        x = np.linalg.solve(A, g.ravel())
    phi = O.solve(g, bcs, Ls, O.FD2)
    assert O.rel_max_error(phi.ravel(), x) < 1e-12


# --------------------------------------------------------------------------
# the library-FFT realisation equals the dense definition
# --------------------------------------------------------------------------

@pytest.mark.parametrize("approx", [O.SPECTRAL, O.FD2])
def test_fft_method_equals_dense_method(approx):
    r = np.random.default_rng(23)
    for bcs in [(O.P, O.DS, O.NS), (O.P, O.P, O.NS), (O.DR, O.NR, O.P), (O.NS, O.NS, O.NS), (O.DS, O.DR, O.NR)]:
        ns = (12, 9, 10)
        g = r.standard_normal(tuple(reversed(ns)))
        Ls = (1.0, 1.2, 0.9)
        a = O.solve(g, bcs, Ls, approx, method="dense")
        b = O.solve(g, bcs, Ls, approx, method="fft")
        assert O.rel_max_error(b, a) < 1e-13


def test_one_and_two_dims():
    r = np.random.default_rng(2)
    g1 = r.standard_normal(16)
    for bc in BCS:
        phi = O.solve(g1, [bc], [1.0], O.FD2)
        res = O.laplacian_fd2(phi, [bc], [1.0]) - O.project_range(g1, [bc])
        assert np.max(np.abs(res)) < 1e-12 * _norm_L([bc], [16], [1.0]) * np.max(np.abs(phi))


@pytest.mark.parametrize("bc", BCS)
def test_fd2_converges_at_second_order_to_continuous_solution(bc):
    """On each Sec. 2.1 grid, the FD2 solve of g = lap(f) for a smooth
    eigenfunction f of the continuous problem converges to f like dx^2
    (this pins the grid spacing of every grid type)."""
    L = 1.6
    errs = []
    for n in (16, 32, 64):
        x = _grid(bc, n, L)
        if bc == O.P:
            f, lam = np.cos(2 * np.pi * x / L), -(2 * np.pi / L) ** 2
        elif bc in (O.DR, O.DS):
            f, lam = np.sin(np.pi * x / L), -(np.pi / L) ** 2
        else:
            f, lam = np.cos(np.pi * x / L), -(np.pi / L) ** 2
        errs.append(np.max(np.abs(O.solve(lam * f, [bc], [L], O.FD2) - f)))
    ratios = np.array(errs[1:]) / np.array(errs[:-1])
    assert np.all((ratios > 0.22) & (ratios < 0.28)), ratios
