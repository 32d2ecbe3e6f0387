"""Pins of the variable-coefficient oracle (CPU): for constant a the operator
is a times the Table 4 staggered-Dirichlet stencil; it is symmetric and
negative definite for any positive a; the eigenpairs of the constant case
are the Table 1 DST-II basis; the PCG solution satisfies the discrete
equation independently of the algorithm; dense solves agree."""

import numpy as np
import pytest

from oracle import poisson as O
from oracle import vc_operator as V


def test_constant_coefficient_is_scaled_fd2_laplacian():
    r = np.random.default_rng(0)
    phi = r.standard_normal((5, 6, 7))
    Ls = (1.0, 1.3, 0.7)
    np.testing.assert_allclose(V.apply_operator(phi, np.full_like(phi, 2.5), Ls),
                               2.5 * O.laplacian_fd2(phi, (O.DS,) * 3, Ls), rtol=1e-12, atol=1e-9)


def test_constant_coefficient_eigenvalues_are_table4():
    n, L, a = 9, 1.4, 3.0
    basis = O.backward_matrix(O.DS, n)
    lam = O.eigenvalues(O.DS, n, L, O.FD2)
    for k in range(n):
        v = basis[:, k]
        np.testing.assert_allclose(V.apply_operator(v, np.full(n, a), [L]), a * lam[k] * v, atol=1e-9)


def _dense(shape, a, Ls):
    N = int(np.prod(shape))
    A = np.zeros((N, N))
    for i in range(N):
        e = np.zeros(N)
        e[i] = 1.0
        A[:, i] = V.apply_operator(e.reshape(shape), a, Ls).ravel()
    return A


def test_operator_symmetric_negative_definite():
    r = np.random.default_rng(1)
    shape = (4, 5, 6)
    a = np.exp(r.standard_normal(shape))
    A = _dense(shape, a, (1.0, 0.8, 1.2))
    np.testing.assert_allclose(A, A.T, atol=1e-10 * np.abs(A).max())
    assert np.max(np.linalg.eigvalsh(A)) < 0


def test_harmonic_face_coefficient_by_hand_1d():
    a = np.array([1.0, 4.0, 2.0])
    phi = np.array([0.5, -1.0, 2.0])
    dx = 1.0 / 3
    h01 = 2 * 1.0 * 4.0 / 5.0
    h12 = 2 * 4.0 * 2.0 / 6.0
    expect = np.array([
        (h01 * (phi[1] - phi[0]) - 1.0 * (phi[0] + phi[0])) / dx ** 2,
        (h12 * (phi[2] - phi[1]) - h01 * (phi[1] - phi[0])) / dx ** 2,
        (2.0 * (-phi[2] - phi[2]) - h12 * (phi[2] - phi[1])) / dx ** 2,
    ])
    np.testing.assert_allclose(V.apply_operator(phi, a, [1.0]), expect, rtol=1e-14)


@pytest.mark.parametrize("contrast", [1.0, 30.0])
def test_pcg_solves_discrete_equation_and_matches_dense(contrast):
    r = np.random.default_rng(2)
    shape = (6, 7, 8)
    s = r.standard_normal(shape)
    a = np.exp(np.log(contrast) * (s - s.min()) / (s.max() - s.min()))
    g = r.standard_normal(shape)
    Ls = (1.0, 1.0, 1.0)
    phi, it, rel = V.pcg(g, a, Ls, tol=1e-12)
    assert rel <= 1e-12
    res = V.apply_operator(phi, a, Ls) - g
    assert np.linalg.norm(res) <= 1e-11 * np.linalg.norm(g)
    x = np.linalg.solve(_dense(shape, a, Ls), g.ravel())
    assert O.rel_max_error(phi.ravel(), x) < 1e-10
    if contrast == 1.0:
        assert it <= 2          # the preconditioner is the exact inverse


def test_sparse_probe_reproduces_operator():
    from tests._vc import sparse_operator
    r = np.random.default_rng(4)
    shape = (5, 6, 7)
    a = np.exp(r.standard_normal(shape))
    Ls = (1.0, 0.9, 1.1)
    A = sparse_operator(a, Ls)
    np.testing.assert_allclose(A.toarray(), _dense(shape, a, Ls), rtol=0, atol=1e-12 * np.abs(A).max())


def test_pcg_matches_sparse_lu_on_a_larger_grid():
    import scipy.sparse.linalg as spla
    from tests._vc import sparse_operator
    r = np.random.default_rng(5)
    shape = (12, 14, 16)
    s = r.standard_normal(shape)
    a = 100.0 ** ((s - s.min()) / (s.max() - s.min()) - 0.5)
    g = r.standard_normal(shape)
    Ls = (1.5, 1.0, 0.75)
    phi, it, rel = V.pcg(g, a, Ls, tol=1e-12, maxit=300)
    x = spla.splu(sparse_operator(a, Ls)).solve(g.ravel())
    assert rel <= 1e-12 and it < 300
    assert O.rel_max_error(phi.ravel(), x) < 1e-9
