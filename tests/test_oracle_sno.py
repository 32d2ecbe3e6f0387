"""Pins of the spectral-neural-operator oracle (CPU).

* The truncated sine matrices against scipy's DST-II / DST-III.
* The separable analysis / synthesis against brute-force sums over 3D sine
  basis functions.
* The forward pass against a cell-by-cell evaluation written from the
  definition with explicit loops (tiny sizes).
* The backward pass against central finite differences of the loss, for
  every parameter group.
* bfloat16 rounding against torch's conversion.
"""

import itertools

import numpy as np
import pytest
import scipy.fft as sf

from oracle import sno as S


def test_sine_matrices_match_scipy_dst():
    n, K = 11, 4
    A, Sinv = S.sine_matrices(n, K)
    x = np.random.default_rng(0).standard_normal(n)
    np.testing.assert_allclose(A @ x, sf.dst(x, type=2)[:K] / n, rtol=1e-13, atol=1e-14)
    c = np.random.default_rng(1).standard_normal(K)
    # DST-III of the zero-padded coefficients is twice the synthesis
    np.testing.assert_allclose(Sinv @ c, 0.5 * sf.dst(np.pad(c, (0, n - K)), type=3), rtol=1e-13, atol=1e-14)
    np.testing.assert_allclose(A @ Sinv, np.eye(K), atol=1e-14)


def test_analysis_synthesis_brute_force():
    r = np.random.default_rng(2)
    shape, K = (5, 4, 6), 3
    v = r.standard_normal(shape)
    nz, ny, nx = shape

    def basis(m, j, n):
        return np.sin(np.pi * (m + 1) * (2 * j + 1) / (2 * n))

    vh = S.analysis(v[None], K)[0]
    u = r.standard_normal((K, K, K))
    syn = S.synthesis(u[None], shape)[0]
    for mz, my, mx in itertools.product(range(K), repeat=3):
        ref = sum(v[z, y, x] * basis(mz, z, nz) * basis(my, y, ny) * basis(mx, x, nx)
                  for z in range(nz) for y in range(ny) for x in range(nx)) * 8.0 / (nx * ny * nz)
        assert abs(vh[mz, my, mx] - ref) < 1e-12
    for z, y, x in itertools.product(range(nz), range(ny), range(nx)):
        ref = sum(u[mz, my, mx] * basis(mz, z, nz) * basis(my, y, ny) * basis(mx, x, nx)
                  for mz in range(K) for my in range(K) for mx in range(K))
        assert abs(syn[z, y, x] - ref) < 1e-12


def _random_case(seed, B=2, C=3, K=2, L=2, shape=(4, 3, 5)):
    r = np.random.default_rng(seed)
    theta = 0.5 * r.standard_normal(S.n_params(C, K, L))
    feats = r.standard_normal((B, 3) + shape)
    return theta, feats, (C, K, L)


def test_forward_cell_by_cell():
    theta, feats, (C, K, L) = _random_case(3, B=1)
    P, p, layers, Q, q = S.unpack(theta, C, K, L)
    nz, ny, nx = feats.shape[-3:]

    def basis(m, j, n):
        return np.sin(np.pi * (m + 1) * (2 * j + 1) / (2 * n))

    cells = list(itertools.product(range(nz), range(ny), range(nx)))
    modes = list(itertools.product(range(K), repeat=3))
    v = {cell: [sum(P[c, f] * feats[0, f][cell] for f in range(3)) + p[c] for c in range(C)] for cell in cells}
    for l, (W, b, R) in enumerate(layers):
        vh = {m: [sum(v[cell][i] * basis(m[0], cell[0], nz) * basis(m[1], cell[1], ny) * basis(m[2], cell[2], nx)
                      for cell in cells) * 8.0 / (nx * ny * nz) for i in range(C)] for m in modes}
        uh = {m: [sum(R[(m[0] * K + m[1]) * K + m[2], o, i] * vh[m][i] for i in range(C)) for o in range(C)]
              for m in modes}
        new = {}
        for cell in cells:
            out = []
            for o in range(C):
                spec = sum(uh[m][o] * basis(m[0], cell[0], nz) * basis(m[1], cell[1], ny) * basis(m[2], cell[2], nx)
                           for m in modes)
                pre = sum(W[o, i] * v[cell][i] for i in range(C)) + b[o] + spec
                out.append(S.gelu(pre) if l < L - 1 else pre)
            new[cell] = out
        v = new
    y_ref = np.array([sum(Q[c] * v[cell][c] for c in range(C)) + q[0] for cell in cells]).reshape(nz, ny, nx)
    y, _ = S.forward(theta, feats, C, K, L)
    np.testing.assert_allclose(y[0], y_ref, rtol=1e-12, atol=1e-12)


def test_backward_matches_finite_differences():
    theta, feats, (C, K, L) = _random_case(4)
    t = np.random.default_rng(5).standard_normal((feats.shape[0],) + feats.shape[-3:])

    def loss(th):
        y, _ = S.forward(th, feats, C, K, L)
        return S.loss_and_grad(y, t)[0]

    y, cache = S.forward(theta, feats, C, K, L)
    _, dy = S.loss_and_grad(y, t)
    grad = S.backward(theta, cache, dy, C, K, L)
    # every parameter group: P, p, (W, b, R) per layer, Q, q
    sizes = [C * 3, C] + [C * C, C, K ** 3 * C * C] * L + [C, 1]
    starts = np.cumsum([0] + sizes[:-1])
    r = np.random.default_rng(6)
    h = 1e-6
    for st, sz in zip(starts, sizes):
        for idx in st + r.choice(sz, size=min(sz, 4), replace=False):
            e = np.zeros_like(theta)
            e[idx] = h
            fd = (loss(theta + e) - loss(theta - e)) / (2 * h)
            assert abs(fd - grad[idx]) <= 1e-6 * max(1.0, abs(fd)), (idx, fd, grad[idx])


def test_gelu_grad_finite_differences():
    x = np.linspace(-4, 4, 41)
    h = 1e-6
    np.testing.assert_allclose(S.gelu_grad(x), (S.gelu(x + h) - S.gelu(x - h)) / (2 * h), atol=1e-8)


def test_bf16_round_matches_torch():
    torch = pytest.importorskip("torch")
    r = np.random.default_rng(7)
    x = np.concatenate([r.standard_normal(10000).astype(np.float32) * 10.0 ** r.integers(-8, 8, 10000),
                        np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -2.5, 0.0], np.float32)])
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy()
    np.testing.assert_array_equal(S.bf16_round(x), ref)


def test_features_are_scale_invariant_in_g():
    r = np.random.default_rng(8)
    shape = (4, 5, 6)
    g, a, phi0 = r.standard_normal(shape), np.exp(r.standard_normal(shape)), r.standard_normal(shape)
    f1, rp1 = S.features(g, a, phi0)
    f2, rp2 = S.features(3.0 * g, a, 3.0 * phi0)
    np.testing.assert_allclose(f1, f2, rtol=1e-13)
    assert abs(rp2 - 3.0 * rp1) < 1e-12
