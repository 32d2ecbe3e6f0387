"""FP64 CPU oracle of the spectral neural operator used with the PCG.

TEST INFRASTRUCTURE ONLY (same rules as oracle/poisson.py): only tests/,
__graft_entry__.smoke() and bench.py's CPU legs may import it; it shares no
code with the CUDA library.

The paper (Sec. 1) names the fast Poisson solve as a preconditioner for
div(a grad phi) = g; the learned operator below is this project's addition
on top of that PCG, not a method of the paper.  It maps per-cell features
of one problem to a correction of the FFT-Poisson solution:

  features  F = [g / rms(g), (log a - mean) / std(log a), phi0 / rms(phi0)],
            phi0 = (1/mean a) L_h^{-1} g, L_h the FD2 Laplacian with staggered
            Dirichlet walls (Table 4): the solution for the mean coefficient
  lifting   v_0 = P F + p                                (C x 3, C)
  layer l   vhat = S(v_l)  (truncated DST-II, K modes per axis)
            uhat[o, m] = sum_i R_l[m, o, i] vhat[i, m]    (m: K^3 modes)
            pre_l = W_l v_l + b_l + S_inv(uhat)
            v_{l+1} = gelu(pre_l) (l < L-1), pre_l (last layer)
  output    y = Q v_L + q
  guess     phi_init = phi0 + rms(phi0) y

The sine basis matches the walls (phi = 0 on every face, staggered grid).
Along an axis with n cells, S[m, j] = (2/n) sin(pi (m+1)(2j+1) / (2n)) and
S_inv[j, m] = sin(pi (m+1)(2j+1) / (2n)) for m < K: coefficients that do
not depend on the resolution, and S S_inv = I.  gelu is the tanh form
0.5 x (1 + tanh(sqrt(2/pi) (x + 0.044715 x^3))).

Arrays: activations (B, C, nz, ny, nx), x fastest, like the solver's fields.
Parameters: one flat vector in the order P, p, then per layer W, b, R
(R as (K^3, C, C) with the mode index m = (mz*K + my)*K + mx), then Q, q.
"""

from __future__ import annotations

import numpy as np

GELU_C = np.sqrt(2.0 / np.pi)


def n_params(C, K, L, F=3):
    return C * F + C + L * (C * C + C + K ** 3 * C * C) + C + 1


def unpack(theta, C, K, L, F=3):
    """Views of the flat parameter vector (see the module docstring)."""
    theta = np.asarray(theta, dtype=np.float64)
    assert theta.size == n_params(C, K, L, F)
    o = 0

    def take(shape):
        nonlocal o
        size = int(np.prod(shape))
        out = theta[o:o + size].reshape(shape)
        o += size
        return out

    P = take((C, F))
    p = take((C,))
    layers = []
    for _ in range(L):
        W = take((C, C))
        b = take((C,))
        R = take((K ** 3, C, C))
        layers.append((W, b, R))
    Q = take((C,))
    q = take((1,))
    return P, p, layers, Q, q


def sine_matrices(n, K):
    """Truncated DST-II analysis S (K x n) and synthesis S_inv (n x K)."""
    j = np.arange(n)
    m = np.arange(K)
    s = np.sin(np.pi * np.outer(m + 1, 2 * j + 1) / (2.0 * n))
    return (2.0 / n) * s, s.T.copy()


def _along(x, M, axis):
    """Apply matrix M (out x in) along `axis` of x."""
    x = np.moveaxis(x, axis, -1)
    y = x @ M.T
    return np.moveaxis(y, -1, axis)


def analysis(v, K):
    """S along x, y, z of v (..., nz, ny, nx) -> (..., K, K, K)."""
    nz, ny, nx = v.shape[-3:]
    for axis, n in ((-1, nx), (-2, ny), (-3, nz)):
        v = _along(v, sine_matrices(n, K)[0], axis)
    return v


def synthesis(vh, shape):
    """S_inv along x, y, z of vh (..., K, K, K) -> (..., nz, ny, nx)."""
    K = vh.shape[-1]
    nz, ny, nx = shape
    for axis, n in ((-1, nx), (-2, ny), (-3, nz)):
        vh = _along(vh, sine_matrices(n, K)[1], axis)
    return vh


def analysis_T(d, shape):
    """Adjoint of `analysis`: S^T along every axis, (..., K,K,K) -> grid."""
    K = d.shape[-1]
    nz, ny, nx = shape
    for axis, n in ((-1, nx), (-2, ny), (-3, nz)):
        d = _along(d, sine_matrices(n, K)[0].T, axis)
    return d


def synthesis_T(d, K):
    """Adjoint of `synthesis`: S_inv^T along every axis, grid -> (..., K,K,K)."""
    nz, ny, nx = d.shape[-3:]
    for axis, n in ((-1, nx), (-2, ny), (-3, nz)):
        d = _along(d, sine_matrices(n, K)[1].T, axis)
    return d


def gelu(x):
    return 0.5 * x * (1.0 + np.tanh(GELU_C * (x + 0.044715 * x ** 3)))


def gelu_grad(x):
    t = np.tanh(GELU_C * (x + 0.044715 * x ** 3))
    return 0.5 * (1.0 + t) + 0.5 * x * (1.0 - t * t) * GELU_C * (1.0 + 3 * 0.044715 * x * x)


def _mix(R, vh):
    """uhat[b, o, m] = sum_i R[m, o, i] vhat[b, i, m] on (B, C, K, K, K)."""
    B, C = vh.shape[:2]
    K = vh.shape[-1]
    flat = vh.reshape(B, C, K ** 3)
    return np.einsum("moi,bim->bom", R, flat).reshape(B, C, K, K, K)


def forward(theta, feats, C, K, L):
    """y (B, nz, ny, nx) and the cache for `backward`."""
    feats = np.asarray(feats, dtype=np.float64)
    P, p, layers, Q, q = unpack(theta, C, K, L, feats.shape[1])
    shape = feats.shape[-3:]
    v = np.einsum("cf,bf...->bc...", P, feats) + p[None, :, None, None, None]
    cache = {"feats": feats, "v": [], "vh": [], "pre": []}
    for l, (W, b, R) in enumerate(layers):
        vh = analysis(v, K)
        pre = (np.einsum("oi,bi...->bo...", W, v) + b[None, :, None, None, None]
               + synthesis(_mix(R, vh), shape))
        cache["v"].append(v)
        cache["vh"].append(vh)
        cache["pre"].append(pre)
        v = gelu(pre) if l < L - 1 else pre
    cache["vL"] = v
    y = np.einsum("c,bc...->b...", Q, v) + q[0]
    return y, cache


def backward(theta, cache, dy, C, K, L):
    """Gradient of sum(dy * y) with respect to theta (flat, same order)."""
    feats = cache["feats"]
    F = feats.shape[1]
    P, p, layers, Q, q = unpack(theta, C, K, L, F)
    shape = feats.shape[-3:]
    grads = []
    dQ = np.einsum("bzyx,bczyx->c", dy, cache["vL"])
    dq = np.array([dy.sum()])
    dv = Q[None, :, None, None, None] * dy[:, None]
    layer_grads = []
    for l in range(L - 1, -1, -1):
        W, b, R = layers[l]
        pre, v, vh = cache["pre"][l], cache["v"][l], cache["vh"][l]
        dpre = dv * gelu_grad(pre) if l < L - 1 else dv
        dW = np.einsum("bozyx,bizyx->oi", dpre, v)
        db = dpre.sum(axis=(0, 2, 3, 4))
        duh = synthesis_T(dpre, K)
        B = dpre.shape[0]
        duh_f = duh.reshape(B, C, K ** 3)
        vh_f = vh.reshape(B, C, K ** 3)
        dR = np.einsum("bom,bim->moi", duh_f, vh_f)
        dvh = np.einsum("moi,bom->bim", R, duh_f).reshape(B, C, K, K, K)
        dv = np.einsum("oi,bo...->bi...", W, dpre) + analysis_T(dvh, shape)
        layer_grads.append((dW, db, dR))
    dP = np.einsum("bczyx,bfzyx->cf", dv, feats)
    dp = dv.sum(axis=(0, 2, 3, 4))
    grads = [dP.ravel(), dp]
    for dW, db, dR in reversed(layer_grads):
        grads += [dW.ravel(), db, dR.ravel()]
    grads += [dQ, dq]
    return np.concatenate(grads)


def loss_and_grad(y, t):
    """Relative squared error sum (y - t)^2 / sum t^2 over the batch, and dL/dy."""
    den = float(np.sum(t * t))
    diff = y - t
    return float(np.sum(diff * diff)) / den, 2.0 * diff / den


def bf16_round(x):
    """Round FP32 values to bfloat16 (nearest, ties to even), returned as FP32."""
    x = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    u = x.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) >> 16 << 16
    return u.astype(np.uint32).view(np.float32)


def features(g, a, phi0):
    """Per-cell features of one problem (3, nz, ny, nx) and rms(phi0)."""
    g = np.asarray(g, dtype=np.float64)
    la = np.log(np.asarray(a, dtype=np.float64))
    phi0 = np.asarray(phi0, dtype=np.float64)
    rg = np.sqrt(np.mean(g * g))
    rp = np.sqrt(np.mean(phi0 * phi0))
    sd = np.std(la)
    return np.stack([g / rg, (la - la.mean()) / (sd if sd > 0 else 1.0), phi0 / rp]), rp
