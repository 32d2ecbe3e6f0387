"""FP64 CPU oracle for the variable-coefficient problem div(a grad phi) = g.

TEST INFRASTRUCTURE ONLY (same rules as oracle/poisson.py): only tests/,
__graft_entry__.smoke() and bench.py's CPU legs may import it; it shares no
code with the CUDA library.

Sec. 1 of the paper notes that the fast solver on a regular grid can serve
as a preconditioner for problems with non-constant coefficients,
div(a(x) grad phi) = g.  The paper gives no discretisation; the reading used
here (and by the CUDA path) is the cell-centred second-order one that
reduces to the Dirichlet-staggered FD2 Laplacian of Table 4 when a is
constant:

  (A phi)_i = sum_d [ a_{i+1/2} (phi_{i+e_d} - phi_i) - a_{i-1/2} (phi_i - phi_{i-e_d}) ] / dx_d^2

with the harmonic mean a_{i+1/2} = 2 a_i a_{i+e_d} / (a_i + a_{i+e_d}) on
interior faces, and on a boundary face the cell's own a with the ghost value
phi_ghost = -phi_i (phi = 0 on the face, staggered Dirichlet).  dx_d = L_d/n_d.

The solver is preconditioned CG on -A (symmetric positive definite) with the
preconditioner M^{-1} r = -(1/a_ref) L_h^{-1} r, L_h the FD2 staggered
Dirichlet Laplacian (oracle/poisson.py), in the flexible (Polak-Ribiere)
form.
"""

from __future__ import annotations

import numpy as np

from oracle import poisson as O


def _shift(a, axis, step):
    """a shifted by `step` cells along `axis`; out-of-range entries are NaN."""
    out = np.full_like(a, np.nan)
    n = a.shape[axis]
    src = [slice(None)] * a.ndim
    dst = [slice(None)] * a.ndim
    if step > 0:
        src[axis] = slice(step, n)
        dst[axis] = slice(0, n - step)
    else:
        src[axis] = slice(0, n + step)
        dst[axis] = slice(-step, n)
    out[tuple(dst)] = a[tuple(src)]
    return out


def apply_operator(phi, a, Ls):
    """(A phi) for cell coefficients a (same shape as phi; x is the last axis)."""
    phi = np.asarray(phi, dtype=np.float64)
    a = np.asarray(a, dtype=np.float64)
    d = phi.ndim
    out = np.zeros_like(phi)
    for ax_phys in range(d):
        ax = d - 1 - ax_phys
        dx = Ls[ax_phys] / phi.shape[ax]
        for step in (+1, -1):
            pn = _shift(phi, ax, step)
            an = _shift(a, ax, step)
            inside = ~np.isnan(pn)
            face = np.where(inside, 2.0 * a * np.where(inside, an, 1.0) / (a + np.where(inside, an, 1.0)), a)
            nb = np.where(inside, pn, -phi)
            out += face * (nb - phi) / dx ** 2
    return out


def precondition(r, Ls, a_ref):
    """M^{-1} r = -(1/a_ref) L_h^{-1} r with the DS FD2 Laplacian (Table 4)."""
    d = r.ndim
    return -O.solve(r, (O.DS,) * d, Ls, O.FD2) / a_ref


def pcg(g, a, Ls, a_ref=None, tol=1e-8, maxit=500, x0=None):
    """Flexible PCG for A phi = g.  Returns (phi, iterations, relative residual)."""
    g = np.asarray(g, dtype=np.float64)
    a = np.asarray(a, dtype=np.float64)
    a_ref = float(np.mean(a)) if a_ref is None else a_ref
    b = -g
    x = np.zeros_like(g) if x0 is None else np.array(x0, dtype=np.float64)
    r = b + apply_operator(x, a, Ls)          # b - K x with K = -A
    bnorm = np.linalg.norm(b)
    if bnorm == 0:
        return x, 0, 0.0
    z = precondition(r, Ls, a_ref)
    p = z.copy()
    rz = float(np.sum(r * z))
    for it in range(1, maxit + 1):
        q = -apply_operator(p, a, Ls)
        alpha = rz / float(np.sum(p * q))
        x += alpha * p
        r -= alpha * q
        rel = np.linalg.norm(r) / bnorm
        if rel <= tol:
            return x, it, rel
        z_new = precondition(r, Ls, a_ref)
        rz_new = float(np.sum(r * z_new))
        beta = float(np.sum(r * (z_new - z))) / rz
        p = z_new + beta * p
        z, rz = z_new, rz_new
    return x, maxit, np.linalg.norm(r) / bnorm
