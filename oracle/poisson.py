"""FP64 CPU oracle for the direct FFT Poisson solve of PoisFFT (arXiv 1409.8116).

TEST INFRASTRUCTURE ONLY.  This module exists to check the CUDA library; it is
not part of it.  Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``
(its CPU-baseline and reference legs) may import or run it.  It shares no code,
tables or helpers with ``paper_1409_8116_gb300`` and imports nothing from it.

What it computes -- the three-step algorithm of Sec. 2.1 ("the whole algorithm
of the Poisson solver can be summarized as"), extended to several dimensions
as a sequence of 1D transforms (Sec. 2.3):

1. For every axis, the forward transform of Table 2 chosen by that axis's
   boundary condition (BC), with the transform formulas of Table 1 and the
   DFT of Eq. (DFT), which carries the 1/n factor.
2. Division by the eigenvalue lambda = lambda_x + lambda_y + lambda_z
   (Sec. 2.3), with the 1D eigenvalues of Table 3 (pseudo-spectral) or
   Table 4 (second-order finite differences).
3. If every axis has a zero eigenvalue (periodic or Neumann), the singular
   all-zero mode is set to 0 (the paper is silent here; see READINGS).
4. For every axis, the backward transform of Table 2 (IDFT of Eq. (IDFT), or
   the scaled real transforms), then the real part.

Two realisations of the per-axis transform step are offered:

* ``method="dense"`` (the definition): the n x n matrix of the Table 1 /
  Eq. (DFT) formula, built entry by entry, applied along the axis with a
  matrix product.  Cost O(N * sum(n)).
* ``method="fft"``: the same Table 1 transforms through ``scipy.fft``
  (library FFT primitives, whose unnormalised definitions coincide with
  Table 1).  Used only where the dense form would take minutes (256^3 and
  up).  Pinned against the dense form in the tests.

Sines and cosines of the matrices are evaluated with exactly reduced
arguments: sin(pi*m/d) with the integer m reduced modulo 2d and folded into
the first quadrant before libm is called.

READINGS of points where the paper is silent, garbled or ambiguous:

* Table 3, periodic row: the printed threshold "k < [n/2]-1" would give
  m = 5 for n = 8, k = 3.  Reading: lambda_k = -(2 pi m_k / L)^2 with
  m_k = min(k, n - k), the aliased wavenumber of smallest magnitude.
* Zero mode: singular iff every axis is P, NR or NS.  The all-zero
  coefficient is set to 0, which removes the null-space component of g
  and fixes phi to zero (trapezoid-weighted along NR axes) mean.
* dx per grid (Sec. 2.1 grids): P and staggered dx = L/n, Dirichlet
  regular dx = L/(n+1), Neumann regular dx = L/(n-1).
* Normalisation: 1/n on the forward DFT (Eq. DFT) and the Table 2 factors
  on the backward real transforms.
"""

from __future__ import annotations

import math

import numpy as np

# Boundary-condition codes (Table 2 rows): periodic, Dirichlet regular,
# Dirichlet staggered, Neumann regular, Neumann staggered.
P, DR, DS, NR, NS = 0, 1, 2, 3, 4
BC_NAMES = {P: "P", DR: "DR", DS: "DS", NR: "NR", NS: "NS"}
SPECTRAL, FD2 = 0, 1


# ---------------------------------------------------------------------------
# exactly reduced trigonometry
# ---------------------------------------------------------------------------

def _sincos_pi_frac(m, d):
    """Return (sin(pi*m/d), cos(pi*m/d)) for integer array m and integer d > 0.

    m is reduced exactly modulo 2d; the angle is folded into [0, pi/4] by
    quadrant and octant symmetries before libm sin/cos are called in FP64.
    """
    m = np.asarray(m, dtype=np.int64)
    d = int(d)
    r = np.mod(m, 2 * d)                       # angle = pi*r/d in [0, 2pi)
    q = (2 * r) // d                           # quadrant 0..3
    rr = 2 * r - q * d                         # angle = q*pi/2 + pi*rr/(2d), rr in [0, d)
    flip = 2 * rr > d                          # fold (pi/4, pi/2) onto [0, pi/4)
    rf = np.where(flip, d - rr, rr)
    phi = np.pi * rf.astype(np.float64) / (2.0 * d)
    s0, c0 = np.sin(phi), np.cos(phi)
    s1 = np.where(flip, c0, s0)                # sin of pi*rr/(2d)
    c1 = np.where(flip, s0, c0)
    sin_t = np.choose(q, [s1, c1, -s1, -c1])
    cos_t = np.choose(q, [c1, -s1, -c1, s1])
    return sin_t, cos_t


def sinpi(m, d):
    return _sincos_pi_frac(m, d)[0]


def cospi(m, d):
    return _sincos_pi_frac(m, d)[1]


# ---------------------------------------------------------------------------
# Table 1 / Eq. (DFT): the 1D transform matrices
# ---------------------------------------------------------------------------

def dft_matrix(n):
    """Eq. (DFT): F[k, j] = (1/n) exp(-2 pi i k j / n)."""
    k = np.arange(n)[:, None]
    j = np.arange(n)[None, :]
    s, c = _sincos_pi_frac(2 * k * j, n)
    return (c - 1j * s) / n


def idft_matrix(n):
    """Eq. (IDFT): B[j, k] = exp(+2 pi i k j / n)."""
    j = np.arange(n)[:, None]
    k = np.arange(n)[None, :]
    s, c = _sincos_pi_frac(2 * k * j, n)
    return c + 1j * s


def dst1_matrix(n):
    """Table 1, DST-I: f^_k = 2 sum_j f_j sin(pi (j+1)(k+1)/(n+1))."""
    k = np.arange(n)[:, None]
    j = np.arange(n)[None, :]
    return 2.0 * sinpi((j + 1) * (k + 1), n + 1)


def dst2_matrix(n):
    """Table 1, DST-II: f^_k = 2 sum_j f_j sin(pi (j+1/2)(k+1)/n)."""
    k = np.arange(n)[:, None]
    j = np.arange(n)[None, :]
    return 2.0 * sinpi((2 * j + 1) * (k + 1), 2 * n)


def dst3_matrix(n):
    """Table 1, DST-III: f^_k = (-1)^k f_{n-1} + 2 sum_{j<=n-2} f_j sin(pi (j+1)(k+1/2)/n)."""
    k = np.arange(n)[:, None]
    j = np.arange(n)[None, :]
    m = 2.0 * sinpi((j + 1) * (2 * k + 1), 2 * n)
    m[:, n - 1] = np.where(np.arange(n) % 2 == 0, 1.0, -1.0)
    return m


def dct1_matrix(n):
    """Table 1, DCT-I: f^_k = f_0 + (-1)^k f_{n-1} + 2 sum_{j=1}^{n-2} f_j cos(pi j k/(n-1))."""
    if n < 2:
        raise ValueError("DCT-I needs n >= 2")
    k = np.arange(n)[:, None]
    j = np.arange(n)[None, :]
    m = 2.0 * cospi(j * k, n - 1)
    m[:, 0] = 1.0
    m[:, n - 1] = np.where(np.arange(n) % 2 == 0, 1.0, -1.0)
    return m


def dct2_matrix(n):
    """Table 1, DCT-II: f^_k = 2 sum_j f_j cos(pi (j+1/2) k/n)."""
    k = np.arange(n)[:, None]
    j = np.arange(n)[None, :]
    return 2.0 * cospi((2 * j + 1) * k, 2 * n)


def dct3_matrix(n):
    """Table 1, DCT-III: f^_k = f_0 + 2 sum_{j=1}^{n-1} f_j cos(pi j (k+1/2)/n)."""
    k = np.arange(n)[:, None]
    j = np.arange(n)[None, :]
    m = 2.0 * cospi(j * (2 * k + 1), 2 * n)
    m[:, 0] = 1.0
    return m


def forward_matrix(bc, n):
    """Table 2, 'forward' column."""
    if bc == P:
        return dft_matrix(n)
    if bc == DR:
        return dst1_matrix(n)
    if bc == DS:
        return dst2_matrix(n)
    if bc == NR:
        return dct1_matrix(n)
    if bc == NS:
        return dct2_matrix(n)
    raise ValueError(f"unknown bc {bc}")


def backward_matrix(bc, n):
    """Table 2, 'backward' column, including its scale factor."""
    if bc == P:
        return idft_matrix(n)
    if bc == DR:
        return dst1_matrix(n) / (2.0 * (n + 1))
    if bc == DS:
        return dst3_matrix(n) / (2.0 * n)
    if bc == NR:
        return dct1_matrix(n) / (2.0 * (n - 1))
    if bc == NS:
        return dct3_matrix(n) / (2.0 * n)
    raise ValueError(f"unknown bc {bc}")


# ---------------------------------------------------------------------------
# grids and eigenvalues (Sec. 2.1 grids; Tables 3 and 4)
# ---------------------------------------------------------------------------

def grid_spacing(bc, n, L):
    """dx of the Sec. 2.1 grids: periodic x_j = jL/n, Dirichlet regular
    x_j = (j+1)L/(n+1), Neumann regular x_j = jL/(n-1), staggered
    x_j = (j+1/2)L/n."""
    if bc in (P, DS, NS):
        return L / n
    if bc == DR:
        return L / (n + 1)
    if bc == NR:
        return L / (n - 1)
    raise ValueError(f"unknown bc {bc}")


def eigenvalues(bc, n, L, approx):
    """1D Laplacian eigenvalues: Table 3 (SPECTRAL) or Table 4 (FD2)."""
    k = np.arange(n)
    if approx == SPECTRAL:
        if bc == P:
            m = np.minimum(k, n - k)           # reading of the garbled threshold
            return -(2.0 * math.pi * m / L) ** 2
        if bc in (DR, DS):
            return -(math.pi * (k + 1) / L) ** 2
        if bc in (NR, NS):
            return -(math.pi * k / L) ** 2
    elif approx == FD2:
        dx = grid_spacing(bc, n, L)
        if bc == P:
            s = sinpi(k, n)
        elif bc == DR:
            s = sinpi(k + 1, 2 * (n + 1))
        elif bc == DS:
            s = sinpi(k + 1, 2 * n)
        elif bc == NR:
            s = sinpi(k, 2 * (n - 1))
        elif bc == NS:
            s = sinpi(k, 2 * n)
        else:
            raise ValueError(f"unknown bc {bc}")
        return -(2.0 * s / dx) ** 2
    raise ValueError(f"unknown approx {approx} / bc {bc}")


def is_singular(bcs):
    """Every axis has lambda_0 = 0 (P, NR, NS) -> the zero mode is singular."""
    return all(b in (P, NR, NS) for b in bcs)


# ---------------------------------------------------------------------------
# the solve
# ---------------------------------------------------------------------------

def _apply_matrix(mat, a, axis):
    """Apply a 1D transform matrix along one array axis (matrix product)."""
    if a.ndim == 1:
        return mat @ a
    moved = np.moveaxis(a, axis, -2)
    out = np.matmul(mat, moved)
    return np.moveaxis(out, -2, axis)


def _fft_forward(bc, a, axis):
    import scipy.fft as sf
    n = a.shape[axis]
    if bc == P:
        return sf.fft(a, axis=axis, workers=-1) / n
    if bc == DR:
        return sf.dst(a, type=1, axis=axis, workers=-1)
    if bc == DS:
        return sf.dst(a, type=2, axis=axis, workers=-1)
    if bc == NR:
        return sf.dct(a, type=1, axis=axis, workers=-1)
    if bc == NS:
        return sf.dct(a, type=2, axis=axis, workers=-1)
    raise ValueError(bc)


def _fft_backward(bc, a, axis):
    import scipy.fft as sf
    n = a.shape[axis]
    if bc == P:
        return sf.ifft(a, axis=axis, workers=-1) * n
    if bc == DR:
        return sf.dst(a, type=1, axis=axis, workers=-1) / (2.0 * (n + 1))
    if bc == DS:
        return sf.dst(a, type=3, axis=axis, workers=-1) / (2.0 * n)
    if bc == NR:
        return sf.dct(a, type=1, axis=axis, workers=-1) / (2.0 * (n - 1))
    if bc == NS:
        return sf.dct(a, type=3, axis=axis, workers=-1) / (2.0 * n)
    raise ValueError(bc)


def _check_args(g, bcs, Ls):
    d = g.ndim
    if not (1 <= d <= 3):
        raise ValueError("dims must be 1..3")
    if len(bcs) != d or len(Ls) != d:
        raise ValueError("one bc and one L per axis")
    for a in range(d):
        n = g.shape[d - 1 - a]
        if bcs[a] == NR and n < 2:
            raise ValueError("Neumann regular needs n >= 2")


def eigenvalue_grid(shape, bcs, Ls, approx):
    """lambda_{k1 k2 k3} = lambda_{k1} + lambda_{k2} + lambda_{k3} (Sec. 2.3),
    as an array of the given numpy shape (x is the last numpy axis)."""
    d = len(shape)
    lam = np.zeros(shape)
    for a in range(d):
        ax = d - 1 - a
        la = eigenvalues(bcs[a], shape[ax], Ls[a], approx)
        bshape = [1] * d
        bshape[ax] = shape[ax]
        lam = lam + la.reshape(bshape)
    return lam


def spectrum(g, bcs, Ls, approx, method="dense"):
    """Steps 1-3: the coefficients psi^ = g^ / lambda (zero mode fixed).

    g is a numpy array of shape (nz, ny, nx) / (ny, nx) / (nx,), x fastest;
    bcs[a], Ls[a] for axis a = 0 (x), 1 (y), 2 (z).
    """
    g = np.asarray(g, dtype=np.float64)
    _check_args(g, bcs, Ls)
    d = g.ndim
    a = g.astype(np.complex128) if P in bcs else g.copy()
    for ax_phys in range(d):
        ax = d - 1 - ax_phys
        bc = bcs[ax_phys]
        if method == "dense":
            a = _apply_matrix(forward_matrix(bc, g.shape[ax]), a, ax)
        else:
            a = _fft_forward(bc, a, ax)
    lam = eigenvalue_grid(g.shape, bcs, Ls, approx)
    zero = (0,) * d
    if is_singular(bcs):
        lam[zero] = 1.0
        psi = a / lam
        psi[zero] = 0.0
    else:
        psi = a / lam
    return psi


def synthesis(psi, bcs, method="dense"):
    """Step 4: backward transforms of Table 2 along every axis."""
    d = psi.ndim
    a = psi
    for ax_phys in range(d):
        ax = d - 1 - ax_phys
        bc = bcs[ax_phys]
        if method == "dense":
            a = _apply_matrix(backward_matrix(bc, psi.shape[ax]), a, ax)
        else:
            a = _fft_backward(bc, a, ax)
    return a


def solve(g, bcs, Ls, approx, method="dense", return_imag=False):
    """phi with lap_h(phi) = g on the grid (Sec. 2.1 algorithm, Sec. 2.3 in nD).

    Returns the real FP64 solution; with return_imag=True also the largest
    |imaginary part| left by the complex periodic path.
    """
    psi = spectrum(g, bcs, Ls, approx, method)
    phi = synthesis(psi, bcs, method)
    if np.iscomplexobj(phi):
        imag = float(np.max(np.abs(phi.imag))) if phi.size else 0.0
        phi = np.ascontiguousarray(phi.real)
    else:
        imag = 0.0
    return (phi, imag) if return_imag else phi


# ---------------------------------------------------------------------------
# the discrete operator itself (Eq. FD2-Laplace / FD2-matrix), for checks
# ---------------------------------------------------------------------------

def _ghost_pad(a, bc, axis):
    """Extend a by one ghost layer on each side of `axis` by the BC rule.

    Rules (reading of how Eq. FD2-Laplace meets each boundary; they are the
    ones whose eigenvectors are the Table 2 bases):
      P:  wrap around;
      DR: phi_{-1} = phi_n = 0 (the boundary nodes carry phi = 0);
      DS: phi_{-1} = -phi_0, phi_n = -phi_{n-1} (zero on the cell face);
      NR: phi_{-1} = phi_1, phi_n = phi_{n-2} (even reflection at a node);
      NS: phi_{-1} = phi_0, phi_n = phi_{n-1} (zero gradient on the face).
    """
    n = a.shape[axis]
    take = lambda i: np.take(a, [i], axis=axis)
    if bc == P:
        lo, hi = take(n - 1), take(0)
    elif bc == DR:
        lo, hi = np.zeros_like(take(0)), np.zeros_like(take(0))
    elif bc == DS:
        lo, hi = -take(0), -take(n - 1)
    elif bc == NR:
        lo, hi = take(1 if n > 1 else 0), take(n - 2 if n > 1 else 0)
    elif bc == NS:
        lo, hi = take(0), take(n - 1)
    else:
        raise ValueError(bc)
    return np.concatenate([lo, a, hi], axis=axis)


def laplacian_fd2(phi, bcs, Ls):
    """Direct application of the second-order stencil of Eq. (FD2-Laplace)
    per axis with the ghost rules above: (phi_{j+1} - 2 phi_j + phi_{j-1})/dx^2.
    Independent of every transform in this module."""
    phi = np.asarray(phi, dtype=np.float64)
    d = phi.ndim
    out = np.zeros_like(phi)
    for ax_phys in range(d):
        ax = d - 1 - ax_phys
        n = phi.shape[ax]
        dx = grid_spacing(bcs[ax_phys], n, Ls[ax_phys])
        pad = _ghost_pad(phi, bcs[ax_phys], ax)
        lo = np.take(pad, np.arange(0, n), axis=ax)
        hi = np.take(pad, np.arange(2, n + 2), axis=ax)
        out += (hi - 2.0 * phi + lo) / dx ** 2
    return out


def null_weights_1d(bc, n):
    """Weights of the discrete mean that the zero-mode fix sets to zero along
    one axis: the k = 0 row of the Table 2 forward transform (all ones for
    P/NS, trapezoid 1/2, 1, ..., 1, 1/2 for NR), normalised to sum 1."""
    if bc in (P, NS):
        w = np.ones(n)
    elif bc == NR:
        w = np.ones(n)
        w[0] = w[-1] = 0.5
    else:
        raise ValueError("axis has no null space")
    return w / w.sum()


def null_weights(shape, bcs):
    d = len(shape)
    w = np.ones(shape)
    for a in range(d):
        ax = d - 1 - a
        bshape = [1] * d
        bshape[ax] = shape[ax]
        w = w * null_weights_1d(bcs[a], shape[ax]).reshape(bshape)
    return w


def project_range(g, bcs):
    """The part of g that lies in the range of the singular operator, i.e.
    what the zero-mode fix leaves of g: g - (weighted mean of g) * 1."""
    g = np.asarray(g, dtype=np.float64)
    if not is_singular(bcs):
        return g
    w = null_weights(g.shape, bcs)
    return g - float(np.sum(w * g))


def weighted_mean(phi, bcs):
    """Weighted mean of phi with the null_weights of a singular problem."""
    return float(np.sum(null_weights(phi.shape, bcs) * phi))


def rel_max_error(x, ref):
    """||x - ref||_inf / ||ref||_inf (normwise max relative error)."""
    x = np.asarray(x, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    den = float(np.max(np.abs(ref))) if ref.size else 0.0
    num = float(np.max(np.abs(x - ref))) if ref.size else 0.0
    return num / den if den > 0 else num
