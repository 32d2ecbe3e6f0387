"""Seeded synthetic inputs for the Poisson-solve workloads.

This module is shared by the tests, the bench and the oracle checks.  It holds
input recipes only (random fields and the workload table); it contains none
of the solver's arithmetic and imports neither the oracle nor the CUDA
library.  All draws use numpy's PCG64 generator with a fixed seed.

The paper measures on no public data set: its runs are 512^3 and 256^3 grids
with periodic or staggered-Neumann conditions (Sec. 4) and a 16.3 M-cell
urban flow model (Sec. 5).  The workloads below are synthetic stand-ins with
the grid sizes and boundary-condition mixes of those runs.

Boundary-condition codes: 0 periodic (P), 1 Dirichlet regular (DR),
2 Dirichlet staggered (DS), 3 Neumann regular (NR), 4 Neumann staggered (NS).
Approximation codes: 0 pseudo-spectral (Table 3), 1 second-order finite
differences (Table 4).
"""

from __future__ import annotations

import math

import numpy as np

P, DR, DS, NR, NS = 0, 1, 2, 3, 4
SPECTRAL, FD2 = 0, 1


def rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def uniform_meanfree(shape, seed, dtype=np.float64):
    """i.i.d. U[-1, 1], arithmetic mean subtracted."""
    g = rng(seed).uniform(-1.0, 1.0, size=shape)
    g -= g.mean()
    return g.astype(dtype)


def normal_meanfree(shape, seed, dtype=np.float64):
    """i.i.d. N(0, 1), arithmetic mean subtracted."""
    g = rng(seed).standard_normal(size=shape, dtype=np.float64 if dtype == np.float64 else np.float32)
    g = g.astype(np.float64 if dtype == np.float64 else np.float32)
    g -= g.mean(dtype=np.float64)
    return g.astype(dtype)


def normal(shape, seed, dtype=np.float64):
    """i.i.d. N(0, 1) (no mean removal)."""
    g = rng(seed).standard_normal(size=shape, dtype=np.float64 if dtype == np.float64 else np.float32)
    return g.astype(dtype)


def smooth_random_field(shape, seed, slope=-3.0, noise=1e-3, dtype=np.float32):
    """Gaussian random field with power spectrum ~ |k|^slope plus white noise.

    White N(0,1) noise is filtered in Fourier space by |k|^(slope/2) (integer
    wavenumbers, k = 0 removed), scaled to unit variance, then noise*N(0,1)
    is added and the arithmetic mean subtracted.  Computed in FP32 slabs so
    that 1024^3 fits in a few host copies of the field.
    """
    import scipy.fft as sf

    gen = rng(seed)
    f = gen.standard_normal(size=shape, dtype=np.float32)
    spec = sf.rfftn(f, workers=-1)
    del f
    kk = [np.fft.fftfreq(n, 1.0 / n).astype(np.float32) for n in shape[:-1]]
    kk.append(np.fft.rfftfreq(shape[-1], 1.0 / shape[-1]).astype(np.float32))
    d = len(shape)
    # filter slab by slab along the first axis to bound temporaries
    tail = None
    if d >= 2:
        grids = np.meshgrid(*kk[1:], indexing="ij")
        tail = sum(gk.astype(np.float32) ** 2 for gk in grids)
        del grids
    for i0 in range(shape[0]):
        k2 = kk[0][i0] ** 2 + (tail if tail is not None else 0.0)
        k2 = np.asarray(k2, dtype=np.float32)
        with np.errstate(divide="ignore"):
            amp = np.where(k2 > 0, k2 ** np.float32(slope / 4.0), np.float32(0.0))
        spec[i0] *= amp
    field = sf.irfftn(spec, s=shape, workers=-1).astype(np.float32)
    del spec
    field /= np.float32(field.std(dtype=np.float64))
    field += np.float32(noise) * gen.standard_normal(size=shape, dtype=np.float32)
    field -= np.float32(field.mean(dtype=np.float64))
    return field.astype(dtype)


# Workload table.  n = (nx, ny, nz) as in the C interface; arrays are numpy
# shapes (nz, ny, nx), x fastest.
WORKLOADS = {
    # 32^3, periodic x,y,z, pseudo-spectral, FP64 on [0, 2 pi)^3
    "p3_spectral_32_f64": dict(
        n=(32, 32, 32), bcs=(P, P, P), Ls=(2 * math.pi,) * 3, approx=SPECTRAL,
        dtype="f64", gen=("uniform_meanfree", 1)),
    # 256^3 FP32 FD2, x periodic, y staggered Dirichlet, z staggered Neumann, dx = 1/256
    "mixed_fd2_256_f32": dict(
        n=(256, 256, 256), bcs=(P, DS, NS), Ls=(1.0, 1.0, 1.0), approx=FD2,
        dtype="f32", gen=("normal_meanfree", 2)),
    # 512^3 FP32 FD2, periodic x,y, staggered Neumann z: a profiling-size case
    # of the 1024^3 workload (fits a few GB on the device, still >> L2)
    "ppn_fd2_512_f32": dict(
        n=(512, 512, 512), bcs=(P, P, NS), Ls=(1.0, 1.0, 1.0), approx=FD2,
        dtype="f32", gen=("normal_meanfree", 3)),
    # 256 x 256 x 1024: the 1024-point z sweeps of the 1024^3 workload on a
    # field small enough for full profiler captures
    "ppn_fd2_256x256x1024_f32": dict(
        n=(256, 256, 1024), bcs=(P, P, NS), Ls=(1.0, 1.0, 4.0), approx=FD2,
        dtype="f32", gen=("normal_meanfree", 3)),
    # 512 x 512 x 1024: profiling case of the 1024-point z kernels with a
    # field (1 GiB) far larger than L2
    "ppn_fd2_512x512x1024_f32": dict(
        n=(512, 512, 1024), bcs=(P, P, NS), Ls=(1.0, 1.0, 2.0), approx=FD2,
        dtype="f32", gen=("normal_meanfree", 3)),
    # 1024^3 FP32 FD2, periodic x,y, staggered Neumann z, L = 1 per axis
    "ppn_fd2_1024_f32": dict(
        n=(1024, 1024, 1024), bcs=(P, P, NS), Ls=(1.0, 1.0, 1.0), approx=FD2,
        dtype="f32", gen=("smooth_random_field", 3)),
}

# Batched workload: 512 independent problems (see batch_problems), FP32, FD2.
BATCHES = {
    "batched_512_f32": dict(count=512, seed=4, dtype="f32", approx=FD2),
}


# Variable-coefficient problems div(a grad phi) = g (staggered Dirichlet on
# every wall) solved by CG preconditioned with the FD2 Poisson solve.
VC_PROBLEMS = {
    # 256^3 cells on the unit cube, a = exp(c s), s a unit-variance Gaussian
    # random field of correlation length 1/16, max(a)/min(a) = 100
    "pcg_vc_256_f64": dict(n=(256, 256, 256), Ls=(1.0, 1.0, 1.0), contrast=100.0, seed=5, tol=1e-8),
}


# Learned form: training pairs on a coarser grid from the same coefficient
# recipe (contrast drawn log-uniformly in [10, 100] per pair), evaluated on
# the 256^3 problem above and on held-out pairs of the training grid.
LEARNED = {
    "learned_pcg_256": dict(eval="pcg_vc_256_f64", n_train=(64, 64, 64), pairs=2000, holdout=16, seed=11,
                            contrast=(10.0, 100.0), arch=dict(channels=16, modes=12, layers=4),
                            batch=8, epochs=20, lr=2e-3, pair_tol=1e-6),
}


def learned_samples(n, count, seed, contrast=(10.0, 100.0)):
    """(a, g) host pairs for training: a = lognormal_coefficient with a
    contrast drawn log-uniformly from `contrast`, g standard normal; pair k
    uses coefficient seed 1000 + k and right-hand-side seed 5000 + k."""
    shape = tuple(reversed(n))
    r = rng(seed)
    out = []
    for k in range(count):
        c = float(np.exp(r.uniform(np.log(contrast[0]), np.log(contrast[1]))))
        out.append((lognormal_coefficient(shape, 1000 + k, c), normal(shape, 5000 + k)))
    return out


def gaussian_random_field(shape, seed, corr_len, Ls=None):
    """Unit-variance Gaussian random field with Gaussian covariance
    exp(-r^2 / (2 corr_len^2)) on a periodic box of lengths Ls (default 1 per
    axis): white N(0,1) noise filtered in Fourier space by the square root of
    the covariance's spectrum, exp(-|k|^2 corr_len^2 / 4) with k = 2 pi m / L,
    then scaled to unit sample variance (FP64)."""
    import scipy.fft as sf

    d = len(shape)
    Ls = Ls or (1.0,) * d
    f = rng(seed).standard_normal(size=shape)
    spec = sf.rfftn(f, workers=-1)
    k2 = 0.0
    for ax, n in enumerate(shape):
        L = Ls[d - 1 - ax]                              # numpy axis 0 is z (the last physical axis)
        m = np.fft.rfftfreq(n, 1.0 / n) if ax == d - 1 else np.fft.fftfreq(n, 1.0 / n)
        k = 2 * np.pi * m / L
        k2 = k2 + (k ** 2).reshape([-1 if i == ax else 1 for i in range(d)])
    spec *= np.exp(-k2 * corr_len ** 2 / 4.0)
    field = sf.irfftn(spec, s=shape, workers=-1)
    field -= field.mean()
    return field / field.std()


def lognormal_coefficient(shape, seed, contrast, corr_len=1.0 / 16):
    """Cell coefficients a = exp(c s) with s a unit-variance Gaussian random
    field of correlation length corr_len (gaussian_random_field) and c chosen
    so that max(a) / min(a) = contrast (c = ln(contrast) / (max s - min s)).
    FP32 (the coefficient is stored in FP32 by the solver)."""
    s = gaussian_random_field(shape, seed, corr_len)
    c = np.log(float(contrast)) / (s.max() - s.min())
    return np.exp(c * s).astype(np.float32)


def smooth_numbers(lo, hi, primes=(2, 3, 5, 7)):
    """Integers in [lo, hi] whose prime factors all lie in `primes`."""
    out = []
    for n in range(lo, hi + 1):
        m = n
        for p in primes:
            while m % p == 0:
                m //= p
        if m == 1:
            out.append(n)
    return out


def batch_problems(count=512, seed=4, n2d=(64, 2048), n3d=(32, 256), max_points=None):
    """Independent problems of the batched workload: half 2D with n in
    [64, 2048] per axis, half 3D with n in [32, 256] per axis, every n
    {2,3,5,7}-smooth; each axis draws its BC from all five kinds (P, DST-I,
    DST-II, DCT-I, DCT-II); FD2 eigenvalues; L = 1 per axis.  Returns a list
    of dicts (dims, n (x first), bcs, Ls, seed of g)."""
    r = rng(seed)
    s2 = smooth_numbers(*n2d)
    s3 = smooth_numbers(*n3d)
    probs = []
    while len(probs) < count:
        dims = 2 if r.random() < 0.5 else 3
        pool = s2 if dims == 2 else s3
        n = tuple(int(pool[r.integers(len(pool))]) for _ in range(dims))
        if max_points is not None and int(np.prod(n)) > max_points:
            continue
        bcs = tuple(int(r.integers(5)) for _ in range(dims))
        probs.append(dict(dims=dims, n=n, bcs=bcs, Ls=(1.0,) * dims, gseed=int(r.integers(1 << 31))))
    return probs


def make_input(name_or_spec, shape=None, dtype=None):
    """Seeded right-hand side g for a workload (numpy array, shape (nz,ny,nx))."""
    spec = WORKLOADS[name_or_spec] if isinstance(name_or_spec, str) else name_or_spec
    nx, ny, nz = spec["n"]
    shp = shape if shape is not None else (nz, ny, nx)
    dt = dtype if dtype is not None else (np.float64 if spec["dtype"] == "f64" else np.float32)
    kind, seed = spec["gen"]
    if kind == "uniform_meanfree":
        return uniform_meanfree(shp, seed, dt)
    if kind == "normal_meanfree":
        return normal_meanfree(shp, seed, dt)
    if kind == "smooth_random_field":
        return smooth_random_field(shp, seed, dtype=dt)
    raise ValueError(kind)
