"""Training and use of the spectral neural operator that supplies the
initial guess of the FFT-preconditioned CG for div(a grad phi) = g.

The paper (Sec. 1) names the fast Poisson solve as a preconditioner for
variable coefficients; the network is this library's addition on top of
that PCG.  Every numerical step runs in the library's kernels: this module
only orders the calls (pair generation with the library's own PCG, the
network's forward and backward passes, the loss and the Adam step) and
holds device memory in torch tensors.

    pairs = generate_pairs(n, Ls, samples)          # (feats, targets) on the device
    theta, hist = train(pairs, n, epochs=20)         # FP32 parameters (numpy)
    sno = load_network(n, theta)                     # batch-1 inference object
    pcg.learned_guess(sno, phi, g, corrections=1)    # then pcg.solve(phi, g, ...)
"""

from __future__ import annotations

import math
import time

import numpy as np

from . import binding as pb

DEFAULT_ARCH = dict(channels=16, modes=12, layers=4)


def init_params(channels=16, modes=12, layers=4, seed=0):
    """Seeded initial parameters (FP32): normal weights scaled by their fan-in,
    zero biases, a small output layer so that the first guesses stay near
    the FFT-Poisson solution."""
    C, K, L = channels, modes, layers
    r = np.random.default_rng(seed)
    parts = [r.standard_normal(C * 3) / math.sqrt(3.0), np.zeros(C)]
    for _ in range(L):
        parts += [r.standard_normal(C * C) / math.sqrt(C), np.zeros(C),
                  r.standard_normal(K ** 3 * C * C) / (C * K ** 1.5)]
    parts += [0.1 * r.standard_normal(C) / math.sqrt(C), np.zeros(1)]
    theta = np.concatenate(parts).astype(np.float32)
    assert theta.size == pb.sno_num_params(C, K, L)
    return theta


def generate_pairs(n, Ls, samples, tol=1e-6, maxit=3000, stream=None):
    """Training pairs from the library's PCG.

    samples: iterable of (a, g) host arrays (shape (n2, n1, n0); a float32 > 0,
    g float64).  For each, the PCG solves div(a grad phi) = g to `tol`, and
    the features of g and the target (phi - phi0) / rms(phi0) are stored.
    Returns (feats [count, 3, N] float32, targets [count, N] float32, info)
    with torch device tensors."""
    import torch

    samples = list(samples)
    N = int(np.prod(n))
    feats = torch.empty((len(samples), 3, N), dtype=torch.float32, device="cuda")
    targets = torch.empty((len(samples), N), dtype=torch.float32, device="cuda")
    iters = []
    pcg = None
    try:
        for k, (a, g) in enumerate(samples):
            ad = torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32)).cuda()
            gd = torch.as_tensor(np.ascontiguousarray(g, dtype=np.float64)).cuda()
            if pcg is None:
                pcg = pb.PCG(n, Ls, ad)
            else:
                pcg.set_coefficient(ad)
            phi = torch.zeros_like(gd)
            it, rel = pcg.solve(phi, gd, tol=tol, maxit=maxit, stream=stream)
            if rel > tol:
                raise RuntimeError(f"PCG did not reach {tol} for training sample {k} ({rel:.2e})")
            iters.append(it)
            pcg.features(gd, feats[k], phi=phi, target=targets[k], stream=stream)
        torch.cuda.synchronize()
    finally:
        if pcg is not None:
            pcg.close()
    return feats, targets, {"pcg_iterations": iters}


def train(pairs, n, channels=16, modes=12, layers=4, batch=8, epochs=20, lr=2e-3, lr_final=1e-4, seed=0,
          holdout=0, log=None):
    """Adam on the relative squared error of the target, cosine learning-rate
    decay from lr to lr_final; the last `holdout` pairs are only evaluated.
    Returns (theta FP32 numpy, history dict)."""
    import torch

    feats, targets = pairs[0], pairs[1]
    count = feats.shape[0] - holdout
    if count < batch:
        raise ValueError("fewer training pairs than one batch")
    net = pb.SNO(n, batch=batch, channels=channels, modes=modes, layers=layers, train=True)
    theta = init_params(channels, modes, layers, seed)
    net.set_params(theta)
    P = theta.size
    grad = torch.zeros(P, dtype=torch.float32, device="cuda")
    N = int(np.prod(n))
    y = torch.empty((batch, N), dtype=torch.float32, device="cuda")
    dy = torch.empty_like(y)
    order_rng = np.random.default_rng(seed + 1)
    steps_per_epoch = count // batch
    total = steps_per_epoch * epochs
    hist = {"train_loss": [], "holdout_loss": [], "seconds": 0.0}
    step = 0
    t0 = time.perf_counter()
    idx_buf = torch.empty(batch, dtype=torch.int64, device="cuda")
    fb = torch.empty((batch, 3, N), dtype=torch.float32, device="cuda")
    tb = torch.empty((batch, N), dtype=torch.float32, device="cuda")
    for ep in range(epochs):
        perm = order_rng.permutation(count)
        run = 0.0
        for s in range(steps_per_epoch):
            sel = perm[s * batch:(s + 1) * batch]
            idx_buf.copy_(torch.from_numpy(sel))
            torch.index_select(feats, 0, idx_buf, out=fb)
            torch.index_select(targets, 0, idx_buf, out=tb)
            net.forward(y, fb)
            last = s == steps_per_epoch - 1
            loss = net.loss(y, tb, dy, read=last)
            net.backward(grad, dy, fb)
            step += 1
            lr_t = lr_final + 0.5 * (lr - lr_final) * (1 + math.cos(math.pi * step / total))
            net.adam(grad, lr_t, step)
            if last:
                run = loss
        hist["train_loss"].append(run)
        if holdout:
            hist["holdout_loss"].append(evaluate(net, feats[count:], targets[count:], batch))
        if log:
            log(f"epoch {ep + 1}/{epochs}: batch loss {run:.4f}"
                + (f", holdout {hist['holdout_loss'][-1]:.4f}" if holdout else ""))
    torch.cuda.synchronize()
    hist["seconds"] = time.perf_counter() - t0
    out = np.empty(P, dtype=np.float32)
    net.get_params(out)
    net.close()
    return out, hist


def evaluate(net, feats, targets, batch):
    """Mean relative squared error of the network over pairs (whole batches)."""
    import torch

    N = feats.shape[-1]
    y = torch.empty((batch, N), dtype=torch.float32, device="cuda")
    vals = []
    for s in range(feats.shape[0] // batch):
        fb = feats[s * batch:(s + 1) * batch].contiguous()
        tb = targets[s * batch:(s + 1) * batch].contiguous()
        net.forward(y, fb)
        vals.append(net.loss(y, tb))
    return float(np.mean(vals)) if vals else float("nan")


def load_network(n, theta, channels=16, modes=12, layers=4):
    """Batch-1 inference object on grid n with parameters theta."""
    net = pb.SNO(n, batch=1, channels=channels, modes=modes, layers=layers, train=False)
    net.set_params(np.ascontiguousarray(theta, dtype=np.float32))
    return net
