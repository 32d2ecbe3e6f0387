"""The learned form of the PCG on the GPU: the spectral neural operator's
kernels against the FP64 oracle (oracle/sno.py), the features and the
assembled guess against the Poisson oracle, and a small end-to-end run
(pairs from the library's PCG, training, PCG from the learned guess).

Tolerances: activations and sums are FP32 with bfloat16 weights (both sides
use the same bfloat16-rounded parameters), so forward outputs agree to
~1e-6 relative and gradients (sums over all cells) to ~1e-5; the tests
allow 2e-5 and 2e-4."""

import numpy as np
import pytest

import workloads as W
from oracle import poisson as O
from oracle import sno as S
from oracle import vc_operator as V
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


def _case(seed, n=(12, 10, 8), B=2, C=4, K=3, L=3):
    r = np.random.default_rng(seed)
    theta = S.bf16_round(0.4 * r.standard_normal(S.n_params(C, K, L)))
    shape = tuple(reversed(n))
    feats = r.standard_normal((B, 3) + shape).astype(np.float32)
    return theta, feats, (C, K, L)


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-30))


@pytest.mark.parametrize("n,B,C,K,L", [((12, 10, 8), 2, 4, 3, 3), ((33, 7, 16), 1, 16, 6, 4), ((64, 64, 64), 1, 16, 12, 4)])
def test_forward_matches_oracle(pb, n, B, C, K, L):
    theta, feats, _ = _case(1, n, B, C, K, L)
    y_ref, _ = S.forward(theta.astype(np.float64), feats.astype(np.float64), C, K, L)
    with pb.SNO(n, batch=B, channels=C, modes=K, layers=L) as net:
        net.set_params(theta)
        y = torch.empty((B, int(np.prod(n))), dtype=torch.float32, device="cuda")
        net.forward(y, torch.from_numpy(feats).cuda())
        torch.cuda.synchronize()
    assert _rel(y.cpu().numpy().reshape(y_ref.shape), y_ref) < 2e-5


def test_backward_and_loss_match_oracle(pb):
    n, B, C, K, L = (12, 10, 8), 2, 4, 3, 3
    theta, feats, _ = _case(2, n, B, C, K, L)
    shape = tuple(reversed(n))
    t = np.random.default_rng(3).standard_normal((B,) + shape).astype(np.float32)
    y_ref, cache = S.forward(theta.astype(np.float64), feats.astype(np.float64), C, K, L)
    loss_ref, dy_ref = S.loss_and_grad(y_ref, t.astype(np.float64))
    g_ref = S.backward(theta.astype(np.float64), cache, dy_ref, C, K, L)
    N = int(np.prod(n))
    with pb.SNO(n, batch=B, channels=C, modes=K, layers=L, train=True) as net:
        net.set_params(theta)
        fd = torch.from_numpy(feats).cuda()
        y = torch.empty((B, N), dtype=torch.float32, device="cuda")
        dy = torch.empty_like(y)
        grad = torch.full((theta.size,), float("nan"), dtype=torch.float32, device="cuda")
        net.forward(y, fd)
        loss = net.loss(y, torch.from_numpy(t.reshape(B, N)).cuda(), dy)
        net.backward(grad, dy, fd)
        torch.cuda.synchronize()
        g = grad.cpu().numpy()
    assert abs(loss - loss_ref) <= 1e-5 * loss_ref
    assert _rel(dy.cpu().numpy().reshape(dy_ref.shape), dy_ref) < 2e-5
    sizes = [C * 3, C] + [C * C, C, K ** 3 * C * C] * L + [C, 1]
    names = ["P", "p"] + [f"{w}{l}" for l in range(L) for w in ("W", "b", "R")] + ["Q", "q"]
    at = 0
    for name, sz in zip(names, sizes):
        err = float(np.max(np.abs(g[at:at + sz] - g_ref[at:at + sz])) / np.max(np.abs(g_ref[at:at + sz])))
        assert err < 2e-4, (name, err)
        at += sz


def test_adam_step_formula(pb):
    n, B, C, K, L = (8, 8, 8), 1, 2, 2, 1
    P = pb.sno_num_params(C, K, L)
    r = np.random.default_rng(4)
    theta = r.standard_normal(P).astype(np.float32)
    g1, g2 = r.standard_normal(P).astype(np.float32), r.standard_normal(P).astype(np.float32)
    lr, b1, b2, eps = 1e-2, 0.9, 0.999, 1e-8
    m = np.zeros(P, np.float64)
    v = np.zeros(P, np.float64)
    th = theta.astype(np.float64)
    with pb.SNO(n, batch=B, channels=C, modes=K, layers=L, train=True) as net:
        net.set_params(theta)
        for step, g in enumerate((g1, g2), start=1):
            net.adam(torch.from_numpy(g).cuda(), lr, step, b1, b2, eps)
            m = b1 * m + (1 - b1) * g
            v = b2 * v + (1 - b2) * g.astype(np.float64) ** 2
            lr_t = lr * np.sqrt(1 - b2 ** step) / (1 - b1 ** step)
            th = th - lr_t * m / (np.sqrt(v) + eps)
        out = np.empty(P, np.float32)
        net.get_params(out)
    assert np.max(np.abs(out - th)) < 1e-5


def test_features_and_guess_match_oracle(pb):
    n = (20, 16, 12)
    shape = tuple(reversed(n))
    Ls = (1.0, 0.8, 0.6)
    a = W.lognormal_coefficient(shape, 9, 30.0)
    g = W.normal(shape, 10)
    abar = float(np.mean(a.astype(np.float64)))
    phi0 = O.solve(g, (O.DS,) * 3, Ls, O.FD2) / abar
    phi, _, _ = V.pcg(g, a.astype(np.float64), Ls, tol=1e-10)
    f_ref, rp = S.features(g, a, phi0)
    t_ref = (phi - phi0) / rp
    N = int(np.prod(n))
    with pb.PCG(n, Ls, torch.from_numpy(a).cuda()) as pcg:
        gd = torch.from_numpy(g).cuda()
        feats = torch.empty((3, N), dtype=torch.float32, device="cuda")
        target = torch.empty(N, dtype=torch.float32, device="cuda")
        pcg.features(gd, feats, phi=torch.from_numpy(phi).cuda(), target=target)
        torch.cuda.synchronize()
        f = feats.cpu().numpy().reshape((3,) + shape)
        for k in range(3):
            assert _rel(f[k], f_ref[k]) < 2e-5, k
        assert _rel(target.cpu().numpy().reshape(shape), t_ref) < 2e-4
        # a network whose output is identically zero gives phi0 itself
        C, K, L = 4, 3, 2
        with pb.SNO(n, batch=1, channels=C, modes=K, layers=L) as net:
            net.set_params(np.zeros(pb.sno_num_params(C, K, L), np.float32))
            guess = torch.full_like(gd, float("nan"))
            pcg.learned_guess(net, guess, gd, corrections=0)
            torch.cuda.synchronize()
            assert _rel(guess.cpu().numpy(), phi0) < 2e-5
            # one correction: phi0 + L^-1 (g - A phi0) / abar
            pcg.learned_guess(net, guess, gd, corrections=1)
            torch.cuda.synchronize()
            r1 = g - V.apply_operator(phi0, a.astype(np.float64), Ls)
            ref1 = phi0 + O.solve(r1, (O.DS,) * 3, Ls, O.FD2) / abar
            assert _rel(guess.cpu().numpy(), ref1) < 1e-4


def test_train_and_learned_guess_reduces_iterations(pb):
    from paper_1409_8116_gb300 import learned

    n = (32, 32, 32)
    shape = tuple(reversed(n))
    Ls = (1.0, 1.0, 1.0)
    rng = np.random.default_rng(11)

    def sample(k):
        contrast = float(np.exp(rng.uniform(np.log(10.0), np.log(100.0))))
        return W.lognormal_coefficient(shape, 1000 + k, contrast), W.normal(shape, 5000 + k)

    samples = [sample(k) for k in range(72)]
    feats, targets, info = learned.generate_pairs(n, Ls, samples[:64], tol=1e-6)
    arch = dict(channels=8, modes=6, layers=4)
    theta, hist = learned.train((feats, targets), n, batch=8, epochs=40, lr=3e-3, seed=1, **arch)
    assert hist["train_loss"][-1] < 0.7 * hist["train_loss"][0]
    net = learned.load_network(n, theta, **arch)
    its_zero, its_phi0, its_learned = [], [], []
    for a, g in samples[64:]:
        with pb.PCG(n, Ls, torch.from_numpy(a).cuda()) as pcg:
            gd = torch.from_numpy(g).cuda()
            phi = torch.zeros_like(gd)
            its_zero.append(pcg.solve(phi, gd, tol=1e-8)[0])
            pcg.learned_guess(learned.load_network(n, np.zeros_like(theta), **arch), phi, gd, corrections=0)
            its_phi0.append(pcg.solve(phi, gd, tol=1e-8)[0])
            pcg.learned_guess(net, phi, gd, corrections=1)
            it, rel = pcg.solve(phi, gd, tol=1e-8)
            assert rel <= 1e-8
            its_learned.append(it)
    net.close()
    assert np.mean(its_learned) < np.mean(its_zero), (its_learned, its_zero, its_phi0)
