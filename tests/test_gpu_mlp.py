"""Warm-start network: the library's BF16 tensor-core training kernels against the FP64 oracle,
and the gain of the trained warm start over the plain BP + CSI start."""
import numpy as np
import pytest

import scenes
from oracle import mlp as omlp

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def net_and_data():
    from paper_2602_13805_gb300 import build
    from paper_2602_13805_gb300.warmstart import WarmStartMLP
    build.build()
    sizes = [256, 192, 160, 96]
    net = WarmStartMLP(sizes, batch_max=64, seed=1)
    rng = np.random.default_rng(2)
    X = rng.standard_normal((48, 256)).astype(np.float32)
    T = rng.standard_normal((48, 96)).astype(np.float32)
    yield net, X, T
    net.close()


def test_mlp_gradient_parity(net_and_data):
    net, X, T = net_and_data
    # a larger batch first, then B = 48: padded batch columns must not leak into the gradients
    Xb = torch.from_numpy(np.random.default_rng(5).standard_normal((64, 256)).astype(np.float32)).cuda()
    Tb = torch.from_numpy(np.random.default_rng(6).standard_normal((64, 96)).astype(np.float32)).cuda()
    net.loss_grad(Xb, Tb)
    loss = float(net.loss_grad(torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda()))
    params, grads = [], []
    for l in range(3):
        W, b, dW, db = net.get_params(l)
        params.append((W.astype(np.float64), b.astype(np.float64)))
        grads.append((dW, db))
    le, ge = omlp.loss_grad(params, X, T, bf16=True)        # same BF16 rounding points as the GPU
    lf, gf = omlp.loss_grad(params, X, T, bf16=False)       # plain FP64
    assert abs(loss - le) < 1e-5 * le
    for l in range(3):
        e_w, e_b = _rel(grads[l][0], ge[l][0]), _rel(grads[l][1], ge[l][1])
        f_w = _rel(grads[l][0], gf[l][0])
        print(f"layer {l}: dW rel {e_w:.2e} (bf16 oracle) {f_w:.2e} (fp64 oracle), db rel {e_b:.2e}")
        assert e_w < 1e-3 and e_b < 1e-3
        # against plain FP64 the BF16 casts of activations and cotangents (2^-9 relative each) add up
        # over three layers, and random targets make these gradients sums of cancelling terms
        assert f_w < 1e-1
    assert abs(loss - lf) < 1e-2 * lf


def test_mlp_forward_parity(net_and_data):
    net, X, T = net_and_data
    y = net.forward(torch.from_numpy(X).cuda()).cpu().numpy()
    params = [(net.get_params(l)[0].astype(np.float64), net.get_params(l)[1].astype(np.float64)) for l in range(3)]
    ye, _ = omlp.forward(params, X, bf16=True)
    assert _rel(y, ye) < 1e-4


def test_mlp_adam_step(net_and_data):
    net, X, T = net_and_data
    Xd, Td = torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda()
    W0 = [net.get_params(l)[0] for l in range(3)]
    net.set_params(0, W0[0], net.get_params(0)[1])          # resets the step count and moments of layer 0
    for l in (1, 2):
        net.set_params(l, W0[l], net.get_params(l)[1])
    lr = 1e-3
    net.train_step(Xd, Td, lr)
    torch.cuda.synchronize()
    for l in range(3):
        W1, _, dW, _ = net.get_params(l)
        # first Adam step: m_hat = g, v_hat = g^2, so W1 = W0 - lr g / (|g| + eps)
        ref = W0[l] - lr * dW / (np.abs(dW) + 1e-8)
        assert np.abs(W1 - ref).max() < 1e-6


def test_warm_start_gain():
    from paper_2602_13805_gb300 import pdf
    from paper_2602_13805_gb300.warmstart import WarmStartMLP, evaluate, generate, train
    w = scenes.workload("c4")
    prob = pdf.Problem.from_workload(w)
    train_set = generate(prob, w, 512, seed0=1000)
    test_set = generate(prob, w, 4, seed0=0)
    sizes = [2 * w.ni * w.nr, 1024, 1024, 1024, 2 * (1 + w.ni) * w.kx * w.ky]
    net = WarmStartMLP(sizes, batch_max=128, seed=0)
    hist = train(net, train_set, steps=400, batch=128, lr=1e-3, log_every=100)
    print("train loss", hist, "data seconds", train_set.seconds)
    res = evaluate(prob, net, test_set, w, iters=100, every=5)
    for r in res:
        print(r)
    assert hist[-1][1] < 0.5 * hist[0][1]
    # the trained start beats BP + CSI in physics loss at iteration 0 on held-out scenes
    assert np.mean([r["loss0_warm"] for r in res]) < np.mean([r["loss0_plain"] for r in res])
    net.close()
    prob.close()


def test_features_match_the_definition():
    # each scene's field divided by its RMS magnitude, (Re, Im) interleaved; a zero scene unscaled
    from paper_2602_13805_gb300.warmstart import features
    rng = np.random.default_rng(3)
    E = (rng.standard_normal((5, 16, 32)) + 1j * rng.standard_normal((5, 16, 32))) * rng.uniform(0.1, 10, (5, 1, 1))
    E[3] = 0.0
    E = E.astype(np.complex64)
    X = features(torch.from_numpy(E).cuda()).cpu().numpy()
    flat = E.reshape(5, -1).astype(np.complex128)
    rms = np.linalg.norm(flat, axis=1) / np.sqrt(flat.shape[1])
    rms[3] = 1.0
    ref = np.stack([(flat / rms[:, None]).real, (flat / rms[:, None]).imag], axis=-1).reshape(5, -1)
    assert np.abs(X - ref).max() <= 1e-6 * np.abs(ref).max()
