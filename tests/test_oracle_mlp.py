"""Pins of the warm-start network oracle: central differences and PyTorch autograd."""
import numpy as np
import pytest

from oracle import mlp


def _net(rng, sizes):
    return [(rng.standard_normal((o, i)) / np.sqrt(i), 0.1 * rng.standard_normal(o)) for i, o in zip(sizes[:-1], sizes[1:])]


def test_bf16_rounding():
    x = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 2 ** -7, 1.0 + 3 * 2 ** -8, -2.5, 3.0e-3], np.float32)
    r = mlp.bf16_round(x)
    assert r[0] == 1.0 and r[1] == 1.0                   # tie rounds to even (down)
    assert r[2] == 1.0 + 2 ** -7
    assert r[3] == 1.0 + 2 ** -6                         # tie rounds to even (up)
    assert r[4] == -2.5
    assert abs(r[5] - 3.0e-3) < 3.0e-3 * 2 ** -8


def test_gradient_central_differences():
    rng = np.random.default_rng(0)
    sizes = [6, 8, 7, 5]
    params = _net(rng, sizes)
    X = rng.standard_normal((4, 6))
    T = rng.standard_normal((4, 5))
    _, grads = mlp.loss_grad(params, X, T)
    h = 1e-6
    for l in range(3):
        W, b = params[l]
        for idx in [(0, 0), (2, 3), (4, 1)]:
            if idx[0] >= W.shape[0] or idx[1] >= W.shape[1]:
                continue
            Wp, Wm = W.copy(), W.copy()
            Wp[idx] += h
            Wm[idx] -= h
            pp = [p if k != l else (Wp, b) for k, p in enumerate(params)]
            pm = [p if k != l else (Wm, b) for k, p in enumerate(params)]
            fd = (mlp.loss_grad(pp, X, T)[0] - mlp.loss_grad(pm, X, T)[0]) / (2 * h)
            assert abs(fd - grads[l][0][idx]) < 1e-7 * max(1.0, abs(fd))
        bp, bm = b.copy(), b.copy()
        bp[1] += h
        bm[1] -= h
        fd = (mlp.loss_grad([p if k != l else (W, bp) for k, p in enumerate(params)], X, T)[0] -
              mlp.loss_grad([p if k != l else (W, bm) for k, p in enumerate(params)], X, T)[0]) / (2 * h)
        assert abs(fd - grads[l][1][1]) < 1e-7 * max(1.0, abs(fd))


def test_matches_torch_autograd():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(1)
    sizes = [5, 9, 4]
    params = _net(rng, sizes)
    X = rng.standard_normal((3, 5))
    T = rng.standard_normal((3, 4))
    loss, grads = mlp.loss_grad(params, X, T)
    tp = [(torch.tensor(W, requires_grad=True), torch.tensor(b, requires_grad=True)) for W, b in params]
    a = torch.tensor(X)
    for l, (W, b) in enumerate(tp):
        a = a @ W.T + b
        if l + 1 < len(tp):
            a = torch.relu(a)
    L = torch.mean((a - torch.tensor(T)) ** 2)
    L.backward()
    assert abs(L.item() - loss) < 1e-14
    for (W, b), (dW, db) in zip(tp, grads):
        assert np.abs(W.grad.numpy() - dW).max() < 1e-14
        assert np.abs(b.grad.numpy() - db).max() < 1e-14
