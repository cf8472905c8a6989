"""Pins for the fp64 proposal-network oracle: library convolution and autograd in
float64, central finite differences, the library Adam, and bf16 rounding."""
import numpy as np
import pytest
import torch

from oracle import cnn


def _params(seed=0, scale=1.0):
    rng = np.random.default_rng(seed)
    p = {}
    for name, shape in cnn.SHAPES:
        fan_in = int(np.prod(shape[1:])) if len(shape) > 1 else 1
        p[name] = rng.uniform(-1, 1, shape) * scale * np.sqrt(6.0 / fan_in) + (0.05 if len(shape) == 1 else 0.0)
    return p


def _batch(seed=1, B=3):
    rng = np.random.default_rng(seed)
    th = rng.integers(0, 256, (B, 2, 36, 64))
    x = np.stack([cnn.pair_input(a, b) for a, b in th])
    y = (np.arange(B) % 2).astype(np.float64)
    return x, y


def test_conv_matches_library():
    rng = np.random.default_rng(2)
    x = rng.normal(size=(2, 3, 9, 16))
    W = rng.normal(size=(5, 3, 3, 3))
    b = rng.normal(size=5)
    ref = torch.nn.functional.conv2d(torch.from_numpy(x), torch.from_numpy(W), torch.from_numpy(b), stride=2,
                                     padding=1).numpy()
    assert np.allclose(cnn.conv_s2(x, W, b), ref, atol=1e-12, rtol=0)
    assert cnn.conv_s2(np.zeros((1, 2, 36, 64)), np.zeros((16, 2, 3, 3)), np.zeros(16)).shape == (1, 16, 18, 32)


def _torch_loss(flat, x, y, w):
    p = {}
    o = 0
    for name, shape in cnn.SHAPES:
        n = int(np.prod(shape))
        p[name] = flat[o:o + n].reshape(shape)
        o += n
    F = torch.nn.functional
    a = F.relu(F.conv2d(x, p["W1"], p["b1"], stride=2, padding=1))
    a = F.relu(F.conv2d(a, p["W2"], p["b2"], stride=2, padding=1))
    a = F.relu(F.conv2d(a, p["W3"], p["b3"], stride=2, padding=1))
    g = a.mean(dim=(2, 3))
    h = F.relu(F.linear(g, p["F1"], p["c1"]))
    z = F.linear(h, p["F2"], p["c2"])[:, 0]
    return F.binary_cross_entropy_with_logits(z, y, pos_weight=torch.tensor(w, dtype=torch.float64)), z


def test_forward_and_backward_match_autograd():
    p = _params()
    x, y = _batch()
    flat = cnn.flatten(p)
    loss, grad = cnn.loss_and_grad(flat, x, y, pos_weight=7.5)
    tf = torch.tensor(flat, requires_grad=True)
    tl, tz = _torch_loss(tf, torch.from_numpy(x), torch.from_numpy(y), 7.5)
    tl.backward()
    assert abs(loss - tl.item()) < 1e-12 * max(1.0, abs(loss))
    assert np.allclose(cnn.forward(p, x)["z"], tz.detach().numpy(), atol=1e-12, rtol=0)
    ref = tf.grad.numpy()
    assert np.abs(grad - ref).max() <= 1e-10 * np.abs(ref).max()


def test_gradient_central_differences():
    p = _params(seed=4)
    x, y = _batch(seed=5, B=2)
    flat = cnn.flatten(p)
    _, grad = cnn.loss_and_grad(flat, x, y, pos_weight=3.0)
    rng = np.random.default_rng(6)
    off = 0
    for name, shape in cnn.SHAPES:
        n = int(np.prod(shape))
        for i in rng.choice(n, size=min(n, 12), replace=False):
            j = off + int(i)
            h = 1e-5
            fp = flat.copy()
            fp[j] += h
            fm = flat.copy()
            fm[j] -= h
            num = (cnn.loss_and_grad(fp, x, y, 3.0)[0] - cnn.loss_and_grad(fm, x, y, 3.0)[0]) / (2 * h)
            assert abs(num - grad[j]) <= 1e-6 * max(1e-3, abs(grad[j])), (name, int(i))
        off += n


def test_adam_matches_library():
    rng = np.random.default_rng(7)
    w = rng.normal(size=50)
    m = np.zeros(50)
    v = np.zeros(50)
    tw = torch.tensor(w.copy(), requires_grad=True)
    opt = torch.optim.Adam([tw], lr=1e-3, betas=(0.9, 0.999), eps=1e-8)
    for step in range(1, 6):
        g = rng.normal(size=50)
        w, m, v = cnn.adam(w, g, m, v, step)
        opt.zero_grad()
        tw.grad = torch.tensor(g)
        opt.step()
        assert np.allclose(w, tw.detach().numpy(), atol=1e-15, rtol=1e-12)


def test_bf16_round_matches_library():
    rng = np.random.default_rng(8)
    a = np.concatenate([rng.normal(size=10000) * 10 ** rng.uniform(-6, 6, 10000), [0.0, -0.0, 1.0, -3.5]])
    ref = torch.from_numpy(a.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(cnn.bf16_round(a), ref)


def test_pair_input_exact_in_bf16():
    t = np.arange(256).reshape(1, 256)
    x = cnn.pair_input(t, t)
    assert np.array_equal(cnn.bf16_round(x), x)
    assert x.min() == -2.0 and x.max() == 127 / 64
