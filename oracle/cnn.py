"""fp64 oracle of the learned boundary proposal network.  TEST INFRASTRUCTURE ONLY.

The paper's pipelines run a DNN on sampled frames (Sec. 3.1 face detection,
Sec. 5.1.2 DNN) but fix no network for shot proposals.  This is the network
used here:
  input  x: 2 x 36 x 64, channel 0 = (Y_prev - 128) / 64, channel 1 = (Y_cur - 128) / 64,
            Y = luma thumbnail (every s-th row and column of the frame);
  a1 = relu(conv3x3/s2/p1(x;  W1: 16 x 2,  b1))     -> 16 x 18 x 32
  a2 = relu(conv3x3/s2/p1(a1; W2: 32 x 16, b2))     -> 32 x 9 x 16
  a3 = relu(conv3x3/s2/p1(a2; W3: 32 x 32, b3))     -> 32 x 5 x 8
  g  = mean over the 5 x 8 positions of a3         -> 32
  h  = relu(F1 g + c1)                             -> 64
  z  = F2 h + c2                                   -> logit
Loss: binary cross-entropy with logits, positive weight w:
  l = -(w y log sigmoid(z) + (1 - y) log(1 - sigmoid(z))), averaged over the batch.
Optimiser: Adam (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected).

`rnd` (optional) rounds the values the GPU keeps in bf16 (layer inputs a1, a2,
a3 and the activation gradients of the convolutions), so that gradients can be
compared on the same rounded values.  Everything else is fp64.
Pins: tests/test_oracle_cnn.py (torch float64 conv2d and autograd, central
finite differences).
"""
from __future__ import annotations

import numpy as np

SHAPES = [("W1", (16, 2, 3, 3)), ("b1", (16,)), ("W2", (32, 16, 3, 3)), ("b2", (32,)),
          ("W3", (32, 32, 3, 3)), ("b3", (32,)), ("F1", (64, 32)), ("c1", (64,)), ("F2", (1, 64)), ("c2", (1,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def unflatten(flat: np.ndarray) -> dict:
    p, o = {}, 0
    for name, shape in SHAPES:
        n = int(np.prod(shape))
        p[name] = np.asarray(flat[o:o + n], dtype=np.float64).reshape(shape)
        o += n
    return p


def flatten(p: dict) -> np.ndarray:
    return np.concatenate([np.asarray(p[name], dtype=np.float64).ravel() for name, _ in SHAPES])


def bf16_round(a: np.ndarray) -> np.ndarray:
    """Round to the nearest bfloat16 (ties to even), returned as fp64."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = ((u + 0x7FFF + lsb) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def pair_input(thumb_prev: np.ndarray, thumb_cur: np.ndarray) -> np.ndarray:
    """2 x 36 x 64 network input of a thumbnail pair (exact in bf16)."""
    return np.stack([(thumb_prev.astype(np.float64) - 128.0) / 64.0, (thumb_cur.astype(np.float64) - 128.0) / 64.0])


def _out(n: int) -> int:
    return (n + 2 - 3) // 2 + 1


def conv_s2(x: np.ndarray, W: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Batched 3x3 convolution, stride 2, zero padding 1.  x: B x C x H x W."""
    B, C, H, Wd = x.shape
    Ho, Wo = _out(H), _out(Wd)
    xp = np.zeros((B, C, H + 2, Wd + 2))
    xp[:, :, 1:H + 1, 1:Wd + 1] = x
    out = np.zeros((B, W.shape[0], Ho, Wo))
    for di in range(3):
        for dj in range(3):
            patch = xp[:, :, di:di + 2 * Ho - 1:2, dj:dj + 2 * Wo - 1:2]  # B x C x Ho x Wo
            out += np.einsum("bchw,oc->bohw", patch, W[:, :, di, dj])
    return out + b[None, :, None, None]


def conv_s2_backward(x: np.ndarray, W: np.ndarray, dy: np.ndarray):
    """Gradients of conv_s2 w.r.t. its input, weights and bias."""
    B, C, H, Wd = x.shape
    Ho, Wo = dy.shape[2], dy.shape[3]
    xp = np.zeros((B, C, H + 2, Wd + 2))
    xp[:, :, 1:H + 1, 1:Wd + 1] = x
    dxp = np.zeros_like(xp)
    dW = np.zeros_like(W)
    for di in range(3):
        for dj in range(3):
            sl = (slice(None), slice(None), slice(di, di + 2 * Ho - 1, 2), slice(dj, dj + 2 * Wo - 1, 2))
            dW[:, :, di, dj] = np.einsum("bohw,bchw->oc", dy, xp[sl])
            dxp[sl] += np.einsum("bohw,oc->bchw", dy, W[:, :, di, dj])
    db = dy.sum(axis=(0, 2, 3))
    return dxp[:, :, 1:H + 1, 1:Wd + 1], dW, db


def forward(p: dict, x: np.ndarray, rnd=None) -> dict:
    """x: B x 2 x 36 x 64.  Returns every intermediate and the logits z (B)."""
    r = rnd if rnd is not None else (lambda a: a)
    t = {"x": x}
    t["u1"] = conv_s2(x, p["W1"], p["b1"])
    t["a1"] = r(np.maximum(t["u1"], 0))
    t["u2"] = conv_s2(t["a1"], p["W2"], p["b2"])
    t["a2"] = r(np.maximum(t["u2"], 0))
    t["u3"] = conv_s2(t["a2"], p["W3"], p["b3"])
    t["a3"] = r(np.maximum(t["u3"], 0))
    t["g"] = t["a3"].mean(axis=(2, 3))
    t["v"] = t["g"] @ p["F1"].T + p["c1"]
    t["h"] = np.maximum(t["v"], 0)
    t["z"] = (t["h"] @ p["F2"].T + p["c2"])[:, 0]
    return t


def bce_with_logits(z: np.ndarray, y: np.ndarray, pos_weight: float):
    """Mean loss and dl/dz."""
    # log sigmoid(z) = -softplus(-z); log(1 - sigmoid(z)) = -softplus(z)
    sp_neg = np.logaddexp(0.0, -z)
    sp_pos = np.logaddexp(0.0, z)
    loss = (pos_weight * y * sp_neg + (1 - y) * sp_pos).mean()
    sig = 1.0 / (1.0 + np.exp(-z))
    dz = (pos_weight * y * (sig - 1) + (1 - y) * sig) / len(z)
    return loss, dz


def backward(p: dict, t: dict, dz: np.ndarray, rnd=None) -> dict:
    """Gradients of the loss w.r.t. every parameter, given dl/dz per sample."""
    r = rnd if rnd is not None else (lambda a: a)
    g = {}
    dz2 = dz[:, None]
    g["F2"] = dz2.T @ t["h"]
    g["c2"] = dz2.sum(axis=0)
    dh = dz2 @ p["F2"]
    dv = dh * (t["v"] > 0)
    g["F1"] = dv.T @ t["g"]
    g["c1"] = dv.sum(axis=0)
    dgv = dv @ p["F1"]
    da3 = np.broadcast_to(dgv[:, :, None, None] / 40.0, t["a3"].shape)
    du3 = r(da3 * (t["u3"] > 0))
    da2, g["W3"], g["b3"] = conv_s2_backward(t["a2"], p["W3"], du3)
    du2 = r(da2 * (t["u2"] > 0))
    da1, g["W2"], g["b2"] = conv_s2_backward(t["a1"], p["W2"], du2)
    du1 = r(da1 * (t["u1"] > 0))
    _, g["W1"], g["b1"] = conv_s2_backward(t["x"], p["W1"], du1)
    return g


def loss_and_grad(flat: np.ndarray, x: np.ndarray, y: np.ndarray, pos_weight: float, rnd=None):
    p = unflatten(flat)
    t = forward(p, x, rnd)
    loss, dz = bce_with_logits(t["z"], y, pos_weight)
    return loss, flatten(backward(p, t, dz, rnd))


def adam(flat: np.ndarray, grad: np.ndarray, m: np.ndarray, v: np.ndarray, step: int, lr: float = 1e-3,
         b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8):
    """One Adam update (step counts from 1).  Returns new (params, m, v)."""
    m = b1 * m + (1 - b1) * grad
    v = b2 * v + (1 - b2) * grad * grad
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return flat - lr * mh / (np.sqrt(vh) + eps), m, v
