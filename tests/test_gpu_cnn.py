"""Proposal network on the GPU against the fp64 oracle (on the same bf16-rounded
weights; activations rounded to bf16 where the GPU stores them)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import cnn as ocnn  # noqa: E402
import ctypes  # noqa: E402


def _cudart():
    return ctypes.CDLL("libcudart.so.13")


@pytest.fixture(scope="module")
def scn():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1805_07339_b300 import scn as s
    return s


def he_params(seed):
    """He-uniform weights, small non-zero biases (fp32)."""
    rng = np.random.default_rng(seed)
    out = []
    for name, shape in ocnn.SHAPES:
        if len(shape) > 1:
            fan_in = int(np.prod(shape[1:]))
            out.append(rng.uniform(-1, 1, shape) * np.sqrt(6.0 / fan_in))
        else:
            out.append(rng.uniform(-0.1, 0.1, shape))
    return np.concatenate([o.ravel() for o in out]).astype(np.float32)


def rounded(params):
    """The oracle's view of the GPU weights: matrices rounded to bf16, biases fp32."""
    p = ocnn.unflatten(params.astype(np.float64))
    for k in ("W1", "W2", "W3", "F1", "F2"):
        p[k] = ocnn.bf16_round(p[k])
    return p


def thumbs_and_pairs(seed, F, B):
    rng = np.random.default_rng(seed)
    # smooth-ish thumbnails (random levels plus noise) like downsampled frames
    base = rng.integers(16, 236, (F, 1, 1))
    th = np.clip(base + rng.normal(0, 12, (F, 36, 64)) + np.linspace(-20, 20, 64)[None, None, :], 0, 255)
    th = th.astype(np.uint8)
    prev = rng.integers(0, F, B).astype(np.int32)
    cur = rng.integers(0, F, B).astype(np.int32)
    return th, prev, cur


def oracle_x(th, prev, cur):
    return np.stack([ocnn.pair_input(th[a], th[b]) for a, b in zip(prev, cur)])


@pytest.mark.parametrize("B", [1, 2, 3, 37, 300, 1501])
def test_forward_matches_oracle(scn, B):
    """Fused forward (one launch, activations on chip): odd counts leave a
    half-filled last pair slot; 1501 pairs give most CTAs several iterations."""
    params = he_params(B)
    th, prev, cur = thumbs_and_pairs(B + 1, 64, B)
    net = scn.scn_cnn_create(8)  # the fused forward does not depend on max_batch
    try:
        scn.scn_cnn_set_params(net, params)
        z = torch.full((B + 1,), float("nan"), dtype=torch.float32, device="cuda")
        scn.scn_cnn_forward(net, torch.from_numpy(th).cuda(), B, z,
                            prev=torch.from_numpy(prev).cuda(), cur=torch.from_numpy(cur).cuda())
        assert scn.scn_cnn_sync_status(net) == scn.SCN_OK
        t = ocnn.forward(rounded(params), oracle_x(th, prev, cur), rnd=ocnn.bf16_round)
        got = z.cpu().numpy().astype(np.float64)
        assert np.all(np.isfinite(got[:B])) and np.isnan(got[B])  # nothing written past n
        scale = max(1.0, np.abs(t["z"]).max())
        assert np.abs(got[:B] - t["z"]).max() <= 2e-2 * scale
        # the bulk agrees far more closely than the bound (bf16 rounding flips are rare)
        assert np.median(np.abs(got[:B] - t["z"])) <= 2e-3 * scale
    finally:
        scn.scn_cnn_destroy(net)


@pytest.mark.parametrize("B", [1, 37, 300])
def test_training_forward_activations_match_oracle(scn, B):
    """The layered forward that training runs keeps a1, a2, a3 for the backward
    pass; they match the oracle's bf16-rounded activations."""
    params = he_params(B)
    th, prev, cur = thumbs_and_pairs(B + 1, 64, B)
    net = scn.scn_cnn_create(B)
    try:
        scn.scn_cnn_set_params(net, params)
        y = torch.zeros(B, dtype=torch.float32, device="cuda")
        scn.scn_cnn_gradients(net, torch.from_numpy(th).cuda(), y, B, 1.0,
                              prev=torch.from_numpy(prev).cuda(), cur=torch.from_numpy(cur).cuda())
        assert scn.scn_cnn_sync_status(net) == scn.SCN_OK
        t = ocnn.forward(rounded(params), oracle_x(th, prev, cur), rnd=ocnn.bf16_round)
        for layer, key, P, C in [(1, "a1", 576, 16), (2, "a2", 144, 32), (3, "a3", 40, 32)]:
            ptr = scn.scn_cnn_activation(net, layer)
            nbytes = B * P * C * 2
            buf = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
            torch.cuda.synchronize()
            assert _cudart().cudaMemcpy(ctypes.c_void_p(buf.data_ptr()), ctypes.c_void_p(ptr),
                                        ctypes.c_size_t(nbytes), 3) == 0  # device to device
            a = buf.view(torch.bfloat16).float().cpu().numpy().reshape(B, P, C).astype(np.float64)
            ref = t[key].transpose(0, 2, 3, 1).reshape(B, P, C)
            err = np.abs(a - ref)
            tol = 2 ** -7 * np.abs(ref) + 1e-2 * max(1.0, np.abs(ref).max()) * 2 ** -7 * 8
            assert np.mean(err <= tol) > 0.999, (layer, err.max())
            assert err.max() <= 0.05 * max(1.0, np.abs(ref).max()), (layer, err.max())
    finally:
        scn.scn_cnn_destroy(net)


def test_forward_rejects_misaligned_thumbnails(scn):
    net = scn.scn_cnn_create(8)
    try:
        th = torch.zeros(3 * 2304 + 16, dtype=torch.uint8, device="cuda")
        z = torch.empty(2, dtype=torch.float32, device="cuda")
        with pytest.raises(scn.ScnError):
            scn.scn_cnn_forward(net, th[1:], 2, z)
    finally:
        scn.scn_cnn_destroy(net)


def test_forward_consecutive_pairs(scn):
    params = he_params(9)
    th, _, _ = thumbs_and_pairs(10, 50, 1)
    net = scn.scn_cnn_create(16)  # several chunks
    try:
        scn.scn_cnn_set_params(net, params)
        z = torch.empty(49, dtype=torch.float32, device="cuda")
        scn.scn_cnn_forward(net, torch.from_numpy(th).cuda(), 49, z)
        prev = np.arange(49, dtype=np.int32)
        t = ocnn.forward(rounded(params), oracle_x(th, prev, prev + 1), rnd=ocnn.bf16_round)
        assert np.abs(z.cpu().numpy() - t["z"]).max() <= 2e-2 * max(1.0, np.abs(t["z"]).max())
        assert np.allclose(scn.scn_cnn_get_params(net), params)
    finally:
        scn.scn_cnn_destroy(net)


def _rel_cos(a, b):
    a = a.astype(np.float64).ravel()
    b = b.astype(np.float64).ravel()
    rel = np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)
    cos = a @ b / max(np.linalg.norm(a) * np.linalg.norm(b), 1e-30)
    return rel, cos


@pytest.mark.parametrize("B,seed", [(64, 3), (256, 4)])
def test_gradients_match_oracle(scn, B, seed):
    params = he_params(seed)
    th, prev, cur = thumbs_and_pairs(seed + 10, 96, B)
    rng = np.random.default_rng(seed)
    y = (rng.random(B) < 0.3).astype(np.float32)
    net = scn.scn_cnn_create(B)
    try:
        scn.scn_cnn_set_params(net, params)
        grads = torch.zeros(scn.scn_cnn_num_params(), dtype=torch.float32, device="cuda")
        loss = torch.zeros(1, dtype=torch.float32, device="cuda")
        scn.scn_cnn_gradients(net, torch.from_numpy(th).cuda(), torch.from_numpy(y).cuda(), B, 4.0, loss=loss,
                              grads=grads, prev=torch.from_numpy(prev).cuda(), cur=torch.from_numpy(cur).cuda())
        assert scn.scn_cnn_sync_status(net) == scn.SCN_OK
        p = rounded(params)
        t = ocnn.forward(p, oracle_x(th, prev, cur), rnd=ocnn.bf16_round)
        rloss, dz = ocnn.bce_with_logits(t["z"], y.astype(np.float64), 4.0)
        rg = ocnn.flatten(ocnn.backward(p, t, dz, rnd=ocnn.bf16_round))
        assert abs(loss.item() - rloss) <= 1e-2 * max(1.0, rloss)
        g = grads.cpu().numpy()
        off = 0
        for name, shape in ocnn.SHAPES:
            n = int(np.prod(shape))
            rel, cos = _rel_cos(g[off:off + n], rg[off:off + n])
            assert rel <= 2e-2 and cos >= 0.999, (name, rel, cos)
            off += n
    finally:
        scn.scn_cnn_destroy(net)


def test_train_step_is_adam_on_the_gradients(scn):
    B = 32
    params = he_params(21)
    th, prev, cur = thumbs_and_pairs(22, 40, B)
    y = (np.arange(B) % 4 == 0).astype(np.float32)
    net = scn.scn_cnn_create(B)
    try:
        scn.scn_cnn_set_params(net, params)
        args = (torch.from_numpy(th).cuda(), torch.from_numpy(y).cuda(), B, 3.0)
        kw = dict(prev=torch.from_numpy(prev).cuda(), cur=torch.from_numpy(cur).cuda())
        grads = torch.zeros(scn.scn_cnn_num_params(), dtype=torch.float32, device="cuda")
        scn.scn_cnn_gradients(net, *args, grads=grads, **kw)
        g1 = grads.cpu().numpy().astype(np.float64)
        scn.scn_cnn_train_step(net, *args, 1e-3, **kw)
        p1 = scn.scn_cnn_get_params(net).astype(np.float64)
        ref, m, v = ocnn.adam(params.astype(np.float64), g1, np.zeros_like(g1), np.zeros_like(g1), 1)
        assert np.abs(p1 - ref).max() <= 1e-6 + 1e-5 * np.abs(ref).max()
        # a few more steps lower the loss on this batch
        loss = torch.zeros(1, dtype=torch.float32, device="cuda")
        scn.scn_cnn_gradients(net, *args, loss=loss, **kw)
        l0 = loss.item()
        for _ in range(30):
            scn.scn_cnn_train_step(net, *args, 3e-3, **kw)
        scn.scn_cnn_gradients(net, *args, loss=loss, **kw)
        assert loss.item() < l0
        assert scn.scn_cnn_sync_status(net) == scn.SCN_OK
    finally:
        scn.scn_cnn_destroy(net)
