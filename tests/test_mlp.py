"""The policy network's training kernels against the CPU oracle: logits
(BF16 tensor-core forward vs the oracle's BF16/FP32 and FP64 forms), the loss
gradient (vs the oracle's FP64 backward, BF16-aware tolerance), and that Adam
steps learn a learnable task."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1802_06215_b300 import _dsp, build
    build.build()
    return torch, _dsp


def bf16_exact(a):
    """Rounds to values that bfloat16 holds exactly (so the BF16 copies equal
    the FP32 masters)."""
    a = np.asarray(a, np.float32).copy()
    u = a.view(np.uint32)
    u += 0x7FFF + ((u >> 16) & 1)
    u &= 0xFFFF0000
    return a


def make_weights(seed):
    rng = np.random.default_rng(seed)
    w = {"W1": rng.normal(0, np.sqrt(2 / 64), (64, 256)), "b1": rng.normal(0, 0.1, 256),
         "W2": rng.normal(0, np.sqrt(2 / 256), (256, 256)), "b2": rng.normal(0, 0.1, 256),
         "W3": rng.normal(0, np.sqrt(2 / 256), (256, 32)), "b3": rng.normal(0, 0.1, 32)}
    return {k: bf16_exact(v).astype(np.float64) for k, v in w.items()}


def test_forward_matches_oracle(env):
    torch, _dsp = env
    w = make_weights(1)
    h = _dsp.dsp_mlp_create(512, 0)
    _dsp.dsp_mlp_set_weights(h, _dsp.pack_params(w))
    rng = np.random.default_rng(2)
    for B in (1, 37, 300):
        X = bf16_exact(rng.normal(0, 1, (B, 64)))
        Xd = torch.tensor(X, device="cuda")
        L = torch.zeros((B, 32), dtype=torch.float32, device="cuda")
        _dsp.dsp_mlp_forward(h, Xd.data_ptr(), B, L.data_ptr())
        torch.cuda.synchronize()
        g = L.cpu().numpy().astype(np.float64)
        ob = oracle.mlp_forward(w, X, bf16=True)
        oe = oracle.mlp_forward(w, X)
        scale = np.max(np.abs(oe))
        assert np.max(np.abs(g - ob)) <= 1e-2 * scale, B
        assert np.max(np.abs(g - oe)) <= 3e-2 * scale, B
    _dsp.dsp_mlp_destroy(h)


def test_gradient_matches_oracle(env):
    """Batches of 1000, 300 and 1 rows on one network, in that order: ragged
    last tiles, and smaller batches after larger ones (the weight gradients
    reduce over the batch padded to the tile, so the padding must read as
    0)."""
    torch, _dsp = env
    w = make_weights(3)
    h = _dsp.dsp_mlp_create(1024, 0)
    _dsp.dsp_mlp_set_weights(h, _dsp.pack_params(w))
    rng = np.random.default_rng(4)
    na = 20
    for B in (1000, 300, 1):
        # Labels: the network's second-best action for half the rows, random
        # for the rest. Per-example gradients then add up instead of
        # cancelling (with purely random labels the batch gradient is a
        # small difference of large terms and BF16 rounding of each term
        # dominates it).
        X = bf16_exact(rng.normal(0, 1, (B, 64)))
        lg = oracle.mlp_forward(w, X)[:, :na]
        y = np.argsort(lg, axis=1)[:, -2].astype(np.int32)
        y[::2] = rng.integers(0, na, (B + 1) // 2)
        Xd = torch.tensor(X, device="cuda")
        yd = torch.tensor(y, device="cuda")
        loss, flat = _dsp.dsp_mlp_grad(h, Xd.data_ptr(), yd.data_ptr(), B, na)
        g = _dsp.unpack_params(flat)
        # BF16-aware: the oracle's FP64 backward at the BF16 forward's activations
        oloss, og = oracle.mlp_loss_grad(w, X, y, na, bf16_forward=True)
        assert abs(loss - oloss) <= 1e-2 * abs(oloss), B
        rels = {k: float(np.linalg.norm(g[k] - og[k]) / np.linalg.norm(og[k])) for k in og}
        assert all(r <= 1e-2 for r in rels.values()), (B, rels)
        # and the exact FP64 gradient within what the BF16 forward moves the
        # logits by (a few per cent, see test_forward_matches_oracle)
        _, ge = oracle.mlp_loss_grad(w, X, y, na)
        rele = {k: float(np.linalg.norm(g[k] - ge[k]) / np.linalg.norm(ge[k])) for k in ge}
        assert all(r <= 8e-2 for r in rele.values()), (B, rele)
    _dsp.dsp_mlp_destroy(h)


def test_training_learns(env):
    """Labels are the argmax of a fixed linear map of the features over 20
    classes: 400 Adam steps drive the loss down and the accuracy up."""
    torch, _dsp = env
    rng = np.random.default_rng(5)
    T = rng.normal(0, 1, (64, 20))
    N = 8192
    X = rng.normal(0, 1, (N, 64)).astype(np.float32)
    y = np.argmax(X @ T, axis=1).astype(np.int32)
    Xd = torch.tensor(X, device="cuda")
    yd = torch.tensor(y, device="cuda")
    h = _dsp.dsp_mlp_create(1024, 7)
    first = None
    for it in range(400):
        k = (it * 1024) % N
        loss = _dsp.dsp_mlp_train_step(h, Xd[k:k + 1024].data_ptr(), yd[k:k + 1024].data_ptr(), 1024, 20, 1e-3)
        first = loss if first is None else first
    L = torch.zeros((1024, 32), dtype=torch.float32, device="cuda")
    _dsp.dsp_mlp_forward(h, Xd[:1024].data_ptr(), 1024, L.data_ptr())
    acc = (L[:, :20].argmax(1).cpu().numpy() == y[:1024]).mean()
    assert loss < 0.5 * first and acc > 0.8, (first, loss, acc)
    _dsp.dsp_mlp_destroy(h)
