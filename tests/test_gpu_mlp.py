"""The warm-start network on the GPU: forward, loss and gradient against the FP64 oracle
(finite differences), BF16 weights, and training on a smooth target."""
import numpy as np
import pytest

from oracle import mlp_oracle as M

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def K():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1612_04082_gb300 as K
    return K


def bf16_round(a):
    """Round-to-nearest-even FP32 -> BF16 -> FP32 (definition of the format)."""
    u = np.asarray(a, np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) >> 16 << 16
    return u.astype(np.uint32).view(np.float32)


def test_gradient_matches_fd_of_oracle(K):
    rng = np.random.default_rng(5)
    dims = (11, 32, 32, 3)
    with K.Mlp(11, 32, 3, 3, seed=7) as net:
        net.set_bf16(False)
        p = (0.3 * rng.normal(size=net.num_params)).astype(np.float32)
        net.set_params(p)
        X = rng.normal(size=(64, 11)).astype(np.float32)
        Y = rng.normal(size=(64, 3)).astype(np.float32)
        loss, g = net.loss_grad(X, Y)
    p64, X64, Y64 = p.astype(np.float64), X.astype(np.float64), Y.astype(np.float64)
    assert loss == pytest.approx(M.loss(p64, dims, X64, Y64), rel=1e-5)
    idx = sorted(rng.choice(len(p), 300, replace=False).tolist())
    fd = M.fd_grad(p64, dims, X64, Y64, idx, eps=1e-6)
    assert np.linalg.norm(g[idx] - fd) / np.linalg.norm(fd) < 1e-4


def test_forward_fp32_and_bf16_match_oracle(K):
    rng = np.random.default_rng(6)
    dims = (11, 64, 64, 64, 3)
    with K.Mlp(11, 64, 4, 3, seed=3) as net:
        p = net.get_params()
        X = rng.normal(size=(70000, 11)).astype(np.float32)  # more than one 65536-row chunk
        net.set_bf16(False)
        y32 = net.forward(X)
        net.set_bf16(True)
        y16 = net.forward(X)
    ref32 = M.forward(p.astype(np.float64), dims, X.astype(np.float64))
    ref16 = M.forward(bf16_round(p).astype(np.float64), dims, X.astype(np.float64))
    assert np.linalg.norm(y32 - ref32) / np.linalg.norm(ref32) < 1e-5
    assert np.linalg.norm(y16 - ref16) / np.linalg.norm(ref16) < 1e-5
    assert np.linalg.norm(y16 - ref32) / np.linalg.norm(ref32) > 1e-4  # the rounding is really applied


def test_training_fits_smooth_target(K):
    rng = np.random.default_rng(8)
    X = rng.normal(size=(16384, 11)).astype(np.float32)
    Y = np.stack([np.sin(X[:, 0] + X[:, 1]), X[:, 2] * X[:, 3], np.tanh(2 * X[:, 4]) + 0.1 * X[:, 5]], 1)
    Y = (3.0 * Y + 5.0).astype(np.float32)  # targets off zero and scaled: standardisation matters
    with K.Mlp(11, 128, 4, 3) as net:
        before = np.mean((net.forward(X) - Y) ** 2)
        st = net.train(X, Y, epochs=40, batch=1024, lr=2e-3)
        after = np.mean((net.forward(X) - Y) ** 2)
        xm, xs, ym, ys = net.normalizers()
    assert st["steps"] == 40 * 16
    assert after < 0.02 * before and after < 0.05 * np.var(Y)
    assert np.allclose(ym, Y.mean(0), rtol=1e-4) and np.allclose(ys, Y.std(0), rtol=1e-3)
