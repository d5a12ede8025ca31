"""Learned-smoother network kernels against the FP64 oracle (tests/test_oracle_cnn
pins the oracle).  BF16 activations with FP32 accumulation: each tensor is
required within 2e-2 relative (Frobenius) error and cosine similarity 0.999."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle import cnn as ocnn  # noqa: E402


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__ as g
    g.build_library()
    import paper_2412_20205_gb300 as p
    assert torch.cuda.is_available()
    return p


def _weights(seed):
    rng = np.random.default_rng(seed)
    W1 = rng.standard_normal((16, 1, 3, 3)) * 0.4
    W2 = rng.standard_normal((16, 16, 3, 3)) * 0.12
    W3 = rng.standard_normal((1, 16, 3, 3)) * 0.12
    return W1, W2, W3


def _flat(Ws):
    W1, W2, W3 = Ws
    return np.concatenate([W1.reshape(16, 9).ravel(), W2.reshape(16, 16, 9).ravel(), W3.reshape(16, 9).ravel()])


def _close(a, b):
    a, b = np.ravel(a), np.ravel(b)
    rel = np.linalg.norm(a - b) / np.linalg.norm(b)
    cos = np.dot(a, b) / (np.linalg.norm(a) * np.linalg.norm(b))
    return rel < 2e-2 and cos > 0.999, (rel, cos)


@pytest.mark.parametrize("B,H,W", [(2, 37, 45), (1, 16, 16), (3, 9, 130)])
def test_forward_and_gradients_match_oracle(pkg, B, H, W):
    rng = np.random.default_rng(B * 100 + H)
    r = rng.standard_normal((B, H, W))
    e = rng.standard_normal((B, H, W)) * 0.1
    Ws = _weights(H)
    assert pkg.igamg_cnn_num_weights() == 2592
    dev = "cuda"
    tr = torch.tensor(r, dtype=torch.float32, device=dev)
    te = torch.tensor(e, dtype=torch.float32, device=dev)
    tw = torch.tensor(_flat(Ws), dtype=torch.float32, device=dev)
    ws = torch.empty(pkg.igamg_cnn_workspace_bytes(B, H, W), dtype=torch.uint8, device=dev)
    y = torch.empty_like(tr)
    pkg.igamg_cnn_forward(B, H, W, tr, tw, y, ws)
    yref, _ = ocnn.forward(r, Ws)
    ok, info = _close(y.cpu().numpy(), yref)
    assert ok, info
    grad = torch.empty(2592, dtype=torch.float32, device=dev)
    loss = torch.empty(1, dtype=torch.float32, device=dev)
    pkg.igamg_cnn_grad(B, H, W, tr, te, tw, grad, loss, ws)
    lref, gref = ocnn.loss_and_grads(r, e, Ws)
    torch.cuda.synchronize()
    assert abs(float(loss.item()) - lref) <= 2e-2 * lref
    g = grad.cpu().numpy()
    for name, got, ref in [("W1", g[:144], gref[0].reshape(16, 9)), ("W2", g[144:2448], gref[1].reshape(16, 16, 9)),
                           ("W3", g[2448:], gref[2].reshape(16, 9))]:
        ok, info = _close(got, ref)
        assert ok, (name, info)


def test_adam_matches_oracle_and_gradient_is_deterministic(pkg):
    rng = np.random.default_rng(7)
    w = rng.standard_normal(2592)
    g = rng.standard_normal(2592)
    tw = torch.tensor(w, dtype=torch.float32, device="cuda")
    tg = torch.tensor(g, dtype=torch.float32, device="cuda")
    tm = torch.zeros_like(tw)
    tv = torch.zeros_like(tw)
    m, v = np.zeros(2592), np.zeros(2592)
    for step in (1, 2, 3):
        pkg.igamg_adam_step(tw, tg, tm, tv, step, 1e-3)
        w, m, v = ocnn.adam_step(w, g, m, v, step, 1e-3)
    assert np.allclose(tw.cpu().numpy(), w, rtol=1e-5, atol=1e-6)
    # two gradient evaluations give identical bits (fixed-order reductions)
    B, H, W = 2, 33, 40
    r = torch.randn(B, H, W, device="cuda")
    e = torch.randn(B, H, W, device="cuda")
    ww = torch.tensor(_flat(_weights(3)), dtype=torch.float32, device="cuda")
    ws = torch.empty(pkg.igamg_cnn_workspace_bytes(B, H, W), dtype=torch.uint8, device="cuda")
    outs = []
    for _ in range(2):
        grad = torch.empty(2592, device="cuda")
        loss = torch.empty(1, device="cuda")
        pkg.igamg_cnn_grad(B, H, W, r, e, ww, grad, loss, ws)
        outs.append(grad.clone())
    assert torch.equal(outs[0], outs[1])
