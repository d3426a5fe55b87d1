"""GPU: the secure CNN through HeLinearFn (torch.autograd.Function over the C ABI).
Every ring value of every linear layer -- forward outputs, the gradient
encodings, grad_X, grad_W, grad_b -- is bit-exact with the oracle's fixed-point
network; the decoded gradients agree with central finite differences of the
float64 plaintext network within 1e-2 (relative)."""
import numpy as np
import pytest
import torch

from oracle import cnn
from paper_2403_11166_gb300 import inputs
from tests.gpu_util import to_np

pytestmark = pytest.mark.gpu
LOSS_SCALE = 2.0 ** 12


@pytest.fixture(scope="module")
def ag():
    from paper_2403_11166_gb300 import autograd
    return autograd


def _float_loss(p, x, labels, dev):
    t = {k: torch.as_tensor(v, dtype=torch.float64, device=dev) for k, v in p.items()}
    xt = torch.as_tensor(x, dtype=torch.float64, device=dev)
    h = torch.nn.functional.conv2d(xt, t["w1"], t["b1"], padding=1)
    h = torch.where(h >= 0, h, torch.zeros_like(h))
    h = torch.nn.functional.conv2d(h, t["w2"], t["b2"], padding=1)
    h = torch.nn.functional.avg_pool2d(h, 2).reshape(x.shape[0], -1)
    logits = h @ t["w3"].T + t["b3"]
    return torch.nn.functional.cross_entropy(logits, torch.as_tensor(labels, device=dev))


def _run(ag, cfg, B, H, channels, classes, seed, dlogits_fn):
    sess = ag.HeSession(*cfg, seed=seed)
    sess.record = True
    p = inputs.cnn_params(seed, channels=channels, height=H, width=H, classes=classes)
    model = ag.SecureCNN(sess, B, p, H, H)
    g = inputs.rng(seed + 1)
    x = np.floor(np.clip(g.standard_normal((B, channels[0], H, H)), -8, 8) * 4096) / 4096
    logits = model(torch.as_tensor(x, device=sess.device))
    dl = dlogits_fn(logits.detach().cpu().numpy())
    logits.backward(torch.as_tensor(dl, device=sess.device))
    torch.cuda.synchronize()
    assert sess.ctx.sync_status() == 0
    return sess, model, p, x, logits, dl


def _check_ring(sess, p, x, dl):
    want = cnn.train_step(p, x, dl)
    tr = {(e["name"], e["pass"]): e for e in sess.trace}
    pairs = [(("conv1", "fwd"), "X", "X1"), (("conv1", "fwd"), "Y", "Y1"), (("conv2", "fwd"), "X", "X2"),
             (("conv2", "fwd"), "Y", "Y2"), (("fc", "fwd"), "X", "X3"), (("fc", "fwd"), "Y", "Y3"),
             (("fc", "bwd"), "G", "G3"), (("fc", "bwd"), "GW", "GW3"), (("fc", "bwd"), "GB", "GB3"),
             (("fc", "bwd"), "GX", "GX3"), (("conv2", "bwd"), "G", "G2"), (("conv2", "bwd"), "GW", "GW2"),
             (("conv2", "bwd"), "GB", "GB2"), (("conv2", "bwd"), "GX", "GX2"), (("conv1", "bwd"), "G", "G1"),
             (("conv1", "bwd"), "GW", "GW1"), (("conv1", "bwd"), "GB", "GB1")]
    for key, field, ok in pairs:
        got = to_np(tr[key][field]).reshape(-1)
        assert (got == np.asarray(want[ok], dtype=np.uint64).reshape(-1)).all(), (key, field)
    return want


def test_small_cnn_ring_exact(ag):
    rng = np.random.default_rng(3)
    sess, model, p, x, logits, dl = _run(ag, (12, 3, 60), 4, 8, (3, 4, 8), 5, 11,
                                         lambda lg: rng.standard_normal(lg.shape) * 64.0)
    _check_ring(sess, p, x, dl)
    assert model.w1.grad is not None and model.b3.grad is not None


def test_cnn_32x32_b64_ring_exact_and_finite_differences(ag):
    """The training workload: conv3x3 3->16, ReLU, conv3x3 16->32, avgpool 2,
    FC 8192->10, batch 64, N = 8192, three 60-bit primes, t = 2^41."""
    B, H, classes = 64, 32, 10
    labels = np.random.default_rng(5).integers(0, classes, B)

    def dl_fn(lg):   # gradient of LOSS_SCALE * mean cross-entropy
        z = lg - lg.max(axis=1, keepdims=True)
        sm = np.exp(z) / np.exp(z).sum(axis=1, keepdims=True)
        sm[np.arange(B), labels] -= 1.0
        return sm * (LOSS_SCALE / B)

    sess, model, p, x, logits, dl = _run(ag, (13, 3, 60), B, H, (3, 16, 32), classes, 21, dl_fn)
    want = _check_ring(sess, p, x, dl)
    dev = sess.device
    # float64 plaintext network: autograd gradient and central finite differences
    t = {k: torch.as_tensor(v, dtype=torch.float64, device=dev).requires_grad_(True) for k, v in p.items()}
    loss = _float_loss(t, x, labels, dev)
    grads = torch.autograd.grad(loss, [t[k] for k in p])
    ref = {k: gk.detach() for k, gk in zip(p, grads)}
    he_grad = {"w1": model.w1.grad, "w2": model.w2.grad, "w3": model.w3.grad,
               "b1": model.b1.grad, "b2": model.b2.grad, "b3": model.b3.grad}
    rs = np.random.default_rng(9)
    for k in ("w1", "w2", "w3", "b3"):
        g = he_grad[k] / LOSS_SCALE
        rel = float(torch.linalg.norm(g - ref[k]) / torch.linalg.norm(ref[k]))
        assert rel < 1e-2, (k, rel)
        for _ in range(3):
            v = torch.as_tensor(rs.standard_normal(p[k].shape), device=dev)
            h = 1e-6 / float(torch.linalg.norm(v))     # small enough not to cross ReLU kinks
            pp = {kk: torch.as_tensor(vv, dtype=torch.float64, device=dev) for kk, vv in p.items()}
            up, dn = dict(pp), dict(pp)
            up[k] = pp[k] + h * v
            dn[k] = pp[k] - h * v
            fd = float((_float_loss(up, x, labels, dev) - _float_loss(dn, x, labels, dev)) / (2 * h))
            gv = float((g * v).sum())
            assert abs(fd - gv) <= 1e-2 * abs(fd) + 1e-9, (k, fd, gv)
