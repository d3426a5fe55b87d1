"""Pin for oracle.cnn: the fixed-point network's decoded gradients agree with
float64 torch autograd of the same network (an independent implementation of
conv / pooling / matmul and their derivatives) to fixed-point precision, and
its forward values match the float network."""
import numpy as np
import torch

from oracle import cnn
from paper_2403_11166_gb300 import inputs


def _float_model(p, x):
    t = {k: torch.tensor(v, dtype=torch.float64, requires_grad=True) for k, v in p.items()}
    xt = torch.tensor(x, dtype=torch.float64)
    h = torch.nn.functional.conv2d(xt, t["w1"], t["b1"], padding=1)
    h = torch.where(h >= 0, h, torch.zeros_like(h))
    h = torch.nn.functional.conv2d(h, t["w2"], t["b2"], padding=1)
    h = torch.nn.functional.avg_pool2d(h, 2).reshape(x.shape[0], -1)
    return t, h @ t["w3"].T + t["b3"]


def test_fixed_point_gradients_match_float_autograd():
    p = inputs.cnn_params(1, channels=(3, 4, 8), height=8, width=8, classes=5)
    rng = np.random.default_rng(2)
    x = np.floor(np.clip(rng.standard_normal((6, 3, 8, 8)), -8, 8) * 4096) / 4096
    t, logits = _float_model(p, x)
    R = rng.standard_normal(logits.shape) * 64.0        # a scaled loss gradient
    (logits * torch.tensor(R)).sum().backward()
    r = cnn.train_step(p, x, R)
    assert np.abs(r["logits"] - logits.detach().numpy()).max() < 5e-3
    for k in ("w1", "w2", "w3", "b1", "b2", "b3"):
        want = t[k].grad.numpy()
        got = r["grads"][k]
        rel = np.linalg.norm(got - want) / max(np.linalg.norm(want), 1e-12)
        assert rel < 1e-2, (k, rel)


def test_floor_truncation_bias_reading():
    """The reason for rounding gradients: with floor, a constant small negative
    gradient truncates to -1 unit everywhere (bias), with rounding to 0."""
    g = np.full((4, 4), -1e-5)
    assert (cnn._dec(cnn._enc(g, 12, 41), 12, 41) == -1 / 4096).all()
    assert (cnn._dec(cnn._enc_round(g, 12, 41), 12, 41) == 0).all()
