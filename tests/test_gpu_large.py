"""GPU: conv3x3 128->128 on 16x16, batch 128, N = 8192 (the large workload):
forward (Alg. 1), grad_X and grad_W (Alg. 2 + local terms) through the session
used by the autograd wrapper; reconstructions checked exactly against the
oracle's defining sums on sampled elements spread over every block."""
import numpy as np
import pytest
import torch

from oracle import ring
from paper_2403_11166_gb300 import inputs
from tests.gpu_util import to_np

pytestmark = pytest.mark.gpu
T = 41


def test_conv128_fwd_bwd_sampled():
    from paper_2403_11166_gb300 import autograd, he
    sess = autograd.HeSession(13, 3, 60, T, seed=8)
    Ly = he.Layer(he.CONV, 128, 128, 128, 16, 16, 3, 1)
    g = inputs.rng(9)
    W = inputs.gaussian_fixed(g, (128, 128, 3, 3))
    x = inputs.gaussian_fixed(g, (128, 128, 16, 16))
    gy = inputs.gaussian_fixed(g, (128, 128, 16, 16))
    x0, x1 = inputs.split_shares(g, x)
    g0, g1 = inputs.split_shares(g, gy)
    dev = sess.device
    td = lambda a: torch.as_tensor(np.ascontiguousarray(a).astype(np.int64) if a.dtype != np.uint64 else a.view(np.int64), device=dev)
    Wr = td(W) & sess.mask
    y0, y1 = sess.forward(Ly, Wr, None, td(x0), td(x1))
    gx0, gx1, gw, gb = sess.backward(Ly, Wr, td(x0), td(x1), td(g0), td(g1), True)
    torch.cuda.synchronize()
    assert sess.ctx.sync_status() == 0
    Y = to_np(sess.reconstruct(y0, y1)).reshape(128, 128, 16, 16)
    GX = to_np(sess.reconstruct(gx0, gx1)).reshape(128, 128, 16, 16)
    GW = to_np(gw).reshape(128, 128, 3, 3)
    r = np.random.default_rng(10)
    idx = [tuple(int(v) for v in (r.integers(128), r.integers(128), r.integers(16), r.integers(16))) for _ in range(48)]
    idx += [(0, 0, 0, 0), (127, 127, 15, 15), (5, 64, 0, 15), (77, 3, 15, 0)]
    assert [int(Y[i]) for i in idx] == ring.ring_conv2d_at(W, x, 1, T, idx)
    assert [int(GX[i]) for i in idx] == ring.ring_conv2d_dgrad_at(W, gy, 1, T, idx)
    idw = [tuple(int(v) for v in (r.integers(128), r.integers(128), r.integers(3), r.integers(3))) for _ in range(24)]
    idw += [(0, 0, 0, 0), (127, 127, 2, 2)]
    assert [int(GW[i]) for i in idw] == ring.ring_conv2d_wgrad_at(gy, x, 1, 3, T, idw)
    GB = to_np(gb)
    with np.errstate(over="ignore"):
        want_gb = gy.astype(np.int64).view(np.uint64).sum(axis=(0, 2, 3), dtype=np.uint64) & np.uint64((1 << T) - 1)
    assert (GB == want_gb).all()
