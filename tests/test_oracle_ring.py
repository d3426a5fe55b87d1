"""Pins for the direct ring operators: against Python-integer brute force and
against float64 PyTorch conv / matmul on small fixed-point values (no wrap)."""
import numpy as np
import torch

from oracle import ring

T = 41
MASK = (1 << T) - 1


def _brute_conv(w, x, pad):
    xp = np.pad(x, ((0, 0), (0, 0), (pad, pad), (pad, pad)))
    B, C, H, W = xp.shape
    O, _, S, _ = w.shape
    out = np.zeros((B, O, H - S + 1, W - S + 1), dtype=object)
    for b in range(B):
        for o in range(O):
            for i in range(H - S + 1):
                for j in range(W - S + 1):
                    acc = 0
                    for c in range(C):
                        for u in range(S):
                            for v in range(S):
                                acc += int(w[o, c, u, v]) * int(xp[b, c, i + u, j + v])
                    out[b, o, i, j] = acc & MASK
    return out


def test_conv_matches_bruteforce_with_wrap():
    g = np.random.default_rng(0)
    x = g.integers(0, 1 << T, size=(2, 3, 5, 4), dtype=np.uint64)
    w = g.integers(-(1 << 15), 1 << 15, size=(2, 3, 3, 3), dtype=np.int64)
    got = ring.ring_conv2d(w, x, 1, T)
    assert (got.astype(object) == _brute_conv(w, x.astype(object), 1)).all()


def test_float_equivalence_small_values():
    g = np.random.default_rng(1)
    x = g.integers(-50, 50, size=(2, 4, 6, 6))
    w = g.integers(-50, 50, size=(3, 4, 3, 3))
    gy = g.integers(-50, 50, size=(2, 3, 6, 6))
    xt, wt, gyt = (torch.tensor(a, dtype=torch.float64) for a in (x, w, gy))
    xt.requires_grad_(True)
    wt.requires_grad_(True)
    y = torch.nn.functional.conv2d(xt, wt, padding=1)
    y.backward(gyt)
    signed = lambda a: (a.astype(np.int64) << 23) >> 23
    assert (signed(ring.ring_conv2d(w, x, 1, T)) == y.detach().numpy()).all()
    assert (signed(ring.ring_conv2d_dgrad(w, gy, 1, T)) == xt.grad.numpy()).all()
    assert (signed(ring.ring_conv2d_wgrad(gy, x, 1, 3, T)) == wt.grad.numpy()).all()

    xf = g.integers(-50, 50, size=(5, 7))
    wf = g.integers(-50, 50, size=(4, 7))
    gyf = g.integers(-50, 50, size=(5, 4))
    xt, wt = (torch.tensor(a, dtype=torch.float64, requires_grad=True) for a in (xf, wf))
    yt = xt @ wt.T
    yt.backward(torch.tensor(gyf, dtype=torch.float64))
    assert (signed(ring.ring_matmul(wf, xf, T)) == yt.detach().numpy()).all()
    assert (signed(ring.ring_matmul_dgrad(wf, gyf, T)) == xt.grad.numpy()).all()
    assert (signed(ring.ring_matmul_wgrad(gyf, xf, T)) == wt.grad.numpy()).all()


def test_sampled_operators_match_full():
    g = np.random.default_rng(3)
    x = g.integers(0, 1 << T, size=(3, 4, 7, 6), dtype=np.uint64)
    w = g.integers(0, 1 << T, size=(5, 4, 3, 3), dtype=np.uint64)
    gy = g.integers(0, 1 << T, size=(3, 5, 7, 6), dtype=np.uint64)
    full_y = ring.ring_conv2d(w, x, 1, T)
    full_gx = ring.ring_conv2d_dgrad(w, gy, 1, T)
    full_gw = ring.ring_conv2d_wgrad(gy, x, 1, 3, T)
    idx = [(0, 0, 0, 0), (2, 4, 6, 5), (1, 2, 3, 0), (0, 3, 6, 2)]
    assert ring.ring_conv2d_at(w, x, 1, T, idx) == [int(full_y[i]) for i in idx]
    idx_x = [(0, 0, 0, 0), (2, 3, 6, 5), (1, 1, 3, 4)]
    assert ring.ring_conv2d_dgrad_at(w, gy, 1, T, idx_x) == [int(full_gx[i]) for i in idx_x]
    idx_w = [(0, 0, 0, 0), (4, 3, 2, 2), (2, 1, 0, 2)]
    assert ring.ring_conv2d_wgrad_at(gy, x, 1, 3, T, idx_w) == [int(full_gw[i]) for i in idx_w]
