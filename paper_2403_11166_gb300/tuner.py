"""Autotuner of the batched HE linear layers (measurement-driven).

Search space: the context knobs (NTT register-block radix 2^4 / 2^5, output
columns per thread of the multiply-accumulate: 2, 4, 8, and its operand
staging: per-thread cp.async ring or producer-warp bulk copies) and, per
distinct layer shape, the planner's cheapest-first partitions (tile shapes:
batch / channel blocks and spatial tiles).  For every knob setting each shape's
candidates are timed as a single layer (per-layer calls, CUDA events on the
launch stream, median of `reps`), the fastest is kept, and the whole batch is
then timed as a captured CUDA graph; the best setting wins.  A batch may mix
roles (forward, input gradient, weight gradient: a training step's products);
candidates are then chosen per (shape, role).  Results do not depend on any of
these choices (the tests check that); only speed does.
"""
from __future__ import annotations

import itertools
import statistics
from typing import Dict, List, Optional, Tuple

import torch

from . import he


def _shape_key(L: he.Layer) -> Tuple:
    return (L.kind, L.batch, L.c_in, L.c_out, L.height, L.width, L.kernel, L.pad)


def _layer_buffers(ctx: he.Context, L: he.Layer, seed: int):
    g = torch.Generator(device="cpu").manual_seed(seed)
    wshape = (L.c_out, L.c_in) if L.kind == he.FC else (L.c_out, L.c_in, L.kernel, L.kernel)
    xshape = (L.batch, L.c_in) if L.kind == he.FC else (L.batch, L.c_in, L.height, L.width)
    dev = f"cuda:{ctx.device}"
    W = torch.randint(-(1 << 14), 1 << 14, wshape, generator=g, dtype=torch.int64).to(dev)
    x0 = torch.randint(0, 1 << ctx.t_bits, xshape, generator=g, dtype=torch.int64).to(dev)
    x1 = torch.randint(0, 1 << ctx.t_bits, xshape, generator=g, dtype=torch.int64).to(dev)
    return W, x0, x1


def _grad_buffers(ctx: he.Context, L: he.Layer, seed: int):
    """Two Z_t shares shaped like the layer's output (grad_Y)."""
    g = torch.Generator(device="cpu").manual_seed(seed + 7919)
    if L.kind == he.FC:
        yshape = (L.batch, L.c_out)
    else:
        yshape = (L.batch, L.c_out, L.height + 2 * L.pad - L.kernel + 1, L.width + 2 * L.pad - L.kernel + 1)
    dev = f"cuda:{ctx.device}"
    return tuple(torch.randint(0, 1 << ctx.t_bits, yshape, generator=g, dtype=torch.int64).to(dev) for _ in range(2))


def time_layer(ctx: he.Context, sk: he.SecretKey, L: he.Layer, part, reps: int = 5, role: int = he.ROLE_FWD) -> float:
    """Median ms of one pass of layer L's product of `role` through the per-layer
    calls: encode, encrypt, Alg. 1, decrypt (forward, input gradient), or both
    encryptions, Alg. 2, decrypt (weight gradient)."""
    plan = he.Plan(ctx, L, role, part)
    S = plan.sizes
    W, x0, x1 = _layer_buffers(ctx, L, 1)
    g0, g1 = _grad_buffers(ctx, L, 1)
    ws = plan.new_ws(max(S.ws_encrypt, S.ws_forward, S.ws_backward, S.ws_decrypt))
    ct_out = plan.new_ct(S.ct_out)
    y0 = torch.empty(S.out_elems, dtype=torch.int64, device=W.device)
    y1 = torch.empty_like(y0)
    if role == he.ROLE_WGRAD:
        ct_x1, ct_g1 = plan.new_ct(S.ct_in), plan.new_ct(S.pt)

        def run(i):
            he.encrypt_share(ctx, sk, plan, he.OPERAND_INPUT, x1, 10 + i, ct_x1, ws)
            he.encrypt_share(ctx, sk, plan, he.OPERAND_KERNEL, g1, 30 + i, ct_g1, ws)
            he.he_linear_backward(ctx, None, plan, None, None, ct_x1, ct_g1, g0, x0, 0, 20 + i, None, None, ct_out,
                                  y0, ws)
            he.decrypt_to_share(ctx, sk, plan, ct_out, y1, False, ws)
    else:
        pt, ct_in = plan.new_pt(S.pt), plan.new_ct(S.ct_in)
        v0, v1 = (x0, x1) if role == he.ROLE_FWD else (g0, g1)

        def run(i):
            he.encode_weights(ctx, plan, he.OPERAND_KERNEL, W, pt)
            he.encrypt_share(ctx, sk, plan, he.OPERAND_INPUT, v1, 10 + i, ct_in, ws)
            he.he_linear_forward(ctx, plan, ct_in, pt, v0, None, 20 + i, ct_out, y0, ws)
            he.decrypt_to_share(ctx, sk, plan, ct_out, y1, False, ws)
    run(0)
    times = []
    stream = torch.cuda.current_stream()
    for i in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        run(i + 1)
        b.record(stream)
        b.synchronize()
        times.append(a.elapsed_time(b))
    return statistics.median(times)


class GraphBatch:
    """A committed Batch of the given layers/partitions (and roles: forward by
    default) with its buffers and a captured CUDA graph of one pass."""

    def __init__(self, ctx: he.Context, sk: he.SecretKey, layers: List[he.Layer], parts: List[Optional[tuple]],
                 capture: bool = True, seed: int = 0, roles: Optional[List[int]] = None):
        self.ctx = ctx
        roles = roles or [he.ROLE_FWD] * len(layers)
        self.plans = [he.Plan(ctx, L, r, p) for L, r, p in zip(layers, roles, parts)]
        self.batch = he.Batch(ctx, self.plans)
        self.bufs = []
        for i, (L, r, p) in enumerate(zip(layers, roles, self.plans)):
            W, x0, x1 = _layer_buffers(ctx, L, seed + i)
            y0 = torch.empty(p.sizes.out_elems, dtype=torch.int64, device=W.device)
            y1 = torch.empty_like(y0)
            if r == he.ROLE_FWD:
                self.batch.bind(i, W, x1, x0, None, y0, y1)
                self.bufs.append((W, x0, x1, y0, y1))
            else:
                g0, g1 = _grad_buffers(ctx, L, seed + i)
                if r == he.ROLE_DGRAD:
                    self.batch.bind(i, W, g1, g0, None, y0, y1)
                else:
                    self.batch.bind_wgrad(i, g0, g1, x0, x1, y0, y1)
                self.bufs.append((W, x0, x1, g0, g1, y0, y1))
        self.ws = torch.empty((self.batch.workspace_bytes + 7) // 8, dtype=torch.int64, device=f"cuda:{ctx.device}")
        self.batch.commit(sk, self.ws, 1000, 5000)
        self.graph = None
        if capture:
            s = torch.cuda.Stream()
            s.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(s):
                self.batch.forward(stream=s)
            torch.cuda.current_stream().wait_stream(s)
            torch.cuda.synchronize()
            self.graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(self.graph):
                self.batch.forward()
        self.products = sum(p.sizes.products * (2 if r == he.ROLE_WGRAD else 1) for p, r in zip(self.plans, roles))

    def run(self):
        if self.graph is not None:
            self.graph.replay()
        else:
            self.batch.forward()

    def time(self, reps: int = 5) -> float:
        self.run()
        torch.cuda.synchronize()
        stream = torch.cuda.current_stream()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            self.run()
        b.record(stream)
        b.synchronize()
        return a.elapsed_time(b) / reps


def tune_batch(ctx: he.Context, sk: he.SecretKey, layers: List[he.Layer], topk: int = 3, reps: int = 3,
               radices=(4, 5), columns=(2, 4, 8), stagings=(0, 1), roles: Optional[List[int]] = None) -> Dict:
    """Returns {"ntt_log_radix", "mac_columns", "mac_staging", "partitions" (per entry), "ms", "table"}
    and leaves the context tuned to the winner.  `roles` (per entry, default all
    forward) lets one batch hold a training step's forward and backward products."""
    roles = roles or [he.ROLE_FWD] * len(layers)
    keys = [(_shape_key(L), r) for L, r in zip(layers, roles)]
    shapes: Dict[Tuple, Tuple[he.Layer, int]] = {}
    for k, L, r in zip(keys, layers, roles):
        shapes.setdefault(k, (L, r))
    table = []
    best = None
    for radix, cols, staging in itertools.product(radices, columns, stagings):
        ctx.tune(he.TUNE_NTT_LOG_RADIX, radix)
        ctx.tune(he.TUNE_MAC_COLUMNS, cols)
        ctx.tune(he.TUNE_MAC_STAGING, staging)
        chosen = {}
        for key, (L, r) in shapes.items():
            cands = he.plan_candidates(ctx, L, r, topk)
            timed = [(time_layer(ctx, sk, L, c, reps, r), c) for c in cands]
            timed.sort()
            chosen[key] = timed[0][1]
            table.append({"radix": radix, "columns": cols, "staging": staging, "shape": key[0], "role": key[1],
                          "candidates": [{"partition": c, "ms": round(t, 4)} for t, c in timed]})
        gb = GraphBatch(ctx, sk, layers, [chosen[k] for k in keys], roles=roles)
        ms = gb.time(reps)
        del gb
        torch.cuda.empty_cache()
        table.append({"radix": radix, "columns": cols, "staging": staging, "batch_graph_ms": round(ms, 4)})
        if best is None or ms < best["ms"]:
            best = {"ntt_log_radix": radix, "mac_columns": cols, "mac_staging": staging,
                    "partitions": [chosen[k] for k in keys], "ms": ms}
    ctx.tune(he.TUNE_NTT_LOG_RADIX, best["ntt_log_radix"])
    ctx.tune(he.TUNE_MAC_COLUMNS, best["mac_columns"])
    ctx.tune(he.TUNE_MAC_STAGING, best["mac_staging"])
    best["table"] = table
    return best
