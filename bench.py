#!/usr/bin/env python
"""Benchmark of the HE linear-layer hot path (one JSON line on stdout).

Workload: the forward homomorphic product of a conv 3x3, 16 -> 16 channels,
32 x 32 input, pad 1, batch 64 (BFV N = 8192, three 60-bit primes, t = 2^41),
seeded synthetic Gaussian fixed-point data (12 fractional bits).  One step =
the whole forward path of Algorithm 1: encode_weights (MO: pi_W + NTT) and
he_linear_forward_prepare (MO: NTT(Delta <X>_0), mask s, NTT(Delta s), share
s + b) on their own streams, and the layer streamed in row slices through
encrypt_share (DO: pi_v + BFV encryption), he_linear_forward_apply (MO: ct x pt
multiply-accumulate with the add of <X>_0 and the re-mask fused) and
decrypt_to_share (DO), each slice's stages overlapping the neighbours'.  Three
steps are in flight (one device buffer set each, --in-flight): step i + 1's
encoding, preparation and encryption run beside step i's multiply-accumulate
and decryption; the line also gives one step's latency with no such overlap
(ms_per_step_unpipelined).  Metric:
ct x pt products per second (whole job), plus the per-kernel roofline of the
dominant kernel, an end-to-end number with host buffers, and the oracle timed
on the host cores.

    python bench.py [--gpus N --steps K --warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "HE linear-layer ct x pt products/s (conv3x3 16->16, 32x32, B=64, N=8192, fwd)"
UNIT = "products/s"
LOG_N, L, PRIME_BITS, T_BITS = 13, 3, 60, 41
LAYER = dict(batch=64, c_in=16, c_out=16, h=32, w=32, s=3, pad=1)
WORKLOAD = "conv3x3_16to16_32x32_b64_fwd_N8192_L3x60_t41"
IMAD_PER_CLK_SM = 64         # 32-bit integer multiply-add results per clock per SM (16 per sub-partition)
MAX_SM_MHZ = 2070.0          # GB300 maximum SM clock (MEASURED_PEAKS.json sm_max_mhz overrides it)
HEADLINE_PARTITION = (7, 1, 1, 32, 32, 3, 3)   # the planner's choice for the workload (default knobs)


def _record(st):
    import torch
    ev = torch.cuda.Event()
    ev.record(st)
    return ev


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-sweep", action="store_true")
    ap.add_argument("--sweep-only", action="store_true", help="run only the batched NTT sweep")
    ap.add_argument("--sweep-polys", type=int, default=10000)
    ap.add_argument("--sweep-points", default="12x2,12x3,12x4,13x2,13x3,13x4,14x2,14x3,14x4")
    ap.add_argument("--sweep-reps", type=int, default=3)
    ap.add_argument("--ntt-log-radix", type=int, default=0, help="force the NTT radix knob (4 or 5)")
    ap.add_argument("--mac-columns", type=int, default=-1,
                    help="force the MAC knob (0: shared-memory staged; 2, 4, 8: columns per thread)")
    ap.add_argument("--mac-staging", type=int, default=-1,
                    help="force the MAC staging knob (0: per-thread cp.async ring, 1: bulk copies by a producer warp)")
    ap.add_argument("--in-flight", type=int, default=3,
                    help="steps in flight in the timed runs (device buffer sets); 1: each step joins before the next")
    ap.add_argument("--chunks", type=int, default=1,
                    help="stream the layer through encrypt / multiply-accumulate / decrypt in this many row slices")
    ap.add_argument("--no-extras", action="store_true", help="skip the batched / training / large-conv workloads")
    ap.add_argument("--extras-only", action="store_true", help="run only the extra workloads (JSON line)")
    ap.add_argument("--extra", action="append", default=None,
                    help="with --extras-only: run only this extra workload (repeatable)")
    return ap.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(vals, world: int, device="cpu"):
    """Element-wise maximum of `vals` over all ranks (the job's time is the
    slowest rank's); identity for one process."""
    if world <= 1:
        return [float(v) for v in vals]
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v) for v in vals], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.tolist()]


def job_throughput(units_per_rank_step: int, steps: int, world: int, ms_max: float) -> float:
    """Whole-job rate: the units every rank processed over the max-over-ranks time."""
    return units_per_rank_step * steps * world / (ms_max * 1e-3)


# ---------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid: str | None):
        self.uuid = uuid
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        rows = [r.split(", ") for r in out.strip().splitlines() if r.strip()]
        if self.uuid:
            mine = [r for r in rows if r and self.uuid in r[0]]
            rows = mine or rows
        sm = [float(r[1]) for r in rows if len(r) > 8 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if len(r) > 8 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows if len(r) > 8 for i in range(4) if r[5 + i].strip() == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(sm)}


# ---------------------------------------------------------------- roofline accounting
def limb_ntt_mults(n: int) -> float:
    """Accounting: one limb-NTT = (N/2) log2 N Shoup modmuls x 10 32-bit multiplies."""
    return 10.0 * (n // 2) * (n.bit_length() - 1)


def kernel_work(name: str, S, n: int, L_: int):
    """(32-bit multiply ops, algorithmic HBM bytes) of ONE launch of kernel `name`
    in this workload's step."""
    ln = L_ * n
    if name == "ntt_encrypt":
        return S.ct_in * L_ * limb_ntt_mults(n), S.ct_in * (16 * ln + n)            # write ct, read errors
    if name == "ntt_addplain":
        return S.ct_in * L_ * limb_ntt_mults(n), S.ct_in * 16 * ln                  # read c0, write c0'
    if name == "ntt_encode":
        return S.pt * L_ * limb_ntt_mults(n), S.pt * 8 * ln                         # write pt
    if name == "ntt_mask":
        return S.ct_out * L_ * limb_ntt_mults(n), S.ct_out * (8 * n + 16 * ln)      # read mask, rw c0
    if name == "intt_decrypt":
        return S.ct_out * L_ * limb_ntt_mults(n), S.ct_out * (16 * ln + 8 * ln)     # read ct, write residues
    if name == "ntt_mo_prep":   # NTT(Delta x0) per input ct, NTT(Delta s) per output ct
        return (S.ct_in + S.ct_out) * L_ * limb_ntt_mults(n), S.ct_in * 8 * ln + S.ct_out * (8 * n + 8 * ln)
    if name == "mac":           # reads ct_in, NTT(Delta x0), pt, NTT(Delta s); writes ct_out
        return S.products * 2 * ln * 4.0, (S.ct_in * 24 * ln + S.pt * 8 * ln + S.ct_out * 24 * ln)
    return 0.0, 0.0


def roofline(prof: dict, serial: dict, S, n: int, L_: int, steps: int, peaks: dict, clocks: dict,
             unpiped: dict | None = None):
    """Dominant kernel: the largest share of a step when the step's kernels run one
    at a time (`serial`, a profiling pass on one stream after the timed region);
    its achieved rate uses its launch duration in a timed run (CUDA events on its
    own stream): the timed run of unpipelined steps (`unpiped`) when given, where
    the multiply-accumulate and the decryption have the GPU to themselves, else the
    main timed run (`prof`).  Kernels that overlap others (encode / preparation /
    encryption on three streams; with several steps in flight, the next step's
    transforms beside this step's multiply-accumulate and decryption) show longer
    event durations in the main timed run than alone."""
    total = sum(v[1] for v in serial.values()) or 1.0
    table = {}
    for name, (launches, ms) in prof.items():
        mults, byts = kernel_work(name, S, n, L_)
        per = ms / max(1, launches) * 1e-3
        sl, sms = serial.get(name, (0, 0.0))
        alone = sms / max(1, sl) * 1e-3 if sl else None
        ul, ums = (unpiped or {}).get(name, (0, 0.0))
        table[name] = {"launches": launches, "ms_per_launch": per * 1e3,
                       "ms_per_launch_unpipelined": ums / ul if ul else None,
                       "ms_per_launch_alone": alone * 1e3 if alone else None,
                       "share_alone": sms / total,
                       "tmul_per_s": mults / per / 1e12 if mults else None,
                       "gb_per_s": byts / per / 1e9 if byts else None,
                       # accounting fraction of the integer peak, in the step and alone
                       "frac_alu": round(mults / per / 1e12 / peaks["alu_tmul"], 4) if mults else None,
                       "frac_alu_alone": round(mults / alone / 1e12 / peaks["alu_tmul"], 4) if mults and alone else None}
    dom = max((k for k in table if kernel_work(k, S, n, L_)[0] > 0), key=lambda k: table[k]["share_alone"])
    mults, byts = kernel_work(dom, S, n, L_)
    timed = "unpipelined timed run" if table[dom]["ms_per_launch_unpipelined"] else "timed run"
    per = (table[dom]["ms_per_launch_unpipelined"] or table[dom]["ms_per_launch"]) * 1e-3
    alu_peak = peaks["alu_tmul"]
    achieved = mults / per / 1e12
    return dom, table, {
        "kernel": dom, "bound": "alu", "achieved": round(achieved, 3), "peak": round(alu_peak, 3),
        "duration_from": timed, "ms_per_launch": round(per * 1e3, 5),
        "unit": "T 32-bit mult/s", "frac": round(achieved / alu_peak, 4), "traffic": ncu_traffic(dom),
        "peak_source": peaks["alu_source"],
        "hbm": {"achieved_gbs": round(byts / per / 1e9, 1), "peak_gbs": peaks["hbm_gbs"],
                "frac": round(byts / per / 1e9 / peaks["hbm_gbs"], 4), "peak_source": "MEASURED_PEAKS.json (measured)"},
        "algorithmic_mults_per_launch": mults, "algorithmic_bytes_per_launch": byts,
    }


def csrc_digest() -> str:
    """Short digest of the CUDA sources (ties a committed ncu figure to the kernels it was taken on)."""
    import hashlib
    d = os.path.join(ROOT, "paper_2403_11166_gb300", "csrc")
    h = hashlib.sha256()
    for f in sorted(os.listdir(d)):
        if f.endswith((".cu", ".cuh", ".h")):
            h.update(f.encode())
            with open(os.path.join(d, f), "rb") as fh:
                h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel: str):
    """DRAM bytes (read + write) of one launch of `kernel` from profiles/dram_traffic.txt, if that
    line was taken on the current kernel sources; else None."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.txt")
    if not os.path.exists(path):
        return None
    digest = csrc_digest()
    with open(path) as f:
        for line in f:
            parts = line.split()
            if len(parts) >= 3 and not line.startswith("#") and parts[0] == kernel and parts[2] == digest:
                return int(parts[1])
    return None


def sm_count(device: int = 0) -> int:
    """Streaming multiprocessors of the device (152 on a GB300)."""
    import torch
    return int(torch.cuda.get_device_properties(device).multi_processor_count)


def load_peaks(sms: int = 152):
    """HBM peak from MEASURED_PEAKS.json (else the fallback) and the integer
    multiply peak derived from the SM count, 64 IMAD results per clock per SM and
    the maximum SM clock."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    hbm, src, mhz = 6800.0, "fallback", MAX_SM_MHZ
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        hbm = float(d.get("hbm_gbs", hbm))
        mhz = float(d.get("sm_max_mhz", mhz))
        src = "measured"
    alu = sms * IMAD_PER_CLK_SM * mhz * 1e6 / 1e12
    return {"hbm_gbs": hbm, "hbm_source": src, "alu_tmul": alu, "sms": sms,
            "alu_source": f"derived: {sms} SMs (device properties) x {IMAD_PER_CLK_SM} IMAD/clk x {mhz:.0f} MHz"}


def check_peak(peaks: dict, imad32_probe: float) -> str:
    """The derived integer peak against the register-only 32-bit multiply-add
    probe: more than 5 % apart means a wrong SM count, clock or pipe width."""
    gap = abs(imad32_probe - peaks["alu_tmul"]) / peaks["alu_tmul"]
    if gap > 0.05:
        msg = (f"PEAK MISMATCH: derived {peaks['alu_tmul']:.2f} T/s vs probe {imad32_probe:.2f} T/s "
               f"({100 * gap:.1f} % apart)")
        print(msg, file=sys.stderr, flush=True)
        return msg
    return f"ok: probe {imad32_probe:.2f} T/s within {100 * gap:.1f} % of the derived peak"


# ---------------------------------------------------------------- batched NTT sweep (row a10)
def ntt_sweep(he, device: int, polys: int, points: str, reps: int, log_radix: int = 0):
    """Sustained batched forward NTT and inverse NTT over `polys` uniform random
    polynomials per (N, L) point (60-bit primes), CUDA events on the launch stream."""
    import torch
    peaks = load_peaks(sm_count(device))
    out = []
    stream = torch.cuda.current_stream()
    for pt in points.split(","):
        log_n, L_ = (int(v) for v in pt.split("x"))
        ctx = he.Context(log_n, L_, 60, T_BITS, device=device)
        if log_radix:
            ctx.tune(he.TUNE_NTT_LOG_RADIX, log_radix)
        n = 1 << log_n
        q_min = min(ctx.primes()[0])
        a = torch.randint(0, q_min, (polys, L_, n), dtype=torch.int64, device=f"cuda:{device}")
        he.pencil_ntt_batch(ctx, a, inverse=False)
        he.pencil_ntt_batch(ctx, a, inverse=True)
        res = {}
        for inv in (False, True):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(reps):
                he.pencil_ntt_batch(ctx, a, inverse=inv)
            e1.record(stream)
            torch.cuda.synchronize()
            sec = e0.elapsed_time(e1) * 1e-3 / reps
            limb_ntts = polys * L_
            mults = limb_ntts * limb_ntt_mults(n)
            byts = limb_ntts * 16 * n
            res["inv" if inv else "fwd"] = {
                "limb_ntts_per_s": limb_ntts / sec, "ms": sec * 1e3,
                "frac_alu": round(mults / sec / 1e12 / peaks["alu_tmul"], 4),
                "frac_hbm": round(byts / sec / 1e9 / peaks["hbm_gbs"], 4)}
        out.append({"N": n, "L": L_, "polys": polys, "log_radix": ctx.get_tune(he.TUNE_NTT_LOG_RADIX), **res})
        del a
        ctx.close()
    return out


# ---------------------------------------------------------------- other workloads (reported beside the headline)
def batched_uneven(he, device: int, reps: int = 5):
    """96 layers: 32 x FC 512->10 (B 16), 32 x conv3x3 64->64 on 8x8 (B 32, pad 1),
    32 x conv1x1 128->256 on 4x4 (B 8); N = 8192, 3 x 60-bit primes.  Per-layer
    launches (planner partitions, default knobs) vs one captured graph of the
    batched sequence, untuned and autotuned."""
    import torch
    from paper_2403_11166_gb300 import tuner
    layers = ([he.Layer(he.FC, 16, 512, 10)] * 32 + [he.Layer(he.CONV, 32, 64, 64, 8, 8, 3, 1)] * 32
              + [he.Layer(he.CONV, 8, 128, 256, 4, 4, 1, 0)] * 32)
    out = {"layers": len(layers)}
    ctx = he.Context(LOG_N, L, PRIME_BITS, T_BITS, device=device)
    sk = ctx.keygen(77)
    # per-layer launches: 4 C-ABI calls per layer
    plans = [he.Plan(ctx, Ly, he.ROLE_FWD, None) for Ly in layers]
    bufs = []
    for i, (Ly, p) in enumerate(zip(layers, plans)):
        W, x0, x1 = tuner._layer_buffers(ctx, Ly, i)
        S = p.sizes
        bufs.append((W, x0, x1, p.new_pt(S.pt), p.new_ct(S.ct_in), p.new_ct(S.ct_out),
                     torch.empty(S.out_elems, dtype=torch.int64, device=W.device),
                     torch.empty(S.out_elems, dtype=torch.int64, device=W.device),
                     p.new_ws(max(S.ws_encrypt, S.ws_forward, S.ws_decrypt))))
    products = sum(p.sizes.products for p in plans)

    def per_layer(step):
        for i, (p, b) in enumerate(zip(plans, bufs)):
            W, x0, x1, pt, ct_in, ct_out, y0, y1, ws = b
            he.encode_weights(ctx, p, he.OPERAND_KERNEL, W, pt)
            he.encrypt_share(ctx, sk, p, he.OPERAND_INPUT, x1, 1000 + i + (step << 32), ct_in, ws)
            he.he_linear_forward(ctx, p, ct_in, pt, x0, None, 5000 + i + (step << 32), ct_out, y0, ws)
            he.decrypt_to_share(ctx, sk, p, ct_out, y1, False, ws)
    per_layer(0)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for r in range(reps):
        per_layer(r + 1)
    b.record(stream)
    b.synchronize()
    ms_pl = a.elapsed_time(b) / reps
    out["per_layer_launches"] = {"ms_per_step": ms_pl, "products_per_s": products / (ms_pl * 1e-3),
                                 "launches_per_step": len(layers) * 10, "products_per_step": products}
    del bufs, plans
    torch.cuda.empty_cache()
    gb = tuner.GraphBatch(ctx, sk, layers, [None] * len(layers))
    ms_g = gb.time(reps)
    out["batched_graph_untuned"] = {"ms_per_step": ms_g, "products_per_s": gb.products / (ms_g * 1e-3),
                                    "launches_per_step": 12, "products_per_step": gb.products}
    del gb
    torch.cuda.empty_cache()
    t0 = time.perf_counter()
    best = tuner.tune_batch(ctx, sk, layers, topk=3, reps=3)
    tune_s = time.perf_counter() - t0
    gb = tuner.GraphBatch(ctx, sk, layers, best["partitions"])
    ms_t = gb.time(reps)
    out["batched_graph_autotuned"] = {"ms_per_step": ms_t, "products_per_s": gb.products / (ms_t * 1e-3),
                                      "products_per_step": gb.products, "ntt_log_radix": best["ntt_log_radix"],
                                      "mac_columns": best["mac_columns"], "mac_staging": best["mac_staging"],
                                      "partitions": sorted({str(p) for p in best["partitions"]}),
                                      "tuning_seconds": round(tune_s, 1)}
    del gb
    ctx.close()
    torch.cuda.empty_cache()
    return out


def batched_fwd_bwd(he, device: int, reps: int = 5):
    """A training step's HE products of the 96 uneven layers: forward (Alg. 1),
    input gradient (Alg. 1 on the transposed kernel) and weight gradient (Alg. 2)
    of every layer, 288 entries.  Per-layer C-ABI calls (encode, encrypt,
    evaluate, decrypt for each) vs one captured CUDA graph of the batch."""
    import torch
    from paper_2403_11166_gb300 import tuner
    layers = ([he.Layer(he.FC, 16, 512, 10)] * 32 + [he.Layer(he.CONV, 32, 64, 64, 8, 8, 3, 1)] * 32
              + [he.Layer(he.CONV, 8, 128, 256, 4, 4, 1, 0)] * 32)
    ctx = he.Context(LOG_N, L, PRIME_BITS, T_BITS, device=device)
    sk = ctx.keygen(78)
    dev = f"cuda:{device}"
    roles = (he.ROLE_FWD, he.ROLE_DGRAD, he.ROLE_WGRAD)
    entries = [(r, Ly) for Ly in layers for r in roles]
    plans = [he.Plan(ctx, Ly, r, None) for r, Ly in entries]
    g = torch.Generator(device="cpu").manual_seed(79)

    def shares(shape):
        return tuple(torch.randint(0, 1 << T_BITS, shape, generator=g, dtype=torch.int64).to(dev) for _ in range(2))
    data = []
    for i, ((r, Ly), p) in enumerate(zip(entries, plans)):
        W, x0, x1 = tuner._layer_buffers(ctx, Ly, i)
        if Ly.kind == he.FC:
            yshape = (Ly.batch, Ly.c_out)
        else:
            yshape = (Ly.batch, Ly.c_out, Ly.height + 2 * Ly.pad - Ly.kernel + 1,
                      Ly.width + 2 * Ly.pad - Ly.kernel + 1)
        g0, g1 = shares(yshape)
        data.append({"W": W, "x0": x0, "x1": x1, "g0": g0, "g1": g1})
    products = sum(p.sizes.products * (2 if r == he.ROLE_WGRAD else 1) for (r, _), p in zip(entries, plans))
    out = {"layers": len(layers), "entries": len(entries), "products_per_step": products}

    # per-layer calls
    bufs = []
    for (r, Ly), p in zip(entries, plans):
        S = p.sizes
        y = [torch.empty(S.out_elems, dtype=torch.int64, device=dev) for _ in range(2)]
        ws = p.new_ws(max(S.ws_encrypt, S.ws_forward, S.ws_backward, S.ws_decrypt))
        if r == he.ROLE_WGRAD:
            bufs.append((p.new_ct(S.ct_in), p.new_ct(S.pt), p.new_ct(S.ct_out), y[0], y[1], ws))
        else:
            bufs.append((p.new_pt(S.pt), p.new_ct(S.ct_in), p.new_ct(S.ct_out), y[0], y[1], ws))

    def per_layer(step):
        for i, ((r, Ly), p, d, b) in enumerate(zip(entries, plans, data, bufs)):
            e, m = 1000 + i + (step << 32), 5000 + i + (step << 32)
            if r == he.ROLE_WGRAD:
                ct_x1, ct_g1, ct_out, y0, y1, ws = b
                he.encrypt_share(ctx, sk, p, he.OPERAND_INPUT, d["x1"], e, ct_x1, ws)
                he.encrypt_share(ctx, sk, p, he.OPERAND_KERNEL, d["g1"], e + (1 << 31), ct_g1, ws)
                he.he_linear_backward(ctx, None, p, None, None, ct_x1, ct_g1, d["g0"], d["x0"], 0, m, None, None,
                                      ct_out, y0, ws)
            else:
                pt, ct_in, ct_out, y0, y1, ws = b
                v0, v1 = (d["x0"], d["x1"]) if r == he.ROLE_FWD else (d["g0"], d["g1"])
                he.encode_weights(ctx, p, he.OPERAND_KERNEL, d["W"], pt)
                he.encrypt_share(ctx, sk, p, he.OPERAND_INPUT, v1, e, ct_in, ws)
                if r == he.ROLE_FWD:
                    he.he_linear_forward(ctx, p, ct_in, pt, v0, None, m, ct_out, y0, ws)
                else:
                    he.he_linear_backward(ctx, p, None, ct_in, pt, None, None, v0, None, m, 0, ct_out, y0, None,
                                          None, ws)
            he.decrypt_to_share(ctx, sk, p, ct_out, y1, False, ws)
    per_layer(0)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for r in range(reps):
        per_layer(r + 1)
    b.record(stream)
    b.synchronize()
    ms_pl = a.elapsed_time(b) / reps
    out["per_layer_calls"] = {"ms_per_step": ms_pl, "products_per_s": products / (ms_pl * 1e-3)}
    del bufs
    torch.cuda.empty_cache()

    # one batch, one captured graph
    batch = he.Batch(ctx, plans)
    outs = []
    for i, ((r, Ly), p, d) in enumerate(zip(entries, plans, data)):
        y0, y1 = (torch.empty(p.sizes.out_elems, dtype=torch.int64, device=dev) for _ in range(2))
        outs.append((y0, y1))
        if r == he.ROLE_WGRAD:
            batch.bind_wgrad(i, d["g0"], d["g1"], d["x0"], d["x1"], y0, y1)
        elif r == he.ROLE_FWD:
            batch.bind(i, d["W"], d["x1"], d["x0"], None, y0, y1)
        else:
            batch.bind(i, d["W"], d["g1"], d["g0"], None, y0, y1)
    ws = torch.empty((batch.workspace_bytes + 7) // 8, dtype=torch.int64, device=dev)
    batch.commit(sk, ws, 1000, 5000)
    s = torch.cuda.Stream(device=dev)
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        batch.forward(stream=s)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        batch.forward()
    graph.replay()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for r in range(reps):
        graph.replay()
    b.record(stream)
    b.synchronize()
    ms_b = a.elapsed_time(b) / reps
    out["batched_graph"] = {"ms_per_step": ms_b, "products_per_s": products / (ms_b * 1e-3),
                            "workspace_GB": round(batch.workspace_bytes / 1e9, 2)}
    out["status_ok"] = ctx.sync_status() == 0
    del graph, batch, ws
    torch.cuda.empty_cache()
    # autotuned: partitions per (shape, role) and the multiply-accumulate's columns
    t0 = time.perf_counter()
    e_layers, e_roles = [Ly for _, Ly in entries], [r for r, _ in entries]
    best = tuner.tune_batch(ctx, sk, e_layers, topk=3, reps=3, radices=(4,), columns=(2, 4, 8), stagings=(1,),
                            roles=e_roles)
    tune_s = time.perf_counter() - t0
    gb = tuner.GraphBatch(ctx, sk, e_layers, best["partitions"], roles=e_roles)
    ms_t = gb.time(reps)
    out["batched_graph_autotuned"] = {"ms_per_step": ms_t, "products_per_s": gb.products / (ms_t * 1e-3),
                                      "products_per_step": gb.products, "mac_columns": best["mac_columns"],
                                      "tuning_seconds": round(tune_s, 1)}
    out["status_ok"] = out["status_ok"] and ctx.sync_status() == 0
    del gb
    ctx.close()
    torch.cuda.empty_cache()
    return out


def training_step(he, device: int, reps: int = 3):
    """Secure fwd + bwd of the 3-layer CNN (conv3x3 3->16, ReLU, conv3x3 16->32,
    avgpool 2, FC 8192->10; batch 64, 32x32x3, N = 8192) through HeLinearFn."""
    import torch
    from paper_2403_11166_gb300 import autograd, inputs
    sess = autograd.HeSession(LOG_N, L, PRIME_BITS, T_BITS, seed=3, device=device)
    model = autograd.SecureCNN(sess, 64, inputs.cnn_params(3), 32, 32)
    g = inputs.rng(4)
    x = torch.as_tensor(np.floor(np.clip(g.standard_normal((64, 3, 32, 32)), -8, 8) * 4096) / 4096,
                        device=sess.device)
    labels = torch.as_tensor(g.integers(0, 10, 64), device=sess.device)

    def step():
        model.zero_grad(set_to_none=True)
        loss = torch.nn.functional.cross_entropy(model(x), labels) * 4096.0
        loss.backward()
    step()
    torch.cuda.synchronize()
    sess.bytes_do_to_mo = sess.bytes_mo_to_do = 0
    t = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        step()
        b.record()
        b.synchronize()
        t.append(a.elapsed_time(b))
    out = {"ms_per_step": statistics.median(t), "batch": 64,
           "ciphertext_MB_per_step": round((sess.bytes_do_to_mo + sess.bytes_mo_to_do) / reps / 1e6, 1)}
    # one more step with the library's per-kernel events (the HE and ring kernels; the rest is PyTorch)
    sess.ctx.profile(True)
    step()
    torch.cuda.synchronize()
    sess.ctx.profile(False)
    out["library_kernels"] = {name: {"launches": n, "ms": round(ms, 4)}
                              for name, (n, ms) in sess.ctx.profile_read().items() if n}
    return out


def large_conv(he, device: int, reps: int = 3):
    """conv3x3 128->128 on 16x16, batch 128: Alg. 1 forward + grad_X + Alg. 2 grad_W, N = 8192."""
    import torch
    from paper_2403_11166_gb300 import autograd, inputs
    sess = autograd.HeSession(LOG_N, L, PRIME_BITS, T_BITS, seed=5, device=device)
    Ly = he.Layer(he.CONV, 128, 128, 128, 16, 16, 3, 1)
    g = inputs.rng(6)
    dev = sess.device
    W = torch.as_tensor(inputs.gaussian_fixed(g, (128, 128, 3, 3)), device=dev) & sess.mask
    x0, x1 = (torch.as_tensor(a.view(np.int64), device=dev) for a in
              inputs.split_shares(g, inputs.gaussian_fixed(g, (128, 128, 16, 16))))
    g0, g1 = (torch.as_tensor(a.view(np.int64), device=dev) for a in
              inputs.split_shares(g, inputs.gaussian_fixed(g, (128, 128, 16, 16))))

    def fwd_bwd():
        sess.forward(Ly, W, None, x0, x1)
        return sess.backward(Ly, W, x0, x1, g0, g1, True)
    fwd_bwd()
    torch.cuda.synchronize()
    t = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fwd_bwd()
        b.record()
        b.synchronize()
        t.append(a.elapsed_time(b))
    prods = sum(sess.plan(Ly, r).sizes.products * (2 if r == he.ROLE_WGRAD else 1)
                for r in (he.ROLE_FWD, he.ROLE_DGRAD, he.ROLE_WGRAD))
    ms = statistics.median(t)
    return {"ms_fwd_bwd": ms, "products": prods, "products_per_s": prods / (ms * 1e-3),
            "partitions": {r: sess.plan(Ly, v).part for r, v in (("fwd", he.ROLE_FWD), ("dgrad", he.ROLE_DGRAD),
                                                                  ("wgrad", he.ROLE_WGRAD))}}


def pencil_plus(he, device: int, m: int = 8, reps: int = 3):
    """Preprocessing protocol (Alg. 3) for the forward product of the headline layer
    (conv3x3 16->16, 32x32, B = 64, N = 8192) with m masks per party: the one-time
    preprocessing (all m^2 products in one stacked Alg. 1 evaluation) and the
    HE-free online phase, next to the HE online forward it replaces."""
    import torch
    from paper_2403_11166_gb300 import inputs, prep
    ctx = he.Context(LOG_N, L, PRIME_BITS, T_BITS, device=device)
    sk = ctx.keygen(77)
    Ly = he.Layer(he.CONV, LAYER["batch"], LAYER["c_in"], LAYER["c_out"], LAYER["h"], LAYER["w"], LAYER["s"],
                  LAYER["pad"])
    g = inputs.rng(78)
    dev = f"cuda:{device}"
    W = torch.as_tensor(inputs.gaussian_fixed(g, (LAYER["c_out"], LAYER["c_in"], 3, 3)), device=dev)
    xs = (LAYER["batch"], LAYER["c_in"], LAYER["h"], LAYER["w"])
    x1 = torch.as_tensor(inputs.uniform_zt(g, xs).view(np.int64), device=dev)
    U = torch.as_tensor(inputs.uniform_zt(g, (m * LAYER["c_out"], LAYER["c_in"], 3, 3)).view(np.int64), device=dev)
    V = torch.as_tensor(inputs.uniform_zt(g, (m * LAYER["batch"],) + xs[1:]).view(np.int64), device=dev)
    pp = prep.PrepProduct(ctx, sk, Ly, he.ROLE_FWD, m)
    pp.preprocess(U, V, 89, 90)   # warm-up (module loading, first-touch of the workspaces); timed below
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    pp.preprocess(U, V, 91, 92)
    b.record()
    b.synchronize()
    prep_ms = a.elapsed_time(b)
    k = [int(v) for v in inputs.uniform_zt(g, (m,))]
    l = [int(v) for v in inputs.uniform_zt(g, (m,))]
    pp.online(W, x1, k, l)
    torch.cuda.synchronize()
    t = []
    for _ in range(reps):
        a.record()
        pp.online(W, x1, k, l)
        b.record()
        b.synchronize()
        t.append(a.elapsed_time(b))
    # one more online pass with the library's per-kernel events (serialised on the stream)
    ctx.profile(True)
    pp.online(W, x1, k, l)
    torch.cuda.synchronize()
    ctx.profile(False)
    kern = {name: {"launches": n, "ms": round(ms, 4)} for name, (n, ms) in ctx.profile_read().items() if n}
    assert ctx.sync_status() == 0
    out = {"m": m, "preprocessing_ms": prep_ms, "preprocessing_products": pp.products,
           "online_ms": statistics.median(t), "online_products_equivalent": pp.plan_one.sizes.products,
           "online_he_free": True, "online_kernels": kern}
    del pp
    ctx.close()
    torch.cuda.empty_cache()
    return out


# The paper's single-layer shapes (Table V: batch 64, online training of one
# linear layer; conv padding "same"), with its A6000 per-sample times as context.
TABLE5 = [("fc", 256, 100, 1, 1, 6.8), ("fc", 512, 10, 1, 1, 2.6), ("fc", 2048, 1001, 1, 1, 256.1),
          ("conv", 64, 64, 16, 5, 165.0), ("conv", 3, 64, 56, 3, 244.0), ("conv", 64, 3, 56, 3, 237.0)]


def _reconstruction_check(kind, Ly, W, x0, x1, g0, g1, Y, GX, GW) -> dict:
    """Every element of the reconstructed Y, grad_X and grad_W against float64
    PyTorch operators on the plaintext fixed-point values (exact: every partial
    sum is an integer below 2^53), compared mod t."""
    import torch
    import torch.nn.functional as F
    t_mask = (1 << T_BITS) - 1

    def centred(v):
        v = v & t_mask
        return torch.where(v >= (1 << (T_BITS - 1)), v - (1 << T_BITS), v).double()
    x, gy, w = centred(x0 + x1), centred(g0 + g1), centred(W)
    if kind == "fc":
        ry, rgx, rgw = x @ w.T, gy @ w, gy.T @ x
    else:
        ry = F.conv2d(x, w, padding=Ly.pad)
        rgx = torch.nn.grad.conv2d_input(x.shape, w, gy, padding=Ly.pad)
        rgw = torch.nn.grad.conv2d_weight(x, w.shape, gy, padding=Ly.pad)

    def same(got, ref):
        return bool(torch.equal(got.reshape(-1) & t_mask, ref.reshape(-1).round().to(torch.int64) & t_mask))
    return {"y": same(Y, ry), "grad_x": same(GX, rgx), "grad_w": same(GW, rgw)}


def table5_layers(he, device: int, reps: int = 2):
    """Forward + grad_X + grad_W of each layer through the HE path (Alg. 1, Alg. 2),
    N = 8192, batch 64: ms per layer step and per sample, ciphertext bytes per sample."""
    import torch
    from paper_2403_11166_gb300 import autograd, inputs
    out = []
    for kind, ci, co, hw, ks, paper_ms in TABLE5:
        sess = autograd.HeSession(LOG_N, L, PRIME_BITS, T_BITS, seed=11, device=device)
        B = 64
        if kind == "fc":
            Ly = he.Layer(he.FC, B, ci, co, 1, 1, 1, 0)
            xs, ys, ws = (B, ci), (B, co), (co, ci)
        else:
            Ly = he.Layer(he.CONV, B, ci, co, hw, hw, ks, ks // 2)
            xs, ys, ws = (B, ci, hw, hw), (B, co, hw, hw), (co, ci, ks, ks)
        g = inputs.rng(12)
        dev = sess.device
        W = torch.as_tensor(inputs.gaussian_fixed(g, ws), device=dev) & sess.mask
        x0, x1 = (torch.as_tensor(a.view(np.int64), device=dev) for a in
                  inputs.split_shares(g, inputs.gaussian_fixed(g, xs)))
        g0, g1 = (torch.as_tensor(a.view(np.int64), device=dev) for a in
                  inputs.split_shares(g, inputs.gaussian_fixed(g, ys)))

        def step():
            y = sess.forward(Ly, W, None, x0, x1)
            return y, sess.backward(Ly, W, x0, x1, g0, g1, True)
        (y0, y1), (gx0, gx1, gw, _) = step()
        torch.cuda.synchronize()
        checked = _reconstruction_check(kind, Ly, W, x0, x1, g0, g1, sess.reconstruct(y0, y1),
                                        sess.reconstruct(gx0, gx1), gw)
        sess.bytes_do_to_mo = sess.bytes_mo_to_do = 0
        t = []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            step()
            b.record()
            b.synchronize()
            t.append(a.elapsed_time(b))
        assert sess.ctx.sync_status() == 0
        ms = statistics.median(t)
        comm = (sess.bytes_do_to_mo + sess.bytes_mo_to_do) / reps
        out.append({"layer": f"{kind} {ci}->{co}" + (f" {hw}x{hw} k{ks}" if kind == "conv" else ""),
                    "reconstruction_ok": checked,
                    "ms_fwd_bwd": round(ms, 3), "ms_per_sample": round(ms / B, 4),
                    "ciphertext_MB_per_sample": round(comm / B / 1e6, 3),
                    "paper_a6000_ms_per_sample_context": paper_ms})
        del sess
        torch.cuda.empty_cache()
    return out


def pk_and_flooding(he, device: int, reps: int = 10, flood_bits: int = 62):
    """The headline layer (conv3x3 16->16, 32x32, B = 64, N = 8192): the DO's
    encryption of its input share with the secret key and with the public key,
    and the MO's Alg. 1 forward without and with noise flooding."""
    import torch
    from paper_2403_11166_gb300 import inputs
    ctx = he.Context(LOG_N, L, PRIME_BITS, T_BITS, device=device)
    sk = ctx.keygen(81)
    pk = ctx.pk_keygen(sk, 82)
    Ly = he.Layer(he.CONV, LAYER["batch"], LAYER["c_in"], LAYER["c_out"], LAYER["h"], LAYER["w"], LAYER["s"],
                  LAYER["pad"])
    plan = he.Plan(ctx, Ly, he.ROLE_FWD, None)
    S = plan.sizes
    dev = f"cuda:{device}"
    g = inputs.rng(83)
    W = torch.as_tensor(inputs.gaussian_fixed(g, (LAYER["c_out"], LAYER["c_in"], 3, 3)).view(np.int64), device=dev)
    x0, x1 = (torch.as_tensor(a.view(np.int64), device=dev) for a in inputs.split_shares(
        g, inputs.gaussian_fixed(g, (LAYER["batch"], LAYER["c_in"], LAYER["h"], LAYER["w"]))))
    ws = plan.new_ws(max(S.ws_encrypt, S.ws_encrypt_pk, S.ws_forward))
    pt, ct_in, ct_out = plan.new_pt(S.pt), plan.new_ct(S.ct_in), plan.new_ct(S.ct_out)
    y0 = torch.empty(S.out_elems, dtype=torch.int64, device=dev)
    he.encode_weights(ctx, plan, he.OPERAND_KERNEL, W, pt)

    def timed(fn):
        fn(0)
        torch.cuda.synchronize()
        t = []
        for r in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            fn(r + 1)
            b.record()
            b.synchronize()
            t.append(a.elapsed_time(b))
        return statistics.median(t)
    ms_sk = timed(lambda r: he.encrypt_share(ctx, sk, plan, he.OPERAND_INPUT, x1, 100 + r, ct_in, ws))
    ms_pk = timed(lambda r: he.encrypt_share_pk(ctx, pk, plan, he.OPERAND_INPUT, x1, 100 + r, ct_in, ws))
    fwd = lambda r: he.he_linear_forward(ctx, plan, ct_in, pt, x0, None, 200 + r, ct_out, y0, ws)
    ms_fwd = timed(fwd)
    ctx.flooding(flood_bits)
    ms_fwd_flood = timed(fwd)
    ctx.flooding(0)
    ok = ctx.sync_status() == 0
    return {"ct_in": S.ct_in, "encrypt_sk_ms": ms_sk, "encrypt_pk_ms": ms_pk,
            "encrypt_sk_ct_per_s": S.ct_in / (ms_sk * 1e-3), "encrypt_pk_ct_per_s": S.ct_in / (ms_pk * 1e-3),
            "forward_ms": ms_fwd, "forward_flooded_ms": ms_fwd_flood, "flood_bits": flood_bits, "status_ok": ok}


def compact_send(he, device: int, reps: int = 10):
    """Returned ciphertexts with the coefficients that carry no output dropped
    (compact_returned on the MO, decrypt_compact_to_share on the DO), forward
    product of the headline conv layer and of the paper's fc 2048->1001 (batch
    64), N = 8192: bytes returned per evaluation and the two calls' time beside
    the whole-ciphertext decryption."""
    import torch
    from paper_2403_11166_gb300 import inputs
    ctx = he.Context(LOG_N, L, PRIME_BITS, T_BITS, device=device)
    sk = ctx.keygen(91)
    dev = f"cuda:{device}"
    layers = {"conv3x3 16->16 32x32 b64": (he.Layer(he.CONV, 64, 16, 16, 32, 32, 3, 1), (16, 16, 3, 3),
                                           (64, 16, 32, 32)),
              "fc 2048->1001 b64": (he.Layer(he.FC, 64, 2048, 1001, 1, 1, 1, 0), (1001, 2048), (64, 2048))}
    out = {}
    for name, (Ly, wshape, xshape) in layers.items():
        plan = he.Plan(ctx, Ly, he.ROLE_FWD, None)
        S = plan.sizes
        g = inputs.rng(92)
        W = torch.as_tensor(inputs.gaussian_fixed(g, wshape).view(np.int64), device=dev)
        x0, x1 = (torch.as_tensor(a.view(np.int64), device=dev) for a in
                  inputs.split_shares(g, inputs.gaussian_fixed(g, xshape)))
        ws = plan.new_ws(max(S.ws_encrypt, S.ws_forward, S.ws_decrypt))
        pt, ct_in, ct_out = plan.new_pt(S.pt), plan.new_ct(S.ct_in), plan.new_ct(S.ct_out)
        y0, y1, y1c = (torch.empty(S.out_elems, dtype=torch.int64, device=dev) for _ in range(3))
        c0c = torch.empty((L, S.out_elems), dtype=torch.int64, device=dev)
        he.encode_weights(ctx, plan, he.OPERAND_KERNEL, W, pt)
        he.encrypt_share(ctx, sk, plan, he.OPERAND_INPUT, x1, 93, ct_in, ws)
        he.he_linear_forward(ctx, plan, ct_in, pt, x0, None, 94, ct_out, y0, ws)

        def timed(fn):
            fn()
            torch.cuda.synchronize()
            t = []
            for _ in range(reps):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record()
                fn()
                b.record()
                b.synchronize()
                t.append(a.elapsed_time(b))
            return statistics.median(t)
        ms_dec = timed(lambda: he.decrypt_to_share(ctx, sk, plan, ct_out, y1, True, ws))
        ms_cmp = timed(lambda: he.compact_returned(ctx, plan, ct_out, c0c))
        ms_decc = timed(lambda: he.decrypt_compact_to_share(ctx, sk, plan, ct_out, c0c, y1c, True, ws))
        torch.cuda.synchronize()
        full = 8 * 2 * L * (1 << LOG_N) * S.ct_out
        compact = 8 * (L * (1 << LOG_N) * S.ct_out + L * S.out_elems)
        out[name] = {"ct_out": S.ct_out, "out_elems": S.out_elems, "returned_MB": round(full / 1e6, 2),
                     "returned_compact_MB": round(compact / 1e6, 2), "ratio": round(compact / full, 3),
                     "decrypt_ms": ms_dec, "compact_ms": ms_cmp, "decrypt_compact_ms": ms_decc,
                     "same_share": bool(torch.equal(y1, y1c)), "status_ok": ctx.sync_status() == 0}
    return out


def _layer_fwd_bwd(he, device: int, cfg, Ly, xs, ys, ws, reps: int, seed: int):
    """Alg. 1 forward + input gradient + Alg. 2 weight gradient of one layer through
    the HE session (the calls HeLinearFn makes), median ms over `reps` steps."""
    import torch
    from paper_2403_11166_gb300 import autograd, inputs
    sess = autograd.HeSession(*cfg, T_BITS, seed=seed, device=device)
    g = inputs.rng(seed + 1)
    dev = sess.device
    W = torch.as_tensor(inputs.gaussian_fixed(g, ws), device=dev) & sess.mask
    x0, x1 = (torch.as_tensor(a.view(np.int64), device=dev) for a in inputs.split_shares(g, inputs.gaussian_fixed(g, xs)))
    g0, g1 = (torch.as_tensor(a.view(np.int64), device=dev) for a in inputs.split_shares(g, inputs.gaussian_fixed(g, ys)))

    def fwd_bwd():
        sess.forward(Ly, W, None, x0, x1)
        return sess.backward(Ly, W, x0, x1, g0, g1, True)
    fwd_bwd()
    torch.cuda.synchronize()
    t = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fwd_bwd()
        b.record()
        b.synchronize()
        t.append(a.elapsed_time(b))
    ok = sess.ctx.sync_status() == 0
    prods = {r: sess.plan(Ly, v).sizes.products * (2 if v == he.ROLE_WGRAD else 1)
             for r, v in (("fwd", he.ROLE_FWD), ("dgrad", he.ROLE_DGRAD), ("wgrad", he.ROLE_WGRAD))}
    ms = statistics.median(t)
    out = {"ms_fwd_bwd": round(ms, 4), "products": sum(prods.values()), "products_by_role": prods,
           "products_per_s": sum(prods.values()) / (ms * 1e-3), "status_ok": ok,
           "partitions": {r: sess.plan(Ly, v).part for r, v in (("fwd", he.ROLE_FWD), ("dgrad", he.ROLE_DGRAD),
                                                                ("wgrad", he.ROLE_WGRAD))}}
    del sess
    torch.cuda.empty_cache()
    return out


def headline_fwd_bwd(he, device: int, reps: int = 10):
    """The headline layer (conv3x3 16->16, 32x32, B = 64, N = 8192): forward +
    input gradient + weight gradient, the metric's "fwd+bwd ms"."""
    Ly = he.Layer(he.CONV, LAYER["batch"], LAYER["c_in"], LAYER["c_out"], LAYER["h"], LAYER["w"], LAYER["s"],
                  LAYER["pad"])
    B, ci, co, h, w = LAYER["batch"], LAYER["c_in"], LAYER["c_out"], LAYER["h"], LAYER["w"]
    return _layer_fwd_bwd(he, device, (LOG_N, L, PRIME_BITS), Ly, (B, ci, h, w), (B, co, h, w), (co, ci, 3, 3),
                          reps, 21)


def fc784_n4096(he, device: int, reps: int = 20):
    """FC 784 -> 100, batch 32, N = 4096, two 54-bit primes (the small workload):
    the forward step of the headline's form (encode, MO preparation, encryption,
    multiply-accumulate, decryption; products/s) and forward + backward ms."""
    import torch
    from paper_2403_11166_gb300 import inputs
    ctx = he.Context(12, 2, 54, T_BITS, device=device)
    sk = ctx.keygen(31)
    Ly = he.Layer(he.FC, 32, 784, 100)
    plan = he.Plan(ctx, Ly, he.ROLE_FWD, None)
    S = plan.sizes
    g = inputs.rng(32)
    dev = f"cuda:{device}"
    W = torch.as_tensor(inputs.gaussian_fixed(g, (100, 784)), device=dev)
    x0, x1 = (torch.as_tensor(a.view(np.int64), device=dev) for a in
              inputs.split_shares(g, inputs.gaussian_fixed(g, (32, 784))))
    pt, ct_in, ct_out = plan.new_pt(S.pt), plan.new_ct(S.ct_in), plan.new_ct(S.ct_out)
    ws = plan.new_ws(max(S.ws_encrypt, S.ws_forward, S.ws_decrypt))
    y0 = torch.empty(S.out_elems, dtype=torch.int64, device=dev)
    y1 = torch.empty_like(y0)

    def step(i):
        he.encode_weights(ctx, plan, he.OPERAND_KERNEL, W, pt)
        he.encrypt_share(ctx, sk, plan, he.OPERAND_INPUT, x1, 100 + i, ct_in, ws)
        he.he_linear_forward(ctx, plan, ct_in, pt, x0, None, 200 + i, ct_out, y0, ws)
        he.decrypt_to_share(ctx, sk, plan, ct_out, y1, False, ws)
    for i in range(3):
        step(i)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for i in range(reps):
        step(10 + i)
    b.record()
    b.synchronize()
    ms = a.elapsed_time(b) / reps
    def centred(v):
        v = v & ((1 << T_BITS) - 1)
        return torch.where(v >= (1 << (T_BITS - 1)), v - (1 << T_BITS), v).double()
    # self-check: the reconstruction is the plaintext product (exact in float64)
    ok = bool(torch.equal(centred(y0 + y1).view(32, 100), centred(x0 + x1) @ W.double().T))
    out = {"forward": {"ms_per_step": round(ms, 4), "products_per_step": S.products,
                       "products_per_s": S.products / (ms * 1e-3), "partition": plan.part,
                       "ct_in": S.ct_in, "pt": S.pt, "ct_out": S.ct_out, "reconstruction_ok": ok,
                       "status_ok": ctx.sync_status() == 0}}
    del ctx
    torch.cuda.empty_cache()
    out["fwd_bwd"] = _layer_fwd_bwd(he, device, (12, 2, 54), Ly, (32, 784), (32, 100), (100, 784), reps, 33)
    return out


EXTRAS = {"headline_fwd_bwd": headline_fwd_bwd, "fc784_b32_n4096": fc784_n4096,
          "batched_uneven": batched_uneven, "batched_fwd_bwd": batched_fwd_bwd, "training_step_cnn": training_step,
          "large_conv_128_fwd_bwd": large_conv, "pencil_plus_fwd_m8": pencil_plus,
          "paper_table5_layers_b64": table5_layers, "public_key_and_flooding": pk_and_flooding,
          "compact_send_form": compact_send}


def extras(he, device: int, names=None):
    return {k: fn(he, device) for k, fn in EXTRAS.items() if not names or k in names}


# ---------------------------------------------------------------- oracle timing (host cores)
def oracle_sample(seed: int = 0, part_tuple=(1, 2, 3, 32, 32, 3, 3), min_seconds: float = 0.0):
    """Times the oracle on one instance of every stage of the workload (repeated
    until `min_seconds` have passed, median per stage) and scales by the stage
    counts of the partition.  Returns (products/s, seconds of the full workload
    step, description, seconds spent)."""
    from oracle import bfv, protocol
    from oracle.packing import Partition, counts
    from oracle.params import BfvParams
    from paper_2403_11166_gb300 import inputs

    t_all = time.perf_counter()
    p = BfvParams(log_n=LOG_N, num_primes=L, prime_bits=PRIME_BITS, t_bits=T_BITS)
    layer = protocol.Layer("conv", B=LAYER["batch"], Ci=LAYER["c_in"], Co=LAYER["c_out"], h=LAYER["h"],
                           w=LAYER["w"], s=LAYER["s"], pad=LAYER["pad"])
    part = Partition(*part_tuple)
    c = counts(protocol.geometry(layer, protocol.FWD), part)
    g = inputs.rng(seed)
    W = inputs.gaussian_fixed(g, layer.w_shape())
    x = inputs.gaussian_fixed(g, layer.x_shape())
    x0, x1 = inputs.split_shares(g, x)
    sk = bfv.keygen(p, 5)
    from oracle.packing import pack_input
    V0 = protocol.role_input(layer, protocol.FWD, x0)
    times = {k: [] for k in ("enc", "encode", "add", "mul", "mask", "dec")}
    while True:
        t0 = time.perf_counter()
        cts = protocol.encrypt_inputs(p, sk, layer, protocol.FWD, part, x1, 9, indices=[0])
        t1 = time.perf_counter()
        pts = protocol.encode_kernel(p, layer, protocol.FWD, part, W, indices=[0])
        t2 = time.perf_counter()
        ct = bfv.add_plain(p, cts[0], pack_input(V0, protocol.geometry(layer, protocol.FWD), part, p.n, 0, 0))
        t3 = time.perf_counter()
        prod = bfv.mul_plain(p, ct, pts[0])
        acc = bfv.add_ct(p, prod, prod)
        t4 = time.perf_counter()
        out = bfv.sub_plain(p, acc, protocol.mask_polynomial(p, layer, protocol.FWD, part, 3, 0))
        t5 = time.perf_counter()
        bfv.decrypt(p, sk, out)
        t6 = time.perf_counter()
        for k, v in zip(times, (t1 - t0, t2 - t1, t3 - t2, t4 - t3, t5 - t4, t6 - t5)):
            times[k].append(v)
        if time.perf_counter() - t_all >= min_seconds:
            break
    med = {k: statistics.median(v) for k, v in times.items()}
    t_enc, t_encode, t_add, t_mul, t_mask, t_dec = (med[k] for k in times)
    step = (c.ct_in * (t_enc + t_add) + c.pt * t_encode + c.products * t_mul + c.ct_out * (t_mask + t_dec))
    desc = (f"oracle (Python, exact big integers) timed on {len(times['enc'])} rounds of: one ct_in encryption "
            f"({t_enc:.2f}s), one add_plain, one pt encoding, one ct x pt product + accumulate, one re-mask and "
            f"one decryption ({t_dec:.2f}s) at N=8192, L=3; median per stage "
            f"scaled by the partition's counts ({c.ct_in} ct_in, {c.pt} pt, {c.products} products, "
            f"{c.ct_out} ct_out)")
    return c.products / step, step, desc, time.perf_counter() - t_all


def cpu_ntt_baseline(seconds: float = 6.0):
    """The plain CPU NTT build (C, OpenMP) on this host: limb-NTTs/s at 1 thread and
    at all threads, forward, 60-bit primes, N in {4096, 8192, 16384}."""
    from oracle import cpu_ntt
    from oracle.params import min_primitive_root_2n, ntt_primes
    cores = cpu_ntt.max_threads()
    out = {"cores": cores}
    budget = seconds / 6
    for log_n in (12, 13, 14):
        n = 1 << log_n
        q = ntt_primes(60, 1, 2 * n)[0]
        eng = cpu_ntt.CpuNtt(q, min_primitive_root_2n(q, 2 * n), log_n)
        res = {}
        for label, threads in (("threads_1", 1), ("threads_all", cores)):
            count = 8 * threads
            a = np.random.default_rng(log_n).integers(0, q, size=(count, n), dtype=np.uint64)
            eng.run(a, threads=threads)
            done, t0 = 0, time.perf_counter()
            while time.perf_counter() - t0 < budget:
                eng.run(a, threads=threads)
                done += count
            res[label] = done / (time.perf_counter() - t0)
        out[f"N{n}"] = res
    return out


def cpu_pipeline(he, device: int):
    """The plain C/OpenMP build of the HE pipeline (oracle/cpu_he.c: encode,
    encrypt, Alg. 1 / Alg. 2 evaluation, decrypt; bit-exact with the oracle) on
    the host cores, on the partitions the GPU planner picks for each (layer, role).
    ms per step at one thread (the small workloads) and at every thread.  The
    96-layer batch is timed on one layer of each shape and role (the other 31
    copies are identical: x 32) and the conv 128->128 layer at batch 16 with the
    batch-128 partitions (scaled by the product count); both are marked."""
    from oracle.cpu_he import CpuHe, max_threads
    from oracle.packing import Partition, counts
    from oracle.params import BfvParams
    from oracle.protocol import DGRAD, FWD, WGRAD
    from oracle.protocol import Layer as OL
    from oracle.protocol import geometry
    from paper_2403_11166_gb300 import inputs
    cores = max_threads()
    roles = {he.ROLE_FWD: FWD, he.ROLE_DGRAD: DGRAD, he.ROLE_WGRAD: WGRAD}
    engines, gctx = {}, {}

    def engine(cfg):
        if cfg not in engines:
            engines[cfg] = CpuHe(BfvParams(log_n=cfg[0], num_primes=cfg[1], prime_bits=cfg[2]), 5)
            gctx[cfg] = he.Context(*cfg, T_BITS, device=device)
        return engines[cfg], gctx[cfg]

    def olayer(Ly):
        if Ly.kind == he.FC:
            return OL("fc", B=Ly.batch, Ci=Ly.c_in, Co=Ly.c_out)
        return OL("conv", B=Ly.batch, Ci=Ly.c_in, Co=Ly.c_out, h=Ly.height, w=Ly.width, s=Ly.kernel, pad=Ly.pad)

    def run(cfg, entries, threads, part_from=None):
        """entries: (he.Layer, he role); returns (seconds, products)."""
        che, ctx = engine(cfg)
        g = inputs.rng(3)
        total, prods = 0.0, 0
        for Ly, r in entries:
            L_ = olayer(Ly)
            src = part_from(Ly, r) if part_from else Ly
            part = Partition(*he.Plan(ctx, src, r, None).part)
            c = counts(geometry(L_, roles[r]), part)
            if r == he.ROLE_WGRAD:
                x0, x1 = inputs.split_shares(g, inputs.gaussian_fixed(g, L_.x_shape()))
                g0, g1 = inputs.split_shares(g, inputs.gaussian_fixed(g, L_.y_shape()))
                t0 = time.perf_counter()
                che.layer_alg2(L_, part, g0, g1, x0, x1, 1, 2, 3, threads=threads)
                total += time.perf_counter() - t0
                prods += 2 * c.products
            else:
                W = inputs.gaussian_fixed(g, L_.w_shape())
                v0, v1 = inputs.split_shares(g, inputs.gaussian_fixed(g, L_.x_shape() if r == he.ROLE_FWD
                                                                      else L_.y_shape()))
                t0 = time.perf_counter()
                che.layer_alg1(L_, roles[r], part, W, v1, v0, 1, 2, threads=threads)
                total += time.perf_counter() - t0
                prods += c.products
        return total, prods

    def line(sec, prods, threads, note=None):
        d = {"ms": round(sec * 1e3, 2), "products": prods, "products_per_s": prods / sec, "threads": threads}
        if note:
            d["note"] = note
        return d
    cfg60, cfg54 = (LOG_N, L, PRIME_BITS), (12, 2, 54)
    fb = (he.ROLE_FWD, he.ROLE_DGRAD, he.ROLE_WGRAD)
    head = he.Layer(he.CONV, LAYER["batch"], LAYER["c_in"], LAYER["c_out"], LAYER["h"], LAYER["w"], LAYER["s"],
                    LAYER["pad"])
    fc1 = he.Layer(he.FC, 32, 784, 100)
    out = {"cores": cores, "kind": "plain C + OpenMP build of the pipeline (oracle/cpu_he.c, oracle/cpu_ntt.c)"}
    t0 = time.perf_counter()
    out["conv16_b64_fwd"] = {"threads_1": line(*run(cfg60, [(head, he.ROLE_FWD)], 1), 1),
                             "threads_all": line(*run(cfg60, [(head, he.ROLE_FWD)], cores), cores)}
    out["conv16_b64_fwd_bwd"] = {"threads_all": line(*run(cfg60, [(head, r) for r in fb], cores), cores)}
    out["fc784_b32_n4096_fwd"] = {"threads_1": line(*run(cfg54, [(fc1, he.ROLE_FWD)], 1), 1),
                                  "threads_all": line(*run(cfg54, [(fc1, he.ROLE_FWD)], cores), cores)}
    out["fc784_b32_n4096_fwd_bwd"] = {"threads_all": line(*run(cfg54, [(fc1, r) for r in fb], cores), cores)}
    cnn = [(he.Layer(he.CONV, 64, 3, 16, 32, 32, 3, 1), he.ROLE_FWD), (he.Layer(he.CONV, 64, 3, 16, 32, 32, 3, 1),
                                                                      he.ROLE_WGRAD)]
    cnn += [(he.Layer(he.CONV, 64, 16, 32, 32, 32, 3, 1), r) for r in fb]
    cnn += [(he.Layer(he.FC, 64, 8192, 10), r) for r in fb]
    out["cnn3_b64_fwd_bwd"] = {"threads_all": line(*run(cfg60, cnn, cores), cores)}
    shapes = [he.Layer(he.FC, 16, 512, 10), he.Layer(he.CONV, 32, 64, 64, 8, 8, 3, 1),
              he.Layer(he.CONV, 8, 128, 256, 4, 4, 1, 0)]
    sec, prods = run(cfg60, [(Ly, r) for Ly in shapes for r in fb], cores)
    out["batched_96_layers_fwd_bwd"] = {"threads_all": line(sec * 32, prods * 32, cores,
                                                            "one layer of each shape and role timed, x 32")}
    big = he.Layer(he.CONV, 128, 128, 128, 16, 16, 3, 1)
    small = he.Layer(he.CONV, 16, 128, 128, 16, 16, 3, 1)
    sec, prods = run(cfg60, [(small, r) for r in fb], cores, part_from=lambda Ly, r: big)
    full = 0
    for r in fb:
        part = Partition(*he.Plan(gctx[cfg60], big, r, None).part)
        full += counts(geometry(olayer(big), roles[r]), part).products * (2 if r == he.ROLE_WGRAD else 1)
    out["conv128_b128_fwd_bwd"] = {"threads_all": line(sec * full / prods, full, cores,
                                                       f"timed at batch 16 with the batch-128 partitions "
                                                       f"({prods} products), scaled to {full}")}
    out["seconds"] = round(time.perf_counter() - t0, 1)
    for c in gctx.values():
        c.close()
    return out


def run_reference(args):
    """The oracle (the only reference implementation of the paper there is) on the
    host cores, on the partition the GPU arm times: every step times one round of
    each stage (one encryption, add_plain, encoding, product, re-mask and
    decryption) and scales the stage times by the partition's counts."""
    world, rank, _ = dist_env()
    if rank != 0:
        return
    vals, steps_s = [], []
    desc, spent = "", 0.0
    for i in range(args.warmup + args.steps):
        v, st, desc, sp = oracle_sample(seed=i, part_tuple=HEADLINE_PARTITION)
        if i >= args.warmup:
            vals.append(v)
            steps_s.append(st)
            spent += sp
    value = statistics.median(vals)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": statistics.median(steps_s) * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64 (RNS mod q_i), u64 mod 2^41",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "partition": dict(zip(("bb", "cib", "cob", "th", "tw", "kth", "ktw"),
                                                                HEADLINE_PARTITION)),
                       "inputs": "larger than L2 (ct_in 63 MB per step)"},
            "extrapolated_from_stage_medians": True,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": desc,
                             "seconds": round(spent, 1)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- our arm
def run_ours(args):
    import torch
    import torch.nn.functional as F

    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))
    torch.cuda.set_device(local)
    if rank == 0:
        from paper_2403_11166_gb300 import build
        build.build()
    if world > 1:
        torch.distributed.barrier()
    from paper_2403_11166_gb300 import he, inputs

    dev = f"cuda:{local}"
    stream = torch.cuda.current_stream()
    if args.sweep_only:
        sw = ntt_sweep(he, local, args.sweep_polys, args.sweep_points, args.sweep_reps, args.ntt_log_radix)
        if rank == 0:
            print(json.dumps({"ntt_sweep": sw}), flush=True)
        return
    if args.extras_only:
        ex = extras(he, local, args.extra)
        if rank == 0:
            print(json.dumps(ex), flush=True)
        return
    ctx = he.Context(LOG_N, L, PRIME_BITS, T_BITS, device=local)
    if args.ntt_log_radix:
        ctx.tune(he.TUNE_NTT_LOG_RADIX, args.ntt_log_radix)
    if args.mac_columns >= 0:
        ctx.tune(he.TUNE_MAC_COLUMNS, args.mac_columns)
    if args.mac_staging >= 0:
        ctx.tune(he.TUNE_MAC_STAGING, args.mac_staging)
    sk = ctx.keygen(1234 + rank)
    layer = he.Layer(he.CONV, LAYER["batch"], LAYER["c_in"], LAYER["c_out"], LAYER["h"], LAYER["w"], LAYER["s"],
                     LAYER["pad"])
    plan = he.Plan(ctx, layer, he.ROLE_FWD, None)
    if plan.part != HEADLINE_PARTITION and args.mac_columns < 0 and args.mac_staging < 0:
        print(f"note: the planner chose {plan.part}, not {HEADLINE_PARTITION} (the reference arm's)", file=sys.stderr)
    S = plan.sizes
    g = inputs.rng(100 + rank)
    W = inputs.gaussian_fixed(g, (LAYER["c_out"], LAYER["c_in"], 3, 3))
    x = inputs.gaussian_fixed(g, (LAYER["batch"], LAYER["c_in"], LAYER["h"], LAYER["w"]))
    bias = inputs.gaussian_fixed(g, (LAYER["c_out"],), frac_bits=24)
    x0, x1 = inputs.split_shares(g, x)

    def to_i64(a):
        a = np.ascontiguousarray(a)
        return torch.from_numpy((a if a.dtype == np.int64 else a.view(np.int64)).copy())

    host = {"W": to_i64(W).pin_memory(), "x0": to_i64(x0).pin_memory(), "x1": to_i64(x1).pin_memory(),
            "bias": to_i64(bias.astype(np.uint64) & np.uint64((1 << T_BITS) - 1)).pin_memory()}
    # one set of per-step inputs and outputs per step in flight: the end-to-end loop
    # copies the next step's inputs in and earlier steps' shares out while a step computes
    D = args.in_flight
    sets = []
    for _ in range(D):
        b = {k: v.to(dev) for k, v in host.items()}
        b["y0"] = torch.empty(S.out_elems, dtype=torch.int64, device=dev)
        b["y1"] = torch.empty_like(b["y0"])
        sets.append(b)
    d = sets[0]
    y0, y1 = d["y0"], d["y1"]
    pt = plan.new_pt(S.pt)
    ct_in = plan.new_ct(S.ct_in)
    ct_out = plan.new_ct(S.ct_out)
    ws = plan.new_ws(S.ws_encrypt)
    ws_dec = plan.new_ws(S.ws_decrypt)
    hy0 = torch.empty(S.out_elems, dtype=torch.int64).pin_memory()
    hy1 = torch.empty_like(hy0).pin_memory()

    ws_mo = plan.new_ws(S.ws_forward)

    # The MO encodes its weights and, independently, prepares its
    # ciphertext-independent terms (the mask s, NTT(Delta <X>_0), NTT(Delta s))
    # while the DO encrypts its share.  The layer then streams through the rest
    # of the protocol in `chunks` slices of its output rows (batch blocks): the
    # MO's multiply-accumulate of slice c overlaps the DO's encryption of slice
    # c + 1 and the DO's decryption of slice c - 1.  A timed run of steps forks
    # the step streams from the launch stream once and joins them at its end.
    M_rows = plan.rows
    nch = max(1, min(args.chunks, M_rows))
    bounds = [M_rows * c // nch for c in range(nch + 1)]
    slices = [plan.slice(bounds[c], bounds[c + 1] - bounds[c]) for c in range(nch)] if nch > 1 else [plan]
    mo_enc, mo_prep, mo_app = (torch.cuda.Stream(device=dev) for _ in range(3))
    do_dec = torch.cuda.Stream(device=dev)
    streams = (mo_enc, mo_prep, stream, mo_app, do_dec)
    fork = torch.cuda.Event()
    # D steps in flight: step i works in device buffer set i % D (plaintexts,
    # input and output ciphertexts, the MO's prepared terms) and writes the shares
    # of input set i % D, so step i + 1's encoding, preparation and encryption run
    # while step i multiplies and decrypts.  Step i + D reuses set i % D only after
    # step i's multiply-accumulate (for pt, ct_in, the prepared terms) and
    # decryption (for ct_out) are done with it.
    work = [{"pt": pt, "ct_in": ct_in, "ct_out": ct_out, "ws_mo": ws_mo}] + [
        {"pt": plan.new_pt(S.pt), "ct_in": plan.new_ct(S.ct_in), "ct_out": plan.new_ct(S.ct_out),
         "ws_mo": plan.new_ws(S.ws_forward)} for _ in range(D - 1)]
    evs = [{"enc": torch.cuda.Event(), "prep": torch.cuda.Event(), "ct": [torch.cuda.Event() for _ in slices],
            "out": [torch.cuda.Event() for _ in slices], "app": torch.cuda.Event(), "dec": torch.cuda.Event()}
           for _ in range(D)]
    used = [False] * D

    def begin():
        """Every step stream starts after the work already on the launch stream."""
        fork.record(stream)
        for st in streams:
            st.wait_event(fork)

    def end(i):
        """The launch stream waits for step i (and so for every earlier step)."""
        stream.wait_event(evs[i % D]["dec"])

    def step(i, b=None, serial=False, wait_in=None):
        p = i % D
        b = sets[p] if b is None else b
        w, e = work[p], evs[p]
        if serial:
            begin()
        if used[p]:   # step i - D is done with this buffer set
            for st in (mo_enc, mo_prep, stream):
                st.wait_event(e["app"])
            mo_app.wait_event(e["dec"])
        if wait_in is not None:   # this step's inputs have been copied in
            for st in (mo_enc, mo_prep, stream):
                st.wait_event(wait_in)
        he.encode_weights(ctx, plan, he.OPERAND_KERNEL, b["W"], w["pt"], stream=mo_enc)
        e["enc"].record(mo_enc)
        he.he_linear_forward_prepare(ctx, plan, b["x0"], b["bias"], 5000 + i, b["y0"], w["ws_mo"], stream=mo_prep)
        e["prep"].record(mo_prep)
        for c, sl in enumerate(slices):            # DO: encrypt slice by slice
            he.encrypt_share(ctx, sk, sl, he.OPERAND_INPUT, b["x1"], 1000 + i, w["ct_in"], ws, stream=stream)
            e["ct"][c].record(stream)
        mo_app.wait_event(e["enc"])
        mo_app.wait_event(e["prep"])
        for c, sl in enumerate(slices):            # MO: multiply-accumulate each slice as it arrives
            mo_app.wait_event(e["ct"][c])
            he.he_linear_forward_apply(ctx, sl, w["ct_in"], w["pt"], w["ct_out"], w["ws_mo"], stream=mo_app)
            e["out"][c].record(mo_app)
        e["app"].record(mo_app)
        for c, sl in enumerate(slices):            # DO: decrypt each slice as it comes back
            do_dec.wait_event(e["out"][c])
            he.decrypt_to_share(ctx, sk, sl, w["ct_out"], b["y1"], False, ws_dec, stream=do_dec)
        e["dec"].record(do_dec)
        used[p] = True
        if serial:
            end(i)

    begin()
    for i in range(args.warmup):
        step(i)
    end(args.warmup - 1)
    torch.cuda.synchronize()
    # self-check: reconstruction equals the plaintext convolution (exact in float64)
    y0, y1 = sets[(args.warmup - 1) % D]["y0"], sets[(args.warmup - 1) % D]["y1"]
    rec = ((y0 + y1) & ((1 << T_BITS) - 1)).view(LAYER["batch"], LAYER["c_out"], LAYER["h"], LAYER["w"])
    rec = torch.where(rec >= (1 << (T_BITS - 1)), rec - (1 << T_BITS), rec).double()
    ref = F.conv2d(torch.from_numpy(x).double().to(dev), torch.from_numpy(W).double().to(dev),
                   torch.from_numpy(bias).double().to(dev), padding=1)
    parity_ok = bool(torch.equal(rec, ref))

    # multiply-pipe probe: measured 32-bit IMAD and 64-bit Shoup rates (register-only)
    sms = sm_count(local)
    probe = {}
    for which, key in ((0, "imad32"), (1, "shoup64"), (2, "madwide32"), (3, "mac128")):
        ms_p, steps_p = ctx.mul_probe(which, 1 << 14, sms * 8, 256)
        ms_p, steps_p = ctx.mul_probe(which, 1 << 14, sms * 8, 256)
        probe[key] = steps_p / (ms_p * 1e-3) / 1e12
    uuid = None
    try:
        uuid = str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        pass
    clocks = ClockSampler(uuid)
    # ---- timed region (inputs resident in HBM)
    ctx.profile(True)
    clocks.start()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    t_issue = time.perf_counter()
    begin()
    for i in range(args.steps):
        step(args.warmup + i)
    end(args.warmup + args.steps - 1)
    t_issue = time.perf_counter() - t_issue   # host time to issue the steps (the GPU runs behind it)
    e1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    ms = e0.elapsed_time(e1)
    ck = clocks.stop()
    ctx.profile(False)
    prof = ctx.profile_read()
    # the same steps with no overlap between consecutive steps (each step's streams
    # fork from and join back into the launch stream): the latency of one step
    torch.cuda.synchronize()
    u0, u1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ctx.profile(True)
    u0.record(stream)
    for i in range(args.steps):
        step(args.warmup + i, serial=True)
    u1.record(stream)
    torch.cuda.synchronize()
    ms_serial = u0.elapsed_time(u1)
    ctx.profile(False)
    unpiped = ctx.profile_read()
    # serial profiling pass (not timed): the same steps with every kernel on the launch stream
    ctx.profile(True)
    for i in range(3):
        he.encode_weights(ctx, plan, he.OPERAND_KERNEL, d["W"], pt, stream=stream)
        he.he_linear_forward_prepare(ctx, plan, d["x0"], d["bias"], 7000 + i, y0, ws_mo, stream=stream)
        he.encrypt_share(ctx, sk, plan, he.OPERAND_INPUT, d["x1"], 3000 + i, ct_in, ws, stream=stream)
        he.he_linear_forward_apply(ctx, plan, ct_in, pt, ct_out, ws_mo, stream=stream)
        he.decrypt_to_share(ctx, sk, plan, ct_out, y1, False, ws_dec, stream=stream)
    torch.cuda.synchronize()
    ctx.profile(False)
    serial = ctx.profile_read()
    # ---- end to end: host buffers; every step's inputs are copied in from pinned
    # host memory and both shares copied back inside the region, inputs on one
    # copy stream and shares on another (the two directions of the host link run
    # at once); double-buffered: step i + 1's inputs go in and step i - 1's shares
    # come out while step i computes
    h2d = sum(v.numel() * 8 for v in host.values())
    d2h = 2 * S.out_elems * 8
    copy_in, copy_out = torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev)
    ev_in = [torch.cuda.Event() for _ in range(D)]
    ev_done = [torch.cuda.Event() for _ in range(D)]
    ev_copied = torch.cuda.Event()
    # the same copies with the GPU otherwise idle: the host link's own rate (the
    # first pass, untimed, also warms the copy path: the first copies from these
    # pinned buffers ran at a third of the later rate)
    def idle_copies(reps):
        for _ in range(reps):
            with torch.cuda.stream(copy_in):
                for k in host:
                    sets[0][k].copy_(host[k], non_blocking=True)
            with torch.cuda.stream(copy_out):
                hy0.copy_(sets[-1]["y0"], non_blocking=True)
                hy1.copy_(sets[-1]["y1"], non_blocking=True)

    torch.cuda.synchronize()
    idle_reps = 10
    idle_copies(idle_reps)
    torch.cuda.synchronize()
    i0, i1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    i0.record(stream)
    copy_in.wait_event(i0)
    copy_out.wait_event(i0)
    idle_copies(idle_reps)
    stream.wait_event(_record(copy_in))
    stream.wait_event(_record(copy_out))
    i1.record(stream)
    torch.cuda.synchronize()
    copy_idle_ms = i0.elapsed_time(i1) / idle_reps
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    copy_in.wait_event(f0)
    copy_out.wait_event(f0)

    # events around every copy on its copy stream: the copies' own time per step
    cp_ev = []

    def timed_copy(st, fn):
        a, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(st)
        with torch.cuda.stream(st):
            fn()
        b_.record(st)
        cp_ev.append((a, b_))

    def h2d_into(b):
        timed_copy(copy_in, lambda: [sets[b][k].copy_(host[k], non_blocking=True) for k in host])
        ev_in[b].record(copy_in)

    h2d_into(0)
    begin()
    base = 12_000   # (a multiple of D: step base + i uses work set i % D)
    for i in range(args.steps):
        b = i % D
        if i + 1 < args.steps:
            nb = (i + 1) % D
            if i + 1 >= D:
                copy_in.wait_event(ev_done[nb])   # step i + 1 - D (and its copy out) has finished with that set
            h2d_into(nb)
        step(base + i, sets[b], wait_in=ev_in[b])   # (work set and input set: both i % D)
        copy_out.wait_event(evs[b]["dec"])
        timed_copy(copy_out, lambda: (hy0.copy_(sets[b]["y0"], non_blocking=True),
                                      hy1.copy_(sets[b]["y1"], non_blocking=True)))
        ev_done[b].record(copy_out)
    end(base + args.steps - 1)
    ev_copied.record(copy_out)
    stream.wait_event(ev_copied)
    stream.wait_event(_record(copy_in))
    f1.record(stream)
    torch.cuda.synchronize()
    ms_e2e = f0.elapsed_time(f1)
    copy_ms = sum(a.elapsed_time(b_) for a, b_ in cp_ev) / args.steps
    copy_gbs = (h2d + d2h) / (copy_ms * 1e-3) / 1e9 if copy_ms > 0 else None
    ms, ms_e2e, ms_serial = max_over_ranks([ms, ms_e2e, ms_serial], world, dev)
    value = job_throughput(S.products, args.steps, world, ms)
    peaks = load_peaks(sms)
    dom, table, roof = roofline(prof, serial, S, ctx.n, ctx.L, args.steps, peaks, ck, unpiped)
    roof["probe"] = {"imad32_T_per_s": round(probe["imad32"], 3), "shoup64_T_per_s": round(probe["shoup64"], 3),
                     "madwide32_T_per_s": round(probe["madwide32"], 3), "mac128_T_per_s": round(probe["mac128"], 3),
                     "note": f"register-only chains, 8 per thread, {sms * 8} x 256 threads, measured before the timed region"}
    roof["peak_check"] = check_peak(peaks, probe["imad32"])
    launches = sum(v[0] for v in prof.values())
    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        # several steps in flight (step i + 1's encoding, preparation and encryption overlap step i's
        # multiply-accumulate and decryption); one step alone, streams joined after every step:
        "ms_per_step_unpipelined": round(ms_serial / args.steps, 4),
        "dtype": "u64 (RNS mod q_i), u64 mod 2^41", "data": "synthetic",
        "config": {"workload": WORKLOAD, "partition": dict(zip(("bb", "cib", "cob", "th", "tw", "kth", "ktw"),
                                                            plan.part)),
                   "ct_in": S.ct_in, "pt": S.pt, "ct_out": S.ct_out, "products_per_step": S.products,
                   "l2": "inputs larger than L2 (ct_in %.0f MB per step)" % (S.ct_in * S.ct_words * 8 / 1e6),
                   "parallelism": f"replicas x{world} (independent layers, no collective)",
                   "streamed_slices": nch, "steps_in_flight": D},
        "parity_selfcheck": parity_ok,
        "host_issue_ms_per_step": round(t_issue * 1e3 / args.steps, 4),
        "roofline": roof,
        "kernels": table,
        "clocks": ck,
        "gpu_launches": launches,
        "e2e": {"value": job_throughput(S.products, args.steps, world, ms_e2e), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": round(ms_e2e / args.steps, 4),
                # the copies' own time per step (events on the copy stream) and the host link rate they reached;
                # overlap = the part of the copy time hidden behind the step
                "copy_ms_per_step": round(copy_ms, 4), "copy_gb_per_s": round(copy_gbs, 1) if copy_gbs else None,
                # both directions at once with the GPU idle (the link's rate): bound = max(step, this)
                "copy_idle_ms_per_step": round(copy_idle_ms, 4),
                "copy_idle_gb_per_s": round((h2d + d2h) / (copy_idle_ms * 1e-3) / 1e9, 1) if copy_idle_ms > 0 else None,
                "overlap": round(max(0.0, min(1.0, (ms / args.steps + copy_ms - ms_e2e / args.steps) / copy_ms)), 3)
                if copy_ms > 0 else None},
    }
    if not args.no_extras and world == 1:
        line["workloads"] = extras(he, local)
    if not args.no_sweep and world == 1:   # (a multi-GPU run keeps to the timed layer step)
        line["ntt_sweep"] = ntt_sweep(he, local, args.sweep_polys, args.sweep_points, args.sweep_reps,
                                      args.ntt_log_radix)
    if world == 1 and not args.no_cpu_baseline:
        v, st, desc, spent = oracle_sample(part_tuple=plan.part, min_seconds=12.0)
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": desc,
                                "seconds": round(spent, 1), "host_cores_available": len(os.sched_getaffinity(0)),
                                "plain_cpu_ntt_limb_ntts_per_s": cpu_ntt_baseline(),
                                "plain_cpu_pipeline": cpu_pipeline(he, local)}
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
