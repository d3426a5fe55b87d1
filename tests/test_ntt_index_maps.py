"""CPU check of the index maps of the GPU transform's rounds (the fold engine of
csrc/ntt.cuh, restated here): T = N / E threads each hold E = 2^LOGE words; round
S0 runs K = min(LOGE, LOGN - S0) radix-2 stages on G = 2^(LOGE - K) groups per
thread, group g at positions ((g >> LOGD) << (LOGD + K)) + (g mod 2^LOGD) + l 2^LOGD
(LOGD = LOGN - S0 - K).  For every size and radix the kernels use:

* every round touches each position exactly once;
* the rounds marked warp-local (full rounds with LOGD <= 5, and the last, partial
  round with its groups numbered warp by warp) keep warp w inside positions
  [32 E w, 32 E (w + 1)), so an exchange between two such rounds needs only the
  warp's own barrier; once a round is warp-local, all later ones are;
* the forward epilogue's and the inverse prologue's groups of consecutive
  positions (numbered 32 (E / W) w + 32 j + lane) stay inside the same range and
  cover every position once;
* the padded shared-memory slot x + 2 (x >> 5) keeps the warps' ranges disjoint."""
import pytest


def slot(x):
    return x + 2 * (x >> 5)


def rounds(logn, loge):
    return list(range(0, logn, loge))


def round_positions(logn, loge, s0):
    n, e = 1 << logn, 1 << loge
    t = n >> loge
    k = min(loge, logn - s0)
    groups = 1 << (loge - k)
    logd = logn - s0 - k
    local = k < loge or logd <= 5

    def grp(tau, gg):
        if groups == 1:
            return tau
        return ((tau >> 5) << (5 + loge - k)) + (gg << 5) + (tau & 31)

    pos = {}
    for tau in range(t):
        for gg in range(groups):
            g = grp(tau, gg)
            base = ((g >> logd) << (logd + k)) + (g & ((1 << logd) - 1))
            pos.setdefault(tau, []).extend(base + (l << logd) for l in range(1 << k))
    return pos, local, e


def in_warp_range(tau, e, p):
    w = tau >> 5
    return 32 * e * w <= p < 32 * e * (w + 1)


@pytest.mark.parametrize("logn,loge", [(12, 4), (12, 5), (13, 4), (13, 5), (14, 4), (14, 5)])
def test_rounds_are_bijections_and_warp_local_where_marked(logn, loge):
    n = 1 << logn
    locals_ = []
    for s0 in rounds(logn, loge):
        pos, local, e = round_positions(logn, loge, s0)
        assert sorted(p for v in pos.values() for p in v) == list(range(n))
        if local:
            assert all(in_warp_range(tau, e, p) for tau, v in pos.items() for p in v)
        locals_.append(local)
    assert not locals_[0]                       # the first round spans the whole polynomial
    assert locals_ == sorted(locals_)           # warp-local from some round on


@pytest.mark.parametrize("logn,loge", [(12, 4), (12, 5), (13, 4), (13, 5), (14, 4), (14, 5)])
def test_epilogue_and_prologue_groups_stay_in_the_warp(logn, loge):
    n, e = 1 << logn, 1 << loge
    t = n >> loge
    nr = (logn + loge - 1) // loge
    kl = logn - (nr - 1) * loge
    fused = kl <= 2
    widths = ([1 << kl] + ([4] if (1 << kl) < 4 else [])) if fused else [2, 4]
    for gw in widths:
        seen = []
        for tau in range(t):
            if fused:
                starts = [((tau >> 5) * (32 * e // gw) + (tau & 31) + 32 * j) * gw for j in range(e // gw)]
            else:
                starts = [(tau >> 5) * 32 * e + gw * ((tau & 31) + 32 * j) for j in range(e // gw)]
            for s in starts:
                for i in range(gw):
                    assert in_warp_range(tau, e, s + i)
                    seen.append(s + i)
        assert sorted(seen) == list(range(n))
    # the inverse prologue of the unfused case: position (tau >> 5) 32 E + lane + 32 l
    if not fused:
        seen = [(tau >> 5) * 32 * e + (tau & 31) + 32 * l for tau in range(t) for l in range(e)]
        assert sorted(seen) == list(range(n))


def test_padded_slots_keep_warp_ranges_disjoint():
    for e in (16, 32):
        for w in range(8):
            lo, hi = 32 * e * w, 32 * e * (w + 1) - 1
            assert slot(hi) < slot(32 * e * (w + 1))
            assert slot(lo) > (slot(lo - 1) if lo else -1)
            # pairs and quads of consecutive positions never straddle a padding gap
            for x in range(lo, hi + 1, 4):
                assert slot(x + 3) - slot(x) == 3
