"""Philox4x64-10 (oracle; test infrastructure only).

Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3",
SC'11.  A 256-bit counter c = (c0, c1, c2, c3) and a 128-bit key k = (k0, k1)
map to four 64-bit words through ten rounds.  One round multiplies c0 and c2
by fixed odd constants, keeping both halves of each 128-bit product, and mixes
the high halves with c1, c3 and the round key; the key advances by fixed Weyl
increments between rounds.

The paper leaves its random source unspecified (Alg. 1 "chooses random mask",
Sec. 2.2 encryption); the counter-based generator makes every draw a pure
function of (seed, stream, index) so that the GPU and this oracle agree
bit-for-bit.  Pinned against numpy.random.Philox (an independent
implementation of the same generator) in tests/test_oracle_philox.py.
"""
from __future__ import annotations

from typing import List, Sequence

MASK64 = (1 << 64) - 1
PHILOX_M0 = 0xD2E7470EE14C6C93
PHILOX_M1 = 0xCA5A826395121157
PHILOX_W0 = 0x9E3779B97F4A7C15
PHILOX_W1 = 0xBB67AE8584CAA73B
ROUNDS = 10


def philox4x64(counter: Sequence[int], key: Sequence[int], rounds: int = ROUNDS) -> List[int]:
    c0, c1, c2, c3 = (int(x) & MASK64 for x in counter)
    k0, k1 = (int(x) & MASK64 for x in key)
    for r in range(rounds):
        if r:
            k0 = (k0 + PHILOX_W0) & MASK64
            k1 = (k1 + PHILOX_W1) & MASK64
        p0 = PHILOX_M0 * c0
        p1 = PHILOX_M1 * c2
        hi0, lo0 = p0 >> 64, p0 & MASK64
        hi1, lo1 = p1 >> 64, p1 & MASK64
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return [c0, c1, c2, c3]


# ---------------------------------------------------------------------------
# Stream layout shared (by specification, not by code) with the CUDA library.
# key = (seed, domain); counter = (block, index_a, index_b, 0).
# ---------------------------------------------------------------------------
DOMAIN_SECRET = 1      # ternary secret key:    ctr = (i // 4, 0, 0, 0),  word i % 4
DOMAIN_A = 2           # encryption mask a:     ctr = (i // 2, ct, limb, 0), words 2(i%2), 2(i%2)+1
DOMAIN_E = 3           # encryption error e:    ctr = (i // 4, ct, 0, 0),  word i % 4
DOMAIN_MASK = 4        # re-mask, per output element: ctr = (flat // 4, 0, 0, 0), word flat % 4
DOMAIN_MASK_PAD = 5    # re-mask, unused ct coefficients: ctr = (i // 4, ct_out, 0, 0), word i % 4
DOMAIN_FLOOD = 6       # flooding noise of returned cts: ctr = (i // 4, ct_out, 0, 0), word i % 4
DOMAIN_PK_A = 7        # public key's a:        ctr = (i // 2, 0, limb, 0), words 2(i%2), 2(i%2)+1
DOMAIN_PK_E = 8        # public key's error e:  ctr = (i // 4, 0, 0, 0),  word i % 4
DOMAIN_PK_U = 9        # public-key encryption u (ternary): ctr = (i // 4, ct, 0, 0), word i % 4
DOMAIN_PK_E2 = 10      # public-key encryption e2: ctr = (i // 4, ct, 0, 0), word i % 4
                       # (its e1 is the symmetric encryption's e: DOMAIN_E)


def word(seed: int, domain: int, block: int, a: int = 0, b: int = 0, lane: int = 0) -> int:
    return philox4x64((block, a, b, 0), (seed, domain))[lane]
