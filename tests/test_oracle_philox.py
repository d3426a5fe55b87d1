"""Pins for oracle.philox against numpy.random.Philox (independent implementation of
Philox4x64-10).  numpy advances its counter by one before producing a block, so
Philox(counter=c - 1) yields block c."""
import random

import numpy as np
import pytest

from oracle.philox import philox4x64


def numpy_block(counter, key):
    c = sum(int(x) << (64 * i) for i, x in enumerate(counter))
    k = sum(int(x) << (64 * i) for i, x in enumerate(key))
    bg = np.random.Philox(counter=(c - 1) % (1 << 256), key=k)
    return [int(x) for x in bg.random_raw(4)]


def test_known_answer_zero():
    # published known-answer vector of Philox4x64-10 for counter = key = 0
    assert philox4x64((0, 0, 0, 0), (0, 0)) == [
        0x16554D9ECA36314C, 0xDB20FE9D672D0FDC, 0xD7E772CEE186176B, 0x7E68B68AEC7BA23B]


@pytest.mark.parametrize("trial", range(40))
def test_matches_numpy(trial):
    r = random.Random(trial)
    ctr = [r.getrandbits(64) if r.random() < 0.7 else r.randrange(8) for _ in range(4)]
    key = [r.getrandbits(64), r.randrange(16)]
    assert philox4x64(ctr, key) == numpy_block(ctr, key)
