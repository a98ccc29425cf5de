"""Pins of the oracle's Philox4x32-10 against an independent implementation.

Triton ships its own Philox4x32 (``triton.language.philox_impl``, 10 rounds by
default); its interpreter runs it on the CPU with numpy.  The oracle's generator
(written from Salmon et al., SC'11) must agree with it word for word on
counters and keys that exercise every input word and the carries of the key
schedule.
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))


def _triton_philox(rows):
    pytest.importorskip("triton")
    r = subprocess.run([sys.executable, os.path.join(HERE, "_triton_philox.py")],
                       input=json.dumps(rows), capture_output=True, text=True, timeout=600)
    if r.returncode != 0:
        pytest.skip("triton interpreter unavailable: " + r.stderr.strip().splitlines()[-1])
    return np.array(json.loads(r.stdout), dtype=np.int64)


def test_philox_matches_triton_reference():
    rng = np.random.default_rng(12345)
    rows = [[0, 0, 0, 0, 0, 0], [0xFFFFFFFF] * 6]
    rows += [[i, 0, 0, 0, 0, 0] for i in range(1, 9)]
    rows += [[0, 0, 0, 0, 1 << s, 0] for s in range(0, 32, 7)]
    rows += [[0, 0, 0, 0, 0, 1 << s] for s in range(0, 32, 7)]
    rows += rng.integers(0, 1 << 32, size=(200, 6), dtype=np.uint64).astype(np.int64).tolist()
    ref = _triton_philox(rows)
    ours = np.array([oracle.philox(r[:4], r[4:]) for r in rows], dtype=np.int64)
    assert np.array_equal(ours, ref)


def test_philox_words_are_uniform():
    # 4 x 20000 words: each of the 32 bit positions is set about half the time
    key = oracle.seed_key(0xDEADBEEFCAFEF00D)
    w = np.array([oracle.philox([i, 7, 0, oracle.TAG_MOVE], key) for i in range(20000)],
                 dtype=np.uint64).ravel()
    bits = ((w[:, None] >> np.arange(32, dtype=np.uint64)) & 1).mean(axis=0)
    sigma = 0.5 / np.sqrt(len(w))
    assert np.all(np.abs(bits - 0.5) < 5 * sigma)


def test_philox_block_is_the_generator_counter_by_counter():
    """The block form (used for bulk device comparisons) is the single-call
    generator at counters ctr[0] + i, wrapping at 2^32 in word 0 only."""
    ctr, key = [0xFFFFFFF0, 7, 9, 2], [0xDEADBEEF, 0x12345678]
    b = oracle.philox_block(ctr, key, 64)
    for i in range(64):
        c = [(ctr[0] + i) & 0xFFFFFFFF] + ctr[1:]
        assert np.array_equal(b[i], oracle.philox(c, key)), i
