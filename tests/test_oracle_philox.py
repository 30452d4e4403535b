"""Pins the oracle's Philox4x32-10 to an independent library implementation.

triton ships its own Philox4x32 (10 rounds, key = (seed low word, seed high
word)); its CPU interpreter runs it without a GPU. Agreement on random
counters and keys fixes the multipliers, the Weyl key schedule, the round
wiring and the word order of the oracle's generator (Salmon et al., SC'11).
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from oracle import oracle as O

_SCRIPT = r"""
import json, os, sys
os.environ["TRITON_INTERPRET"] = "1"
import torch, triton, triton.language as tl

@triton.jit
def _k(out_ptr, c_ptr, seed, N: tl.constexpr):
    o = tl.arange(0, N)
    c0 = tl.load(c_ptr + 4 * o + 0); c1 = tl.load(c_ptr + 4 * o + 1)
    c2 = tl.load(c_ptr + 4 * o + 2); c3 = tl.load(c_ptr + 4 * o + 3)
    a, b, c, d = tl.random.philox(seed, c0, c1, c2, c3, 10)
    tl.store(out_ptr + 4 * o + 0, a); tl.store(out_ptr + 4 * o + 1, b)
    tl.store(out_ptr + 4 * o + 2, c); tl.store(out_ptr + 4 * o + 3, d)

cases = json.loads(sys.stdin.read())
res = []
for seed, ctrs in cases:
    c = torch.tensor([[x - (1 << 32) if x >= (1 << 31) else x for x in row] for row in ctrs],
                     dtype=torch.int32).reshape(-1)
    out = torch.zeros(len(ctrs) * 4, dtype=torch.int32)
    _k[(1,)](out, c, seed, len(ctrs))
    res.append([[v & 0xffffffff for v in out.tolist()[4 * i:4 * i + 4]] for i in range(len(ctrs))])
print(json.dumps(res))
"""


def test_philox_matches_triton_library():
    pytest.importorskip("triton")
    rng = np.random.default_rng(2024)
    cases = []
    for n in range(6):
        seed = int(rng.integers(0, 2**63)) if n else 0
        ctrs = rng.integers(0, 2**32, size=(16, 4), dtype=np.uint64).tolist()
        ctrs[0] = [0, 0, 0, 0]
        ctrs[1] = [0xFFFFFFFF] * 4
        cases.append([seed, [[int(x) for x in r] for r in ctrs]])
    env = dict(os.environ, TRITON_INTERPRET="1")
    p = subprocess.run([sys.executable, "-c", _SCRIPT], input=json.dumps(cases),
                       capture_output=True, text=True, env=env, timeout=600)
    if p.returncode != 0:
        pytest.skip("triton interpreter unavailable: " + p.stderr[-300:])
    ref = json.loads(p.stdout.strip().splitlines()[-1])
    for (seed, ctrs), want in zip(cases, ref):
        key = [seed & 0xFFFFFFFF, seed >> 32]
        for ctr, w in zip(ctrs, want):
            assert O.philox(ctr, key).tolist() == w, (seed, ctr)


def test_philox_is_counter_sensitive():
    # Every input word must reach every output word (no dropped term).
    base = O.philox([1, 2, 3, 4], [5, 6])
    for pos in range(4):
        c = [1, 2, 3, 4]
        c[pos] ^= 1
        d = O.philox(c, [5, 6])
        assert np.all(d != base)
    for pos in range(2):
        k = [5, 6]
        k[pos] ^= 1
        assert np.all(O.philox([1, 2, 3, 4], k) != base)
