"""The oracle's Philox4x32-10 against an independent implementation of the published generator
(Salmon et al., SC'11): the one in the Triton library (triton.language.random), run on the CPU by
Triton's interpreter in a child process.  It takes the key as (seed low word, seed high word), as the
oracle does, and uses the generator's published multipliers and Weyl increments; equal outputs on
many counters and keys pin the oracle's constants and round structure."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from oracle import philox as P

_CHILD = r'''
import json, os, sys
os.environ["TRITON_INTERPRET"] = "1"
import torch, triton, triton.language as tl

@triton.jit
def gen(seed, c0_ptr, c1_ptr, c2_ptr, c3_ptr, o_ptr, n: tl.constexpr):
    i = tl.arange(0, n)
    r0, r1, r2, r3 = tl.philox(seed, tl.load(c0_ptr + i), tl.load(c1_ptr + i), tl.load(c2_ptr + i),
                               tl.load(c3_ptr + i), 10)
    tl.store(o_ptr + 4 * i, r0)
    tl.store(o_ptr + 4 * i + 1, r1)
    tl.store(o_ptr + 4 * i + 2, r2)
    tl.store(o_ptr + 4 * i + 3, r3)

req = json.loads(sys.stdin.read())
res = []
for seed, cs in req:
    c = [torch.tensor([int(v) for v in col], dtype=torch.int64).to(torch.uint32) for col in zip(*cs)]
    out = torch.zeros(4 * len(cs), dtype=torch.int64).to(torch.uint32)
    gen[(1,)](seed, *c, out, n=len(cs))
    res.append([int(v) for v in out.to(torch.int64) & 0xFFFFFFFF])
print(json.dumps(res))
'''


def test_philox4x32_matches_triton():
    pytest.importorskip("triton")
    pytest.importorskip("torch")
    rng = np.random.default_rng(2)
    M = 0xFFFFFFFF
    counters = [[0, 0, 0, 0], [1, 0, 0, 0], [M, M, M, M], [0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344]]
    counters += [[int(v) for v in rng.integers(0, 1 << 32, 4, dtype=np.uint64)] for _ in range(12)]
    seeds = [0, 1, (1 << 64) - 1, 0xA4093822299F31D0, int(rng.integers(0, 1 << 62))]
    req = [[s, counters] for s in seeds]
    env = dict(os.environ, TRITON_INTERPRET="1")
    r = subprocess.run([sys.executable, "-c", _CHILD], input=json.dumps(req), capture_output=True, text=True,
                       env=env, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    got = json.loads(r.stdout.strip().splitlines()[-1])
    for (seed, cs), words in zip(req, got):
        for k, c in enumerate(cs):
            ref = P.philox4(c, (seed & M, seed >> 32))
            assert words[4 * k:4 * k + 4] == ref, (seed, c)
            v = P.philox4x32_vec(*[np.array([x], dtype=np.uint64) for x in c], seed & M, seed >> 32)
            assert [int(x[0]) for x in v] == ref
