"""Pins for the oracle's Philox4x32-10 stream, source bits and Box-Muller noise.

Philox is pinned against an independent implementation (Triton's
``tl.philox``, run by Triton's CPU interpreter in a subprocess). The noise
is pinned by its distribution (Kolmogorov-Smirnov against N(0,1), moments). splitmix64,
which seeds the codes, is pinned by known-answer outputs of its reference implementation.
"""
import json
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest
from scipy import stats

TRITON_SCRIPT = textwrap.dedent(
    """
    import os, json, sys
    os.environ["TRITON_INTERPRET"] = "1"
    import torch, triton, triton.language as tl

    @triton.jit
    def k(out_ptr, c_ptr, seed, N: tl.constexpr):
        i = tl.arange(0, N)
        c0 = tl.load(c_ptr + i * 4 + 0)
        c1 = tl.load(c_ptr + i * 4 + 1)
        c2 = tl.load(c_ptr + i * 4 + 2)
        c3 = tl.load(c_ptr + i * 4 + 3)
        a, b, c, d = tl.philox(seed, c0, c1, c2, c3)
        tl.store(out_ptr + i * 4 + 0, a)
        tl.store(out_ptr + i * 4 + 1, b)
        tl.store(out_ptr + i * 4 + 2, c)
        tl.store(out_ptr + i * 4 + 3, d)

    cfg = json.loads(sys.stdin.read())
    ctr = torch.tensor(cfg["ctr"], dtype=torch.int64).to(torch.int32)
    out = torch.zeros_like(ctr)
    k[(1,)](out, ctr, cfg["seed"], N=ctr.shape[0] // 4)
    print(json.dumps([int(x) & 0xFFFFFFFF for x in out.tolist()]))
    """
)


def test_philox_matches_independent_implementation(orc):
    pytest.importorskip("triton")
    rng = np.random.default_rng(3)
    ctr = rng.integers(0, 2**32, size=(16, 4), dtype=np.uint64).astype(np.uint32)
    ctr[0] = 0
    ctr[1] = [1, 0, 0, 0]
    ctr[2] = [0xFFFFFFFF] * 4
    seed = 0x1DBC | (2 << 32)
    env = dict(os.environ, TRITON_INTERPRET="1")
    proc = subprocess.run([sys.executable, "-c", TRITON_SCRIPT], input=json.dumps(
        {"ctr": [int(x) for x in ctr.reshape(-1)], "seed": seed}), capture_output=True, text=True, env=env,
        timeout=600)
    if proc.returncode != 0:
        pytest.skip("triton interpreter unavailable: " + proc.stderr[-300:])
    ref = np.array(json.loads(proc.stdout.strip().splitlines()[-1]), dtype=np.uint64).astype(np.uint32)
    got = orc.philox(ctr, (seed & 0xFFFFFFFF, seed >> 32)).reshape(-1)
    assert (got == ref).all()


def test_source_bit_layout(orc):
    seed, cw0, k = 0x1234_0000_5678, 5, 300
    u = orc.source_bits(seed, cw0, 2, k)
    key = (seed & 0xFFFFFFFF, seed >> 32)
    for b in range(2):
        cw = cw0 + b
        for j in [0, 1, 31, 32, 127, 128, 255, 299]:
            blk = orc.philox(np.array([[j // 128, cw & 0xFFFFFFFF, cw >> 32, 0]], dtype=np.uint32), key)[0]
            assert u[b, j] == (int(blk[(j % 128) // 32]) >> (j % 32)) & 1


def test_source_bits_are_balanced(orc):
    u = orc.source_bits(7, 0, 64, 8448)
    p = u.mean()
    n = u.size
    assert abs(p - 0.5) < 5 * 0.5 / np.sqrt(n)
    # different codewords draw different bits
    assert (u[0] != u[1]).mean() > 0.45


def test_box_muller_distribution(orc):
    x = np.zeros((64, 4096), dtype=np.float64)  # 64 "codewords" of 4096 real symbols
    y = orc.awgn(x, 1, 2.0, 99, 0)  # N0 = 2 -> unit variance per dimension
    g = y.reshape(-1)
    n = g.size
    assert abs(g.mean()) < 5 / np.sqrt(n)
    assert abs(g.var() - 1.0) < 5 * np.sqrt(2.0 / n)
    assert stats.kstest(g, "norm").pvalue > 1e-4
    # complex noise: both dimensions, N0/2 each, uncorrelated
    xc = np.zeros((32, 2048, 2))
    yc = orc.awgn(xc, 4, 0.5, 5, 100)
    re, im = yc[..., 0].reshape(-1), yc[..., 1].reshape(-1)
    nn = re.size
    for d in (re, im):
        assert abs(d.var() - 0.25) < 5 * 0.25 * np.sqrt(2.0 / nn)
    assert abs(np.corrcoef(re, im)[0, 1]) < 5 / np.sqrt(nn)


def test_box_muller_pair_values(orc):
    # u1 = 1/2, u2 = 0: r = sqrt(2 ln 2), angle 0
    g0, g1 = orc.gauss_pair(0x80000000 - 128, 0)
    u1 = ((0x80000000 - 128) >> 9) + 0.5
    u1 /= 2**23
    assert np.float32(u1) == u1  # the uniform is an exact binary32 number
    assert g0 == pytest.approx(np.sqrt(-2 * np.log(u1)), rel=1e-15)
    assert g1 == pytest.approx(0.0, abs=1e-15)
    # u2 = 1/4: angle pi/2
    g0, g1 = orc.gauss_pair(0x80000000 - 128, 0x40000000)
    assert g0 == pytest.approx(0.0, abs=1e-12)
    assert g1 == pytest.approx(np.sqrt(-2 * np.log(u1)), rel=1e-15)


def test_splitmix64_known_answer():
    """The oracle's splitmix64 (it seeds the base matrices' shifts and block placement) against the first
    outputs of the algorithm's reference implementation (S. Vigna, splitmix64.c, which accompanies the
    xoshiro generators) started from state 0."""
    import ctypes as C

    import oracle
    L = oracle.lib()
    st = C.c_uint64(0)
    got = [L.orc_splitmix64_next(C.byref(st)) for _ in range(3)]
    assert got == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    assert st.value == (3 * 0x9E3779B97F4A7C15) % (1 << 64)  # the Weyl sequence's state after three draws
