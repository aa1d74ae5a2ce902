"""Pins for the oracle's Gray QAM mapper, AWGN scaling and APP demapper.

Closed forms: BPSK L = 4y/N0, QPSK L = 2 sqrt(2) y/N0; the max-log bound
|exact - maxlog| <= ln 2^(m-1); separability of square QAM; and the uncoded
bit error rate of BPSK (Q(sqrt(2 Eb/N0))) and of Gray 16-QAM with max-log
decisions (per-bit 4-PAM error probabilities), within binomial confidence.
"""
import itertools
import math

import numpy as np
import pytest
from scipy import special


def Q(x):
    return 0.5 * special.erfc(x / math.sqrt(2.0))


def all_labels(m):
    return np.array(list(itertools.product([0, 1], repeat=m)), dtype=np.uint8)


@pytest.mark.parametrize("m", [2, 4, 6, 8])
def test_unit_energy_and_gray(orc, m):
    lab = all_labels(m)
    x = orc.map_bits(lab, m)[:, 0, :]  # one symbol per row
    es = (x ** 2).sum(axis=1).mean()
    assert es == pytest.approx(1.0, rel=1e-14)
    h = m // 2
    sc = orc.qam_scale(m)
    # per dimension: levels are the odd integers, each label distinct, Gray adjacency
    for dim in (0, 1):
        bits = lab[:, dim::2]
        lev = np.rint(x[:, dim] / sc).astype(int)
        assert np.allclose(x[:, dim] / sc, lev, atol=1e-12)
        table = {}
        for bb, lv in zip(map(tuple, bits), lev):
            assert table.setdefault(bb, lv) == lv
        assert sorted(set(table.values())) == list(range(-(2 ** h - 1), 2 ** h, 2))
        inv = {lv: bb for bb, lv in table.items()}
        levels = sorted(inv)
        for a, b in zip(levels[:-1], levels[1:]):
            assert sum(i != j for i, j in zip(inv[a], inv[b])) == 1
        # first bit of a dimension is the sign bit
        for bb, lv in table.items():
            assert (lv > 0) == (bb[0] == 0)


def test_bpsk_and_qpsk_closed_forms(orc):
    rng = np.random.default_rng(1)
    N0 = 0.7
    y = rng.normal(size=(3, 50))
    for method in (orc.DEMAP_EXACT, orc.DEMAP_MAXLOG):
        L = orc.demap(y, 1, N0, method, clamp=1e9)
        assert np.allclose(L, 4 * y / N0, rtol=1e-12, atol=1e-12)
    yc = rng.normal(size=(3, 40, 2))
    for method in (orc.DEMAP_EXACT, orc.DEMAP_MAXLOG):
        L = orc.demap(yc, 2, N0, method, clamp=1e9).reshape(3, 40, 2)
        assert np.allclose(L[..., 0], 2 * math.sqrt(2) * yc[..., 0] / N0, rtol=1e-12, atol=1e-12)
        assert np.allclose(L[..., 1], 2 * math.sqrt(2) * yc[..., 1] / N0, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("m", [4, 6, 8])
def test_exact_vs_maxlog_bound_and_separability(orc, m):
    rng = np.random.default_rng(m)
    N0 = 0.3
    y = rng.normal(scale=0.8, size=(2, 200, 2))
    Le = orc.demap(y, m, N0, orc.DEMAP_EXACT, clamp=1e9)
    Lm = orc.demap(y, m, N0, orc.DEMAP_MAXLOG, clamp=1e9)
    assert np.all(np.abs(Le - Lm) <= math.log(2 ** (m - 1)) + 1e-9)
    assert np.abs(Le - Lm).max() > 1e-3  # the two really differ
    # I-bits do not depend on the Q coordinate, and vice versa
    y2 = y.copy()
    y2[..., 1] = rng.normal(size=y2[..., 1].shape)
    Le2 = orc.demap(y2, m, N0, orc.DEMAP_EXACT, clamp=1e9)
    Le = Le.reshape(2, 200, m)
    Le2 = Le2.reshape(2, 200, m)
    assert np.allclose(Le[..., 0::2], Le2[..., 0::2], rtol=1e-9, atol=1e-9)
    assert not np.allclose(Le[..., 1::2], Le2[..., 1::2])


def test_clamp(orc):
    y = np.array([[5.0, -5.0, 0.01]])
    L = orc.demap(y, 1, 0.1, orc.DEMAP_EXACT, clamp=20.0)
    assert L[0, 0] == 20.0 and L[0, 1] == -20.0 and L[0, 2] == pytest.approx(0.4)


def binom_ok(errors, n, p, z=5.0):
    sd = math.sqrt(n * p * (1 - p))
    return abs(errors - n * p) <= z * sd + 1


@pytest.mark.parametrize("ebn0", [0.0, 2.0, 4.0])
def test_uncoded_bpsk_ber(orc, ebn0):
    B, n = 200, 4000
    bits = orc.source_bits(21, 0, B, n)
    x = orc.map_bits(bits, 1)
    N0 = orc.n0_from_ebn0(ebn0, n, n, 1)  # rate 1, one bit per symbol
    y = orc.awgn(x, 1, N0, 77, 0)
    L = orc.demap(y, 1, N0, orc.DEMAP_EXACT)
    err = int(((L < 0) != (bits == 1)).sum())
    p = Q(math.sqrt(2 * 10 ** (ebn0 / 10)))
    assert binom_ok(err, B * n, p)


@pytest.mark.parametrize("k_over_n,ebn0", [(0.5, 2.0), (1 / 3, 4.0), (0.8, 1.0)])
def test_n0_carries_the_code_rate(orc, k_over_n, ebn0):
    """Reading R5: N0 = 1/(r m Eb/N0) with r = k/n_tx, so a transmitted BPSK bit sees Es/N0 = r Eb/N0 and its
    hard-decision error rate is Q(sqrt(2 r Eb/N0)) (uncoded bits sent at the code's rate)."""
    B, n = 200, 3000
    k = round(k_over_n * n)
    bits = orc.source_bits(23, 0, B, n)
    x = orc.map_bits(bits, 1)
    N0 = orc.n0_from_ebn0(ebn0, k, n, 1)
    y = orc.awgn(x, 1, N0, 79, 0)
    err = int(((y < 0) != (bits == 1)).sum())
    p = Q(math.sqrt(2 * (k / n) * 10 ** (ebn0 / 10)))
    assert binom_ok(err, B * n, p)
    # and a rate-1 reading would be far off
    assert not binom_ok(err, B * n, Q(math.sqrt(2 * 10 ** (ebn0 / 10))))


@pytest.mark.parametrize("ebn0", [2.0, 6.0])
def test_uncoded_16qam_maxlog_ber(orc, ebn0):
    B, n = 100, 8000
    bits = orc.source_bits(31, 0, B, n)
    x = orc.map_bits(bits, 4)
    N0 = orc.n0_from_ebn0(ebn0, n, n, 4)
    y = orc.awgn(x, 4, N0, 78, 0)
    L = orc.demap(y, 4, N0, orc.DEMAP_MAXLOG)
    wrong = (L < 0) != (bits == 1)
    d = 1 / math.sqrt(10)
    s = math.sqrt(N0 / 2)
    p_sign = 0.5 * (Q(d / s) + Q(3 * d / s))
    p_mag = 0.5 * (2 * Q(d / s) + Q(3 * d / s) - Q(5 * d / s))
    nb = B * n // 4
    for pos, p in [(0, p_sign), (1, p_sign), (2, p_mag), (3, p_mag)]:
        assert binom_ok(int(wrong[:, pos::4].sum()), nb, p)


def test_awgn_variance_and_mean(orc):
    bits = orc.source_bits(1, 0, 50, 4000)
    x = orc.map_bits(bits, 4)
    N0 = 0.2
    y = orc.awgn(x, 4, N0, 9, 0)
    noise = (y - x).reshape(-1)
    assert abs(noise.var() - N0 / 2) < 5 * (N0 / 2) * math.sqrt(2 / noise.size)


def test_placement(orc):
    ltx = np.arange(1, 7, dtype=np.float64).reshape(1, 6)
    out = orc.place_llr(ltx, 2, 10)
    assert out.tolist() == [[0, 0, 1, 2, 3, 4, 5, 6, 0, 0]]
