"""Oracle pins for polar coding: encoder structure, Bhattacharyya construction
identities, CRC by independent long division, SC on noiseless input, and SCL
with a list covering every information word equal to brute-force maximum
likelihood in the max-log (correlation discrepancy) metric. CPU only."""
import itertools

import numpy as np
import pytest

from tests import inputs


def test_encoder_is_kronecker_power_and_involution(orc):
    F = np.array([[1, 0], [1, 1]], dtype=np.uint8)
    G = F
    for _ in range(2):
        G = np.kron(G, F) % 2  # F^(x)3, N = 8
    rng = inputs.rng(2)
    u = (rng.random((20, 8)) < 0.5).astype(np.uint8)
    x = orc.polar_encode(u)
    assert np.array_equal(x, (u.astype(int) @ G.astype(int)) % 2)
    u16 = (rng.random((10, 16)) < 0.5).astype(np.uint8)
    assert np.array_equal(orc.polar_encode(orc.polar_encode(u16)), u16)  # G_N^2 = I over GF(2)


@pytest.mark.parametrize("n,snr", [(3, 0.0), (6, 1.5), (10, -1.0)])
def test_bhattacharyya_identities(orc, n, snr):
    z = orc.polar_bhatt(n, snr)
    z0 = np.exp(-10 ** (snr / 10))
    N = 1 << n
    # (2z - z^2) + z^2 = 2z: the recursion conserves the sum
    assert z.sum() == pytest.approx(N * z0, rel=1e-12)
    assert z[-1] == pytest.approx(z0 ** N, rel=1e-12, abs=1e-300)
    assert z[0] == pytest.approx(1 - (1 - z0) ** N, rel=1e-12)
    # a bit channel with more "plus" transforms in the same places is better
    assert z[N - 1] <= z[N - 2] <= z[N // 2]


def test_info_set(orc):
    info, frozen = orc.polar_info_set(6, 32, 1.0)
    z = orc.polar_bhatt(6, 1.0)
    assert len(info) == 32 and (np.diff(info) > 0).all()
    assert frozen.sum() == 32 and not frozen[info].any()
    assert z[info].max() <= z[frozen.astype(bool)].min()


def gf2_remainder(bits, g, r):
    # long division of bits * x^r by g over GF(2), coefficient lists MSB first
    poly = [(g >> (r - i)) & 1 for i in range(r + 1)]
    work = list(bits) + [0] * r
    for i in range(len(bits)):
        if work[i]:
            for j in range(r + 1):
                work[i + j] ^= poly[j]
    return np.array(work[-r:], dtype=np.uint8)


@pytest.mark.parametrize("g,r", [(0x107, 8), (0x1021 | (1 << 16), 16), (0b1011, 3)])
def test_crc_by_long_division(orc, g, r):
    rng = inputs.rng(r)
    for length in (1, 7, 40, 123):
        bits = (rng.random(length) < 0.5).astype(np.uint8)
        rem = orc.crc(bits, g, r)
        assert np.array_equal(rem, gf2_remainder(bits, g, r))
        # a message followed by its remainder divides evenly
        assert not orc.crc(np.concatenate([bits, rem]), g, r).any()


def test_sc_noiseless(orc):
    n, K = 7, 64
    info, frozen = orc.polar_info_set(n, K, 2.0)
    rng = inputs.rng(3)
    u = np.zeros((5, 1 << n), dtype=np.uint8)
    u[:, info] = (rng.random((5, K)) < 0.5)
    x = orc.polar_encode(u)
    llr = 8.0 * (1.0 - 2.0 * x)
    for L in (1, 4):
        uh, pm = orc.polar_scl(llr, frozen, info, L)
        assert np.array_equal(uh, u) and (pm == 0).all()


@pytest.mark.parametrize("n,K", [(3, 3), (4, 5), (5, 4)])
def test_full_list_is_maxlog_ml(orc, n, K):
    # with every information word kept, SCL returns the codeword of least correlation discrepancy
    # sum_j |L_j| [x_j != hard(L_j)], and its path metric is that discrepancy
    N = 1 << n
    info, frozen = orc.polar_info_set(n, K, 0.0)
    rng = inputs.rng(10 * n + K)
    words = []
    for bits in itertools.product([0, 1], repeat=K):
        u = np.zeros(N, dtype=np.uint8)
        u[info] = bits
        words.append((u, orc.polar_encode(u)))
    for _ in range(15):
        llr = rng.normal(size=N) * 2.0
        uh, pm = orc.polar_scl(llr[None], frozen, info, 1 << K)
        mets = [float(np.sum(np.abs(llr) * (x != (llr < 0)))) for _, x in words]
        best = int(np.argmin(mets))
        assert pm[0] == pytest.approx(mets[best], abs=1e-9)
        assert np.array_equal(uh[0], words[best][0]) or mets[best] == sorted(mets)[1]


def test_crc_aided_selection(orc):
    # CRC-aided list decoding at moderate noise returns a CRC-valid word more often than plain SCL picks the
    # transmitted one; and at high SNR both return the transmitted word
    n, K, r, g = 7, 40, 8, 0x107
    info, frozen = orc.polar_info_set(n, K, 1.0)
    rng = inputs.rng(4)
    B = 60
    data = (rng.random((B, K - r)) < 0.5).astype(np.uint8)
    u = np.zeros((B, 1 << n), dtype=np.uint8)
    for b in range(B):
        u[b, info] = np.concatenate([data[b], orc.crc(data[b], g, r)])
    x = orc.polar_encode(u)
    clean = 6.0 * (1.0 - 2.0 * x)
    uh, _ = orc.polar_scl(clean, frozen, info, 8, g, r)
    assert np.array_equal(uh, u)
    noisy = 1.0 * (1.0 - 2.0 * x) + rng.normal(size=x.shape) * 1.2
    plain, _ = orc.polar_scl(noisy, frozen, info, 8)
    ca, _ = orc.polar_scl(noisy, frozen, info, 8, g, r)
    ok_plain = sum(np.array_equal(plain[b], u[b]) for b in range(B))
    ok_ca = sum(np.array_equal(ca[b], u[b]) for b in range(B))
    assert ok_ca >= ok_plain
    valid = [not orc.crc(np.concatenate([ca[b, info][:K - r], ca[b, info][K - r:]]), g, r).any() for b in range(B)]
    assert sum(valid) >= ok_ca
