"""Oracle pins for the demapper with prior, the a-priori LLR source and the
EXIT quantities (mutual information, J function). CPU only."""
import math

import numpy as np
import pytest

from tests import inputs


def symbols(m, B=3, S=40, seed=5):
    rng = inputs.rng(seed)
    shape = (B, S) if m == 1 else (B, S, 2)
    return rng.normal(size=shape) * (1.2 if m > 2 else 1.0)


def priors(m, B=3, S=40, seed=6, scale=4.0):
    return inputs.rng(seed).normal(size=(B, S * m)) * scale


@pytest.mark.parametrize("m", [1, 2, 4, 6, 8])
@pytest.mark.parametrize("method", [0, 1])
def test_zero_prior_is_plain_demapper(orc, m, method):
    y = symbols(m)
    for mode in (0, 1):
        a = orc.demap_prior(y, m, 0.7, None, method=method, mode=mode)
        b = orc.demap(y, m, 0.7, method=method)
        assert np.allclose(a, b, rtol=1e-12, atol=1e-12)
        z = orc.demap_prior(y, m, 0.7, np.zeros((y.shape[0], y.shape[1] * m)), method=method, mode=mode)
        assert np.allclose(z, b, rtol=1e-12, atol=1e-12)


def test_bpsk_closed_form(orc):
    y, la, n0 = symbols(1), priors(1), 0.8
    app = orc.demap_prior(y, 1, n0, la, mode=0, clamp=1e9)
    ext = orc.demap_prior(y, 1, n0, la, mode=1, clamp=1e9)
    assert np.allclose(ext, 4.0 * y / n0, rtol=1e-12, atol=1e-12)
    assert np.allclose(app, 4.0 * y / n0 + la, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("method", [0, 1])
def test_qpsk_extrinsic_ignores_prior(orc, method):
    # the I and Q bits of a QPSK symbol are independent: a prior on one says
    # nothing about the other, and the extrinsic LLR is the channel LLR
    y, la, n0 = symbols(2), priors(2), 0.6
    ext = orc.demap_prior(y, 2, n0, la, method=method, mode=1, clamp=1e9)
    ref = np.empty_like(ext)
    ref[:, 0::2] = 2.0 * math.sqrt(2.0) * y[..., 0] / n0
    ref[:, 1::2] = 2.0 * math.sqrt(2.0) * y[..., 1] / n0
    assert np.allclose(ext, ref, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("m", [4, 6, 8])
@pytest.mark.parametrize("method", [0, 1])
def test_app_minus_extrinsic_is_prior(orc, m, method):
    y, la = symbols(m, S=20), priors(m, S=20)
    app = orc.demap_prior(y, m, 0.5, la, method=method, mode=0, clamp=1e9)
    ext = orc.demap_prior(y, m, 0.5, la, method=method, mode=1, clamp=1e9)
    assert np.allclose(app - ext, la, rtol=1e-9, atol=1e-9)


def gray_points(m):
    # the constellation of the oracle's mapper, point index p = label bits MSB first
    P = 1 << m
    bits = ((np.arange(P)[:, None] >> (m - 1 - np.arange(m))[None, :]) & 1).astype(np.uint8)
    x = orc_map_points(bits, m)
    return bits, x


def orc_map_points(bits, m):
    import oracle
    x = oracle.map_bits(bits, m)  # each row of m bits is one symbol
    return x[:, 0, 0] + 1j * x[:, 0, 1]


@pytest.mark.parametrize("m", [4, 6])
def test_app_by_probabilities(orc, m):
    # Bayes in the probability domain: P(b_i = 0 | y) = sum_{x: b_i = 0} p(y|x) P(x) / sum_x p(y|x) P(x),
    # with P(x) = prod_j P(b_j(x)) and P(b = 0) = 1 / (1 + e^-La)
    bits, pts = gray_points(m)
    y, la, n0 = symbols(m, B=1, S=12), priors(m, B=1, S=12, scale=2.0), 0.9
    app = orc.demap_prior(y, m, n0, la, mode=0, clamp=1e9)
    for s in range(12):
        yc = y[0, s, 0] + 1j * y[0, s, 1]
        pb0 = 1.0 / (1.0 + np.exp(-la[0, s * m:(s + 1) * m]))
        px = np.prod(np.where(bits == 0, pb0[None, :], 1.0 - pb0[None, :]), axis=1)
        w = np.exp(-np.abs(yc - pts) ** 2 / n0) * px
        for i in range(m):
            ref = math.log(w[bits[:, i] == 0].sum()) - math.log(w[bits[:, i] == 1].sum())
            assert app[0, s * m + i] == pytest.approx(ref, rel=1e-9, abs=1e-9)


def test_apriori_is_consistent_gaussian(orc):
    from oracle import exit as oexit
    B, N, sigma = 4, 50000, 1.7
    bits = (inputs.rng(9).random((B, N)) < 0.5).astype(np.uint8)
    L = orc.apriori(bits, sigma, seed=77, cw0=3)
    s = 1.0 - 2.0 * bits
    u = s * L  # N(sigma^2/2, sigma^2) for either bit value
    tol = 5.0 / math.sqrt(B * N)
    assert abs(u.mean() - 0.5 * sigma ** 2) < 5 * sigma * tol
    assert abs(u.std() - sigma) < 5 * sigma * tol
    # consistency E[exp(-u)] = 1 (the symmetry of a true LLR)
    assert abs(np.exp(-u).mean() - 1.0) < 0.05
    # the estimate of I approaches J(sigma)
    assert abs(oexit.mutual_info(L, bits) - oexit.J(sigma)) < 0.004
    # a different counter draws different noise, the same one the same noise
    assert not np.array_equal(L, orc.apriori(bits, sigma, seed=77, cw0=4))
    assert np.array_equal(L, orc.apriori(bits, sigma, seed=77, cw0=3))


def test_mutual_info_limits():
    from oracle import exit as oexit
    bits = (inputs.rng(1).random((2, 1000)) < 0.5).astype(np.uint8)
    sure = 30.0 * (1.0 - 2.0 * bits)
    assert oexit.mutual_info(sure, bits) == pytest.approx(1.0, abs=1e-12)
    assert oexit.mutual_info(np.zeros_like(sure), bits) == pytest.approx(0.0, abs=1e-15)
    assert oexit.mutual_info(-sure, bits) < -40.0  # confidently wrong LLRs
    assert oexit.J(0.0) == 0.0
    assert oexit.J(40.0) == pytest.approx(1.0, abs=1e-9)
    js = [oexit.J(s) for s in np.linspace(0.1, 8.0, 40)]
    assert all(a < b for a, b in zip(js, js[1:]))
    # J(sigma) for small sigma: I ~ sigma^2 / (8 ln 2) (second-order expansion of the capacity of a weak
    # consistent Gaussian LLR)
    assert oexit.J(0.05) == pytest.approx(0.05 ** 2 / (8 * math.log(2)), rel=2e-3)
