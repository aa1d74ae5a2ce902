"""Oracle pins for code-block shortening with filler bits (oracle/shorten.py).

Pinned against what the construction fixes, with nothing taken from the oracle's
own arithmetic: H c = 0 on a parity-check matrix built here from numpy rolls,
zero fillers and the information bits in place; the shortened code equals the
mother code with the filler columns deleted, whose GF(2) rank (eliminated here)
gives dimension k; noiseless decoding in one iteration; the transmit-layout
bit selection equals the 5G form that keeps the fillers as <NULL> entries and
skips them; with no fillers everything reduces to the mother code. CPU only.
"""
import numpy as np
import pytest

from oracle import ratematch as rm
from oracle import shorten as sh
from tests import inputs
from tests.test_oracle_code import dense_H


def gf2_rank(M: np.ndarray) -> int:
    M = (np.asarray(M, dtype=np.uint8) & 1).copy()
    rank, rows, cols = 0, M.shape[0], M.shape[1]
    for c in range(cols):
        piv = np.nonzero(M[rank:, c])[0]
        if len(piv) == 0:
            continue
        p = rank + piv[0]
        M[[rank, p]] = M[[p, rank]]
        hit = np.nonzero(M[:, c])[0]
        hit = hit[hit != rank]
        M[hit] ^= M[rank]
        rank += 1
        if rank == rows:
            break
    return rank


CASES = [(2, 8, 2, 60), (2, 16, 2, 150), (1, 8, 2, 170), (2, 8, 0, 80)]  # (bg, Z, punct_cols, k)


@pytest.mark.parametrize("bg,Z,punct,k", CASES)
def test_shortened_codewords(orc, bg, Z, punct, k):
    code = orc.Code(bg, Z, punct_cols=punct)
    s = sh.ShortCode(code, k)
    u = inputs.info_bits(7, 9, k)
    cw = s.encode(u)
    H = dense_H(code.S, Z)
    assert not ((H.astype(np.int64) @ cw.T.astype(np.int64)) & 1).any()  # H c = 0
    assert np.array_equal(cw[:, :k], u)                                   # systematic
    assert not cw[:, k:code.k].any()                                      # fillers are 0
    assert s.n_fill == code.k - k and s.n_tx == code.n - code.p0 - s.n_fill
    # the transmit layout skips exactly the fillers and the punctured columns
    sent = np.zeros(code.n, dtype=bool)
    sent[s.tx_pos] = True
    assert not sent[:code.p0].any() and not sent[k:code.k].any() and sent[code.p0:k].all() and sent[code.k:].all()


@pytest.mark.parametrize("bg,Z,punct,k", CASES[:3])
def test_shortening_deletes_filler_columns(orc, bg, Z, punct, k):
    code = orc.Code(bg, Z, punct_cols=punct)
    s = sh.ShortCode(code, k)
    H = dense_H(code.S, Z)
    keep = np.ones(code.n, dtype=bool)
    keep[k:code.k] = False
    Hs = H[:, keep]
    # dimension of the shortened code = its length minus the rank of its parity-check matrix
    assert Hs.shape[1] - gf2_rank(Hs) == k
    cw = s.encode(inputs.info_bits(8, 5, k))
    assert not ((Hs.astype(np.int64) @ cw[:, keep].T.astype(np.int64)) & 1).any()


@pytest.mark.parametrize("bg,Z,punct,k", CASES)
def test_noiseless_decode(orc, bg, Z, punct, k):
    code = orc.Code(bg, Z, punct_cols=punct)
    s = sh.ShortCode(code, k)
    cw = s.encode(inputs.info_bits(9, 6, k))
    L = s.place_llr(20.0 * (1.0 - 2.0 * s.tx_bits(cw).astype(np.float64)))
    assert np.all(L[:, k:code.k] == 20.0) and np.all(L[:, :code.p0] == 0.0)
    for algo in (orc.ALGO_MINSUM, orc.ALGO_SPA):
        app, hard, its = orc.decode(code.graph, L, algo=algo, iters=10, early_stop=True)
        assert np.array_equal(hard, cw) and (its == 1).all()


def test_noisy_decode_keeps_fillers_zero(orc):
    code = orc.Code(2, 16, punct_cols=2)
    s = sh.ShortCode(code, 140)
    cw = s.encode(inputs.info_bits(10, 40, 140))
    L = s.place_llr(inputs.gaussian_llrs(s.tx_bits(cw), 2.5, 11))
    app, hard, _ = orc.decode(code.graph, L, algo=orc.ALGO_MINSUM, iters=20, prec=1, store=orc.STORE_F16)
    assert not hard[:, 140:code.k].any()
    assert (app[:, 140:code.k] > 0).all()


@pytest.mark.parametrize("k0_null,E", [(0, 300), (0, 1000), (37, 250), (60, 260), (65, 700), (330, 90)])
def test_selection_equals_null_skipping(orc, k0_null, E):
    # BG2-shaped Z = 8, 2 punctured columns (p0 = 16), k = 62: fillers at [62, 80), buffer index 46 .. 63
    code = orc.Code(2, 8, punct_cols=2)
    s = sh.ShortCode(code, 62)
    cw = s.encode(inputs.info_bits(12, 4, 62))
    ncb_null = code.n - code.p0
    ref = sh.select_with_nulls(cw, code.p0, 62, code.k, ncb_null, k0_null, E)
    # the same start on the transmit layout counts the non-NULL entries before it
    null = (np.arange(ncb_null) + code.p0 >= 62) & (np.arange(ncb_null) + code.p0 < code.k)
    k0 = int((~null[:k0_null]).sum())
    got = rm.select(s.tx_bits(cw), 0, s.n_tx, k0, E)
    assert np.array_equal(got, ref)


def test_no_fillers_is_the_mother_code(orc):
    code = orc.Code(2, 16, punct_cols=2)
    s = sh.ShortCode(code, code.k)
    assert s.n_fill == 0 and s.n_tx == code.n_tx
    assert np.array_equal(s.tx_pos, np.arange(code.p0, code.p0 + code.n_tx))
    L = inputs.gaussian_llrs(np.zeros((3, code.n_tx), np.uint8), 1.0, 13)
    assert np.array_equal(s.place_llr(L), orc.place_llr(L, code.p0, code.n))
    u = inputs.info_bits(14, 3, code.k)
    assert np.array_equal(s.encode(u), code.encoder.encode(u))


def test_listing1_sizes(orc):
    # k = 500 information bits, n = 1000 coded bits on a BG2-shaped code with Z = 52 (10 Z = 520 >= 500)
    code = orc.Code(2, 52, punct_cols=2, encoder=False)
    assert code.k == 520 and code.p0 == 104 and code.n == 2704
    s = sh.ShortCode(code, 500)
    assert s.n_fill == 20 and s.n_tx == 2580 and 1000 <= s.n_tx


def test_bad_shortening(orc):
    code = orc.Code(2, 8, punct_cols=2, encoder=False)
    for k in (15, 81):  # below the punctured columns, above kb Z
        with pytest.raises(ValueError):
            sh.ShortCode(code, k)
