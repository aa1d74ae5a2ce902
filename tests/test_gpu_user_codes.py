"""Codes from caller-supplied base matrices on the device: the transmitter's
codewords bit-exact against the oracle's Gauss-Jordan encoder (any invertible
core through its inverse, the dual-diagonal core by its recursion, own
extension shifts other than 0), every decoder on such codes bit-exact against
the oracle's FP32 replay (min-sum) or within 1e-3 of FP64 (sum-product), a
seeded code passed in as a user matrix (and through alist text) giving the
seeded code's results, and an unencodable code refused by the transmitter
but decoded."""
import numpy as np
import pytest

from tests import inputs
from tests.test_user_codes import alist_text, dense_from_base, gf2_rank, random_base

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lx():
    import paper_2203_11854_gb300 as lx
    assert torch.cuda.is_available()
    lx.load_library()
    return lx


def cuda(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def unpack(words: np.ndarray, k: int) -> np.ndarray:
    w = words.view(np.uint32)
    bits = ((w[:, :, None] >> np.arange(32, dtype=np.uint32)) & 1).astype(np.uint8)
    return bits.reshape(w.shape[0], -1)[:, :k]


# (seed, Z, kb, rows, core): Z = 24 and 40 put several codewords in one CTA with warps across codewords
USER = [(11, 16, 8, 10, "random"), (12, 24, 6, 8, "random"), (13, 40, 10, 12, "dual"), (14, 7, 5, 9, "random")]


def invertible_base(seed, Z, kb, rows, core):
    for s in range(seed, seed + 400):
        S = random_base(s, Z, kb, rows, core=core)
        if gf2_rank(dense_from_base(S[:4, kb:kb + 4], Z)) == 4 * Z:
            return S
    raise AssertionError("no invertible core drawn")


@pytest.mark.parametrize("case", USER)
def test_encoder_matches_oracle(lx, orc, case):
    seed, Z, kb, rows, core = case
    S = invertible_base(*case)
    code = lx.qc_ldpc_build_base(S, Z, kb)
    assert code.encodable == 1
    B, cw0 = 37, 1000
    cw = unpack(lx.sim_codewords(code, 5, cw0, B).cpu().numpy(), code.n)
    u = orc.source_bits(5, cw0, B, code.k)
    ref = orc.Encoder(S, kb, Z).encode(u)
    assert np.array_equal(cw, ref)
    assert not orc.Graph(S, Z).syndrome(cw).any()


@pytest.mark.parametrize("case", USER[:2])
@pytest.mark.parametrize("algo,sched", [(0, 0), (0, 1)])
@pytest.mark.parametrize("prec", [0, 1, 2])
def test_minsum_decoders_bit_exact(lx, orc, case, algo, sched, prec):
    seed, Z, kb, rows, core = case
    S = invertible_base(*case)
    code = lx.qc_ldpc_build_base(S, Z, kb)
    B = 23
    u = inputs.info_bits(seed, B, code.k)
    cw = orc.Encoder(S, kb, Z).encode(u)
    L = inputs.gaussian_llrs(cw, 2.0, seed + 1)
    galgo = lx.LAYERED_MINSUM if sched == 0 else lx.FLOOD_MINSUM
    llr, bits, its = lx.ldpc_bp_decode(code, cuda(L), algo=galgo, iters=7, msg_prec=prec, early_stop=True,
                                       llr_out=True)
    app, hard, oits = orc.decode(orc.Graph(S, Z), L.astype(np.float64), algo=0, schedule=sched, iters=7, prec=1,
                                 store=prec, early_stop=True)
    assert np.array_equal(llr.cpu().numpy(), app.astype(np.float32))
    assert np.array_equal(unpack(bits.cpu().numpy(), code.k), hard[:, :code.k])
    assert np.array_equal(its.cpu().numpy(), oits)


@pytest.mark.parametrize("sched", [0, 1])
def test_spa_decoders_close(lx, orc, sched):
    seed, Z, kb, rows, core = USER[0]
    S = invertible_base(*USER[0])
    code = lx.qc_ldpc_build_base(S, Z, kb)
    u = inputs.info_bits(3, 9, code.k)
    L = inputs.gaussian_llrs(orc.Encoder(S, kb, Z).encode(u), 2.0, 4)
    llr, _, _ = lx.ldpc_bp_decode(code, cuda(L), algo=lx.LAYERED_SPA if sched == 0 else lx.FLOOD_SPA, iters=5,
                                  llr_out=True)
    app, _, _ = orc.decode(orc.Graph(S, Z), L.astype(np.float64), algo=1, schedule=sched, iters=5, prec=0, store=0)
    g = np.clip(llr.cpu().numpy().astype(np.float64), -20, 20)
    r = np.clip(app, -20, 20)
    assert (np.abs(g - r) <= 1e-3 * np.maximum(np.abs(r), 1.0)).all()


@pytest.mark.parametrize("via_alist", [False, True])
def test_seeded_code_as_user_matrix(lx, via_alist):
    c = lx.qc_ldpc_build(1, 64, rows_kept=20, punct_cols=2)
    S = c.base()
    if via_alist:
        S = lx.qc_alist_parse(alist_text(dense_from_base(S, 64)), 64)
    u = lx.qc_ldpc_build_base(S, 64, c.kb, punct_cols=2)
    B = 40
    n0 = torch.tensor([0.5], device="cuda")
    ya, ia = lx.sim_tx(c, 9, 0, B, 4, n0)
    yb, ib = lx.sim_tx(u, 9, 0, B, 4, n0)
    assert torch.equal(ya, yb) and torch.equal(ia, ib)
    llr = lx.demap_app(ya, n0, 4)
    for prec in (0, 1):
        ra = lx.ldpc_bp_decode(c, llr, iters=10, msg_prec=prec, early_stop=True, llr_out=True)
        rb = lx.ldpc_bp_decode(u, llr, iters=10, msg_prec=prec, early_stop=True, llr_out=True)
        assert all(torch.equal(a, b) for a, b in zip(ra, rb))


def test_unencodable_code_decodes(lx, orc):
    S = random_base(21, 8, 6, 8, core="dual")
    S[5, 6 + 7] = 3  # extension row 5 reads a later parity column: no transmitter
    code = lx.qc_ldpc_build_base(S, 8, 6)
    assert code.encodable == 0
    n0 = torch.tensor([0.5], device="cuda")
    with pytest.raises(lx.LdpcxError) as e:
        lx.sim_tx(code, 1, 0, 4, 2, n0)
    assert e.value.status == -2
    L = inputs.rng(8).normal(2.0, 2.0, size=(6, code.n_tx)).astype(np.float32)
    llr, _, _ = lx.ldpc_bp_decode(code, cuda(L), iters=4, llr_out=True)
    app, _, _ = orc.decode(orc.Graph(S, 8), L.astype(np.float64), algo=0, schedule=0, iters=4, prec=1, store=0)
    assert np.array_equal(llr.cpu().numpy(), app.astype(np.float32))


def test_flooding_more_columns_than_threads(lx, orc):
    """Flooding on a base matrix with more columns than a CTA has threads (600 columns of Z = 2, rows of degree
    6): a CTA builds its column lists by the counting sort instead of one column per thread; min-sum
    bit-exact against the oracle's FP32 replay, FP32 and FP16 messages, with early stop."""
    g = inputs.rng(61)
    R, C, Z = 300, 600, 2
    S = -np.ones((R, C), dtype=np.int16)
    for r in range(R):
        for c in g.choice(C, size=6, replace=False):
            S[r, c] = g.integers(Z)
    code = lx.qc_ldpc_build_base(S, Z, C - R)
    B = 9
    L = inputs.gaussian_llrs(np.zeros((B, C * Z), np.uint8), 4.0, 62)
    for prec in (0, 1):
        llr, bits, its = lx.ldpc_bp_decode(code, cuda(L), algo=lx.FLOOD_MINSUM, iters=6, msg_prec=prec,
                                           early_stop=True, llr_out=True)
        app, hard, oits = orc.decode(orc.Graph(S, Z), L.astype(np.float64), algo=0, schedule=1, iters=6, prec=1,
                                     store=prec, early_stop=True)
        assert np.array_equal(llr.cpu().numpy(), app.astype(np.float32))
        assert np.array_equal(unpack(bits.cpu().numpy(), code.k), hard[:, :code.k])
        assert np.array_equal(its.cpu().numpy(), oits)
