"""GPU parity of shortened code blocks (filler bits) and of the paper's Listing 1
chain: k = 500 information bits coded into n = 1000 bits, 16-QAM, on a seeded
BG2-shaped code with Z = 52 (kb Z = 520, so 20 filler bits).

Each stage runs through the C ABI and is compared with the oracle
(oracle/shorten.py, oracle/ratematch.py and the C oracle) on the same inputs:
codewords, rate-matched bits, recovered soft buffers and integer counts
bit-exact; symbols within the accuracy of the binary32 noise draws; min-sum
decoding bit-exact against the FP32 replay (APP, hard decisions, iteration
counts), sum-product within 1e-3.
"""
import numpy as np
import pytest

from tests import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lx():
    import paper_2203_11854_gb300 as lx
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    lx.load_library()
    return lx


def cuda(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def unpack(words, nbits):
    w = words.cpu().numpy().view(np.uint32)
    bits = ((w[:, :, None] >> np.arange(32, dtype=np.uint32)) & 1).astype(np.uint8)
    return bits.reshape(w.shape[0], -1)[:, :nbits]


def pack(bits):
    bits = np.asarray(bits, dtype=np.uint32)
    B, n = bits.shape
    nw = (n + 31) // 32
    padded = np.zeros((B, nw * 32), dtype=np.uint32)
    padded[:, :n] = bits
    w = (padded.reshape(B, nw, 32) << np.arange(32, dtype=np.uint32)).sum(axis=2, dtype=np.uint64)
    return w.astype(np.uint32).view(np.int32)


CASES = [(2, 52, 2, 500), (2, 16, 2, 150), (1, 8, 2, 170), (2, 8, 0, 80), (1, 384, 2, 8000)]


def codes(lx, orc, bg, Z, punct, k, encoder=True):
    from oracle import shorten as sh
    mother = lx.qc_ldpc_build(bg, Z, punct_cols=punct)
    sc = lx.qc_ldpc_shorten(mother, k)
    osc = sh.ShortCode(orc.Code(bg, Z, punct_cols=punct, encoder=encoder), k)
    return mother, sc, osc


@pytest.mark.parametrize("bg,Z,punct,k", CASES)
def test_shortened_code_info(lx, orc, bg, Z, punct, k):
    mother, sc, osc = codes(lx, orc, bg, Z, punct, k, encoder=False)
    assert sc.k == k and sc.n_fill == mother.k - k and sc.n_tx == osc.n_tx and sc.n == mother.n
    assert sc.p0 == mother.p0 and sc.edges == mother.edges and mother.n_fill == 0


@pytest.mark.parametrize("bg,Z,punct,k", CASES[:4])
def test_shortened_codewords_match_oracle(lx, orc, bg, Z, punct, k):
    _, sc, osc = codes(lx, orc, bg, Z, punct, k)
    seed, cw0, B = 91, 5, 13
    cw = unpack(lx.sim_codewords(sc, seed, cw0, B), sc.n)
    u = orc.source_bits(seed, cw0, B, k)
    assert np.array_equal(cw, osc.encode(u))
    n0 = cuda(np.full(1, 0.5, np.float32))
    _, info = lx.sim_tx(sc, seed, cw0, B, 2 if sc.n_tx % 2 == 0 else 1, n0)
    assert np.array_equal(unpack(info, k), u)


@pytest.mark.parametrize("bg,Z,punct,k", CASES)
@pytest.mark.parametrize("m", [1, 2, 4, 6])
def test_sim_tx_equals_codewords_ratematch_map(lx, orc, bg, Z, punct, k, m):
    """sim_tx == sim_codewords -> rate_match (k0 = 0, ncb = E = n_tx, qm = 1) -> qam_map_awgn, bit for bit,
    for the shortened code and for its mother code."""
    mother, sc, _ = codes(lx, orc, bg, Z, punct, k, encoder=False)
    seed, cw0, B = 17, 1 << 33, 9
    n0 = cuda(np.linspace(0.2, 0.9, B).astype(np.float32))
    for c in (sc, mother):
        if c.n_tx % m:
            continue
        y, _ = lx.sim_tx(c, seed, cw0, B, m, n0)
        f = lx.rate_match(c, lx.sim_codewords(c, seed, cw0, B), 0, c.n_tx, c.n_tx, 1)
        y2 = lx.qam_map_awgn(f, c.n_tx, m, seed, cw0, n0)
        assert torch.equal(y, y2)


@pytest.mark.parametrize("k0,ncb,E,qm", [(0, 2580, 1000, 4), (0, 2580, 2580, 2), (517, 2580, 3000, 6),
                                         (1999, 2000, 120, 8), (350, 2580, 7740, 1)])
def test_rate_match_shortened_matches_oracle(lx, orc, k0, ncb, E, qm):
    from oracle import ratematch as rm
    _, sc, osc = codes(lx, orc, 2, 52, 2, 500)
    seed, B = 23, 6
    cw_gpu = lx.sim_codewords(sc, seed, 0, B)
    cw = osc.encode(orc.source_bits(seed, 0, B, 500))
    f = unpack(lx.rate_match(sc, cw_gpu, k0, ncb, E, qm), E)
    assert np.array_equal(f, rm.rate_match(osc.tx_bits(cw), 0, ncb, k0, E, qm))
    llr = inputs.gaussian_llrs(f, 1.5, 29)
    v = lx.rate_recover(sc, cuda(llr), k0, ncb, qm).cpu().numpy()
    ref = rm.rate_recover(llr.astype(np.float64), ncb, k0, qm)
    if E <= ncb:
        assert np.array_equal(v, ref.astype(np.float32))  # one term per position: exact
    else:
        assert np.allclose(v, ref, rtol=1e-6, atol=1e-5)


def test_rate_match_rejects_buffer_past_the_fillers(lx, orc):
    _, sc, _ = codes(lx, orc, 2, 52, 2, 500, encoder=False)
    cw = torch.zeros((1, (sc.n + 31) // 32), dtype=torch.int32, device="cuda")
    with pytest.raises(lx.LdpcxError):
        lx.rate_match(sc, cw, 0, sc.n_tx + 1, 100, 1)


@pytest.mark.parametrize("bg,Z,punct,k", CASES)
@pytest.mark.parametrize("algo,schedule,prec", [(0, 0, 0), (0, 0, 1), (0, 0, 2), (0, 1, 1), (1, 0, 0), (1, 1, 1)])
def test_decode_shortened(lx, orc, bg, Z, punct, k, algo, schedule, prec):
    _, sc, osc = codes(lx, orc, bg, Z, punct, k)
    B = 5 if Z >= 128 else 24
    cw = osc.encode(inputs.info_bits(31, B, k))
    # sum-product is compared within a tolerance: a channel past the threshold, as in the mother-code tests
    L_tx = inputs.gaussian_llrs(osc.tx_bits(cw), 2.0 if algo == 0 else 3.0, 32)
    lalgo = {(0, 0): lx.LAYERED_MINSUM, (0, 1): lx.FLOOD_MINSUM, (1, 0): lx.LAYERED_SPA, (1, 1): lx.FLOOD_SPA}
    llr, bits, its = lx.ldpc_bp_decode(sc, cuda(L_tx), algo=lalgo[(algo, schedule)], iters=8, msg_prec=prec,
                                       early_stop=True, llr_out=True)
    app, hard, oits = orc.decode(osc.graph, osc.place_llr(L_tx), algo=algo, schedule=schedule, iters=8,
                                 prec=1 if algo == 0 else 0, store=prec, early_stop=True)
    assert bits.shape[1] == (k + 31) // 32
    if algo == 0:
        assert np.array_equal(llr.cpu().numpy(), app.astype(np.float32))
        assert np.array_equal(unpack(bits, k), hard[:, :k])
        assert np.array_equal(its.cpu().numpy(), oits)
    else:
        g = np.clip(llr.cpu().numpy().astype(np.float64), -20, 20)
        r = np.clip(app, -20, 20)
        assert (np.abs(g - r) <= 1e-3 * np.maximum(np.abs(r), 1.0)).all()
    assert not hard[:, k:k + sc.n_fill].any()  # the fillers decode to their known zeros


def test_mixed_launch_with_a_shortened_group(lx, orc):
    groups = []
    for bg, Z, punct, k, B in [(2, 52, 2, 500, 40), (2, 16, 2, 150, 30), (1, 8, 2, 176, 20)]:
        _, sc, osc = codes(lx, orc, bg, Z, punct, k)
        cw = osc.encode(inputs.info_bits(41 + Z, B, k))
        groups.append((sc, cuda(inputs.gaussian_llrs(osc.tx_bits(cw), 2.2, 42 + Z))))
    res = lx.ldpc_bp_decode_mixed(groups, algo=lx.LAYERED_MINSUM, iters=10, msg_prec=lx.MSG_F16, early_stop=True,
                                  llr_out=True)
    for (c, llr), (lo, b, it) in zip(groups, res):
        ref = lx.ldpc_bp_decode(c, llr, algo=lx.LAYERED_MINSUM, iters=10, msg_prec=lx.MSG_F16, early_stop=True,
                                llr_out=True)
        assert torch.equal(lo, ref[0]) and torch.equal(b, ref[1]) and torch.equal(it, ref[2])


def test_extrinsic_shortened(lx, orc):
    _, sc, osc = codes(lx, orc, 2, 16, 2, 150)
    B = 7
    cw = osc.encode(inputs.info_bits(51, B, 150))
    L_tx = inputs.gaussian_llrs(osc.tx_bits(cw), 1.5, 52)
    app, _, _ = lx.ldpc_bp_decode(sc, cuda(L_tx), algo=lx.LAYERED_MINSUM, iters=4, msg_prec=lx.MSG_F32,
                                  llr_out=True)
    ext = lx.ldpc_extrinsic(sc, app, cuda(L_tx)).cpu().numpy()
    a = app.cpu().numpy()[:, osc.tx_pos]
    ref = np.clip(a - np.clip(L_tx, -20, 20), -20, 20)
    assert np.array_equal(ext, ref.astype(np.float32))


def test_differentiable_decode_refuses_shortened_codes(lx, orc):
    _, sc, _ = codes(lx, orc, 2, 16, 2, 150, encoder=False)
    with pytest.raises(lx.LdpcxError):
        lx.ldpc_bp_ckpt_bytes(sc, 4, iters=5)


@pytest.mark.parametrize("prec", [0, 1])
def test_listing1_chain(lx, orc, prec):
    """Listing 1: BinarySource -> LDPC5GEncoder(k=500, n=1000) -> Mapper(16-QAM) -> AWGN -> Demapper("app")
    -> LDPC5GDecoder -> compute_ber, stage by stage against the oracle."""
    from oracle import ratematch as rm
    _, sc, osc = codes(lx, orc, 2, 52, 2, 500)
    k, n, m, B, seed, cw0 = 500, 1000, 4, 96, 0x1DBC, 7
    ebn0 = 5.0
    n0 = 1.0 / (k / n * m * 10 ** (ebn0 / 10))
    no = cuda(np.full(1, n0, np.float32))
    # source and encoder
    cw_gpu = lx.sim_codewords(sc, seed, cw0, B)
    u = orc.source_bits(seed, cw0, B, k)
    cw = osc.encode(u)
    assert np.array_equal(unpack(cw_gpu, sc.n), cw)
    # 5G rate matching: n = 1000 bits from the start of the circular buffer, interleaved over 4 rows
    f_gpu = lx.rate_match(sc, cw_gpu, 0, sc.n_tx, n, m)
    f = rm.rate_match(osc.tx_bits(cw), 0, osc.n_tx, 0, n, m)
    assert np.array_equal(unpack(f_gpu, n), f)
    # mapper and AWGN on the rate-matched bits
    y = lx.qam_map_awgn(f_gpu, n, m, seed, cw0, no)
    ref_y = orc.awgn(orc.map_bits(f, m), m, float(np.float32(n0)), seed, cw0)
    assert np.allclose(y.cpu().numpy(), ref_y, rtol=0, atol=2e-5)
    # APP demapper, soft rate recovery into the decoder's transmit layout
    llr = lx.demap_app(y, no, m, method=lx.DEMAP_EXACT)
    ref_llr = orc.demap(y.cpu().numpy().astype(np.float64), m, float(np.float32(n0)), orc.DEMAP_EXACT)
    assert np.allclose(llr.cpu().numpy(), ref_llr, rtol=2e-5, atol=1e-4)
    buf = lx.rate_recover(sc, llr, 0, sc.n_tx, m)
    ref_buf = rm.rate_recover(llr.cpu().numpy().astype(np.float64), osc.n_tx, 0, m)
    assert np.array_equal(buf.cpu().numpy(), ref_buf.astype(np.float32))
    # decoder (layered offset min-sum, 20 iterations) against the FP32 replay with the same message store
    app, bits, its = lx.ldpc_bp_decode(sc, buf, algo=lx.LAYERED_MINSUM, iters=20, msg_prec=prec, llr_out=True)
    o_app, o_hard, o_its = orc.decode(osc.graph, osc.place_llr(ref_buf), algo=0, iters=20, prec=1, store=prec)
    assert np.array_equal(app.cpu().numpy(), o_app.astype(np.float32))
    assert np.array_equal(unpack(bits, k), o_hard[:, :k])
    assert np.array_equal(its.cpu().numpy(), o_its)
    # compute_ber: integer counts against the oracle's hard decisions
    counts = torch.zeros(5, dtype=torch.int64, device="cuda")
    lx.sim_count(cuda(pack(u)), bits, its, k, counts)
    c = counts.cpu().tolist()
    err = (o_hard[:, :k] != u)
    assert c[0] == B * k and c[1] == int(err.sum()) and c[2] == B and c[3] == int(err.any(axis=1).sum())
    # the code works: fewer information-bit errors than hard decisions on the demapped channel bits make
    uncoded = int(((llr.cpu().numpy() < 0) != f).sum()) * k / n
    assert c[1] < uncoded


def test_sim_run_shortened(lx, orc):
    _, sc, _ = codes(lx, orc, 2, 52, 2, 500, encoder=False)
    pts = lx.sim_run(sc, [2.0, 4.0], m=4, batch=256, max_batches=2, iters=10, use_graph=False)
    pts_g = lx.sim_run(sc, [2.0, 4.0], m=4, batch=256, max_batches=2, iters=10, use_graph=True)
    for p, q in zip(pts, pts_g):
        assert p["bits"] == 2 * 256 * 500 and p == q
    assert pts[1]["bit_errors"] <= pts[0]["bit_errors"]
