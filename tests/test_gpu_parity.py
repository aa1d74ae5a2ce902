"""GPU parity: the CUDA library (through its C ABI) against the CPU oracle.

Bars:
* min-sum (layered and flooding; FP32 / FP16 / 6-bit messages): output LLRs,
  hard decisions and iteration counts bit-exact against the oracle's FP32
  replay with the same message store;
* sum-product: output LLRs (clamped to +-20) within 1e-3 relative of the
  FP64 oracle;
* transmitter: information bits and noiseless symbols exact up to binary32
  rounding of the level scale, noise within the accuracy of binary32
  logf/sqrtf/sincospif;
* demapper: within 2e-5 relative (+1e-4 absolute) of the FP64 2-D oracle;
* error counts: exact integers.
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


def unpack(words: np.ndarray, k: int) -> np.ndarray:
    w = words.view(np.uint32)
    bits = ((w[:, :, None] >> np.arange(32, dtype=np.uint32)) & 1).astype(np.uint8)
    return bits.reshape(w.shape[0], -1)[:, :k]


CODES = {
    # name: (bg, Z, rows_kept, punct_cols, B) -- B spans several CTAs plus a ragged tail
    "bg2_z8": (2, 8, 0, 0, 100),
    "bg2_z64": (2, 64, 0, 0, 20),
    "bg1_z384": (1, 384, 0, 2, 5),
    "bg1_z128_r13": (1, 128, 13, 2, 9),
    "bg2_z200": (2, 200, 0, 0, 3),
    # truncations of both shapes at rate points of the mixed workload (rows 24, 5, 7, 4); the two
    # shortest send every column (with 2Z punctured, two punctured columns can share each of their
    # few rows and then never resolve, so no codeword would stop early)
    "bg1_z64_r24": (1, 64, 24, 2, 7),
    "bg1_z32_r5": (1, 32, 5, 0, 11),
    "bg2_z64_r7": (2, 64, 7, 2, 5),
    "bg2_z16_r4": (2, 16, 4, 0, 13),
}


# channel strength per code for the early-stop cases: the truncated high-rate
# code needs a stronger channel to converge within a few iterations
STRONG = {"bg1_z128_r13": 5.0, "bg1_z64_r24": 4.0, "bg1_z32_r5": 7.0, "bg2_z64_r7": 6.0, "bg2_z16_r4": 7.0}


def make_case(orc, name, mean, seed):
    bg, Z, rows_kept, punct, B = CODES[name]
    ocode = orc.Code(bg, Z, rows_kept=rows_kept, punct_cols=punct)
    u = inputs.info_bits(seed, B, ocode.k)
    cw = ocode.encoder.encode(u)
    L = inputs.gaussian_llrs(cw, mean, seed + 1)
    L_tx = np.ascontiguousarray(L[:, ocode.p0:ocode.p0 + ocode.n_tx])
    return ocode, u, cw, L_tx


def gpu_code(lx, name):
    bg, Z, rows_kept, punct, _ = CODES[name]
    return lx.qc_ldpc_build(bg, Z, rows_kept=rows_kept, punct_cols=punct)


@pytest.mark.parametrize("name", list(CODES))
@pytest.mark.parametrize("prec", [0, 1, 2])
@pytest.mark.parametrize("early_stop", [False, True])
def test_layered_minsum_bit_exact(lx, orc, name, prec, early_stop):
    ocode, u, cw, L_tx = make_case(orc, name, STRONG.get(name, 2.2) if early_stop else 2.2, 17)
    code = gpu_code(lx, name)
    llr, bits, its = lx.ldpc_bp_decode(code, cuda(L_tx), algo=lx.LAYERED_MINSUM, iters=8, msg_prec=prec,
                                       early_stop=early_stop, llr_out=True)
    app, hard, oits = orc.decode(ocode.graph, orc.place_llr(L_tx, ocode.p0, ocode.n), algo=0, schedule=0, iters=8,
                                 prec=1, store=prec, early_stop=early_stop)
    assert np.array_equal(llr.cpu().numpy(), app.astype(np.float32))
    assert np.array_equal(unpack(bits.cpu().numpy(), ocode.k), hard[:, :ocode.k])
    assert np.array_equal(its.cpu().numpy(), oits)
    if early_stop:
        assert oits.min() < 8  # some codewords stop early: the path is exercised


# flooding: Z = 8 (a warp spans four rows), 64, a truncated Z = 128 code, 200 and 384
@pytest.mark.parametrize("name", ["bg2_z8", "bg2_z64", "bg1_z128_r13", "bg2_z200", "bg1_z384"])
@pytest.mark.parametrize("prec", [0, 1, 2])
@pytest.mark.parametrize("weighted", [False, True])
def test_flooding_minsum_bit_exact(lx, orc, name, prec, weighted):
    ocode, u, cw, L_tx = make_case(orc, name, 2.5, 23)
    code = gpu_code(lx, name)
    w = None
    if weighted:
        w = (0.6 + 0.8 * inputs.rng(5).random((6, code.nnz))).astype(np.float32)
    llr, bits, its = lx.ldpc_bp_decode(code, cuda(L_tx), algo=lx.FLOOD_MINSUM, iters=6, msg_prec=prec,
                                       early_stop=True, llr_out=True, weights=None if w is None else cuda(w))
    app, hard, oits = orc.decode(ocode.graph, orc.place_llr(L_tx, ocode.p0, ocode.n), algo=0, schedule=1, iters=6,
                                 prec=1, store=prec, early_stop=True,
                                 weights=None if w is None else w.astype(np.float64))
    assert np.array_equal(llr.cpu().numpy(), app.astype(np.float32))
    assert np.array_equal(unpack(bits.cpu().numpy(), ocode.k), hard[:, :ocode.k])
    assert np.array_equal(its.cpu().numpy(), oits)


def spa_close(gpu, ref, rel=1e-3):
    """Element-wise |g - r| <= rel * max(|r|, 1) after clamping both to +-20: relative
    below the clamp, with an absolute floor of rel where |r| < 1 (an LLR near 0 has no
    meaningful relative error; 1e-3 in L moves the bit probability by at most 2.5e-4)."""
    g = np.clip(gpu.astype(np.float64), -20, 20)
    r = np.clip(ref, -20, 20)
    return np.abs(g - r) <= rel * np.maximum(np.abs(r), 1.0)


def spa_report(gpu, ref):
    g = np.clip(gpu.astype(np.float64), -20, 20)
    r = np.clip(ref, -20, 20)
    err = np.abs(g - r) / np.maximum(np.abs(r), 1.0)
    return f"max scaled error {err.max():.3g}, {(err > 1e-3).sum()} of {err.size} above 1e-3"


@pytest.mark.parametrize("name", ["bg2_z8", "bg2_z64", "bg2_z200", "bg1_z384"])
@pytest.mark.parametrize("schedule", ["layered", "flooding"])
def test_spa_fp32_within_tolerance(lx, orc, name, schedule):
    ocode, u, cw, L_tx = make_case(orc, name, 3.0, 29)
    code = gpu_code(lx, name)
    algo = lx.LAYERED_SPA if schedule == "layered" else lx.FLOOD_SPA
    llr, bits, _ = lx.ldpc_bp_decode(code, cuda(L_tx), algo=algo, iters=10, msg_prec=0, llr_out=True)
    app, hard, _ = orc.decode(ocode.graph, orc.place_llr(L_tx, ocode.p0, ocode.n), algo=1,
                              schedule=0 if schedule == "layered" else 1, iters=10)
    ok = spa_close(llr.cpu().numpy(), app)
    assert ok.all(), f"{(~ok).sum()} of {ok.size} outside 1e-3"
    assert np.array_equal(unpack(bits.cpu().numpy(), ocode.k), hard[:, :ocode.k])


@pytest.mark.parametrize("name", ["bg2_z8", "bg2_z64", "bg2_z200", "bg1_z384"])
@pytest.mark.parametrize("schedule", ["layered", "flooding"])
def test_spa_fp16_within_tolerance(lx, orc, name, schedule):
    """Sum-product with FP16 messages against the FP64 oracle with the binary16 message store:
    the check-node output is rounded to half (RNE), stored and added to the APP on both sides."""
    ocode, u, cw, L_tx = make_case(orc, name, 3.0, 29)
    code = gpu_code(lx, name)
    algo = lx.LAYERED_SPA if schedule == "layered" else lx.FLOOD_SPA
    llr, bits, _ = lx.ldpc_bp_decode(code, cuda(L_tx), algo=algo, iters=10, msg_prec=lx.MSG_F16, llr_out=True)
    app, hard, _ = orc.decode(ocode.graph, orc.place_llr(L_tx, ocode.p0, ocode.n), algo=1,
                              schedule=0 if schedule == "layered" else 1, iters=10, store=orc.STORE_F16)
    g = llr.cpu().numpy()
    ok = spa_close(g, app)
    assert ok.all(), spa_report(g, app)
    # hard decisions agree wherever the oracle's APP is farther from 0 than the tolerance
    sure = np.abs(app[:, :ocode.k]) > 1e-3
    assert np.array_equal(unpack(bits.cpu().numpy(), ocode.k)[sure], hard[:, :ocode.k][sure])


@pytest.mark.parametrize("prec", [0, 1])
def test_spa_weighted_flooding_within_tolerance(lx, orc, prec):
    """Weighted flooding sum-product (FP32 and FP16 messages) against the FP64 oracle."""
    ocode, u, cw, L_tx = make_case(orc, "bg2_z64", 2.5, 37)
    code = gpu_code(lx, "bg2_z64")
    w = (0.6 + 0.8 * inputs.rng(9).random((8, code.nnz))).astype(np.float32)
    llr, _, _ = lx.ldpc_bp_decode(code, cuda(L_tx), algo=lx.FLOOD_SPA, iters=8, msg_prec=prec, llr_out=True,
                                  weights=cuda(w))
    app, _, _ = orc.decode(ocode.graph, orc.place_llr(L_tx, ocode.p0, ocode.n), algo=1, schedule=1, iters=8,
                           store=orc.STORE_F16 if prec == 1 else orc.STORE_NATIVE, weights=w.astype(np.float64))
    g = llr.cpu().numpy()
    assert spa_close(g, app).all(), spa_report(g, app)


@pytest.mark.parametrize("name", ["bg2_z8", "bg2_z16_r4", "bg2_z64"])
@pytest.mark.parametrize("algo", ["minsum", "spa"])
def test_flooding_codewords_per_cta_agree(lx, orc, name, algo):
    """Flooding with 1, 2, 3, 5 and 8 codewords per CTA (a CTA's threads walk the nodes of all its codewords,
    across codeword boundaries within a warp at small Z) and the automatic choice: identical outputs, with
    early stop (codewords stop in different iterations within one CTA) and weights; min-sum also equals
    the oracle's FP32 replay."""
    bg, Z, rows_kept, punct, _ = CODES[name]
    ocode = orc.Code(bg, Z, rows_kept=rows_kept, punct_cols=punct)
    B = 61  # ragged against every tile size
    u = inputs.info_bits(41, B, ocode.k)
    L = inputs.gaussian_llrs(ocode.encoder.encode(u), STRONG.get(name, 2.2), 42)
    L_tx = np.ascontiguousarray(L[:, ocode.p0:ocode.p0 + ocode.n_tx])
    code = gpu_code(lx, name)
    w = (0.6 + 0.8 * inputs.rng(43).random((8, code.nnz))).astype(np.float32)
    a = lx.FLOOD_MINSUM if algo == "minsum" else lx.FLOOD_SPA
    outs = []
    try:
        for G in (1, 2, 3, 5, 8, 0):
            lx.ldpcx_tune_set(lx.TUNE_CW_PER_CTA, G)
            llr, bits, its = lx.ldpc_bp_decode(code, cuda(L_tx), algo=a, iters=8, msg_prec=1, early_stop=True,
                                               llr_out=True, weights=cuda(w))
            outs.append((llr.cpu().numpy(), bits.cpu().numpy(), its.cpu().numpy()))
    finally:
        lx.ldpcx_tune_set(lx.TUNE_CW_PER_CTA, 0)
    for o in outs[1:]:
        assert np.array_equal(o[0], outs[0][0]) and np.array_equal(o[1], outs[0][1])
        assert np.array_equal(o[2], outs[0][2])
    assert len(np.unique(outs[0][2])) > 1  # codewords of one CTA stop in different iterations
    if algo == "minsum":
        app, hard, oits = orc.decode(ocode.graph, orc.place_llr(L_tx, ocode.p0, ocode.n), algo=0, schedule=1, iters=8,
                                     prec=1, store=1, early_stop=True, weights=w.astype(np.float64))
        assert np.array_equal(outs[0][0], app.astype(np.float32))
        assert np.array_equal(outs[0][2], oits)


def test_tx_noiseless_symbols_and_bits(lx, orc):
    for name, m in [("bg1_z384", 4), ("bg2_z8", 2), ("bg1_z384", 8), ("bg2_z64", 1), ("bg1_z128_r13", 6)]:
        bg, Z, rows_kept, punct, B = CODES[name]
        ocode = orc.Code(bg, Z, rows_kept=rows_kept, punct_cols=punct)
        if ocode.n_tx % m:
            continue
        code = gpu_code(lx, name)
        seed, cw0 = 0x1DBC | (2 << 32), 12345
        y, info = lx.sim_tx(code, seed, cw0, B, m, cuda(np.zeros(1, np.float32)))
        u = orc.source_bits(seed, cw0, B, ocode.k)
        assert np.array_equal(unpack(info.cpu().numpy(), ocode.k), u)
        x = orc.map_bits(ocode.encoder.encode(u), m, ocode.p0, ocode.n_tx)
        assert np.allclose(y.cpu().numpy(), x, rtol=2e-7, atol=0), (name, m)


def test_tx_noise_matches_oracle(lx, orc):
    bg, Z, rows_kept, punct, B = CODES["bg1_z384"]
    ocode = orc.Code(bg, Z, punct_cols=punct)
    code = gpu_code(lx, "bg1_z384")
    seed = 77
    u = orc.source_bits(seed, 3, B, ocode.k)
    cw = ocode.encoder.encode(u)
    for m, n0 in [(4, 0.3), (1, 0.8), (2, 0.5)]:
        y, _ = lx.sim_tx(code, seed, 3, B, m, cuda(np.full(1, n0, np.float32)))
        x = orc.map_bits(cw, m, ocode.p0, ocode.n_tx)
        ref = orc.awgn(x, m, float(np.float32(n0)), seed, 3)
        assert np.allclose(y.cpu().numpy(), ref, rtol=0, atol=2e-5), m
    # per-codeword N0
    n0s = np.linspace(0.1, 1.0, B).astype(np.float32)
    y, _ = lx.sim_tx(code, seed, 3, B, 4, cuda(n0s))
    ref = orc.awgn(orc.map_bits(cw, 4, ocode.p0, ocode.n_tx), 4, n0s.astype(np.float64), seed, 3)
    assert np.allclose(y.cpu().numpy(), ref, rtol=0, atol=2e-5)


@pytest.mark.parametrize("m", [1, 2, 4, 6, 8])
@pytest.mark.parametrize("method", [0, 1])
def test_demap_matches_oracle(lx, orc, m, method):
    B, S = 7, 333
    y = inputs.symbols(41 + m, B, S, m)
    n0 = np.float32(0.5)
    llr = lx.demap_app(cuda(y), cuda(np.full(1, n0, np.float32)), m, method=method, clamp=20.0)
    ref = orc.demap(y.astype(np.float64), m, float(n0), method, 20.0)
    assert np.allclose(llr.cpu().numpy(), ref, rtol=2e-5, atol=1e-4)
    # per-codeword N0
    n0s = np.linspace(0.2, 2.0, B).astype(np.float32)
    llr = lx.demap_app(cuda(y), cuda(n0s), m, method=method, clamp=20.0)
    ref = orc.demap(y.astype(np.float64), m, n0s.astype(np.float64), method, 20.0)
    assert np.allclose(llr.cpu().numpy(), ref, rtol=2e-5, atol=1e-4)


def test_count_exact(lx):
    B, k = 1000, 8448
    kw = (k + 31) // 32
    ref = inputs.packed_bits(1, B, kw, k)
    hat = ref.copy()
    rng = inputs.rng(2)
    for b in rng.choice(B, 50, replace=False):
        for _ in range(int(rng.integers(1, 40))):
            j = int(rng.integers(0, k))
            hat[b, j // 32] ^= np.int32(np.uint32(1 << (j % 32)).view(np.int32))
    its = rng.integers(1, 21, size=B).astype(np.int32)
    counts = torch.zeros(5, dtype=torch.int64, device="cuda")
    lx.sim_count(cuda(ref), cuda(hat), cuda(its), k, counts)
    diff = unpack(ref ^ hat, k)
    errs = diff.sum(axis=1)
    assert counts.cpu().tolist() == [B * k, int(errs.sum()), B, int((errs > 0).sum()), int(its.sum())]


def test_sim_run_equals_stepwise_chain(lx):
    code = lx.qc_ldpc_build(2, 64)
    kw = dict(m=2, demap_method=lx.DEMAP_MAXLOG, algo=lx.LAYERED_MINSUM, iters=10, msg_prec=lx.MSG_F16,
              seed=99, cw0=1000, batch=300, max_batches=3)
    ebn0 = [1.0, 2.0]
    res_g = lx.sim_run(code, ebn0, use_graph=True, **kw)
    res_e = lx.sim_run(code, ebn0, use_graph=False, **kw)
    assert res_g == res_e
    # the same chain, one public call at a time
    r = code.k / code.n_tx
    cw = 1000
    for i, eb in enumerate(ebn0):
        counts = torch.zeros(5, dtype=torch.int64, device="cuda")
        n0 = torch.tensor([1.0 / (r * 2 * 10 ** (eb / 10))], dtype=torch.float32, device="cuda")
        for _ in range(3):
            y, info = lx.sim_tx(code, 99, cw, 300, 2, n0)
            llr = lx.demap_app(y, n0, 2, method=lx.DEMAP_MAXLOG)
            _, bits, its = lx.ldpc_bp_decode(code, llr, algo=lx.LAYERED_MINSUM, iters=10, msg_prec=lx.MSG_F16)
            lx.sim_count(info, bits, its, code.k, counts)
            cw += 300
        c = counts.cpu().tolist()
        assert [res_g[i][f] for f in ("bits", "bit_errors", "blocks", "block_errors", "iter_sum")] == c


@pytest.mark.parametrize("kw", [dict(max_batches=4, min_bit_errors=300), dict(max_batches=2, stop_ber=2e-2),
                                dict(max_batches=3, min_bit_errors=50, stop_ber=1e-1)])
def test_sim_run_graph_equals_eager_with_early_ends(lx, kw):
    # graph mode starts the next batch's front before the host reads the counts; a point ended by its
    # error count or a sweep ended by stop_ber discards that front, so the counts must still match eager mode
    code = lx.qc_ldpc_build(2, 32)
    base = dict(m=4, demap_method=lx.DEMAP_MAXLOG, algo=lx.LAYERED_MINSUM, iters=8, msg_prec=lx.MSG_F16,
                seed=17, cw0=5, batch=200)
    ebn0 = [0.0, 1.0, 2.0, 3.0, 4.0]
    res_g = lx.sim_run(code, ebn0, use_graph=True, **base, **kw)
    res_e = lx.sim_run(code, ebn0, use_graph=False, **base, **kw)
    assert res_g == res_e
    assert sum(p["blocks"] for p in res_g) > 0


def test_sim_run_ber_matches_oracle_statistically(lx, orc):
    code = lx.qc_ldpc_build(2, 8)
    ocode = orc.Code(2, 8)
    res = lx.sim_run(code, [1.5], m=2, demap_method=lx.DEMAP_EXACT, algo=lx.LAYERED_MINSUM, iters=20,
                     msg_prec=lx.MSG_F32, seed=5, batch=2000, max_batches=1)
    o = orc.sim(ocode, seed=5, cw0=0, B=2000, ebn0_db=1.5, m=2, demap_method=orc.DEMAP_EXACT, prec=1)
    g_err, o_err = res[0]["bit_errors"], int(o[1])
    n = res[0]["bits"]
    assert n == int(o[0])
    p = (g_err + o_err) / (2 * n)
    assert p > 1e-3
    # same codewords, same noise draws (up to binary32 rounding): nearly identical counts
    assert abs(g_err - o_err) <= 0.02 * max(g_err, o_err) + 20


@pytest.mark.parametrize("prec", [1, 0, 2])
def test_full_size_launch_sampled(lx, orc, prec):
    """The bench launch: BG1-shaped Z=384, B=4096, layered min-sum, 20 iterations, FP16 messages (the
    headline) and the FP32 / 6-bit variants; six sampled codewords against the oracle's FP32 replay."""
    bg, Z, B = 1, 384, 4096
    ocode = orc.Code(bg, Z, punct_cols=2)
    code = lx.qc_ldpc_build(bg, Z, punct_cols=2)
    rng = inputs.rng(8)
    sample = np.sort(rng.choice(B, 6, replace=False))
    sample[-1] = B - 1
    cw = np.zeros((B, ocode.n), dtype=np.uint8)
    u = inputs.info_bits(9, len(sample), ocode.k)
    cw[sample] = ocode.encoder.encode(u)
    L = inputs.gaussian_llrs(cw, 2.0, 10)
    L_tx = np.ascontiguousarray(L[:, ocode.p0:ocode.p0 + ocode.n_tx])
    llr, bits, its = lx.ldpc_bp_decode(code, cuda(L_tx), algo=lx.LAYERED_MINSUM, iters=20, msg_prec=prec,
                                       llr_out=True)
    app, hard, oits = orc.decode(ocode.graph, orc.place_llr(L_tx[sample], ocode.p0, ocode.n), algo=0, iters=20,
                                 prec=1, store=prec)
    assert np.array_equal(llr[torch.from_numpy(sample).cuda()].cpu().numpy(), app.astype(np.float32))
    assert np.array_equal(unpack(bits.cpu().numpy()[sample], ocode.k), hard[:, :ocode.k])
    assert (its.cpu().numpy() == 20).all()


def test_edge_cases(lx, orc):
    code = lx.qc_ldpc_build(2, 8)
    ocode = orc.Code(2, 8)
    # B = 0 is a no-op
    empty = torch.zeros((0, code.n_tx), dtype=torch.float32, device="cuda")
    lx.ldpc_bp_decode(code, empty)
    assert lx.ldpcx_sync_status()[0] == 0
    # non-finite inputs: NaN decodes as 0, +-inf as +-clamp, and the condition is latched
    L = inputs.gaussian_llrs(np.zeros((3, code.n), np.uint8), 3.0, 4)
    L[0, 5] = np.nan
    L[1, 7] = np.inf
    L[2, 9] = -np.inf
    llr, bits, its = lx.ldpc_bp_decode(code, cuda(L), iters=5, llr_out=True)
    st, flags = lx.ldpcx_sync_status()
    assert st == -6 and flags & lx.FLAG_NONFINITE
    L2 = L.astype(np.float64)
    L2[0, 5] = 0.0
    app, _, _ = orc.decode(ocode.graph, L2, iters=5, prec=1)
    assert np.array_equal(llr.cpu().numpy(), app.astype(np.float32))
    assert lx.ldpcx_sync_status()[0] == 0  # cleared
    # too-small workspace is refused before any launch
    with pytest.raises(lx.LdpcxError):
        lx.ldpc_bp_decode(code, cuda(L), ws=torch.empty(16, dtype=torch.uint8, device="cuda"))
    # one iteration, huge clamp, zero offset
    ocode2, u, cw, L_tx = make_case(orc, "bg2_z64", 1.5, 3)
    code2 = gpu_code(lx, "bg2_z64")
    llr, _, _ = lx.ldpc_bp_decode(code2, cuda(L_tx), iters=1, offset=0.0, clamp=1e4, llr_out=True)
    app, _, _ = orc.decode(ocode2.graph, L_tx.astype(np.float64), iters=1, offset=0.0, clamp=1e4, prec=1)
    assert np.array_equal(llr.cpu().numpy(), app.astype(np.float32))


def test_repeat_calls_are_deterministic(lx, orc):
    ocode, u, cw, L_tx = make_case(orc, "bg1_z384", 1.8, 51)
    code = gpu_code(lx, "bg1_z384")
    a = lx.ldpc_bp_decode(code, cuda(L_tx), msg_prec=1, llr_out=True)[0].cpu().numpy()
    b = lx.ldpc_bp_decode(code, cuda(L_tx), msg_prec=1, llr_out=True)[0].cpu().numpy()
    assert np.array_equal(a, b)


@pytest.mark.parametrize("name", ["bg2_z64", "bg1_z384", "bg2_z200", "bg1_z128_r13", "bg1_z64_r24", "bg1_z32_r5",
                                  "bg2_z64_r7", "bg2_z16_r4"])
@pytest.mark.parametrize("prec", [0, 1, 2])
def test_kernel_variants_agree(lx, orc, name, prec):
    """Per-edge messages, check-node state with the row table, check-node state
    with the compiled-in schedule (one or two check nodes per thread), generic
    and compile-time Z: identical outputs."""
    ocode, u, cw, L_tx = make_case(orc, name, 1.9, 23)
    code = gpu_code(lx, name)
    outs = []
    try:
        for cns, sched, spec, zpt in [(0, 0, 1, 0), (1, 0, 1, 0), (1, 1, 1, 0), (1, 1, 0, 0), (0, 0, 0, 0),
                                      (1, 1, 1, 2), (1, 1, 0, 2), (0, 0, 1, 2), (1, 0, 1, 2)]:
            lx.ldpcx_tune_set(lx.TUNE_CN_STATE, cns)
            lx.ldpcx_tune_set(lx.TUNE_SCHEDULE, sched)
            lx.ldpcx_tune_set(lx.TUNE_SPECIALISED, spec)
            lx.ldpcx_tune_set(lx.TUNE_ZPT, zpt)
            outs.append(lx.ldpc_bp_decode(code, cuda(L_tx), algo=lx.LAYERED_MINSUM, iters=9, msg_prec=prec,
                                          early_stop=True, llr_out=True))
    finally:
        for key in (lx.TUNE_CN_STATE, lx.TUNE_SCHEDULE, lx.TUNE_SPECIALISED):
            lx.ldpcx_tune_set(key, 1)
        lx.ldpcx_tune_set(lx.TUNE_ZPT, 0)
    for o in outs[1:]:
        assert all(torch.equal(a, b) for a, b in zip(o, outs[0]))


@pytest.mark.parametrize("name", ["bg2_z64", "bg1_z384", "bg2_z200"])
@pytest.mark.parametrize("prec", [0, 1])
def test_spa_schedule_variants_agree(lx, orc, name, prec):
    """Layered sum-product: the compiled-in schedule equals the row-table kernel
    bit for bit (same arithmetic, same order)."""
    ocode, u, cw, L_tx = make_case(orc, name, 2.4, 31)
    code = gpu_code(lx, name)
    outs = []
    try:
        for sched, spec in [(0, 1), (1, 1), (1, 0)]:
            lx.ldpcx_tune_set(lx.TUNE_SCHEDULE, sched)
            lx.ldpcx_tune_set(lx.TUNE_SPECIALISED, spec)
            outs.append(lx.ldpc_bp_decode(code, cuda(L_tx), algo=lx.LAYERED_SPA, iters=7, msg_prec=prec,
                                          early_stop=True, llr_out=True))
    finally:
        lx.ldpcx_tune_set(lx.TUNE_SCHEDULE, 1)
        lx.ldpcx_tune_set(lx.TUNE_SPECIALISED, 1)
    for o in outs[1:]:
        assert all(torch.equal(a, b) for a, b in zip(o, outs[0]))
