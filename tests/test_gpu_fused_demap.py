"""The demapper fused into the layered decoders (ldpc_bp_decode_qam): every output equal, bit for bit, to
demap_app followed by ldpc_bp_decode on the same received symbols. The two-step chain is itself compared with
the oracle elsewhere (the demapper within 2e-5 of the FP64 2-D demapper, min-sum bit-exact against the FP32
replay, sum-product within 1e-3), so equality here carries those comparisons over.

Cases cover each layered kernel the host can pick: the compiled schedule of a full BG1-shaped code (check-node
state and the per-edge sum-product kernel), the row-table check-node-state kernel of a truncated code, several
codewords per CTA with a ragged last CTA (small Z), shortened codes (filler bits at +clamp, the transmit layout
skipping them), every constellation size, both demapper methods, one N0 per codeword or one for all, and
non-finite symbols."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lx():
    import paper_2203_11854_gb300 as lx
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    lx.load_library()
    return lx


def build(lx, name):
    if name == "bg1_z384":
        return lx.qc_ldpc_build(1, 384, punct_cols=2)
    if name == "bg1_z36_trunc":
        return lx.qc_ldpc_build(1, 36, rows_kept=20, punct_cols=2)
    if name == "bg2_z8":
        return lx.qc_ldpc_build(2, 8)
    if name == "bg2_z52_short500":
        return lx.qc_ldpc_shorten(lx.qc_ldpc_build(2, 52, punct_cols=2), 500)
    if name == "bg1_z16_short300":
        return lx.qc_ldpc_shorten(lx.qc_ldpc_build(1, 16, punct_cols=2), 300)
    if name == "bg2_z7_short60":
        return lx.qc_ldpc_shorten(lx.qc_ldpc_build(2, 7, punct_cols=2), 60)
    raise KeyError(name)


def channel(lx, code, B, m, ebn0, per_cw, seed=0x5EED):
    r = code.k / code.n_tx
    base = 1.0 / (r * m * 10 ** (ebn0 / 10))
    no = (np.linspace(0.7, 1.3, B) * base if per_cw else np.full(1, base)).astype(np.float32)
    no = torch.from_numpy(no).cuda()
    y, _ = lx.sim_tx(code, seed, 77, B, m, no)
    return y, no


def two_step(lx, code, y, no, m, method, dclamp, dec):
    llr = lx.demap_app(y, no, m, method=method, clamp=dclamp)
    return lx.ldpc_bp_decode(code, llr, **dec, llr_out=True)


def fused(lx, code, y, no, m, method, dclamp, dec):
    return lx.ldpc_bp_decode_qam(code, y, no, m, demap_method=method, demap_clamp=dclamp, **dec, llr_out=True)


def assert_same(a, b):
    for x, z in zip(a, b):
        assert torch.equal(x, z)


DECODERS = [dict(algo=0, msg_prec=1), dict(algo=0, msg_prec=0), dict(algo=0, msg_prec=2), dict(algo=1, msg_prec=1),
            dict(algo=1, msg_prec=0)]


@pytest.mark.parametrize("name,B", [("bg1_z384", 24), ("bg1_z36_trunc", 29), ("bg2_z8", 37),
                                    ("bg2_z52_short500", 21), ("bg1_z16_short300", 33)])
@pytest.mark.parametrize("d", range(len(DECODERS)))
@pytest.mark.parametrize("early_stop", [False, True])
def test_fused_equals_demap_then_decode(lx, name, B, d, early_stop):
    code = build(lx, name)
    dec = dict(DECODERS[d], iters=12, early_stop=early_stop, offset=0.5, clamp=20.0)
    m = 4 if code.n_tx % 4 == 0 else 2
    y, no = channel(lx, code, B, m, 2.5, per_cw=True)
    assert_same(fused(lx, code, y, no, m, lx.DEMAP_MAXLOG, 20.0, dec),
                two_step(lx, code, y, no, m, lx.DEMAP_MAXLOG, 20.0, dec))


@pytest.mark.parametrize("m", [1, 2, 4, 6, 8])
@pytest.mark.parametrize("method", [0, 1])
@pytest.mark.parametrize("per_cw", [False, True])
def test_fused_every_constellation(lx, m, method, per_cw):
    code = build(lx, "bg1_z384")  # n_tx = 25,344: every m divides it
    dec = dict(algo=0, msg_prec=1, iters=8, early_stop=False, offset=0.5, clamp=20.0)
    y, no = channel(lx, code, 9, m, 1.0 + 1.5 * m, per_cw)
    # a demapper clamp below the decoder's exercises both clamps
    for dclamp in (20.0, 7.5):
        assert_same(fused(lx, code, y, no, m, method, dclamp, dec), two_step(lx, code, y, no, m, method, dclamp, dec))


@pytest.mark.parametrize("name,m", [("bg2_z7_short60", 4), ("bg2_z52_short500", 6)])
def test_fused_shortened_symbols_across_the_fillers(lx, name, m):
    """BG2-shaped Z = 7 shortened to k = 60: n_tx = 340, and the transmitted bits before the fillers number
    k - p0 = 46, so 16-QAM symbol 11 takes two bits on each side of them."""
    code = build(lx, name)
    assert code.n_tx % m == 0
    if name == "bg2_z7_short60":
        assert (code.k - code.p0) % m != 0
    dec = dict(algo=0, msg_prec=0, iters=10, early_stop=False, offset=0.5, clamp=20.0)
    y, no = channel(lx, code, 17, m, 3.0, per_cw=False)
    for method in (lx.DEMAP_EXACT, lx.DEMAP_MAXLOG):
        assert_same(fused(lx, code, y, no, m, method, 20.0, dec), two_step(lx, code, y, no, m, method, 20.0, dec))


def test_fused_nonfinite_symbols(lx):
    code = build(lx, "bg2_z8")
    dec = dict(algo=0, msg_prec=1, iters=10, early_stop=False, offset=0.5, clamp=20.0)
    y, no = channel(lx, code, 11, 4, 2.0, per_cw=True)
    y[2, 5, 0] = float("nan")
    y[4, 0, 1] = float("inf")
    y[7, 3, 0] = -float("inf")
    lx.ldpcx_sync_status()
    a = fused(lx, code, y, no, 4, lx.DEMAP_EXACT, 20.0, dec)
    st, flags = lx.ldpcx_sync_status()
    assert st != 0 and flags & 1  # LDPCX_FLAG_NONFINITE
    b = two_step(lx, code, y, no, 4, lx.DEMAP_EXACT, 20.0, dec)
    lx.ldpcx_sync_status()
    assert_same(a, b)


@pytest.mark.parametrize("name,B", [("bg1_z384", 12), ("bg2_z8", 37), ("bg1_z16_short300", 33)])
@pytest.mark.parametrize("prec", [0, 1, 2])
def test_fused_per_edge_minsum(lx, name, B, prec):
    """With the check-node state switched off, min-sum runs the per-edge kernels, which are built once per
    input kind: the symbol-input build equals the LLR-input build after demap_app."""
    code = build(lx, name)
    dec = dict(algo=0, msg_prec=prec, iters=10, early_stop=True, offset=0.5, clamp=20.0)
    m = 4 if code.n_tx % 4 == 0 else 2
    y, no = channel(lx, code, B, m, 2.5, per_cw=True)
    lx.ldpcx_tune_set(lx.TUNE_CN_STATE, 0)
    try:
        assert_same(fused(lx, code, y, no, m, lx.DEMAP_MAXLOG, 20.0, dec),
                    two_step(lx, code, y, no, m, lx.DEMAP_MAXLOG, 20.0, dec))
    finally:
        lx.ldpcx_tune_set(lx.TUNE_CN_STATE, 1)


@pytest.mark.parametrize("prec", [1, 2])
def test_fused_full_size_launch_equals_two_step(lx, prec):
    """The launch the bench step times: BG1-shaped Z = 384, 4096 codewords, 16-QAM max-log at Eb/N0 = 2 dB with
    one N0, layered min-sum for 20 iterations without early stop (FP16; 6-bit as in the 256-QAM sweep's
    variant), bits and iteration counts only. Equal bit for bit to demap_app followed by ldpc_bp_decode,
    whose full-size launch is compared with the oracle's FP32 replay in test_gpu_parity.py."""
    code = build(lx, "bg1_z384")
    B, m = 4096, 4
    dec = dict(algo=0, msg_prec=prec, iters=20, early_stop=False, offset=0.5, clamp=20.0)
    y, no = channel(lx, code, B, m, 2.0, per_cw=False)
    _, bits_f, its_f = lx.ldpc_bp_decode_qam(code, y, no, m, demap_method=lx.DEMAP_MAXLOG, demap_clamp=20.0, **dec)
    llr = lx.demap_app(y, no, m, method=lx.DEMAP_MAXLOG, clamp=20.0)
    _, bits_t, its_t = lx.ldpc_bp_decode(code, llr, **dec)
    assert torch.equal(bits_f, bits_t) and torch.equal(its_f, its_t)
    assert (its_f == 20).all()
