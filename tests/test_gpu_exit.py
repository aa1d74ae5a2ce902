"""GPU parity and behaviour of the demapper with prior, the a-priori LLR
source, the mutual-information estimate, extrinsic LLRs and the transmitted
codewords, against the FP64 oracle; EXIT curves and iterative demapping and
decoding (BICM-ID) on a small code."""
import numpy as np
import pytest

from tests import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lx():
    import paper_2203_11854_gb300 as lx
    assert torch.cuda.is_available()
    lx.load_library()
    return lx


def unpack(words: np.ndarray, n: int) -> np.ndarray:
    w = words.view(np.uint32)
    bits = ((w[:, :, None] >> np.arange(32, dtype=np.uint32)) & 1).astype(np.uint8)
    return bits.reshape(w.shape[0], -1)[:, :n]


@pytest.mark.parametrize("m", [1, 2, 4, 6, 8])
@pytest.mark.parametrize("method", [0, 1])
@pytest.mark.parametrize("mode", [0, 1])
def test_demap_prior_matches_oracle(lx, orc, m, method, mode):
    rng = inputs.rng(40 + m)
    B, S = 5, 301
    y = (rng.normal(size=(B, S) if m == 1 else (B, S, 2)) * 1.1).astype(np.float32)
    la = (rng.normal(size=(B, S * m)) * 3.0).astype(np.float32)
    n0 = np.linspace(0.2, 1.5, B).astype(np.float32)
    got = lx.demap_app_prior(torch.from_numpy(y).cuda(), torch.from_numpy(n0).cuda(), m,
                             torch.from_numpy(la).cuda(), method=method, out_mode=mode).cpu().numpy()
    ref = orc.demap_prior(y.astype(np.float64), m, n0.astype(np.float64), la.astype(np.float64), method=method,
                          mode=mode)
    assert np.allclose(got, ref, rtol=2e-5, atol=2e-4), np.abs(got - ref).max()
    # no prior: the plain demapper
    plain = lx.demap_app(torch.from_numpy(y).cuda(), torch.from_numpy(n0).cuda(), m, method=method).cpu().numpy()
    none = lx.demap_app_prior(torch.from_numpy(y).cuda(), torch.from_numpy(n0).cuda(), m, None, method=method,
                              out_mode=mode).cpu().numpy()
    assert np.array_equal(plain, none) or np.allclose(plain, none, rtol=1e-6, atol=1e-6)


@pytest.mark.parametrize("bg,Z,punct", [(2, 8, 0), (1, 32, 2), (2, 64, 0)])
def test_codewords_match_oracle_encoder(lx, orc, bg, Z, punct):
    code = lx.qc_ldpc_build(bg, Z, punct_cols=punct)
    ocode = orc.Code(bg, Z, punct_cols=punct)
    B = 37
    n0 = torch.tensor([0.5], device="cuda")
    _, info = lx.sim_tx(code, 99, 5, B, 2, n0)
    cw = lx.sim_codewords(code, 99, 5, B).cpu().numpy()
    u = unpack(info.cpu().numpy(), ocode.k)
    ref = ocode.encoder.encode(u)
    assert np.array_equal(unpack(cw, ocode.n), ref)


def test_apriori_and_mutual_info_match_oracle(lx, orc):
    from oracle import exit as oexit
    B, N, off = 6, 5000, 13
    rng = inputs.rng(3)
    words = rng.integers(0, 2 ** 32, size=(B, (off + N + 31) // 32), dtype=np.uint64).astype(np.uint32)
    bits = torch.from_numpy(words.view(np.int32)).cuda()
    ref_bits = unpack(words.view(np.int32), off + N)[:, off:]
    for sigma in (0.0, 0.7, 2.5, 6.0):
        L = lx.llr_apriori(bits, off, N, sigma, seed=1234, cw0=77).cpu().numpy()
        ref = orc.apriori(ref_bits, sigma, seed=1234, cw0=77)
        assert np.allclose(L, ref, rtol=1e-5, atol=1e-5 * max(sigma, 1.0))
        got = lx.llr_mutual_info(torch.from_numpy(L).cuda(), bits, off)
        assert got == pytest.approx(oexit.mutual_info(L.astype(np.float64), ref_bits), abs=1e-6)


def test_extrinsic_is_output_minus_input(lx, orc):
    code = lx.qc_ldpc_build(1, 32, punct_cols=2)
    B = 9
    llr = (inputs.rng(5).normal(size=(B, code.n_tx)) * 3.0 + 1.0).astype(np.float32)
    L = torch.from_numpy(llr).cuda()
    app, _, _ = lx.ldpc_bp_decode(code, L, iters=5, llr_out=True)
    ext = lx.ldpc_extrinsic(code, app, L, clamp=1e4).cpu().numpy()
    ref = app.cpu().numpy()[:, code.p0:code.p0 + code.n_tx] - llr
    assert np.array_equal(ext, ref)
    # inputs beyond the clamp: the decoder saw them clamped, and so does the subtraction
    big = L * 30.0
    app2, _, _ = lx.ldpc_bp_decode(code, big, iters=5, llr_out=True)
    ext2 = lx.ldpc_extrinsic(code, app2, big, clamp=20.0).cpu().numpy()
    ref2 = np.clip(app2.cpu().numpy()[:, code.p0:code.p0 + code.n_tx] - np.clip(llr * 30.0, -20, 20), -20, 20)
    assert np.array_equal(ext2, ref2)


def test_library_J_matches_oracle():
    from oracle import exit as oexit
    from paper_2203_11854_gb300 import exit as lexit
    for s in (0.05, 0.3, 1.0, 2.0, 3.5, 6.0, 10.0):
        assert lexit.J(s) == pytest.approx(oexit.J(s), abs=1e-7)
        assert lexit.J(lexit.J_inv(lexit.J(s))) == pytest.approx(lexit.J(s), abs=1e-9)


def test_exit_curves_and_bicm_id(lx):
    from paper_2203_11854_gb300 import exit as lexit
    code = lx.qc_ldpc_build(2, 64)
    ia = [0.0, 0.2, 0.4, 0.6, 0.8, 0.95, 1.0]
    dec = lexit.decoder_curve(code, ia, B=128, iters=10)
    ie = [e for _, e in dec]
    # more a-priori information never gives less extrinsic information, and an informative input gives
    # more out than it had in once the decoder converges
    assert all(b >= a - 0.01 for a, b in zip(ie, ie[1:]))
    assert ie[-1] > 0.99 and ie[0] < 0.05
    dem = lexit.demapper_curve(code, 4, 3.0, ia, B=128)
    de = [e for _, e in dem]
    # Gray 16-QAM: the extrinsic information rises with the prior (the bits of one dimension share it)
    assert all(b >= a - 0.005 for a, b in zip(de, de[1:])) and de[-1] > de[0]
    # iterative demapping and decoding: the decoder's extrinsic information grows over outer iterations
    tr = lexit.bicm_id(code, 4, 2.0, outer=3, iters=8, B=128)
    assert tr[-1]["i_dec"] >= tr[0]["i_dec"] - 1e-3
    assert tr[-1]["ber"] <= tr[0]["ber"] + 1e-3
