"""Rate matching on the device against the oracle: transmitted bits bit-exact
for repetition, puncturing, every qm and start positions across the buffer;
soft recovery exact on dyadic LLRs (whose sums are exact in binary32) and
within binary32 rounding otherwise; and a whole round trip -- codewords, rate
matching, BPSK over AWGN, recovery, decoding with a code of n_tx = ncb --
recovering the transmitted codewords at a high SNR."""
import numpy as np
import pytest

from oracle import ratematch as rm
from tests import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lx():
    import paper_2203_11854_gb300 as lx
    assert torch.cuda.is_available()
    lx.load_library()
    return lx


def unpack(words: np.ndarray, k: int) -> np.ndarray:
    w = words.view(np.uint32)
    bits = ((w[:, :, None] >> np.arange(32, dtype=np.uint32)) & 1).astype(np.uint8)
    return bits.reshape(w.shape[0], -1)[:, :k]


CASES = [  # (bg, Z, punct, k0 fraction, ncb fraction of n - p0, E as a multiple of ncb, qm)
    (2, 16, 0, 0.0, 1.0, 1.0, 1), (2, 16, 0, 0.3, 1.0, 2.6, 2), (1, 8, 2, 0.55, 0.8, 0.5, 4),
    (1, 24, 2, 0.99, 1.0, 1.3, 6), (2, 32, 2, 0.1, 0.6, 3.1, 8),
]


def params(code, frac_k0, frac_ncb, mult_e, qm):
    ncb = max(qm, int((code.n - code.p0) * frac_ncb))
    k0 = min(ncb - 1, int(frac_k0 * ncb))
    E = max(qm, int(mult_e * ncb) // qm * qm)
    return k0, ncb, E


@pytest.mark.parametrize("case", CASES)
def test_rate_match_bit_exact(lx, case):
    bg, Z, punct, fk, fn, fe, qm = case
    code = lx.qc_ldpc_build(bg, Z, punct_cols=punct)
    k0, ncb, E = params(code, fk, fn, fe, qm)
    B = 37
    cw = lx.sim_codewords(code, 3, 11, B)
    f = lx.rate_match(code, cw, k0, ncb, E, qm)
    ref = rm.rate_match(unpack(cw.cpu().numpy(), code.n), code.p0, ncb, k0, E, qm)
    assert np.array_equal(unpack(f.cpu().numpy(), E), ref)


@pytest.mark.parametrize("case", CASES)
def test_rate_recover(lx, case):
    bg, Z, punct, fk, fn, fe, qm = case
    code = lx.qc_ldpc_build(bg, Z, punct_cols=punct)
    k0, ncb, E = params(code, fk, fn, fe, qm)
    rng = inputs.rng(Z + qm)
    dy = (rng.integers(-64, 65, size=(9, E)) / 8.0).astype(np.float32)  # dyadic: exact sums
    v = lx.rate_recover(code, torch.from_numpy(dy).cuda(), k0, ncb, qm)
    assert np.array_equal(v.cpu().numpy().astype(np.float64), rm.rate_recover(dy, ncb, k0, qm))
    x = rng.normal(size=(9, E)).astype(np.float32)
    v = lx.rate_recover(code, torch.from_numpy(x).cuda(), k0, ncb, qm).cpu().numpy()
    r = rm.rate_recover(x, ncb, k0, qm)
    reps = -(-E // ncb)
    assert np.all(np.abs(v - r) <= reps * 6e-8 * np.maximum(np.abs(r), 1.0) * 4)


def test_round_trip_decodes(lx):
    code = lx.qc_ldpc_build(1, 64, punct_cols=2)
    # the buffer read from its start (systematic bits first), the tail of the parity punctured: rate 1/2
    k0, ncb, E, qm = 0, code.n - code.p0, 2 * (code.n - code.p0) // 3 // 4 * 4, 4
    rx = lx.qc_ldpc_build(1, 64, punct_cols=2, n_tx=ncb)
    B = 64
    cw = lx.sim_codewords(code, 9, 0, B)
    f = lx.rate_match(code, cw, k0, ncb, E, qm)
    bits = torch.from_numpy(unpack(f.cpu().numpy(), E).astype(np.float32)).cuda()
    g = torch.Generator(device="cuda")
    g.manual_seed(4)
    sigma = 0.5
    y = (1.0 - 2.0 * bits) + sigma * torch.randn(bits.shape, device="cuda", generator=g)
    llr = (2.0 / sigma ** 2) * y
    soft = lx.rate_recover(code, llr.contiguous(), k0, ncb, qm)
    _, dec, _ = lx.ldpc_bp_decode(rx, soft, iters=20, msg_prec=lx.MSG_F16)
    sent = unpack(cw.cpu().numpy(), code.k)
    assert np.array_equal(unpack(dec.cpu().numpy(), code.k), sent)


def test_rejects_bad_parameters(lx):
    code = lx.qc_ldpc_build(2, 8)
    cw = torch.zeros((2, (code.n + 31) // 32), dtype=torch.int32, device="cuda")
    for k0, ncb, E, qm in [(0, 0, 8, 1), (5, 5, 8, 1), (0, code.n + 1, 8, 1), (0, 40, 9, 2), (0, 40, 8, 3)]:
        with pytest.raises(lx.LdpcxError):
            lx.rate_match(code, cw, k0, ncb, E, qm)
