"""Polar codes on the device against the oracle: construction (information
set), transmitter (data bits, CRC, encoder, BPSK, AWGN) and CRC-aided SCL:
decoded data bits and path metrics bit-exact against the oracle's FP32 replay
for lists of 1 (SC) to 32, with and without CRC, N from 8 to 1024."""
import numpy as np
import pytest

from tests import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

CRC8 = (0x107, 8)


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


@pytest.mark.parametrize("n,K,design", [(3, 4, 0.0), (6, 32, 1.0), (10, 512, 2.0), (8, 17, -1.5)])
def test_information_set(lx, orc, n, K, design):
    code = lx.polar_build(n, K, design)
    info, _ = orc.polar_info_set(n, K, design)
    assert np.array_equal(code.info, info)


@pytest.mark.parametrize("n,K,crc", [(6, 32, (0, 0)), (9, 200, CRC8)])
def test_transmitter_matches_oracle(lx, orc, n, K, crc):
    code = lx.polar_build(n, K, 1.0, *crc)
    B, seed, cw0 = 9, 21, 100
    n0 = torch.tensor([0.7], device="cuda")
    y, data = lx.polar_sim_tx(code, seed, cw0, B, n0)
    kd = code.k_data
    d = orc.source_bits(seed, cw0, B, kd)
    assert np.array_equal(unpack(data.cpu().numpy(), kd), d)
    info, _ = orc.polar_info_set(n, K, 1.0)
    u = np.zeros((B, 1 << n), dtype=np.uint8)
    for b in range(B):
        bits = d[b] if crc[1] == 0 else np.concatenate([d[b], orc.crc(d[b], *crc)])
        u[b, info] = bits
    x = 1.0 - 2.0 * orc.polar_encode(u)
    ref = orc.awgn(x, 1, 0.7, seed, cw0)
    assert np.allclose(y.cpu().numpy(), ref, rtol=1e-5, atol=2e-5)


@pytest.mark.parametrize("n,K,L,crc", [(3, 4, 1, (0, 0)), (3, 4, 16, (0, 0)), (6, 32, 1, (0, 0)),
                                       (6, 32, 4, CRC8), (8, 100, 8, CRC8), (8, 100, 32, CRC8),
                                       (10, 512, 8, CRC8), (10, 300, 2, (0, 0))])
def test_scl_bit_exact_vs_fp32_replay(lx, orc, n, K, L, crc):
    code = lx.polar_build(n, K, 1.0, *crc)
    info, frozen = orc.polar_info_set(n, K, 1.0)
    N, B = 1 << n, 12
    rng = inputs.rng(100 * n + L)
    # noisy codewords at a moderate SNR: lists disagree with SC often enough to exercise the selection
    d = (rng.random((B, code.k_data)) < 0.5).astype(np.uint8)
    u = np.zeros((B, N), dtype=np.uint8)
    for b in range(B):
        u[b, info] = d[b] if crc[1] == 0 else np.concatenate([d[b], orc.crc(d[b], *crc)])
    x = orc.polar_encode(u)
    llr = (2.0 * (1.0 - 2.0 * x) + 1.6 * rng.normal(size=(B, N))).astype(np.float32)
    llr[0, :3] = 0.0  # zero LLRs: ties in f, decisions and list metrics
    bits, pm = lx.polar_scl_decode(code, torch.from_numpy(llr).cuda(), L)
    uh, opm = orc.polar_scl(llr.astype(np.float64), frozen, info, L, crc[0], crc[1], prec=1)
    assert np.array_equal(unpack(bits.cpu().numpy(), code.k_data), uh[:, info[:code.k_data]])
    assert np.array_equal(pm.cpu().numpy(), opm.astype(np.float32))


def test_scl_corrects_more_than_sc(lx):
    code = lx.polar_build(8, 128, 1.0, *CRC8)
    B = 512
    n0 = torch.tensor([10 ** (-2.0 / 10) / (code.k_data / code.N)], device="cuda")  # Eb/N0 = 2 dB
    y, data = lx.polar_sim_tx(code, 5, 0, B, n0)
    llr = (4.0 / n0) * y
    errs = {}
    for L in (1, 8):
        bits, _ = lx.polar_scl_decode(code, llr.contiguous(), L)
        errs[L] = int((bits != data).any(dim=1).sum())
    assert errs[8] < errs[1]
