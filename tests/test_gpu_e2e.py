"""Trainable constellation (the paper's Listing 2) on the device: the
arbitrary-point mapper and demapper against the FP64 oracle, the BCE kernel,
the hand-written adjoint of the chain against torch FP64 autograd of the
oracle on the same codewords and noise, and a short training run."""
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


@pytest.mark.parametrize("m", [2, 4, 6, 8])
def test_gray_points_reproduce_sim_tx(lx, m):
    from paper_2203_11854_gb300 import e2e
    code = lx.qc_ldpc_build(1, 48, punct_cols=2)
    B, n0 = 7, torch.tensor([0.3], device="cuda")
    y, _ = lx.sim_tx(code, 5, 11, B, m, n0)
    cw = torch.empty((B, (code.n + 31) // 32), dtype=torch.int32, device="cuda")
    yp, _ = lx.sim_tx_points(code, 5, 11, B, m, e2e.qam_points(m), n0, cw_out=cw)
    assert torch.allclose(y, yp, rtol=1e-6, atol=1e-6)
    assert torch.equal(cw, lx.sim_codewords(code, 5, 11, B))


@pytest.mark.parametrize("m", [2, 4, 6, 8])
@pytest.mark.parametrize("method", [0, 1])
def test_demap_points_matches_oracle(lx, orc, m, method):
    rng = inputs.rng(60 + m)
    pts = rng.normal(size=(1 << m, 2)).astype(np.float32)
    y = (rng.normal(size=(4, 211, 2)) * 1.3).astype(np.float32)
    n0 = np.array([0.3, 0.6, 1.0, 2.0], dtype=np.float32)
    got = lx.demap_points(torch.from_numpy(y).cuda(), torch.from_numpy(n0).cuda(), m, torch.from_numpy(pts).cuda(),
                          method=method).cpu().numpy()
    ref = orc.demap_points(y.astype(np.float64), m, n0.astype(np.float64), pts.astype(np.float64), method=method)
    assert np.allclose(got, ref, rtol=2e-5, atol=2e-4), np.abs(got - ref).max()


def test_bce_and_gradient(lx):
    from oracle import e2e as oe
    rng = inputs.rng(4)
    B, N, off = 3, 999, 5
    words = rng.integers(0, 2 ** 32, size=(B, (off + N + 31) // 32), dtype=np.uint64).astype(np.uint32)
    bits = unpack(words.view(np.int32), off + N)[:, off:]
    L = (rng.normal(size=(B, N)) * 6.0).astype(np.float32)
    acc, g = lx.llr_bce(torch.from_numpy(L).cuda(), torch.from_numpy(words.view(np.int32)).cuda(), off, scale=0.5)
    Lt = torch.from_numpy(L.astype(np.float64)).requires_grad_(True)
    loss = oe.bce(Lt, torch.from_numpy(bits))
    loss.backward()
    assert float(acc.cpu()[0]) == pytest.approx(float(loss.detach()), rel=1e-6)
    assert np.allclose(g.cpu().numpy(), 0.5 * Lt.grad.numpy(), rtol=1e-5, atol=1e-7)


@pytest.mark.parametrize("m", [2, 4, 6])
def test_chain_gradient_matches_autograd_oracle(lx, m):
    from oracle import e2e as oe
    from paper_2203_11854_gb300 import e2e
    code = lx.qc_ldpc_build(2, 24)  # n_tx = 1248: whole symbols for m = 2, 4, 6
    B, ebn0 = 6, 1.0
    pts = e2e.normalise(e2e.qam_points(m) + 0.15 * torch.from_numpy(inputs.rng(m).normal(size=(1 << m, 2))).float()
                        .cuda())
    P = pts.clone().requires_grad_(True)
    r = code.k / code.n_tx
    n0 = torch.tensor([1.0 / (r * m * 10.0 ** (ebn0 / 10.0))], dtype=torch.float32, device="cuda")
    loss = e2e.Chain.apply(P, code, m, n0, 77, 3, B, 20.0)
    loss.backward()
    # the oracle on the same codewords and noise: labels from the codewords, noise = y - x
    cw = lx.sim_codewords(code, 77, 3, B).cpu().numpy()
    bits = unpack(cw, code.n)[:, code.p0:code.p0 + code.n_tx]
    S = code.n_tx // m
    lab = (bits.reshape(B, S, m) * (1 << (m - 1 - np.arange(m)))).sum(-1)
    y, _ = lx.sim_tx_points(code, 77, 3, B, m, pts, n0)
    noise = y.cpu().double() - pts.cpu().double()[torch.from_numpy(lab)]
    Po = pts.cpu().double().requires_grad_(True)
    lo = oe.chain_loss(Po, torch.from_numpy(lab), noise, n0.cpu().double().expand(B), m) / (B * code.n_tx)
    lo.backward()
    assert float(loss.detach()) == pytest.approx(float(lo.detach()), rel=1e-5)
    g, go = P.grad.cpu().double().numpy(), Po.grad.numpy()
    assert np.allclose(g, go, rtol=1e-3, atol=1e-3 * np.abs(go).max())


def test_training_lowers_held_out_loss(lx):
    from paper_2203_11854_gb300 import e2e
    code = lx.qc_ldpc_build(2, 64)
    pts, trace = e2e.train_constellation(code, 4, -1.0, steps=120, lr=5e-3, B=32)
    print("held-out BCE:", trace)
    assert trace[-1][1] < trace[0][1]
    assert torch.isfinite(pts).all()
    assert float((pts ** 2).sum(-1).mean()) == pytest.approx(1.0, rel=1e-5)
