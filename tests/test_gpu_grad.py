"""GPU adjoint of weighted flooding sum-product BP (ldpc_bp_backward) against the oracles.

* ldpc_bp_decode_ckpt gives the same output LLRs as ldpc_bp_decode, bit for bit.
* Gradients of the BCE loss with respect to the channel LLRs and the weights
  match the torch-FP64 autograd oracle (1e-3 relative, measured against the
  largest gradient component) and central differences (h = 1e-3) of the FP64
  C oracle on sampled coordinates (1e-3 relative).
* 200 Adam steps on the weights lower the held-out loss and bit error rate
  against unit weights (unweighted BP).
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


def make(orc, bg, Z, B, mean, iters, seed):
    code = orc.Code(bg, Z)
    u = inputs.info_bits(seed, B, code.k)
    cw = code.encoder.encode(u)
    L = inputs.gaussian_llrs(cw, mean, seed + 1)
    w = (0.8 + 0.4 * inputs.rng(seed + 2).random((iters, code.graph.n_cls))).astype(np.float32)
    return code, cw, L, w


def gpu_grads(lx, gcode, L, cw, w, iters):
    from paper_2203_11854_gb300.autograd import LdpcBP
    Lt = torch.from_numpy(L).cuda().requires_grad_(True)
    wt = torch.from_numpy(w).cuda().requires_grad_(True)
    out = LdpcBP.apply(Lt, wt, gcode, iters, 20.0)
    loss = torch.nn.functional.binary_cross_entropy_with_logits(-out, torch.from_numpy(cw).cuda().float())
    loss.backward()
    return float(loss.detach()), Lt.grad.cpu().numpy(), wt.grad.cpu().numpy(), out.detach().cpu().numpy()


def test_ckpt_forward_equals_plain_decode(lx, orc):
    code, cw, L, w = make(orc, 2, 64, 10, 1.5, 8, 3)
    g = lx.qc_ldpc_build(2, 64)
    Lt, wt = torch.from_numpy(L).cuda(), torch.from_numpy(w).cuda()
    out, ckpt = lx.ldpc_bp_decode_ckpt(g, Lt, iters=8, weights=wt)
    ref, _, _ = lx.ldpc_bp_decode(g, Lt, algo=lx.FLOOD_SPA, iters=8, weights=wt, llr_out=True)
    assert torch.equal(out, ref)
    assert ckpt.numel() == lx.ldpc_bp_ckpt_bytes(g, 10, iters=8)


# Z <= 128 runs four threads per check node in the adjoint, 129..256 two, larger Z one; BG1 rows reach degree 19
@pytest.mark.parametrize("bg,Z,B,iters", [(2, 64, 4, 10), (2, 8, 12, 6), (1, 16, 3, 5), (2, 160, 2, 4),
                                          (2, 288, 1, 3)])
def test_gradients_match_autograd_oracle(lx, orc, bg, Z, B, iters):
    from oracle import grad
    code, cw, L, w = make(orc, bg, Z, B, 1.0, iters, 17)
    loss, gL, gw, out = gpu_grads(lx, lx.qc_ldpc_build(bg, Z), L, cw, w, iters)
    rl, rgL, rgw, rapp = grad.loss_and_grads(code.graph, L.astype(np.float64), cw, w.astype(np.float64), iters)
    assert loss == pytest.approx(rl, rel=1e-4)
    for g, r in ((gL, rgL), (gw, rgw)):
        scale = np.abs(r).max()
        assert scale > 0
        err = np.abs(g - r)
        assert err.max() <= 1e-3 * scale, f"max error {err.max():.3g} vs scale {scale:.3g}"
        big = np.abs(r) > 0.05 * scale  # per-coordinate relative check on the significant components
        assert np.all(err[big] <= 1e-3 * np.abs(r[big]) + 1e-5 * scale)


def test_gradients_match_finite_differences(lx, orc):
    from oracle import grad
    iters = 10
    code, cw, L, w = make(orc, 2, 64, 2, 1.0, iters, 23)
    _, gL, gw, _ = gpu_grads(lx, lx.qc_ldpc_build(2, 64), L, cw, w, iters)
    L64, w64 = L.astype(np.float64), w.astype(np.float64)

    def loss_of(Lx, wx):
        app, _, _ = orc.decode(code.graph, Lx, algo=orc.ALGO_SPA, schedule=orc.SCHED_FLOOD, iters=iters, weights=wx)
        return grad.bce_numpy(app, cw)

    rng = inputs.rng(29)
    h = 1e-3
    scale_L, scale_w = np.abs(gL).max(), np.abs(gw).max()
    coords = 0
    while coords < 32:
        b, v = int(rng.integers(0, L.shape[0])), int(rng.integers(0, L.shape[1]))
        if abs(gL[b, v]) < 0.05 * scale_L:
            continue
        Lp, Lm = L64.copy(), L64.copy()
        Lp[b, v] += h
        Lm[b, v] -= h
        fd = (loss_of(Lp, w64) - loss_of(Lm, w64)) / (2 * h)
        assert gL[b, v] == pytest.approx(fd, rel=1e-3, abs=1e-4 * scale_L)
        coords += 1
    coords = 0
    while coords < 32:
        t, c = int(rng.integers(0, iters)), int(rng.integers(0, w.shape[1]))
        if abs(gw[t, c]) < 0.05 * scale_w:
            continue
        wp, wm = w64.copy(), w64.copy()
        wp[t, c] += h
        wm[t, c] -= h
        fd = (loss_of(L64, wp) - loss_of(L64, wm)) / (2 * h)
        assert gw[t, c] == pytest.approx(fd, rel=1e-3, abs=1e-4 * scale_w)
        coords += 1


def test_training_lowers_heldout_loss_and_ber(lx):
    """200 Adam steps (lr 1e-3) on BG2-shaped Z=64, 10 iterations, BPSK at Eb/N0 in [1, 3] dB:
    the trained weights beat unit weights on a fixed held-out batch at 1.5 dB."""
    from paper_2203_11854_gb300.train import train_weighted_bp
    h = train_weighted_bp(bg=2, Z=64, batch=1024, iters=10, steps=200, lr=1e-3, ebn0_range=(1.0, 3.0), seed=5,
                          eval_ebn0=(1.5, 1.5), eval_batch=8192)
    print("held-out loss unit %.3g trained %.3g; BER unit %.3g trained %.3g"
          % (h["loss_unit"], h["loss_trained"], h["ber_unit"], h["ber_trained"]))
    assert h["loss_trained"] < h["loss_unit"]
    assert h["ber_trained"] < h["ber_unit"]
