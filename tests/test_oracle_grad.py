"""Pins for the gradient oracle (weighted flooding sum-product, torch FP64 autograd).

* Its forward equals the C oracle's weighted flooding sum-product (FP64).
* Its gradients equal central finite differences (h = 1e-3, Richardson-combined
  with h/2 to cancel the h^2 term) of the C oracle's loss, to 1e-6 relative, on
  random coordinates of the channel LLRs and of the weights.
* All-ones weights: the loss equals the unweighted decoder's loss.
"""
import numpy as np
import pytest

from tests import inputs


@pytest.fixture(scope="module")
def case(orc):
    from oracle import grad
    code = orc.Code(2, 8)
    u = inputs.info_bits(5, 3, code.k)
    cw = code.encoder.encode(u)
    # BPSK channel at a moderate SNR: LLRs that stay away from the clamps
    L = inputs.gaussian_llrs(cw, 1.2, 6).astype(np.float64)
    iters = 5
    w = 0.7 + 0.6 * inputs.rng(7).random((iters, code.graph.n_cls))
    return code, cw, L, w, iters, grad


def c_oracle_loss(orc, grad, code, L, cw, w, iters):
    app, _, _ = orc.decode(code.graph, L, algo=orc.ALGO_SPA, schedule=orc.SCHED_FLOOD, iters=iters, weights=w)
    return grad.bce_numpy(app, cw), app


def test_forward_matches_c_oracle(orc, case):
    code, cw, L, w, iters, grad = case
    loss, gL, gw, app = grad.loss_and_grads(code.graph, L, cw, w, iters)
    ref_loss, ref_app = c_oracle_loss(orc, grad, code, L, cw, w, iters)
    assert np.allclose(app, ref_app, rtol=1e-10, atol=1e-10)
    assert loss == pytest.approx(ref_loss, rel=1e-12)


def richardson_fd(f, x0, h=1e-3):
    """Central differences at h and h/2 combined to cancel the h^2 term."""
    d1 = (f(x0 + h) - f(x0 - h)) / (2 * h)
    d2 = (f(x0 + h / 2) - f(x0 - h / 2)) / h
    return (4 * d2 - d1) / 3


def test_gradients_match_finite_differences(orc, case):
    code, cw, L, w, iters, grad = case
    loss, gL, gw, _ = grad.loss_and_grads(code.graph, L, cw, w, iters)
    rng = inputs.rng(11)
    checked = 0
    for _ in range(24):
        b, v = int(rng.integers(0, L.shape[0])), int(rng.integers(0, L.shape[1]))

        def f_L(x):
            Lx = L.copy()
            Lx[b, v] = x
            return c_oracle_loss(orc, grad, code, Lx, cw, w, iters)[0]

        assert richardson_fd(f_L, L[b, v]) == pytest.approx(gL[b, v], rel=1e-6, abs=1e-10)
        checked += abs(gL[b, v]) > 1e-6
    for _ in range(24):
        t, c = int(rng.integers(0, iters)), int(rng.integers(0, w.shape[1]))

        def f_w(x):
            wx = w.copy()
            wx[t, c] = x
            return c_oracle_loss(orc, grad, code, L, cw, wx, iters)[0]

        assert richardson_fd(f_w, w[t, c]) == pytest.approx(gw[t, c], rel=1e-6, abs=1e-10)
        checked += abs(gw[t, c]) > 1e-6
    assert checked > 20  # the gradients are not trivially zero


def test_unit_weights_equal_unweighted(orc, case):
    code, cw, L, w, iters, grad = case
    ones = np.ones_like(w)
    loss, _, _, app = grad.loss_and_grads(code.graph, L, cw, ones, iters)
    app0, _, _ = orc.decode(code.graph, L, algo=orc.ALGO_SPA, schedule=orc.SCHED_FLOOD, iters=iters)
    assert np.allclose(app, app0, rtol=1e-10, atol=1e-10)
