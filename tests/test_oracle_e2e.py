"""Oracle pins for the trainable-constellation chain: the arbitrary-point
demapper against the Gray QAM demapper and against its torch restatement,
phase invariance, and the torch autograd gradients against central finite
differences of the C oracle. CPU only."""
import math

import numpy as np
import pytest

from tests import inputs

torch = pytest.importorskip("torch")


@pytest.mark.parametrize("m", [2, 4, 6, 8])
@pytest.mark.parametrize("method", [0, 1])
def test_qam_points_equal_gray_demapper(orc, m, method):
    y = inputs.rng(m).normal(size=(3, 30, 2))
    a = orc.demap_points(y, m, 0.6, orc.qam_points(m), method=method)
    b = orc.demap(y, m, 0.6, method=method)
    assert np.allclose(a, b, rtol=1e-11, atol=1e-11)


def test_phase_rotation_invariance(orc):
    rng = inputs.rng(11)
    m = 4
    pts = rng.normal(size=(1 << m, 2))
    y = rng.normal(size=(2, 25, 2))
    th = 0.7
    R = np.array([[math.cos(th), -math.sin(th)], [math.sin(th), math.cos(th)]])
    a = orc.demap_points(y, m, 0.9, pts)
    b = orc.demap_points(y @ R.T, m, 0.9, pts @ R.T)
    assert np.allclose(a, b, rtol=1e-10, atol=1e-10)


@pytest.mark.parametrize("m", [2, 4, 6])
def test_torch_restatement_equals_c(orc, m):
    from oracle import e2e
    rng = inputs.rng(20 + m)
    pts = rng.normal(size=(1 << m, 2))
    y = rng.normal(size=(3, 17, 2))
    n0 = np.array([0.4, 0.9, 1.7])
    a = e2e.demap(torch.from_numpy(y), torch.from_numpy(pts), torch.from_numpy(n0), m).numpy()
    b = orc.demap_points(y, m, n0, pts)
    assert np.allclose(a, b, rtol=1e-11, atol=1e-11)


def test_autograd_matches_finite_differences(orc):
    from oracle import e2e
    rng = inputs.rng(7)
    m, B, S = 4, 2, 9
    pts = rng.normal(size=(1 << m, 2))
    lab = rng.integers(0, 1 << m, size=(B, S))
    noise = rng.normal(size=(B, S, 2)) * 0.5
    n0 = np.array([0.5, 0.8])
    bits = ((lab[..., None] >> (m - 1 - np.arange(m))) & 1).reshape(B, -1)

    def loss_c(p):  # the C oracle end to end
        y = p[lab] + noise
        L = orc.demap_points(y, m, n0, p)
        return float(np.logaddexp(0.0, -(1.0 - 2.0 * bits) * L).sum())

    P = torch.from_numpy(pts).requires_grad_(True)
    loss = e2e.chain_loss(P, torch.from_numpy(lab), torch.from_numpy(noise), torch.from_numpy(n0), m)
    loss.backward()
    assert float(loss.detach()) == pytest.approx(loss_c(pts), rel=1e-12)
    g = P.grad.numpy()
    h = 1e-6
    for idx in [(0, 0), (3, 1), (7, 0), (12, 1), (15, 0)]:
        e = np.zeros_like(pts)
        e[idx] = h
        fd = (loss_c(pts + e) - loss_c(pts - e)) / (2 * h)
        assert g[idx] == pytest.approx(fd, rel=1e-6, abs=1e-8)
