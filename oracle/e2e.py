"""Gradient oracle of the trainable-constellation chain (TEST INFRASTRUCTURE
ONLY: imported by tests/ alone).

A plain torch float64 restatement, on the CPU with autograd, of the APP
demapper over arbitrary points (the C oracle's orc_demap_points) and of the
binary cross-entropy on LLRs (logits = -L for L = ln P0/P1, Listing 2):

  d_l(y)  = -|y - p_l|^2 / N0
  L_i     = logsumexp_{l: b_i(l)=0} d_l - logsumexp_{l: b_i(l)=1} d_l, clamped
  loss    = sum ln(1 + exp(-(1 - 2c) L))

with the transmitted symbol x = p_{label} and y = x + noise, so the loss
depends on the points through the demapper and through x.
"""
from __future__ import annotations

import torch


def labels(m: int) -> torch.Tensor:
    l = torch.arange(1 << m)
    return ((l[:, None] >> (m - 1 - torch.arange(m))[None, :]) & 1).to(torch.bool)


def demap(y: torch.Tensor, points: torch.Tensor, n0: torch.Tensor, m: int, clamp: float = 20.0) -> torch.Tensor:
    """y [B, S, 2], points [2^m, 2], n0 [B] -> LLRs [B, S*m] (exact log-sum-exp)."""
    d = -((y[:, :, None, :] - points[None, None, :, :]) ** 2).sum(-1) / n0[:, None, None]  # [B, S, P]
    lab = labels(m)  # [P, m]
    neg = torch.tensor(float("-inf"), dtype=d.dtype)
    d0 = torch.where(~lab.T[None, None], d[:, :, None, :], neg)  # [B, S, m, P]
    d1 = torch.where(lab.T[None, None], d[:, :, None, :], neg)
    L = torch.logsumexp(d0, -1) - torch.logsumexp(d1, -1)
    return torch.clamp(L, -clamp, clamp).reshape(y.shape[0], -1)


def bce(llr: torch.Tensor, bits: torch.Tensor) -> torch.Tensor:
    s = 1.0 - 2.0 * bits.to(llr.dtype)
    return torch.nn.functional.softplus(-s * llr).sum()


def chain_loss(points: torch.Tensor, sym_labels: torch.Tensor, noise: torch.Tensor, n0: torch.Tensor, m: int,
               clamp: float = 20.0) -> torch.Tensor:
    """Loss of the chain for symbol labels [B, S] (ints) and noise [B, S, 2]: x = points[label], y = x + noise."""
    x = points[sym_labels]  # [B, S, 2]
    y = x + noise
    llr = demap(y, points, n0, m, clamp)
    bits = labels(m)[sym_labels].reshape(sym_labels.shape[0], -1)
    return bce(llr, bits)
