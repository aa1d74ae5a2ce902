"""End-to-end learning of the constellation (the paper's Listing 2) through
mapper, AWGN and APP demapper, with hand-written adjoints in the library.

The chain for codewords of ``code``: bits c -> symbol x = p[label] ->
y = x + sqrt(N0/2) g -> LLRs L = demap(y; p) -> loss = sum ln(1 + e^{-(1-2c) L})
(binary cross-entropy with logits -L). ``Chain.apply(points, ...)`` is a
torch.autograd.Function whose forward and backward run the library's kernels:
``sim_tx_points``, ``demap_points`` and ``llr_bce`` forward;
``demap_points_backward`` (through the demapper to y and to the points) and
``map_points_backward`` (from dLoss/dx = dLoss/dy to the points) backward.
The points are normalised to unit average energy (the 2^m-entry parameter,
on torch) before they enter the chain.
"""
from __future__ import annotations

import math

import torch

from . import DEMAP_EXACT, demap_points, demap_points_backward, llr_bce, map_points_backward, sim_tx_points


def qam_points(m: int, device="cuda") -> torch.Tensor:
    """Gray QAM as points [2^m, 2] by label (the constellation of sim_tx)."""
    h = m // 2
    P = 1 << m
    out = torch.empty((P, 2), dtype=torch.float64)
    scale = 1.0 / math.sqrt(2.0 * ((1 << (2 * h)) - 1) / 3.0)
    for l in range(P):
        bits = [(l >> (m - 1 - j)) & 1 for j in range(m)]

        def level(a):
            inner = 1 - 2 * a[h - 1]
            for i in range(h - 2, -1, -1):
                inner = (1 - 2 * a[i]) * ((1 << (h - 1 - i)) - inner)
            return inner

        out[l, 0] = level(bits[0::2]) * scale
        out[l, 1] = level(bits[1::2]) * scale
    return out.float().to(device)


def normalise(points: torch.Tensor) -> torch.Tensor:
    return points / torch.sqrt((points ** 2).sum(-1).mean())


class Chain(torch.autograd.Function):
    """loss(points) of one batch: mapper, AWGN, demapper and BCE (mean over the B n_tx bits)."""

    @staticmethod
    def forward(ctx, points, code, m, n0, seed, cw0, B, clamp):
        pts = points.detach().contiguous()
        cw = torch.empty((B, (code.n + 31) // 32), dtype=torch.int32, device=pts.device)
        y, _ = sim_tx_points(code, seed, cw0, B, m, pts, n0, cw_out=cw)
        llr = demap_points(y, n0, m, pts, method=DEMAP_EXACT, clamp=clamp)
        n = B * code.n_tx
        acc, gllr = llr_bce(llr, cw, code.p0, scale=1.0 / n)
        ctx.save_for_backward(pts, y, gllr, cw, n0)
        ctx.code, ctx.m, ctx.clamp = code, m, clamp
        return (acc / n).to(points.dtype).reshape(())

    @staticmethod
    def backward(ctx, grad_loss):
        pts, y, gllr, cw, n0 = ctx.saved_tensors
        gp = torch.zeros_like(pts)
        gy = demap_points_backward(y, n0, ctx.m, pts, gllr, gp, clamp=ctx.clamp)  # through the demapper
        map_points_backward(ctx.code, cw, ctx.m, gy, gp)  # through y = x + noise and the mapper
        return gp * grad_loss.to(gp.dtype), None, None, None, None, None, None, None


def chain_loss(points, code, m: int, ebn0_db: float, *, B: int = 64, seed: int = 0x1DBC, cw0: int = 0,
               clamp: float = 20.0):
    r = code.k / code.n_tx
    n0 = torch.tensor([1.0 / (r * m * 10.0 ** (ebn0_db / 10.0))], dtype=torch.float32, device=points.device)
    return Chain.apply(normalise(points), code, m, n0, seed, cw0, B, clamp)


def train_constellation(code, m: int, ebn0_db: float, *, steps: int = 200, lr: float = 1e-2, B: int = 64,
                        seed: int = 0x1DBC, init=None, eval_batches: int = 4):
    """Adam on the points from the Gray QAM (or init); fresh codewords and noise every step. Returns
    (points, [(step, held-out loss)]) with the held-out loss on fixed codewords disjoint from training."""
    points = (qam_points(m) if init is None else init.clone()).requires_grad_(True)
    opt = torch.optim.Adam([points], lr=lr)
    held = 1 << 40  # codeword counter range of the held-out batches

    def evaluate():
        with torch.no_grad():
            return sum(float(chain_loss(points, code, m, ebn0_db, B=B, seed=seed, cw0=held + i * B))
                       for i in range(eval_batches)) / eval_batches

    trace = [(0, evaluate())]
    for step in range(steps):
        opt.zero_grad()
        loss = chain_loss(points, code, m, ebn0_db, B=B, seed=seed, cw0=step * B)
        loss.backward()
        opt.step()
        if (step + 1) % max(1, steps // 4) == 0:
            trace.append((step + 1, evaluate()))
    return normalise(points.detach()), trace
