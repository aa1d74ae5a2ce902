"""Training per-iteration per-block weights of flooding sum-product BP ("weighted
BP") with the hand-written adjoint -- end-to-end learning as in the paper's
Listing 2 (binary cross-entropy from logits, gradients through the receiver).

Each step draws a fresh batch on the device: Philox source, encoder and BPSK
mapper (sim_tx), AWGN with a per-codeword Eb/N0 uniform in `ebn0_range`, the
APP demapper (demap_app, L = 4y/N0), then LdpcBP with the current weights, the
BCE loss against the transmitted codeword bits (logits = -LLR) and Adam.
The codeword bits come from a noiseless transmission of the same codewords
(N0 = 0 gives y = 1 - 2c).
"""
from __future__ import annotations

import numpy as np
import torch

from . import (DEMAP_EXACT, FLOOD_SPA, demap_app, ldpc_bp_decode, qc_ldpc_build, sim_count, sim_tx)
from .autograd import LdpcBP


def _batch(code, seed, cw0, batch, ebn0, dev):
    r = code.k / code.n_tx
    n0 = (1.0 / (r * 10 ** (ebn0 / 10))).float().to(dev)
    y, info = sim_tx(code, seed, cw0, batch, 1, n0)
    y0, _ = sim_tx(code, seed, cw0, batch, 1, torch.zeros(1, dtype=torch.float32, device=dev))
    cw = (y0 < 0).float()
    llr = demap_app(y, n0, 1, method=DEMAP_EXACT)
    return llr, cw, info


def bit_error_rate(code, weights, iters, batch, ebn0, seed, cw0, dev="cuda"):
    """BER of weighted flooding sum-product on a fresh batch at fixed Eb/N0."""
    e = torch.full((batch,), float(ebn0), dtype=torch.float64)
    llr, _, info = _batch(code, seed, cw0, batch, e, dev)
    _, bits, its = ldpc_bp_decode(code, llr, algo=FLOOD_SPA, iters=iters, weights=weights)
    counts = torch.zeros(5, dtype=torch.int64, device=dev)
    sim_count(info, bits, its, code.k, counts)
    c = counts.cpu().tolist()
    return c[1] / c[0]


def eval_loss(code, weights, iters, batch, ebn0_range, seed, cw0, dev="cuda"):
    """BCE loss of the weighted decoder on a fixed batch (no gradient)."""
    gen = np.random.default_rng(seed)
    ebn0 = torch.from_numpy(gen.uniform(*ebn0_range, size=batch))
    llr, cw, _ = _batch(code, seed, cw0, batch, ebn0, dev)
    with torch.no_grad():
        out, _, _ = ldpc_bp_decode(code, llr, algo=FLOOD_SPA, iters=iters, weights=weights, llr_out=True,
                                   bits_out=False, iters_out=False)
        p0 = code.p0
        return float(torch.nn.functional.binary_cross_entropy_with_logits(-out[:, p0:p0 + code.n_tx], cw))


def train_weighted_bp(bg=2, Z=64, batch=2048, iters=10, steps=200, lr=1e-3, ebn0_range=(1.0, 3.0), seed=5,
                      dev="cuda", eval_ebn0=None, eval_batch=4096):
    code = qc_ldpc_build(bg, Z)
    w = torch.ones((iters, code.nnz), dtype=torch.float32, device=dev, requires_grad=True)
    opt = torch.optim.Adam([w], lr=lr)
    gen = np.random.default_rng(seed)
    hist = {"loss": []}
    cw0 = 0
    for _ in range(steps):
        ebn0 = torch.from_numpy(gen.uniform(*ebn0_range, size=batch))
        llr, cw, _ = _batch(code, seed, cw0, batch, ebn0, dev)
        cw0 += batch
        out = LdpcBP.apply(llr, w, code, iters, 20.0)
        p0 = code.p0
        loss = torch.nn.functional.binary_cross_entropy_with_logits(-out[:, p0:p0 + code.n_tx], cw)
        opt.zero_grad()
        loss.backward()
        opt.step()
        hist["loss"].append(float(loss.detach()))
    hist["weights"] = w.detach()
    if eval_ebn0 is not None:
        ones = torch.ones_like(w.detach())
        lo, hi = eval_ebn0 if isinstance(eval_ebn0, tuple) else (eval_ebn0, eval_ebn0)
        hist["loss_unit"] = eval_loss(code, ones, iters, eval_batch, (lo, hi), seed + 7, 1 << 41, dev)
        hist["loss_trained"] = eval_loss(code, w.detach(), iters, eval_batch, (lo, hi), seed + 7, 1 << 41, dev)
        eval_ebn0 = (lo + hi) / 2
        ones = torch.ones_like(w.detach())
        hist["ber_trained"] = bit_error_rate(code, w.detach(), iters, eval_batch, eval_ebn0, seed + 1, 1 << 40, dev)
        hist["ber_unit"] = bit_error_rate(code, ones, iters, eval_batch, eval_ebn0, seed + 1, 1 << 40, dev)
    return hist
