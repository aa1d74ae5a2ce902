"""Gradient oracle for weighted flooding sum-product BP (test infrastructure).

A vectorised restatement, in torch FP64 on the CPU, of the flooding schedule
of the C oracle (ldpc_oracle.c, decode_one with schedule 1 and algo 1), so that
torch autograd gives the exact derivative of the unrolled decoder -- the
"gradients can be specified" custom op of the paper (Sec. IV-A) used for
end-to-end learning (Sec. III-C, Listing 2):

    V_e  = w[t, cls(e)] * (APP_v - C_e)                 (C = 0 in iteration 0)
    a_e  = clamp(|V_e|, phi(clamp), clamp)
    S_e  = sum over the other edges e' of e's check of phi(a_e')
    C_e  = s_e * phi(clamp(S_e, phi(clamp), clamp)), s_e = prod of the others' signs
    APP  = L + sum over v's edges of C                  (L = clamped channel LLRs)

with phi(x) = ln(1 + 2/(e^x - 1)). The loss helper is the binary cross-entropy
of the output LLRs against the codeword bits (logits = -LLR, Listing 2).
The exclusive sum is computed as the check total minus the own term, which in
FP64 is far below the finite-difference tolerance. Only tests import this.
"""
from __future__ import annotations

import numpy as np
import torch


def phi(x: torch.Tensor) -> torch.Tensor:
    return torch.log1p(2.0 / torch.expm1(x))


def _check_slots(graph):
    """Per-check padded edge table [m, D] (pad = E, a zero slot) and each edge's slot."""
    cn_ptr = np.asarray(graph.cn_ptr, dtype=np.int64)
    deg = cn_ptr[1:] - cn_ptr[:-1]
    D = int(deg.max())
    idx = np.full((graph.m, D), graph.E, dtype=np.int64)
    slot = np.zeros(graph.E, dtype=np.int64)
    for c in range(graph.m):
        e = np.arange(cn_ptr[c], cn_ptr[c + 1])
        idx[c, :len(e)] = e
        slot[e] = np.arange(len(e))
    return torch.from_numpy(idx), torch.from_numpy(slot), D


def weighted_flood_spa(graph, L: torch.Tensor, weights: torch.Tensor, iters: int, clamp: float = 20.0):
    """L: [B, n] placed channel LLRs (float64); weights: [iters, n_cls]. Returns APP [B, n].

    The exclusive sums over the other edges of a check are summed directly, in
    ascending edge order (as the C oracle does), not as total minus own term."""
    cn_ptr = torch.from_numpy(np.asarray(graph.cn_ptr, dtype=np.int64))
    vn = torch.from_numpy(np.asarray(graph.edge_vn, dtype=np.int64))
    cls = torch.from_numpy(np.asarray(graph.edge_cls, dtype=np.int64))
    deg = cn_ptr[1:] - cn_ptr[:-1]
    edge_cn = torch.repeat_interleave(torch.arange(graph.m), deg)
    idx, slot, D = _check_slots(graph)
    B, n = L.shape
    lo = float(np.log1p(2.0 / np.expm1(clamp)))
    Lc = torch.clamp(L, -clamp, clamp)
    app = Lc
    C = torch.zeros(B, graph.E, dtype=L.dtype)
    zero = torch.zeros(B, 1, dtype=L.dtype)
    for t in range(iters):
        V = weights[t][cls] * (app[:, vn] - C)
        a = torch.clamp(V.abs(), lo, clamp)
        f = phi(a)
        F = torch.cat([f, zero], dim=1)[:, idx]  # [B, m, D], padded slots hold 0
        excl = []
        for k in range(D):
            acc = torch.zeros(B, graph.m, dtype=L.dtype)
            for kk in range(D):
                if kk != k:
                    acc = acc + F[:, :, kk]
            excl.append(acc)
        S = torch.stack(excl, dim=2)[:, edge_cn, slot]
        neg = (V < 0).to(L.dtype)
        nneg = torch.zeros(B, graph.m, dtype=L.dtype).index_add_(1, edge_cn, neg)
        sign = 1.0 - 2.0 * torch.remainder(nneg[:, edge_cn] - neg, 2.0)
        C = sign * torch.clamp(phi(torch.clamp(S, lo, clamp)), max=clamp)
        app = Lc + torch.zeros(B, n, dtype=L.dtype).index_add_(1, vn, C)
    return app


def bce_loss(app: torch.Tensor, cw: torch.Tensor) -> torch.Tensor:
    """Mean binary cross-entropy with logits = -APP against codeword bits."""
    return torch.nn.functional.binary_cross_entropy_with_logits(-app, cw.to(app.dtype))


def loss_and_grads(graph, L: np.ndarray, cw: np.ndarray, weights: np.ndarray, iters: int, clamp: float = 20.0):
    """Loss and its gradients with respect to L [B, n] and weights [iters, n_cls] (FP64 autograd)."""
    Lt = torch.tensor(L, dtype=torch.float64, requires_grad=True)
    wt = torch.tensor(weights, dtype=torch.float64, requires_grad=True)
    app = weighted_flood_spa(graph, Lt, wt, iters, clamp)
    loss = bce_loss(app, torch.from_numpy(np.asarray(cw)))
    loss.backward()
    return float(loss.detach()), Lt.grad.numpy(), wt.grad.numpy(), app.detach().numpy()


def bce_numpy(app: np.ndarray, cw: np.ndarray) -> float:
    """The same loss from plain numpy (for finite differences of the C oracle)."""
    x = -app
    y = cw.astype(np.float64)
    return float(np.mean(np.maximum(x, 0) - x * y + np.log1p(np.exp(-np.abs(x)))))
