"""torch.autograd.Function around the checkpointed decoder and its hand-written adjoint.

LdpcBP.apply(llr_ch, weights, code, iters, clamp) runs weighted flooding
sum-product BP on the GPU (ldpc_bp_decode_ckpt), keeping each iteration's
check-to-variable messages; backward() calls ldpc_bp_backward, which walks
the iterations in reverse and recomputes each from its checkpoint. The
gradients flow to the channel LLRs and to the per-iteration per-block weights
(the paper's custom op with specified gradients, Sec. IV-A, used for end-to-end
learning, Sec. III-C). LLR convention: L = ln P(0)/P(1); a binary
cross-entropy "from logits" takes -L (Listing 2).
"""
from __future__ import annotations

import torch

from . import ldpc_bp_backward, ldpc_bp_decode_ckpt


class LdpcBP(torch.autograd.Function):
    @staticmethod
    def forward(ctx, llr_ch, weights, code, iters: int, clamp: float = 20.0):
        llr_ch = llr_ch.contiguous()
        w = weights.contiguous() if weights is not None else None
        out, ckpt = ldpc_bp_decode_ckpt(code, llr_ch, iters=iters, clamp=clamp, weights=w)
        ctx.save_for_backward(llr_ch, w if w is not None else torch.empty(0, device=llr_ch.device), ckpt)
        ctx.code, ctx.iters, ctx.clamp, ctx.has_w = code, iters, clamp, w is not None
        return out

    @staticmethod
    def backward(ctx, grad_out):
        llr_ch, w, ckpt = ctx.saved_tensors
        w = w if ctx.has_w else None
        g_llr, g_w = ldpc_bp_backward(ctx.code, llr_ch, ckpt, grad_out.contiguous().float(), iters=ctx.iters,
                                      clamp=ctx.clamp, weights=w)
        return g_llr, g_w, None, None, None
