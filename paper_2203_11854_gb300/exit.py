"""EXIT charts and iterative demapping-decoding (BICM-ID) on the device.

The paper lists a demapper with prior and EXIT chart simulations among its
FEC features (Section III). Everything here is orchestration of C-ABI calls;
the arithmetic runs in the library's kernels:

* a-priori LLRs of the consistent Gaussian model, L = (s^2/2)(1 - 2c) + s g
  (``llr_apriori``), with s chosen so that their mutual information is I_A:
  s = J^-1(I_A);
* extrinsic LLRs of the demapper (``demap_app_prior``, bit i's own prior left
  out) and of the decoder (``ldpc_extrinsic``: output APP minus its input);
* the mutual information estimate I = 1 - E[log2(1 + e^{-(1-2c) L})]
  (``llr_mutual_info``) against the transmitted codeword bits
  (``sim_codewords``).

J(s) = 1 - E[log2(1 + e^-L)], L ~ N(s^2/2, s^2), is evaluated on the host by
Gauss-Hermite quadrature (numpy) and inverted by bisection.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import (DEMAP_MAXLOG, DEMAP_OUT_EXTRINSIC, LAYERED_MINSUM, MSG_F32, demap_app_prior, ldpc_bp_decode,
               ldpc_bp_workspace, ldpc_extrinsic, llr_apriori, llr_mutual_info, sim_codewords, sim_count, sim_tx)

_GH = np.polynomial.hermite.hermgauss(120)


def J(sigma: float) -> float:
    """Mutual information of a consistent Gaussian LLR with standard deviation sigma."""
    if sigma <= 0.0:
        return 0.0
    x, w = _GH
    l = 0.5 * sigma * sigma + math.sqrt(2.0) * sigma * x  # L = mu + sqrt(2) sigma x, weight e^{-x^2}
    return float(1.0 - np.sum(w * np.logaddexp(0.0, -l)) / (math.sqrt(math.pi) * math.log(2.0)))


def J_inv(info: float, hi: float = 60.0) -> float:
    """sigma with J(sigma) = info (bisection; J increases strictly)."""
    if info <= 0.0:
        return 0.0
    if info >= 1.0:
        return hi
    lo = 0.0
    for _ in range(80):
        mid = 0.5 * (lo + hi)
        if J(mid) < info:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def n0_of(code, m: int, ebn0_db: float) -> float:
    r = code.k / code.n_tx
    return 1.0 / (r * m * 10.0 ** (ebn0_db / 10.0))


def demapper_curve(code, m: int, ebn0_db: float, ia, *, B: int = 256, seed: int = 0x1DBC, cw0: int = 0,
                   method: int = DEMAP_MAXLOG):
    """[(I_A, I_E)] of the demapper at Eb/N0: a-priori LLRs with information I_A on the transmitted bits,
    extrinsic output information I_E."""
    n0 = torch.tensor([n0_of(code, m, ebn0_db)], dtype=torch.float32, device="cuda")
    y, _ = sim_tx(code, seed, cw0, B, m, n0)
    cw = sim_codewords(code, seed, cw0, B)
    out = []
    for i_a in ia:
        la = llr_apriori(cw, code.p0, code.n_tx, J_inv(i_a), seed=seed, cw0=cw0 + (1 << 32))
        le = demap_app_prior(y, n0, m, la, method=method, out_mode=DEMAP_OUT_EXTRINSIC)
        out.append((float(i_a), llr_mutual_info(le, cw, code.p0)))
    return out


def decoder_curve(code, ia, *, B: int = 256, iters: int = 20, algo: int = LAYERED_MINSUM, msg_prec: int = MSG_F32,
                  seed: int = 0x1DBC, cw0: int = 0):
    """[(I_A, I_E)] of the decoder: its channel input is a-priori LLRs with information I_A on the
    transmitted bits; I_E is the information of its extrinsic output (APP minus input)."""
    cw = sim_codewords(code, seed, cw0, B)
    dec = dict(algo=algo, iters=iters, msg_prec=msg_prec)
    ws = torch.empty(max(1, ldpc_bp_workspace(code, B, **dec)), dtype=torch.uint8, device="cuda")
    out = []
    for i_a in ia:
        la = llr_apriori(cw, code.p0, code.n_tx, J_inv(i_a), seed=seed, cw0=cw0 + (2 << 32))
        app, _, _ = ldpc_bp_decode(code, la, **dec, llr_out=True, bits_out=False, iters_out=False, ws=ws)
        le = ldpc_extrinsic(code, app, la)
        out.append((float(i_a), llr_mutual_info(le, cw, code.p0)))
    return out


def bicm_id(code, m: int, ebn0_db: float, *, outer: int = 3, iters: int = 10, B: int = 256,
            algo: int = LAYERED_MINSUM, msg_prec: int = MSG_F32, method: int = DEMAP_MAXLOG, seed: int = 0x1DBC,
            cw0: int = 0):
    """Iterative demapping and decoding: demap with the decoder's extrinsic LLRs as prior (zero at first),
    decode the demapper's extrinsic LLRs, repeat. Returns per outer iteration the information of the
    demapper and decoder extrinsic LLRs and the information-bit error rate of the decoder output."""
    n0 = torch.tensor([n0_of(code, m, ebn0_db)], dtype=torch.float32, device="cuda")
    y, info = sim_tx(code, seed, cw0, B, m, n0)
    cw = sim_codewords(code, seed, cw0, B)
    dec = dict(algo=algo, iters=iters, msg_prec=msg_prec)
    ws = torch.empty(max(1, ldpc_bp_workspace(code, B, **dec)), dtype=torch.uint8, device="cuda")
    prior = None
    trace = []
    for _ in range(outer):
        le_dem = demap_app_prior(y, n0, m, prior, method=method, out_mode=DEMAP_OUT_EXTRINSIC)
        app, bits, its = ldpc_bp_decode(code, le_dem, **dec, llr_out=True, ws=ws)
        prior = ldpc_extrinsic(code, app, le_dem)
        counts = torch.zeros(5, dtype=torch.int64, device="cuda")
        sim_count(info, bits, its, code.k, counts)
        c = counts.cpu().tolist()
        trace.append({"i_dem": llr_mutual_info(le_dem, cw, code.p0), "i_dec": llr_mutual_info(prior, cw, code.p0),
                      "ber": c[1] / c[0], "bler": c[3] / c[2]})
    return trace
