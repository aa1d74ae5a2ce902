"""Synthetic workloads built from the library's own device kernels.

mixed_batch(): the uneven Monte-Carlo batch of one persistent launch -- codes
over lifting sizes {16, 32, 64, 128, 256, 384}, both 5G base-graph shapes and
rates {1/3, 1/2, 2/3, 8/9} set by extension-row truncation, a modulation per
codeword from {QPSK, 16-QAM, 64-QAM} and an Eb/N0 per codeword uniform within
+-1 dB of the waterfall of its (code, modulation).

Rate by truncation: keep 4 + max(0, ceil(Kb/r) + 2 - (Kb + 4)) base rows and
send n_tx = k/r bits from column 2 on (the first 2Z systematic bits are
punctured), rounded down to a multiple of 12 so that every modulation maps
whole symbols. The waterfall of a (code, modulation) is the Eb/N0 where the
block error rate of layered min-sum (20 iterations, early stop) is 0.5, found by
bisection on sim_run.
"""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np
import torch

from . import DEMAP_MAXLOG, LAYERED_MINSUM, MSG_F16, demap_app, qc_ldpc_build, sim_run, sim_tx

Z_SET = (16, 32, 64, 128, 256, 384)
RATES = (Fraction(1, 3), Fraction(1, 2), Fraction(2, 3), Fraction(8, 9))
MODS = (2, 4, 6)


def rows_for_rate(bg: int, r: Fraction) -> int:
    kb = 22 if bg == 1 else 10
    return 4 + max(0, math.ceil(Fraction(kb) / r) + 2 - (kb + 4))


def rate_code(bg: int, Z: int, r: Fraction):
    kb = 22 if bg == 1 else 10
    n_tx = int(Fraction(kb * Z) / r)
    n_tx -= n_tx % 12
    return qc_ldpc_build(bg, Z, rows_kept=rows_for_rate(bg, r), punct_cols=2, n_tx=n_tx)


def waterfall(code, m: int, seed: int = 77, batch: int = 256, lo: float = -2.0, hi: float = 14.0,
              steps: int = 8) -> float:
    """Eb/N0 (dB) with block error rate 0.5 (bisection)."""
    for i in range(steps):
        mid = 0.5 * (lo + hi)
        r = sim_run(code, [mid], m=m, demap_method=DEMAP_MAXLOG, algo=LAYERED_MINSUM, iters=20, msg_prec=MSG_F16,
                    early_stop=True, seed=seed, cw0=i * batch, batch=batch, max_batches=1, use_graph=False)[0]
        if r["block_errors"] / r["blocks"] > 0.5:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def mixed_codes():
    return [((bg, Z, r), rate_code(bg, Z, r)) for Z in Z_SET for bg in (1, 2) for r in RATES]


def mixed_batch(total: int = 8192, seed: int = 11, dev: str = "cuda", codes=None, centres=None):
    """Returns (groups [(code, llr [B_i, n_tx_i])], info [(packed info bits [B_i, kw_i])], description)."""
    codes = codes if codes is not None else mixed_codes()
    if centres is None:
        centres = {(i, m): waterfall(c, m) for i, (_, c) in enumerate(codes) for m in MODS}
    gen = np.random.default_rng(seed)
    pick = gen.integers(0, len(codes), size=total)
    mods = gen.choice(MODS, size=total)
    groups, infos = [], []
    cw0 = 0
    for i, (key, code) in enumerate(codes):
        llrs, bits = [], []
        for m in MODS:
            cnt = int(((pick == i) & (mods == m)).sum())
            if cnt == 0:
                continue
            e = centres[(i, m)] + gen.uniform(-1.0, 1.0, size=cnt)
            r = code.k / code.n_tx
            n0 = torch.from_numpy(1.0 / (r * m * 10 ** (e / 10))).float().to(dev)
            y, info = sim_tx(code, seed, cw0, cnt, m, n0)
            cw0 += cnt
            llrs.append(demap_app(y, n0, m, method=DEMAP_MAXLOG))
            bits.append(info)
        if llrs:
            groups.append((code, torch.cat(llrs)))
            infos.append(torch.cat(bits))
    desc = {"codewords": total, "codes": len(codes), "groups": len(groups),
            "lifting_sizes": list(Z_SET), "rates": [str(r) for r in RATES], "modulations": ["QPSK", "16-QAM", "64-QAM"]}
    return groups, infos, desc
