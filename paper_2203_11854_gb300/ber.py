"""Bit-error-rate curves and the Eb/N0 at a target BER (the Monte-Carlo loop
around the paper's Listing 1, run with sim_run on the device).

Each point decodes a fixed set of codewords (same Philox seed and codeword
range for every decoder variant), so two variants see identical codewords and
noise draws and their curves can be compared point by point. The Eb/N0 at a
target BER is interpolated linearly in log10(BER) between the two bracketing
points.
"""
from __future__ import annotations

import math

from . import DEMAP_MAXLOG, LAYERED_MINSUM, MSG_F16, sim_run


def ber_point(code, ebn0_db: float, *, codewords: int, batch: int = 4096, seed: int = 0x1DBC, cw0: int = 0,
              m: int = 4, algo: int = LAYERED_MINSUM, msg_prec: int = MSG_F16, iters: int = 20,
              demap_method: int = DEMAP_MAXLOG, offset: float = 0.5, clamp: float = 20.0) -> dict:
    """Counts for codewords [cw0, cw0 + codewords) at one Eb/N0 (rounded up to whole batches)."""
    batch = min(batch, codewords)
    nb = (codewords + batch - 1) // batch
    res = sim_run(code, [ebn0_db], m=m, demap_method=demap_method, algo=algo, iters=iters, msg_prec=msg_prec,
                  offset=offset, clamp=clamp, seed=seed, cw0=cw0, batch=batch, max_batches=nb, use_graph=True)[0]
    res["ber"] = res["bit_errors"] / res["bits"]
    res["bler"] = res["block_errors"] / res["blocks"]
    return res


def crossing(points, target: float = 1e-4):
    """Eb/N0 (dB) where the BER of `points` [(ebn0, ber), ...] crosses `target`, by log10 interpolation
    between the first bracketing pair; None if no pair brackets the target."""
    pts = sorted(points)
    for (x1, b1), (x2, b2) in zip(pts[:-1], pts[1:]):
        if b1 >= target > b2 and b1 > 0:
            if b2 <= 0:
                return x2  # no errors at x2: the crossing lies at or before x2
            l1, l2, lt = math.log10(b1), math.log10(b2), math.log10(target)
            return x1 + (lt - l1) * (x2 - x1) / (l2 - l1)
    return None


def bracket(code, grid, *, target: float = 1e-4, codewords: int = 16384, **kw):
    """Coarse sweep over `grid` (ascending Eb/N0); returns the first pair (x1, x2) with
    BER(x1) >= target > BER(x2), and the points measured."""
    pts = []
    for x in grid:
        r = ber_point(code, x, codewords=codewords, **kw)
        pts.append((x, r["ber"]))
        if len(pts) >= 2 and pts[-2][1] >= target > pts[-1][1]:
            return (pts[-2][0], pts[-1][0]), pts
    return None, pts
