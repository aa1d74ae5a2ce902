"""Oracle of circular-buffer rate matching (TEST INFRASTRUCTURE ONLY: imported
by tests/ alone).

The paper lists 5G LDPC codes with rate matching among its FEC features
(Section III). Rate matching is taken here as the parameterised procedure of
the 5G NR LDPC chain; the tables that fix the start position per redundancy
version are not used -- the caller passes the start k0 and the buffer size:

* circular buffer: w = codeword bits [p0, p0 + ncb) (the first p0 systematic
  bits are never sent);
* bit selection: e_k = w[(k0 + k) mod ncb], k = 0 .. E-1 (E > ncb repeats,
  E < ncb punctures the tail of the buffer as seen from k0);
* bit interleaving over qm rows of E/qm columns, written row by row and read
  column by column: f[i qm + j] = e[j (E/qm) + i];
* recovery (soft combining): e_k = f[(k mod (E/qm)) qm + k div (E/qm)], and
  buffer position p collects the sum of the e_k with (k0 + k) mod ncb = p in
  increasing k, 0 where no k lands.

float64 numpy; loops over k, vectorised over codewords.
"""
from __future__ import annotations

import numpy as np


def _check(ncb: int, k0: int, E: int, qm: int) -> None:
    if ncb < 1 or not 0 <= k0 < ncb or E < 1 or qm not in (1, 2, 4, 6, 8) or E % qm:
        raise ValueError("bad rate-matching parameters")


def select(cw: np.ndarray, p0: int, ncb: int, k0: int, E: int) -> np.ndarray:
    """e [B][E] from codeword bits cw [B][n]."""
    cw = np.asarray(cw)
    w = cw[:, p0:p0 + ncb]
    if w.shape[1] != ncb:
        raise ValueError("buffer beyond the codeword")
    e = np.zeros((cw.shape[0], E), dtype=cw.dtype)
    for k in range(E):
        e[:, k] = w[:, (k0 + k) % ncb]
    return e


def interleave(e: np.ndarray, qm: int) -> np.ndarray:
    B, E = e.shape
    C = E // qm
    f = np.zeros_like(e)
    for i in range(C):
        for j in range(qm):
            f[:, i * qm + j] = e[:, j * C + i]
    return f


def deinterleave(f: np.ndarray, qm: int) -> np.ndarray:
    B, E = f.shape
    C = E // qm
    e = np.zeros_like(f)
    for k in range(E):
        e[:, k] = f[:, (k % C) * qm + k // C]
    return e


def rate_match(cw: np.ndarray, p0: int, ncb: int, k0: int, E: int, qm: int) -> np.ndarray:
    """Transmitted bits f [B][E] of codewords cw [B][n]."""
    _check(ncb, k0, E, qm)
    return interleave(select(cw, p0, ncb, k0, E), qm)


def rate_recover(llr: np.ndarray, ncb: int, k0: int, qm: int) -> np.ndarray:
    """Soft buffer [B][ncb] (float64) of received LLRs llr [B][E] in transmission order."""
    llr = np.asarray(llr, dtype=np.float64)
    B, E = llr.shape
    _check(ncb, k0, E, qm)
    e = deinterleave(llr, qm)
    v = np.zeros((B, ncb), dtype=np.float64)
    for k in range(E):
        v[:, (k0 + k) % ncb] += e[:, k]
    return v
