"""Oracle of code-block shortening with filler bits (TEST INFRASTRUCTURE ONLY:
imported by tests/ alone).

The paper's Listing 1 encodes k = 500 information bits into n = 1000 coded bits
with the 5G LDPC encoder (Sec. III-C), and its feature list names 5G LDPC codes
with rate matching (Sec. III-B). A 5G code block carries fewer information
bits than the base graph's kb Z systematic positions; the rest are filler bits.
Restated here from that construction:

* information bits u_0 .. u_{k-1} occupy systematic positions 0 .. k-1, filler
  bits positions k .. kb Z - 1; fillers are 0, known to both ends;
* the codeword is the mother code's systematic encoding of [u | 0 ... 0];
* filler bits are never transmitted: the transmit layout is the list of
  codeword positions p0 .. n-1 (the first p0 are punctured) without the
  fillers, n_tx = n - p0 - (kb Z - k) of them, in increasing order;
* the receiver knows the fillers are 0: their channel LLR is +clamp (the
  largest LLR the decoder admits), punctured positions get 0;
* the decoded information bits are the first k hard decisions.

Rate matching runs on the transmit layout (oracle/ratematch.py with p0 = 0 over
the transmitted bits). The 5G form keeps the fillers in the circular buffer as
<NULL> entries and skips them while reading; `select_with_nulls` restates that
form so tests can check the two against each other.

float64 numpy; plain loops where the definition is a loop.
"""
from __future__ import annotations

import numpy as np

from . import Code


class ShortCode:
    """Mother code `code` carrying k information bits (p0 <= k <= kb Z)."""

    def __init__(self, code: Code, k: int):
        K = code.k  # kb Z systematic positions of the mother code
        if not code.p0 <= k <= K:
            raise ValueError("information bits must cover the punctured columns and fit the systematic part")
        if code.p0 + code.n_tx < K:
            raise ValueError("the fillers must lie inside the transmitted span")
        self.code, self.graph, self.encoder = code, code.graph, code.encoder
        self.n, self.p0, self.K = code.n, code.p0, K
        self.k = k
        self.n_fill = K - k
        self.n_tx = code.n_tx - self.n_fill
        span = np.arange(code.p0, code.p0 + code.n_tx)
        self.tx_pos = span[(span < k) | (span >= K)]  # codeword position of transmitted bit t
        assert len(self.tx_pos) == self.n_tx

    def encode(self, u: np.ndarray) -> np.ndarray:
        """Codewords [B, n] of information bits u [B, k]: fillers 0, then the mother encoder."""
        u = np.asarray(u, dtype=np.uint8).reshape(-1, self.k)
        full = np.zeros((u.shape[0], self.K), dtype=np.uint8)
        full[:, :self.k] = u
        return self.encoder.encode(full)

    def tx_bits(self, cw: np.ndarray) -> np.ndarray:
        """Transmitted bits [B, n_tx] of codewords [B, n]."""
        return np.asarray(cw)[:, self.tx_pos]

    def place_llr(self, llr_tx: np.ndarray, clamp: float = 20.0) -> np.ndarray:
        """Decoder input [B, n] from LLRs [B, n_tx] in transmit order: fillers at +clamp, punctured at 0."""
        llr_tx = np.asarray(llr_tx, dtype=np.float64).reshape(-1, self.n_tx)
        out = np.zeros((llr_tx.shape[0], self.n), dtype=np.float64)
        out[:, self.tx_pos] = llr_tx
        out[:, self.k:self.K] = clamp
        return out


def select_with_nulls(cw: np.ndarray, p0: int, k: int, K: int, ncb_null: int, k0_null: int, E: int) -> np.ndarray:
    """5G-form bit selection: the circular buffer w = codeword positions [p0, p0 + ncb_null) with the filler
    positions [k, K) marked <NULL>; reading starts at buffer index k0_null and skips <NULL> entries until E bits
    are taken (the buffer must hold at least one non-NULL entry)."""
    cw = np.asarray(cw)
    w = cw[:, p0:p0 + ncb_null]
    null = np.zeros(ncb_null, dtype=bool)
    for j in range(ncb_null):
        null[j] = k <= p0 + j < K
    if null.all():
        raise ValueError("empty buffer")
    e = np.zeros((cw.shape[0], E), dtype=cw.dtype)
    taken, j = 0, 0
    while taken < E:
        idx = (k0_null + j) % ncb_null
        if not null[idx]:
            e[:, taken] = w[:, idx]
            taken += 1
        j += 1
    return e
