"""Seeded synthetic inputs shared by the CUDA-path tests and the oracle tests.

This module holds no step of the method: it draws random bits, Gaussian
values and channel symbols with numpy's seeded generator, so that the CUDA
library and the oracle receive identical float32 inputs.
"""
from __future__ import annotations

import numpy as np


def rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(seed)


def info_bits(seed: int, B: int, k: int) -> np.ndarray:
    return rng(seed).integers(0, 2, size=(B, k), dtype=np.uint8)


def gaussian_llrs(cw: np.ndarray, mean: float, seed: int) -> np.ndarray:
    """Consistent Gaussian LLRs of codewords cw [B, n]: mean +-mean, variance 2*mean
    (the LLR law of BPSK on AWGN), as float32."""
    g = rng(seed).standard_normal(size=cw.shape)
    x = mean * (1.0 - 2.0 * cw.astype(np.float64)) + np.sqrt(2.0 * mean) * g
    return x.astype(np.float32)


def symbols(seed: int, B: int, S: int, m: int, spread: float = 1.2) -> np.ndarray:
    """Random received symbols: [B, S] real for m = 1, else [B, S, 2]."""
    shape = (B, S) if m == 1 else (B, S, 2)
    return (spread * rng(seed).standard_normal(size=shape)).astype(np.float32)


def packed_bits(seed: int, B: int, words: int, k: int) -> np.ndarray:
    """Random packed bit vectors [B, words] (int32 view) with bits >= k cleared."""
    w = rng(seed).integers(0, 2**32, size=(B, words), dtype=np.uint64).astype(np.uint32)
    rem = k - 32 * (words - 1)
    if rem < 32:
        w[:, -1] &= np.uint32((1 << rem) - 1)
    return w.view(np.int32)
