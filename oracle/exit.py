"""Oracle of the EXIT-chart quantities (TEST INFRASTRUCTURE ONLY: imported by
tests/ alone).

* mutual_info(llr, bits): the time-average estimate of the mutual information
  between a bit and its consistent LLR, I = 1 - E[log2(1 + exp(-(1 - 2c) L))]
  (ten Brink, IEEE Trans. Commun. 49(10), 2001; Hagenauer, Proc. EUSIPCO 2004),
  in float64 numpy.
* J(sigma): the mutual information of the consistent Gaussian LLR
  L ~ N(sigma^2/2, sigma^2) given c = 0, by adaptive quadrature (scipy.quad) of
  1 - integral of N(l; sigma^2/2, sigma^2) log2(1 + e^-l) dl.
"""
from __future__ import annotations

import math

import numpy as np


def mutual_info(llr: np.ndarray, bits: np.ndarray) -> float:
    x = (1.0 - 2.0 * bits.astype(np.float64)) * llr.astype(np.float64)
    return float(1.0 - np.mean(np.logaddexp(0.0, -x)) / math.log(2.0))


def J(sigma: float) -> float:
    if sigma <= 0.0:
        return 0.0
    from scipy import integrate
    mu, var = 0.5 * sigma * sigma, sigma * sigma

    def f(l):
        return math.exp(-(l - mu) ** 2 / (2.0 * var)) / math.sqrt(2.0 * math.pi * var) * np.logaddexp(0.0, -l)

    lo, hi = mu - 12.0 * sigma, mu + 12.0 * sigma
    val, _ = integrate.quad(f, lo, hi, limit=400, epsabs=1e-13, epsrel=1e-12)
    return 1.0 - val / math.log(2.0)
