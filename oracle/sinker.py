"""Multi-sinker viscosity and forcing of Sec. 2.1.

chi_n(x) = prod_i [1 - exp(-delta max(0, |c_i - x| - omega/2)^2)]
mu(x)    = (mu_max - mu_min)(1 - chi_n(x)) + mu_min,
           mu_min = DR^(-1/2), mu_max = DR^(1/2)
f(x)     = (0, 0, beta (chi_n(x) - 1)),  beta = 10
"""
from __future__ import annotations

import numpy as np


def indicator(x: np.ndarray, centres: np.ndarray, omega: float, delta: float) -> np.ndarray:
    """chi_n at points x of shape (npts, 3)."""
    chi = np.ones(x.shape[0])
    for c in centres:
        dist = np.sqrt(np.sum((x - c[None, :]) ** 2, axis=1))
        s = np.maximum(0.0, dist - omega / 2.0)
        chi *= 1.0 - np.exp(-delta * s * s)
    return chi


def viscosity(x, centres, omega, delta, dr):
    chi = indicator(x, centres, omega, delta)
    mu_min, mu_max = dr ** -0.5, dr ** 0.5
    return (mu_max - mu_min) * (1.0 - chi) + mu_min


def forcing(x, centres, omega, delta, beta=10.0):
    """(npts, 3) body force f = (0, 0, beta (chi - 1))."""
    chi = indicator(x, centres, omega, delta)
    f = np.zeros((x.shape[0], 3))
    f[:, 2] = beta * (chi - 1.0)
    return f
