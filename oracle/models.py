"""Model potentials and the initial packet, written as plain functions of the
coordinates (the oracle never uses a sum-of-products form for V: a DVR
potential is diagonal, Sec. 2.1, so V_II = V(x_I) is all that is needed).

The coupled Morse and Henon-Heiles models are synthetic stand-ins the
workloads define; the double well is the paper's own model (Sec. 3.1).
"""
from __future__ import annotations

import numpy as np


def henon_heiles(q: np.ndarray, lam: float, omega=None) -> np.ndarray:
    """Henon-Heiles chain, q of shape (..., D):
    V = sum_k 1/2 omega_k^2 q_k^2 + lam sum_{k<D} (q_k^2 q_{k+1} - q_{k+1}^3 / 3).
    """
    q = np.asarray(q, dtype=np.float64)
    D = q.shape[-1]
    om = np.ones(D) if omega is None else np.asarray(omega, dtype=np.float64)
    v = 0.5 * np.sum((om * q) ** 2, axis=-1)
    for k in range(D - 1):
        a, b = q[..., k], q[..., k + 1]
        v = v + lam * (a * a * b - b ** 3 / 3.0)
    return v


def coupled_morse(q: np.ndarray, De: float, a: float, qe: float,
                  coupling: float) -> np.ndarray:
    """sum_k De (1 - exp(-a (q_k - qe)))^2 + coupling * sum_{i<j} q_i q_j."""
    q = np.asarray(q, dtype=np.float64)
    D = q.shape[-1]
    v = np.sum(De * (1.0 - np.exp(-a * (q - qe))) ** 2, axis=-1)
    for i in range(D):
        for j in range(i + 1, D):
            v = v + coupling * q[..., i] * q[..., j]
    return v


def double_well(q: np.ndarray, c1: float = 6.4, c2: float = 37.5, c3: float = 10.0) -> np.ndarray:
    """The 2D double well of Sec. 3.1 (Eq. ex_dwell), q of shape (..., 2):
    V = c1 (x-1)^2 (x-2)^2 + c2 (y-2)^2 + c3 x^2 y."""
    q = np.asarray(q, dtype=np.float64)
    x, y = q[..., 0], q[..., 1]
    return c1 * (x - 1.0) ** 2 * (x - 2.0) ** 2 + c2 * (y - 2.0) ** 2 + c3 * x * x * y


def gaussian_1d(x, q0: float, p0: float, width: float) -> np.ndarray:
    """(2 pi s^2)^(-1/4) exp(-(x-q0)^2 / (4 s^2) + i p0 (x - q0)), s = position
    standard deviation (normalised on the real line)."""
    x = np.asarray(x, dtype=np.float64)
    s2 = width * width
    return (2.0 * np.pi * s2) ** -0.25 * np.exp(
        -((x - q0) ** 2) / (4.0 * s2) + 1j * p0 * (x - q0))
