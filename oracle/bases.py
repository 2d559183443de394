"""1D primitive bases of the oracle (FP64).

Sec. 2.1 (Eq. of the direct-product expansion and the DVR remarks): a DVR
basis chi_j has grid points x_j and weights w_j such that the coefficient of a
wavefunction is a_j = sqrt(w_j) psi(x_j); the potential is diagonal.
Sec. 2.2 (Eq. pvN_def): "omega_j = W_j / omega(x_j)" -- the weight used in the
projection is the quadrature weight divided by the weight function of the
DVR polynomials; for both DVRs below it is the factor that turns grid values
into coefficients.
"""
from __future__ import annotations

import numpy as np


def sine_dvr(n: int, xmin: float, xmax: float, mass: float):
    """Sine DVR on the box [xmin, xmax] (a non-periodic DVR, Sec. 2.2: the
    sinc / sine DVRs are admissible under the projected bases).

    Points x_j = xmin + j L/(n+1), j = 1..n, L = xmax - xmin; the DVR is the
    particle-in-a-box basis sin(k pi (x - xmin)/L) diagonalised in position,
    so U_jk = sqrt(2/(n+1)) sin(j k pi/(n+1)) and the kinetic matrix is
    T = U diag(k^2 pi^2 / (2 m L^2)) U^T.  Weight w = L/(n+1).

    Returns (x, w, T) with w an array of equal weights.
    """
    L = xmax - xmin
    j = np.arange(1, n + 1)
    x = xmin + j * L / (n + 1)
    U = np.sqrt(2.0 / (n + 1)) * np.sin(np.outer(j, j) * np.pi / (n + 1))
    ek = (j * np.pi / L) ** 2 / (2.0 * mass)
    T = U @ np.diag(ek) @ U.T
    w = np.full(n, L / (n + 1))
    return x, w, T


def ho_dvr(n: int, mass: float = 1.0, omega: float = 1.0):
    """Harmonic-oscillator (Gauss-Hermite) DVR.

    The position operator in the first n HO eigenfunctions phi_0..phi_{n-1}
    has X_{k,k+1} = sqrt((k+1)/(2 m omega)); its eigenvectors U (columns) and
    eigenvalues x_i are the DVR.  The kinetic energy is taken exactly in the
    HO basis, (p^2)_{kk} = m omega (k + 1/2), (p^2)_{k,k+2} =
    -(m omega / 2) sqrt((k+1)(k+2)), and transformed, T = U^T (p^2/2m) U.
    Eigenvector signs are fixed so that U_{0i} > 0 (chi_i(x_i) > 0).
    Weights w_i = (U_{0i} / phi_0(x_i))^2.
    """
    k = np.arange(n - 1)
    X = np.zeros((n, n))
    X[k, k + 1] = X[k + 1, k] = np.sqrt((k + 1) / (2.0 * mass * omega))
    x, U = np.linalg.eigh(X)
    U = U * np.sign(U[0, :])[None, :]
    P2 = np.zeros((n, n))
    kk = np.arange(n)
    P2[kk, kk] = mass * omega * (kk + 0.5)
    k2 = np.arange(n - 2)
    off = -0.5 * mass * omega * np.sqrt((k2 + 1.0) * (k2 + 2.0))
    P2[k2, k2 + 2] = P2[k2 + 2, k2] = off
    T = U.T @ (P2 / (2.0 * mass)) @ U
    phi0 = (mass * omega / np.pi) ** 0.25 * np.exp(-0.5 * mass * omega * x * x)
    w = (U[0, :] / phi0) ** 2
    return x, w, T
