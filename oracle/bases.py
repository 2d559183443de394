"""1D primitive bases of the oracle (FP64).

Sec. 2.1 (Eq. wavepacket_form): the wavefunction is expanded in direct
products of DVR functions chi_j with grid points x_j, in which the potential is
diagonal.  Sec. 2.2 (Eq. pvN_def): a function f projects onto chi_j with the
coefficient sqrt(w_j) f(x_j), where w_j is the quadrature weight divided by the
weight function of the DVR polynomials; for the DVRs below it is the weight
returned with the grid.
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


def fgh_dvr(n: int, xmin: float, xmax: float, mass: float):
    """Fourier grid Hamiltonian DVR on the periodic box [xmin, xmax) (Sec. 2.2:
    the FGH DVR, whose functions cover the same phase-space area as a
    periodic lattice; the double-well grids of Sec. 3.1).

    Points x_j = xmin + j L/n, j = 0..n-1 (xmax is identified with xmin),
    weight w = L/n.  The kinetic matrix is p^2/2m in the discrete Fourier
    basis transformed to the grid: T = F^H diag(k_l^2 / 2m) F with the unitary
    DFT F and momenta k_l = 2 pi l / L on the centred integer range
    l = -(n-1)//2 .. n//2 (for even n the last one is the Nyquist mode).
    Built here from numpy's FFT of the identity.

    Returns (x, w, T) with w an array of equal weights.
    """
    L = xmax - xmin
    j = np.arange(n)
    x = xmin + j * L / n
    F = np.fft.fft(np.eye(n), axis=0) / np.sqrt(n)   # F[l, j] = exp(-2 pi i l j / n) / sqrt(n)
    l = np.fft.fftfreq(n, d=1.0 / n)                  # integer frequencies in FFT order
    if n % 2 == 0:
        l[n // 2] = n // 2                            # the Nyquist mode taken as +n/2
    k = 2.0 * np.pi * l / L
    T = (F.conj().T @ np.diag(k * k / (2.0 * mass)) @ F).real
    w = np.full(n, L / n)
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


def pw_functions(x, w, xmin, xmax, nx, np_):
    """The momentum-symmetrised Gaussians of Eq. sG_def projected on a DVR with
    points x and weights w (Eq. sG_def of Sec. 2.3, projected as in Eq. psG_def of
    Sec. 2.4), before orthogonalisation.

    Doubly dense phase-space lattice (Delta x Delta p = pi, p_l > 0):
    x_a = xmin + (a + 1/2) Dx with Dx = (xmax - xmin) / nx, p_b = (b + 1/2) Dp
    with Dp = pi / Dx, alpha = Dp / (2 Dx),
        phi_ab(x) = (8 alpha / pi)^(1/4) exp(-alpha (x - x_a)^2)
                    sin(p_b (x - x_a - sqrt(pi / (8 alpha)))),
    and Phi_ji = sqrt(w_j) phi_i(x_j) with i = a np + b (x index slow, p index
    fast).  Returns Phi, shape (len(x), nx np)."""
    x = np.asarray(x, dtype=np.float64)
    L = xmax - xmin
    dx = L / nx
    dp = np.pi / dx
    alpha = dp / (2.0 * dx)
    xa = xmin + (np.arange(nx) + 0.5) * dx
    pb = (np.arange(np_) + 0.5) * dp
    shift = np.sqrt(np.pi / (8.0 * alpha))
    Phi = np.zeros((len(x), nx * np_))
    for a in range(nx):
        for b in range(np_):
            g = (8.0 * alpha / np.pi) ** 0.25 * np.exp(-alpha * (x - xa[a]) ** 2) \
                * np.sin(pb[b] * (x - xa[a] - shift))
            Phi[:, a * np_ + b] = np.sqrt(w) * g
    return Phi


def pw_basis(n, xmin, xmax, mass, nx, np_, dvr="sine"):
    """Projected Weylets on a sine DVR, or on an FGH DVR with dvr="fgh" (Sec. 2.4;
    Sec. 3.1 uses the FGH grid).

    The projected symmetrised Gaussians Phi (``pw_functions``, Eq. sG_def) are
    orthogonalised symmetrically (Loewdin): W = Phi S^(-1/2), S = Phi^T Phi.
    Needs n = nx np.  Returns (x, w, T, W) where x, w, T are the underlying
    DVR's."""
    if nx * np_ != n:
        raise ValueError("the phase-space lattice must have as many functions as DVR points")
    x, w, T = (fgh_dvr if dvr == "fgh" else sine_dvr)(n, xmin, xmax, mass)
    Phi = pw_functions(x, w, xmin, xmax, nx, np_)
    S = Phi.T @ Phi
    lam, U = np.linalg.eigh(S)
    W = Phi @ (U @ np.diag(lam ** -0.5) @ U.T)
    return x, w, T, W


def pvb_basis(n, xmin, xmax, mass, nx, np_, dvr="sine"):
    """Biorthogonal projected von Neumann basis on a sine DVR, or on an FGH
    DVR with dvr="fgh" (Sec. 2.2; Sec. 3.1 uses the FGH grid).

    von Neumann Gaussians on a lattice with Delta x Delta p = 2 pi:
    x_a = xmin + (a + 1/2) Dx, Dx = L / nx, Dp = 2 pi / Dx, momenta
    p_b = -p_max + (b + 1/2) Dp with p_max = np Dp / 2, alpha = Dp / (2 Dx),
        g_ab(x) = (2 alpha / pi)^(1/4) exp(-alpha (x - x_a)^2 + i p_b (x - x_a)).
    Projection (Eq. pvN_def): G_jm = sqrt(w_j) g_m(x_j), m = a np + b.  The
    biorthogonal functions (Eq. pvb_def) have B = G^{-dagger}, so that
    B^dagger G = 1 (<b_n|g_m> = delta).  Needs n = nx np.
    Returns (x, w, T, G, B)."""
    if nx * np_ != n:
        raise ValueError("the phase-space lattice must have as many functions as DVR points")
    x, w, T = (fgh_dvr if dvr == "fgh" else sine_dvr)(n, xmin, xmax, mass)
    L = xmax - xmin
    dx = L / nx
    dp = 2.0 * np.pi / dx
    alpha = dp / (2.0 * dx)
    xa = xmin + (np.arange(nx) + 0.5) * dx
    pmax = np_ * dp / 2.0
    pb = -pmax + (np.arange(np_) + 0.5) * dp
    G = np.zeros((n, n), dtype=np.complex128)
    for a in range(nx):
        for b in range(np_):
            g = (2.0 * alpha / np.pi) ** 0.25 * np.exp(-alpha * (x - xa[a]) ** 2
                                                      + 1j * pb[b] * (x - xa[a]))
            G[:, a * np_ + b] = np.sqrt(w) * g
    B = np.linalg.inv(G).conj().T
    return x, w, T, G, B
