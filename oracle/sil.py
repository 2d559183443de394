"""Short-iterative Lanczos propagator (FP64).

Sec. 3.1 propagates with the short iterative Arnoldi method; for a Hermitian H
Arnoldi's Hessenberg matrix is the symmetric tridiagonal Lanczos matrix.  The
oracle takes a fixed Krylov dimension K (K H.a products per step), orthogonal-
ises every new vector against all previous ones (classical Gram-Schmidt,
applied twice), and exponentiates the K x K tridiagonal matrix through its
eigendecomposition:

    v_1 = a / beta_0,   beta_0 = ||a||
    w = H v_k,  alpha_k = Re <v_k, w>
    w <- w - sum_{i<=k} <v_i, w> v_i      (twice)
    beta_k = ||w||,  v_{k+1} = w / beta_k
    a(t + dt) = beta_0 V_K exp(-i T_K dt) e_1

Breakdown (invariant subspace found): if beta_k <= 1e-12 ||H v_k|| the
Krylov space is truncated to k vectors.
"""
from __future__ import annotations

import numpy as np

BREAKDOWN_REL = 1e-12


def tridiag_exp_e1(alpha, beta, dt):
    """exp(-i T dt) e_1 for the real symmetric tridiagonal T with diagonal
    alpha and off-diagonal beta (len(alpha) - 1 entries)."""
    k = len(alpha)
    T = np.diag(np.asarray(alpha, dtype=np.float64))
    if k > 1:
        b = np.asarray(beta[:k - 1], dtype=np.float64)
        T += np.diag(b, 1) + np.diag(b, -1)
    lam, Z = np.linalg.eigh(T)
    return Z @ (np.exp(-1j * lam * dt) * Z[0, :])


def sil_step(psi, apply, K, dt, return_info=False, tol=0.0):
    """One SIL step of order K; ``apply(v)`` is the (pruned) H.v.  With
    tol > 0 the order is error-controlled (the adaptive-order reading of
    Sec. 3.1's Arnoldi): after Lanczos step k the estimate
    beta_k |[exp(-i T_{k+1} dt) e_1]_k| of the relative error of stopping
    with k + 1 vectors is formed, and the step stops once it is <= tol
    (K stays the maximum)."""
    psi = np.asarray(psi, dtype=np.complex128)
    beta0 = np.linalg.norm(psi)
    if beta0 == 0.0 or len(psi) == 0:
        return (psi.copy(), dict(alpha=[], beta=[], K=0)) if return_info else psi.copy()
    V = [psi / beta0]
    alpha, beta = [], []
    for k in range(K):
        w = apply(V[k])
        hn = np.linalg.norm(w)
        alpha.append(float(np.real(np.vdot(V[k], w))))
        if k == K - 1:
            break
        for _ in range(2):
            c = np.array([np.vdot(v, w) for v in V])
            for ci, v in zip(c, V):
                w = w - ci * v
        b = np.linalg.norm(w)
        if b <= BREAKDOWN_REL * hn:
            break
        beta.append(float(b))
        if tol > 0.0:
            ck = tridiag_exp_e1(alpha, beta, dt)[k]
            if b * abs(ck) <= tol:
                beta.pop()
                break
        V.append(w / b)
    c = tridiag_exp_e1(alpha, beta, dt)
    out = beta0 * sum(ci * v for ci, v in zip(c, V))
    if return_info:
        return out, dict(alpha=alpha, beta=beta, K=len(alpha))
    return out


def rk4_step(psi, apply, dt):
    """One classical fourth-order Runge-Kutta step of i da/dt = H a (the
    alternative integrator to SIL; not in the paper):
    k1 = -i H a, k2 = -i H (a + dt/2 k1), k3 = -i H (a + dt/2 k2),
    k4 = -i H (a + dt k3), a' = a + dt/6 (k1 + 2 k2 + 2 k3 + k4)."""
    a = np.asarray(psi, dtype=np.complex128)
    k1 = -1j * apply(a)
    k2 = -1j * apply(a + 0.5 * dt * k1)
    k3 = -1j * apply(a + 0.5 * dt * k2)
    k4 = -1j * apply(a + dt * k3)
    return a + (dt / 6.0) * (k1 + 2.0 * k2 + 2.0 * k3 + k4)
