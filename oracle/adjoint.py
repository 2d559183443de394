"""Reference gradients of the survival probability P = |<Psi(0)|Psi(T)>|^2
of a pruned propagation, with the sequence of active sets frozen.

With the sets A_0..A_N of an unperturbed run fixed, the propagation is
    psi_{n+1} = R_n SIL(psi_n; A_n, dt),
R_n carrying coefficients from A_n to A_{n+1} (kept where the point stays,
zero where it is new), and C = sum_{I in A_N} conj(a0_I) psi_N,I with a0 the
normalised full packet (Sec. 3.1, Eq. acorr).  Parameters enter through the
potential (lambda, omega_k of the Henon-Heiles chain) and through the packet
centres q0_k (both the initial coefficients on A_0 and the bra a0).

The reference here is the central finite difference with step h of this
frozen-set map, evaluated in FP64 (the adaption is a step function of the
coefficients; freezing the sets makes the map differentiable).
"""
from __future__ import annotations

import numpy as np

from . import propagate, pruned, sil


def run_frozen(prob, A0, a_init, sets, K, dt):
    """Replay the propagation on the recorded sets (sets[0] = A0)."""
    A = np.asarray(A0, dtype=np.int64)
    a = np.asarray(a_init, dtype=np.complex128)
    for n in range(len(sets) - 1):
        vd = prob.vdiag(A)
        a = sil.sil_step(a, lambda v: prob.apply(A, v, vd), K, dt)
        An = np.asarray(sets[n + 1], dtype=np.int64)
        pos, found = pruned.lookup(A, An)
        b = np.zeros(len(An), dtype=np.complex128)
        b[found] = a[pos[found]]
        A, a = An, b
    return A, a


def survival(cfg, params, sets, K=None, dt=None):
    """P(theta) on frozen sets for the Henon-Heiles workload; params =
    (lam, omega_1..omega_D, q0_1..q0_D)."""
    D = cfg["D"]
    lam, om, q0 = params[0], params[1:1 + D], params[1 + D:1 + 2 * D]
    prob = propagate.problem_from_config(cfg, omegas=om, lam=lam)
    f = prob.factors(q0, cfg["p0"], cfg["width"])
    A0 = np.asarray(sets[0], dtype=np.int64)
    a_init = pruned.product_on(A0, prob.dims, f)
    AN, aN = run_frozen(prob, A0, a_init, sets, K or cfg["K"], dt or cfg["dt"])
    C = np.vdot(pruned.product_on(AN, prob.dims, f), aN)
    return abs(C) ** 2, C


def fd_gradient(cfg, params, sets, h=1e-4):
    """Central differences of P on the frozen sets, one parameter at a time."""
    params = np.asarray(params, dtype=np.float64)
    g = np.zeros(len(params))
    for i in range(len(params)):
        p1, p2 = params.copy(), params.copy()
        p1[i] += h
        p2[i] -= h
        g[i] = (survival(cfg, p1, sets)[0] - survival(cfg, p2, sets)[0]) / (2 * h)
    return g
