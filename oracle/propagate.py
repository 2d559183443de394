"""The whole pruned propagation (FP64): initial packet, initial prune, then
per step SIL -> prune -> observables (Sec. 2.5 adaption after every step,
Sec. 3.1 autocorrelation).
"""
from __future__ import annotations

import numpy as np

from . import bases, models, pruned, sil


class DVRProblem:
    """A DVR direct-product problem: per-mode grids, weights, kinetic
    matrices, and the potential as a function of the coordinates."""

    def __init__(self, grids, weights, Ts, vfunc):
        self.grids = [np.asarray(g, dtype=np.float64) for g in grids]
        self.weights = [np.asarray(w, dtype=np.float64) for w in weights]
        self.Ts = [np.asarray(T, dtype=np.float64) for T in Ts]
        self.vfunc = vfunc
        self.dims = tuple(len(g) for g in self.grids)

    def vdiag(self, A):
        return pruned.potential_diag(A, self.dims, self.grids, self.vfunc)

    def apply(self, A, psi, vd=None):
        if vd is None:
            vd = self.vdiag(A)
        return pruned.apply_H(A, psi, self.dims, self.Ts, vd)


def problem_from_config(cfg, omegas=None, lam=None):
    """Build the DVR problem of a workload record (see ``workloads``)."""
    D, n = cfg["D"], cfg["n"]
    if cfg["basis"] == "sine":
        x, w, T = bases.sine_dvr(n, cfg["xmin"], cfg["xmax"], cfg["mass"])
        vf = lambda q: models.coupled_morse(q, cfg["morse_D"], cfg["morse_a"],
                                            cfg["morse_qe"], cfg["coupling"])
    elif cfg["basis"] == "ho":
        x, w, T = bases.ho_dvr(n, cfg.get("mass", 1.0), cfg.get("omega", 1.0))
        lm = cfg["lam"] if lam is None else lam
        vf = lambda q: models.henon_heiles(q, lm, omegas)
    else:
        raise ValueError(cfg["basis"])
    return DVRProblem([x] * D, [w] * D, [T] * D, vf)


def initial_state(prob, q0, p0, width, theta, radius=1, chunk=1 << 22):
    """Projected, normalised product packet (Sec. 2.1) and its initial prune
    (Sec. 2.5 applied to the full lattice).  Returns (A, a, factors) where the
    factors are the per-mode normalised packet vectors (the full-lattice packet
    used by C(t) is their product).  The full lattice is scanned in chunks of
    linear indices so that 6D lattices fit in host memory."""
    f = pruned.packet_factors(prob.grids, prob.weights, q0, p0, width,
                              models.gaussian_1d)
    total = int(np.prod(prob.dims))
    S = []
    for c0 in range(0, total, chunk):
        idx = np.arange(c0, min(total, c0 + chunk), dtype=np.int64)
        a = pruned.product_on(idx, prob.dims, f)
        S.append(idx[pruned.significant(a, theta)])
    A = pruned.adapt_set(np.concatenate(S), prob.dims, radius)
    return A, pruned.product_on(A, prob.dims, f), f


def observables(prob, A, psi, factors, theta, vd=None):
    a0 = pruned.product_on(A, prob.dims, factors)
    nrm2 = float(np.real(np.vdot(psi, psi)))
    Hpsi = prob.apply(A, psi, vd)
    E = float(np.real(np.vdot(psi, Hpsi))) / nrm2 if nrm2 > 0 else 0.0
    wasted = int(np.count_nonzero(~pruned.significant(psi, theta)))
    return dict(C=complex(pruned.autocorrelation(A, psi, a0)), norm2=nrm2,
                E=E, n_active=len(A), n_wasted=wasted)


def run(prob, q0, p0, width, theta, K, dt, nsteps, radius=1,
        record_sets=False, state=None):
    """Propagate ``nsteps`` steps.  Returns a dict with per-step observables
    (index 0 = t = 0 after the initial prune), the final (A, a) and, when
    asked, the active set after each step."""
    if state is None:
        A, a, f = initial_state(prob, q0, p0, width, theta, radius)
    else:
        A, a, f = state
    obs = [observables(prob, A, a, f, theta)]
    sets = [A.copy()] if record_sets else None
    for _ in range(nsteps):
        vd = prob.vdiag(A)
        a = sil.sil_step(a, lambda v: prob.apply(A, v, vd), K, dt)
        A, a = pruned.prune(A, a, prob.dims, theta, radius)
        obs.append(observables(prob, A, a, f, theta))
        if record_sets:
            sets.append(A.copy())
    out = dict(obs=obs, A=A, a=a, factors=f)
    if record_sets:
        out["sets"] = sets
    return out
