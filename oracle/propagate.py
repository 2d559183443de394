"""The whole pruned propagation (FP64): initial packet, initial prune, then
per step SIL -> prune -> observables (Sec. 2.5 adaption after every step,
Sec. 3.1 autocorrelation).
"""
from __future__ import annotations

import numpy as np

from . import bases, models, pruned, sil


class DVRProblem:
    """A DVR direct-product problem: per-mode grids, weights, kinetic
    matrices, and the potential as a function of the coordinates.  The
    adaption lattice has one axis per mode."""

    def __init__(self, grids, weights, Ts, vfunc):
        self.grids = [np.asarray(g, dtype=np.float64) for g in grids]
        self.weights = [np.asarray(w, dtype=np.float64) for w in weights]
        self.Ts = [np.asarray(T, dtype=np.float64) for T in Ts]
        self.vfunc = vfunc
        self.dims = tuple(len(g) for g in self.grids)
        self.axes = self.dims

    def vdiag(self, A):
        return pruned.potential_diag(A, self.dims, self.grids, self.vfunc)

    def apply(self, A, psi, vd=None):
        if vd is None:
            vd = self.vdiag(A)
        return pruned.apply_H(A, psi, self.dims, self.Ts, vd)

    def factors(self, q0, p0, width):
        return pruned.packet_factors(self.grids, self.weights, q0, p0, width,
                                     models.gaussian_1d)


class PWProblem:
    """Projected-Weylet problem (Sec. 2.4): per mode a DVR and the orthogonal
    transformation W to the pW functions; every SoP factor is transformed by
    congruence, h^w = W^T h^chi W (Sec. 2.2, Eq. pvb_H_trafo with B -> W),
    and applied with the pruned sequential transform.  The adaption lattice
    has two axes per mode (x and p indices of the phase-space lattice)."""

    def __init__(self, grids, weights, Ts, Ws, lattices, sop_terms):
        self.grids = [np.asarray(g, dtype=np.float64) for g in grids]
        self.weights = [np.asarray(w, dtype=np.float64) for w in weights]
        self.Ws = [np.asarray(W, dtype=np.float64) for W in Ws]
        self.dims = tuple(len(g) for g in self.grids)
        self.axes = tuple(v for lat in lattices for v in lat)
        self.terms = []
        for coef, facs in sop_terms:     # factors given on the DVR: 'T' or grid values
            tf = {}
            for k, f in facs.items():
                h = Ts[k] if isinstance(f, str) else np.diag(np.asarray(f, dtype=np.float64))
                tf[k] = self.Ws[k].T @ h @ self.Ws[k]
            self.terms.append((coef, tf))

    def vdiag(self, A):
        return None

    def apply(self, A, psi, vd=None):
        return pruned.apply_H_sop(A, psi, self.dims, self.terms)

    def factors(self, q0, p0, width):
        f = pruned.packet_factors(self.grids, self.weights, q0, p0, width, models.gaussian_1d)
        return [self.Ws[k].T @ f[k] for k in range(len(f))]


def morse_sop_terms(grids, De, a, qe, coupling):
    """Coupled Morse as SoP terms on the DVR grids: kinetic per mode, Morse
    per mode, coupling * q_i q_j per pair (used by the phase-space bases)."""
    D = len(grids)
    terms = [(1.0, {k: "T"}) for k in range(D)]
    for k in range(D):
        terms.append((1.0, {k: models.coupled_morse(grids[k][:, None], De, a, qe, 0.0)}))
    for i in range(D):
        for j in range(i + 1, D):
            terms.append((coupling, {i: grids[i], j: grids[j]}))
    return terms


def pw_problem_from_config(cfg, n=None, nx=None, np_=None):
    """pW problem of the 3D coupled Morse workload (or a smaller lattice)."""
    n = cfg["n"] if n is None else n
    nx = cfg["nx_lattice"] if nx is None else nx
    np_ = cfg["np_lattice"] if np_ is None else np_
    D = cfg["D"]
    x, w, T, W = bases.pw_basis(n, cfg["xmin"], cfg["xmax"], cfg["mass"], nx, np_)
    terms = morse_sop_terms([x] * D, cfg["morse_D"], cfg["morse_a"], cfg["morse_qe"],
                            cfg["coupling"])
    return PWProblem([x] * D, [w] * D, [T] * D, [W] * D, [(nx, np_)] * D, terms)


def dwell_pw_problem(cfg):
    """pW problem of the double well (Sec. 3.1): projected Weylets on the FGH
    grids of each mode, the double-well SoP terms transformed by congruence."""
    xs, ws, Ts, Wm, lat = [], [], [], [], []
    for k in range(cfg["D"]):
        x, w, T, Wk = bases.pw_basis(cfg["n"][k], cfg["xmin"][k], cfg["xmax"][k], cfg["mass"],
                                     cfg["nx_lattice"][k], cfg["np_lattice"][k], dvr="fgh")
        xs.append(x); ws.append(w); Ts.append(T); Wm.append(Wk)
        lat.append((cfg["nx_lattice"][k], cfg["np_lattice"][k]))
    c1, c2, c3 = cfg["dw_coef"]
    x, y = xs
    terms = [(1.0, {0: "T"}), (1.0, {1: "T"}), (c1, {0: (x - 1.0) ** 2 * (x - 2.0) ** 2}),
             (c2, {1: (y - 2.0) ** 2}), (c3, {0: x * x, 1: y})]
    return PWProblem(xs, ws, Ts, Wm, lat, terms)


def problem_from_config(cfg, omegas=None, lam=None):
    """Build the problem of a workload record (see ``workloads``)."""
    D, n = cfg["D"], cfg["n"]
    if cfg["basis"] == "pw" and cfg.get("dvr") == "fgh":
        return dwell_pw_problem(cfg)
    if cfg["basis"] == "pw":
        return pw_problem_from_config(cfg)
    if cfg["basis"] == "fgh":
        xs, ws, Ts = [], [], []
        for k in range(D):
            x, w, T = bases.fgh_dvr(n[k], cfg["xmin"][k], cfg["xmax"][k], cfg["mass"])
            xs.append(x); ws.append(w); Ts.append(T)
        c = cfg["dw_coef"]
        return DVRProblem(xs, ws, Ts, lambda q: models.double_well(q, *c))
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
    """Projected (Eq. pvN_def), normalised product packet and its initial prune
    (Sec. 2.5 applied to the full lattice).  Returns (A, a, factors) where the
    factors are the per-mode normalised packet vectors (the full-lattice packet
    used by C(t) is their product).  The full lattice is scanned in chunks of
    linear indices so that 6D lattices fit in host memory."""
    f = prob.factors(q0, p0, width)
    total = int(np.prod(prob.dims))
    S = []
    for c0 in range(0, total, chunk):
        idx = np.arange(c0, min(total, c0 + chunk), dtype=np.int64)
        a = pruned.product_on(idx, prob.dims, f)
        S.append(idx[pruned.significant(a, theta)])
    A = pruned.adapt_set(np.concatenate(S), prob.axes, radius)
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
        record_sets=False, state=None, rel_excl=0.0, integrator="sil", sil_tol=0.0):
    """Propagate ``nsteps`` steps.  Returns a dict with per-step observables
    (index 0 = t = 0 after the initial prune), the final (A, a) and, when
    asked, the active set after each step.  ``radius`` is the neighbour rule
    and ``rel_excl`` the relative exclusion threshold of the adaption;
    ``integrator`` is "sil" (order K, error-controlled below K when
    sil_tol > 0) or "rk4"."""
    if state is None:
        A, a, f = initial_state(prob, q0, p0, width, theta, radius)
    else:
        A, a, f = state
    obs = [observables(prob, A, a, f, theta)]
    sets = [A.copy()] if record_sets else None
    for _ in range(nsteps):
        vd = prob.vdiag(A)
        if integrator == "rk4":
            a = sil.rk4_step(a, lambda v: prob.apply(A, v, vd), dt)
        else:
            a = sil.sil_step(a, lambda v: prob.apply(A, v, vd), K, dt, tol=sil_tol)
        A, a = pruned.prune(A, a, prob.axes, theta, radius, rel_excl)
        obs.append(observables(prob, A, a, f, theta))
        if record_sets:
            sets.append(A.copy())
    out = dict(obs=obs, A=A, a=a, factors=f)
    if record_sets:
        out["sets"] = sets
    return out
