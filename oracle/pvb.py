"""Pruned dynamics in the biorthogonal projected von Neumann basis (Sec. 2.2).

The basis is nonorthogonal: i S da/dt = H a with H = B^dagger H^chi B and
S = B^dagger B (Eq. pvb_H_trafo), both per mode.  On an active set A only
S_AA and H_AA are kept.  H_AA a cannot be formed on the pruned set because
the partially transformed tensors are not sparse (Sec. 2.2.2, drawbacks in
high dimensions), so it is taken on the full grid:
    y = P_A (x_k B_k^dagger) H^chi (x_k B_k) P_A^T a,
and S_AA^{-1} y by conjugate gradients with S_AA v = P_A (x_k S_k) P_A^T v.
The propagator is Lanczos in the S inner product <x, y>_S = x^dagger S_AA y,
for which S_AA^{-1} H_AA is self-adjoint.

Coefficients: a = G^dagger a^chi (Eq. psi_exp_pvb: a_m = <g_m|Psi>), so the
packet's coefficients are the product of G_k^dagger f_k; the autocorrelation
<Psi(0)|Psi(t)> = sum_n conj(<b_n|Psi(0)>) a_n with <b_n|Psi(0)> the product
of B_k^dagger f_k (Sec. 3.1: "multiply the coefficient vector with B^T B").
"""
from __future__ import annotations

import numpy as np

from . import bases, models, pruned, propagate

CG_TOL = 1e-13


def mode_transform(X, M, k):
    """Apply the matrix M along axis k of the full-grid tensor X."""
    Y = np.tensordot(M, X, axes=([1], [k]))
    return np.moveaxis(Y, 0, k)


class PVBProblem:
    """pvB problem of a workload record: the 3D coupled Morse on sine DVRs
    (uniform modes; n, nx, np may be overridden), or the double well of
    Sec. 3.1 on its FGH grids (per-mode sizes, ``dvr="fgh"``)."""

    def __init__(self, cfg, n=None, nx=None, np_=None):
        self.cfg = cfg
        D = cfg["D"]
        if cfg.get("dvr") == "fgh":
            ns, nxs, nps = cfg["n"], cfg["nx_lattice"], cfg["np_lattice"]
            lo, hi, dvr = cfg["xmin"], cfg["xmax"], "fgh"
        else:
            n = cfg["n"] if n is None else n
            nx = cfg["nx_lattice"] if nx is None else nx
            np_ = cfg["np_lattice"] if np_ is None else np_
            ns, nxs, nps = (n,) * D, (nx,) * D, (np_,) * D
            lo, hi, dvr = (cfg["xmin"],) * D, (cfg["xmax"],) * D, "sine"
        self.xs, self.ws, self.Ts, self.Gs, self.Bs = [], [], [], [], []
        for k in range(D):
            x, w, T, G, B = bases.pvb_basis(ns[k], lo[k], hi[k], cfg["mass"], nxs[k], nps[k], dvr)
            self.xs.append(x); self.ws.append(w); self.Ts.append(T)
            self.Gs.append(G); self.Bs.append(B)
        self.Ss = [B.conj().T @ B for B in self.Bs]
        self.smax = max(np.abs(S).max() for S in self.Ss)
        self.dims = tuple(ns)
        self.axes = tuple(v for k in range(D) for v in (nxs[k], nps[k]))
        q = np.stack(np.meshgrid(*self.xs, indexing="ij"), axis=-1)
        if "dw_coef" in cfg:
            self.V = models.double_well(q, *cfg["dw_coef"])
        else:
            self.V = models.coupled_morse(q, cfg["morse_D"], cfg["morse_a"], cfg["morse_qe"],
                                          cfg["coupling"])

    def embed(self, A, a):
        X = np.zeros(int(np.prod(self.dims)), dtype=np.complex128)
        X[A] = a
        return X.reshape(self.dims)

    def H_full(self, X):
        """H^chi on the full DVR grid: kinetic along every mode + V."""
        Y = self.V * X
        for k in range(len(self.dims)):
            Y = Y + mode_transform(X, self.Ts[k], k)
        return Y

    def H_AA(self, A, a):
        X = self.embed(A, a)
        for k in range(len(self.dims)):
            X = mode_transform(X, self.Bs[k], k)
        Y = self.H_full(X)
        for k in range(len(self.dims)):
            Y = mode_transform(Y, self.Bs[k].conj().T, k)
        return Y.ravel()[A]

    def S_AA(self, A, v):
        X = self.embed(A, v)
        for k in range(len(self.dims)):
            X = mode_transform(X, self.Ss[k], k)
        return X.ravel()[A]

    def solve_S(self, A, y):
        """Conjugate gradients for S_AA x = y (Hermitian positive definite),
        relative residual CG_TOL."""
        x = np.zeros_like(y)
        r = y.copy()
        p = r.copy()
        rr = np.vdot(r, r).real
        y2 = max(np.vdot(y, y).real, 1e-300)
        for _ in range(10 * len(y) + 100):
            if rr <= CG_TOL ** 2 * y2:
                break
            Sp = self.S_AA(A, p)
            al = rr / np.vdot(p, Sp).real
            x = x + al * p
            r = r - al * Sp
            rr_new = np.vdot(r, r).real
            p = r + (rr_new / rr) * p
            rr = rr_new
        return x

    def factors(self, q0, p0, width, which):
        """Per-mode normalised DVR packet vectors, mapped by G^dagger (the
        coefficients) or B^dagger (the bra of the autocorrelation)."""
        f = pruned.packet_factors(self.xs, self.ws, q0, p0, width, models.gaussian_1d)
        Ms = self.Gs if which == "G" else self.Bs
        return [M.conj().T @ fk for M, fk in zip(Ms, f)]


def sil_step_S(prob, A, a, K, dt):
    """Lanczos of order K in the S inner product (full re-orthogonalisation,
    classical Gram-Schmidt twice): w = S^-1 H v_k, alpha_k = v_k^dag H v_k,
    <v_i, w>_S = v_i^dag S w, beta_k = ||w||_S."""
    Sa = prob.S_AA(A, a)
    beta0 = np.sqrt(max(np.vdot(a, Sa).real, 0.0))
    if beta0 == 0.0:
        return a.copy()
    V = [a / beta0]
    alpha, beta = [], []
    for k in range(K):
        Hv = prob.H_AA(A, V[k])
        alpha.append(float(np.vdot(V[k], Hv).real))
        if k == K - 1:
            break
        w = prob.solve_S(A, Hv)
        for _ in range(2):
            Sw = prob.S_AA(A, w)
            c = [np.vdot(v, Sw) for v in V]
            for ci, v in zip(c, V):
                w = w - ci * v
        b = np.sqrt(max(np.vdot(w, prob.S_AA(A, w)).real, 0.0))
        if b <= 1e-12 * np.sqrt(max(np.vdot(Hv, Hv).real, 1e-300)) / max(1.0, prob.smax):
            break
        beta.append(b)
        V.append(w / b)
    from .sil import tridiag_exp_e1
    c = tridiag_exp_e1(alpha, beta, dt)
    return beta0 * sum(ci * v for ci, v in zip(c, V))


def run(prob, q0, p0, width, theta, K, dt, nsteps, radius=1):
    """Propagation with adaption on the pvB coefficients (Sec. 2.5)."""
    fa = prob.factors(q0, p0, width, "G")
    fb = prob.factors(q0, p0, width, "B")
    full = np.arange(int(np.prod(prob.dims)), dtype=np.int64)
    a_full = pruned.product_on(full, prob.dims, fa)
    S0 = full[pruned.significant(a_full, theta)]
    A = pruned.adapt_set(S0, prob.axes, radius)
    a = pruned.product_on(A, prob.dims, fa)

    def obs(A, a):
        c = pruned.product_on(A, prob.dims, fb)
        n2 = float(np.vdot(a, prob.S_AA(A, a)).real)
        E = float(np.vdot(a, prob.H_AA(A, a)).real) / n2 if n2 > 0 else 0.0
        return dict(C=complex(np.vdot(c, a)), norm2=n2, E=E, n_active=len(A))

    out = [obs(A, a)]
    for _ in range(nsteps):
        a = sil_step_S(prob, A, a, K, dt)
        A, a = pruned.prune(A, a, prob.axes, theta, radius)
        out.append(obs(A, a))
    return dict(obs=out, A=A, a=a)
