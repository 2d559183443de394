"""Shared set-up of the GPU parity tests."""
import numpy as np

import workloads as W


def lib():
    import paper_1606_04004_gb300 as pq
    return pq


def random_sop(dims, seed, nterms=3):
    """Random diagonal SoP potential terms: (coef, [values or None per mode])."""
    rng = np.random.default_rng(seed)
    terms = []
    for t in range(nterms):
        f = []
        for k, n in enumerate(dims):
            f.append(rng.uniform(-1, 1, n) if rng.random() < 0.7 else None)
        terms.append((float(rng.uniform(-2, 2)), f))
    return terms


def vdiag_of(terms, A, dims):
    """V(x_I) = sum_t c_t prod_k f_tk(i_k) at the active points (the test's
    own evaluation of the random potential, given to the oracle)."""
    from oracle import pruned
    dg = pruned.digits(A, dims)
    v = np.zeros(len(A))
    for c, f in terms:
        p = np.full(len(A), c)
        for k in range(len(dims)):
            if f[k] is not None:
                p = p * np.asarray(f[k])[dg[k]]
        v += p
    return v


def ho_problem(dims, seed, nterms=3):
    """Library basis (HO DVR modes, kinetic + random potential) and the
    oracle's kinetic matrices and potential for the same lattice."""
    from oracle import bases
    pq = lib()
    b = pq.Basis([dict(kind=pq.HO_DVR, n=int(n), mass=1.0, omega=1.0) for n in dims])
    pot = random_sop(dims, seed, nterms)
    terms = [(1.0, ["T" if k == m else None for k in range(len(dims))]) for m in range(len(dims))]
    b.set_sop(terms + pot)
    Ts = [bases.ho_dvr(int(n))[2] for n in dims]
    return b, Ts, pot


def fgh_problem(dims, seed, nterms=3, box=(-1.0, 2.0), mass=3.0):
    """Library basis (FGH DVR modes of any length up to 256, kinetic + random
    potential) and the oracle's kinetic matrices for the same lattice."""
    from oracle import bases
    pq = lib()
    b = pq.Basis([dict(kind=pq.FGH_DVR, n=int(n), xmin=box[0], xmax=box[1], mass=mass)
                  for n in dims])
    pot = random_sop(dims, seed, nterms)
    terms = [(1.0, ["T" if k == m else None for k in range(len(dims))]) for m in range(len(dims))]
    b.set_sop(terms + pot)
    Ts = [bases.fgh_dvr(int(n), box[0], box[1], mass)[2] for n in dims]
    return b, Ts, pot


def state_with(b, A, psi, precision):
    """A library state on basis b loaded with (A, psi)."""
    pq = lib()
    D = b.D
    s = pq.State(b, [0.0] * D, [0.0] * D, [1.0] * D, 1e30, precision=precision)
    s.load(A, psi)
    return s


def rel_bound(Ts, A, psi, dims, vdiag):
    """Per-element scale of H.psi: the same sum with |T|, |psi|, |V| (for
    rounding-error tolerances)."""
    from oracle import pruned
    return pruned.apply_H(A, np.abs(psi).astype(np.complex128), dims, [np.abs(T) for T in Ts],
                          np.abs(vdiag)).real
