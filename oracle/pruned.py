"""Pruned H.a, the adaption set function and the observables (FP64).

Notation follows Sec. 2.1 and Sec. 2.2.2: a multi-index I = i_1..i_D, the
active set A is a subset of the direct-product lattice, stored as sorted
int64 row-major linear indices (last mode fastest).
"""
from __future__ import annotations

import itertools

import numpy as np


def strides_of(dims):
    """Row-major strides of the lattice (last mode has stride 1)."""
    s = [1] * len(dims)
    for k in range(len(dims) - 2, -1, -1):
        s[k] = s[k + 1] * int(dims[k + 1])
    return s


def digits(A, dims):
    """The multi-index digits i_kappa of every active point, shape (D, N)."""
    return np.array(np.unravel_index(np.asarray(A, dtype=np.int64), dims),
                    dtype=np.int64).reshape(len(dims), -1)


DENSE_MAP_LIMIT = 1 << 28


class PositionMap:
    """Position of every lattice point in the sorted active set A (-1 when
    not active): the set semantics of the paper's hash set (Sec. 2.5) as a
    dense table for lattices up to DENSE_MAP_LIMIT points (int32 entries, so
    that a 24^6 lattice takes 0.8 GB), else a binary search in A."""

    def __init__(self, A, nfull):
        self.A = np.asarray(A, dtype=np.int64)
        self.dense = None
        if nfull <= DENSE_MAP_LIMIT and len(self.A) < (1 << 31):
            self.dense = np.full(int(nfull), -1, dtype=np.int32)
            self.dense[self.A] = np.arange(len(self.A), dtype=np.int32)

    def __call__(self, keys):
        if self.dense is not None:
            ok = (keys >= 0) & (keys < len(self.dense))
            p = np.where(ok, self.dense[np.where(ok, keys, 0)], -1).astype(np.int64)
            found = p >= 0
            return np.where(found, p, 0), found
        return lookup(self.A, keys)


def lookup(A, keys):
    """Positions of ``keys`` in the sorted array A and a found-mask."""
    A = np.asarray(A, dtype=np.int64)
    pos = np.searchsorted(A, keys)
    pos_c = np.minimum(pos, max(len(A) - 1, 0))
    found = (pos < len(A)) & (A[pos_c] == keys) if len(A) else np.zeros(len(keys), bool)
    return pos_c, found


def potential_diag(A, dims, grids, vfunc):
    """V_II = V(x_I) at every active point (DVR potential is diagonal,
    Sec. 2.1 and Sec. 2.5)."""
    dg = digits(A, dims)
    q = np.stack([np.asarray(grids[k])[dg[k]] for k in range(len(dims))], axis=-1)
    return vfunc(q)


# Lattices up to this many points take the whole-lattice form of the pruned
# products below (the coefficients embedded in the lattice with exact zeros
# off A, each 1D operator applied along its mode by numpy's tensordot, the
# result read back on A): the same sum as the member-by-member form, whose
# absent members would only add exact zeros.  Larger lattices (24^6) use the
# member-by-member form.
WHOLE_LATTICE_LIMIT = 1 << 22


def _embed(A, x, dims):
    full = np.zeros(int(np.prod(dims)), dtype=np.complex128)
    full[A] = x
    return full.reshape(tuple(int(d) for d in dims))


def _along(h, full, kappa):
    """The matrix h applied along mode kappa of a whole-lattice array."""
    return np.moveaxis(np.tensordot(np.asarray(h), full, axes=([1], [kappa])), 0, kappa)


def apply_H(A, psi, dims, Ts, vdiag):
    """y = P_A H P_A a on the active set, for a DVR Hamiltonian
    H = sum_kappa T^(kappa) (x) 1 + V with diagonal V (Sec. 2.1, Sec. 2.2.2
    pruned sets I, J(i), K(i,j); Appendix, last-dimension transform).

    Written as the definition y_I = sum_{J in A} H_IJ a_J: for a kinetic factor
    along mode kappa, H_IJ = T_{i_kappa j_kappa} when I and J agree in every
    other digit, so J runs over I[kappa -> j] for j = 0..n_kappa-1 and only the
    members of A contribute.  ``vdiag`` holds V(x_I) for I in A.
    """
    A = np.asarray(A, dtype=np.int64)
    psi = np.asarray(psi, dtype=np.complex128)
    y = np.asarray(vdiag, dtype=np.float64) * psi
    if len(A) == 0:
        return y
    if int(np.prod(dims)) <= WHOLE_LATTICE_LIMIT:
        full = _embed(A, psi, dims)
        for k in range(len(dims)):
            y += _along(np.asarray(Ts[k], dtype=np.float64), full, k).reshape(-1)[A]
        return y
    dg = digits(A, dims)
    st = strides_of(dims)
    where = PositionMap(A, int(np.prod(dims)))
    for kappa, n in enumerate(dims):
        T = np.asarray(Ts[kappa], dtype=np.float64)
        ik = dg[kappa]
        for j in range(int(n)):
            target = A + (j - ik) * st[kappa]
            pos, found = where(target)
            y[found] += T[ik[found], j] * psi[pos[found]]
    return y


def apply_H_at(A, psi, dims, Ts, vdiag_at, pos):
    """The same definition as ``apply_H`` evaluated only at the output
    positions ``pos`` (indices into A); ``vdiag_at`` holds V(x_I) there.  Used
    to check large cases on a sample of outputs."""
    A = np.asarray(A, dtype=np.int64)
    psi = np.asarray(psi, dtype=np.complex128)
    pos = np.asarray(pos, dtype=np.int64)
    I = A[pos]
    y = np.asarray(vdiag_at, dtype=np.float64) * psi[pos]
    dg = digits(I, dims)
    st = strides_of(dims)
    for kappa, n in enumerate(dims):
        T = np.asarray(Ts[kappa], dtype=np.float64)
        ik = dg[kappa]
        for j in range(int(n)):
            target = I + (j - ik) * st[kappa]
            p, found = lookup(A, target)
            y[found] += T[ik[found], j] * psi[p[found]]
    return y


def mode_apply(A, x, dims, kappa, h):
    """P_A (h along mode kappa) x: y_I = sum_j h[i_kappa, j] x(I[kappa -> j])
    over I[kappa -> j] in A, for I in A -- one step of the pruned sequential
    transform of Sec. 2.2.2 (the sets I, J(i), K(i,j) restrict both the
    summation and the result to the active set)."""
    A = np.asarray(A, dtype=np.int64)
    x = np.asarray(x, dtype=np.complex128)
    y = np.zeros(len(A), dtype=np.complex128)
    if len(A) == 0:
        return y
    if int(np.prod(dims)) <= WHOLE_LATTICE_LIMIT:
        return _along(h, _embed(A, x, dims), kappa).reshape(-1)[A]
    dg = digits(A, dims)
    st = strides_of(dims)
    where = PositionMap(A, int(np.prod(dims)))
    h = np.asarray(h)
    ik = dg[kappa]
    for j in range(int(dims[kappa])):
        pos, found = where(A + (j - ik) * st[kappa])
        y[found] += h[ik[found], j] * x[pos[found]]
    return y


def apply_H_sop(A, a, dims, terms):
    """Pruned H.a for an SoP Hamiltonian with dense 1D factors (Sec. 2.2.2):
    for every term (coef, {mode: matrix}) the factors are applied one mode at
    a time, last mode first (the order of Eq. matvecprod_sequential), each
    result truncated to the active set; terms with no factor are coef * a."""
    a = np.asarray(a, dtype=np.complex128)
    y = np.zeros(len(a), dtype=np.complex128)
    for coef, facs in terms:
        x = a
        for kappa in sorted(facs, reverse=True):
            x = mode_apply(A, x, dims, kappa, facs[kappa])
        y += coef * x
    return y


# Neighbour rules of Sec. 3.1 ("phase-space ball radius" on the lattice axes).
RADIUS_1 = 1        # +-1 along one axis: 2k neighbours on k axes
RADIUS_SQRT2 = 2    # radius sqrt(2): also +-1 along two axes at once: 2k^2 neighbours
RADIUS_2 = 3        # radius 2: +-1 or 0 along every axis at once: 3^k - 1 neighbours


def neighbour_offsets(axes, radius=RADIUS_1):
    """The phase-space-ball neighbour rule of Sec. 3.1 on a lattice with the
    given axes, as offset vectors with entries in {-1, 0, +1}: radius 1 moves
    along one axis, radius sqrt(2) along one or two axes, radius 2 along any
    number of axes (all 3^k - 1 non-zero offsets)."""
    k = len(axes)
    if radius not in (RADIUS_1, RADIUS_SQRT2, RADIUS_2):
        raise ValueError(f"unknown neighbour rule {radius}")
    maxmoved = {RADIUS_1: 1, RADIUS_SQRT2: 2, RADIUS_2: k}[radius]
    out = []
    for off in itertools.product((-1, 0, 1), repeat=k):
        moved = sum(1 for d in off if d)
        if 1 <= moved <= maxmoved:
            out.append(off)
    return out


def significant(psi, theta):
    """The keep-test of Sec. 2.5: |a_I| >= theta, evaluated as
    fl(fl(re*re) + fl(im*im)) >= fl(theta*theta) in FP64 (FP32 inputs are
    widened exactly first)."""
    p = np.asarray(psi).astype(np.complex128)
    re, im = p.real, p.imag
    mag2 = re * re + im * im
    return mag2 >= np.float64(theta) * np.float64(theta)


def adapt_set(S, axes, radius=1):
    """A' = S union N(S) as a sorted array (N: lattice neighbours, clipped at
    the lattice edges, Sec. 2.5 and Sec. 3.1)."""
    S = np.asarray(S, dtype=np.int64)
    if len(S) == 0:
        return np.zeros(0, np.int64)
    cand = [S]
    dg = digits(S, axes)
    st = strides_of(axes)
    for off in neighbour_offsets(axes, radius):
        ok = np.ones(len(S), dtype=bool)
        delta = 0
        for a, d in enumerate(off):
            if d:
                nd = dg[a] + d
                ok &= (nd >= 0) & (nd < axes[a])
                delta += d * st[a]
        cand.append(S[ok] + delta)
    return np.unique(np.concatenate(cand))


def prune(A, psi, axes, theta, radius=RADIUS_1, rel_excl=0.0):
    """Adaption of Sec. 2.5 (one threshold theta, nearest neighbours of
    Sec. 3.1).  S = {I in A : |a_I| >= theta};  A' = S union N(S), where N adds
    the lattice neighbours (clipped at the lattice edges).  With the relative
    exclusion threshold rel_excl (Sec. 2.5: functions are excluded only when
    their number exceeds a fraction of the set), the members of A outside
    A' stay when there are at most rel_excl * |A| of them.  Coefficients of
    members of A that stay are kept; newly added members start at zero.

    ``axes`` are the lattice axes (one per DVR mode, two -- x and p -- per
    phase-space mode); the row-major linear index over the axes equals the one
    over the modes.  Returns (A', a').
    """
    A = np.asarray(A, dtype=np.int64)
    psi = np.asarray(psi)
    Anew = adapt_set(A[significant(psi, theta)], axes, radius)
    if rel_excl > 0.0:
        _, inside = lookup(Anew, A)
        n_out = int(np.count_nonzero(~inside))
        if n_out <= rel_excl * len(A):
            Anew = np.union1d(Anew, A)
    pos, found = lookup(A, Anew)
    out = np.zeros(len(Anew), dtype=psi.dtype if psi.dtype.kind == "c" else np.complex128)
    out[found] = psi[pos[found]]
    return Anew, out


def packet_factors(grids, weights, q0, p0, width, gfunc):
    """Per-mode coefficient vectors of a product packet, a^k_i =
    sqrt(w_i) g_k(x_i) (DVR projection, Eq. pvN_def of Sec. 2.2), each normalised; the
    normalised full-lattice packet is their direct product."""
    out = []
    for k in range(len(grids)):
        v = np.sqrt(np.asarray(weights[k])) * gfunc(np.asarray(grids[k]), q0[k], p0[k], width[k])
        out.append(v / np.linalg.norm(v))
    return out


def product_on(A, dims, factors):
    """The product state prod_k f^k_{i_k} at the active points."""
    dg = digits(A, dims)
    v = np.ones(len(dg[0]) if len(dims) else 0, dtype=np.complex128)
    for k in range(len(dims)):
        v = v * np.asarray(factors[k])[dg[k]]
    return v


def autocorrelation(A, psi, a0_on_A):
    """C(t) = <Psi(0)|Psi(t)> = sum_{I in A(t)} conj(a0_I) a_I(t) (Eq. acorr)."""
    return np.vdot(a0_on_A, np.asarray(psi, dtype=np.complex128))
