"""Pins of the FP64 oracle against what the paper and the mathematics fix:
closed forms, library routines of a different construction, dense brute
force on tiny lattices.  Each test names the mistake it would catch."""
import itertools

import numpy as np
import pytest
import scipy.linalg

import workloads as W
from oracle import bases, models, pruned, sil, propagate


# ---------------------------------------------------------------- 1D bases

def test_fgh_free_particle_spectrum():
    # Closed form: on a periodic box of length L the FGH DVR is exact for the
    # plane waves it carries, so the eigenvalues of T are (2 pi l / L)^2 / 2m
    # for l = -(n-1)//2 .. n//2 (catches a wrong L, mass, grid or Nyquist term).
    for n, lo, hi, m in [(165, -0.5, 3.7, 200.0), (81, 1.0, 2.9, 200.0), (8, 0.0, 1.0, 1.0)]:
        x, w, T = bases.fgh_dvr(n, lo, hi, m)
        L = hi - lo
        l = np.arange(-((n - 1) // 2), n // 2 + 1)
        ref = np.sort((2 * np.pi * l / L) ** 2 / (2 * m))
        np.testing.assert_allclose(np.sort(np.linalg.eigvalsh(T)), ref, rtol=1e-12,
                                   atol=1e-12 * ref.max())
        np.testing.assert_allclose(np.diff(x), L / n, rtol=1e-12)
        assert x[0] == lo and abs(x[-1] + L / n - hi) < 1e-12
        np.testing.assert_allclose(w, L / n, rtol=1e-15)


def test_fgh_is_circulant_and_gives_ho_levels():
    # a periodic DVR's T depends on (i - j) mod n only; on a wide box it gives
    # the HO levels n + 1/2 (catches an asymmetric or mis-phased kernel).
    x, w, T = bases.fgh_dvr(64, -8.0, 8.0, 1.0)
    for s in range(1, 64):
        np.testing.assert_allclose(np.diag(np.roll(T, s, axis=1)), np.roll(T, s, axis=1)[0, 0],
                                   atol=1e-13)
    ev = np.linalg.eigvalsh(T + np.diag(0.5 * x * x))
    np.testing.assert_allclose(ev[:10], np.arange(10) + 0.5, atol=1e-10)


def test_sine_dvr_free_particle_levels():
    # Closed form: a particle in a box of length L has E_k = (k pi / L)^2 / 2m,
    # and the sine DVR is exact for it for k <= n (catches a wrong U, L or m).
    for n, lo, hi, m in [(32, 0.5, 6.0, 1836.0), (7, -1.0, 2.5, 1.0)]:
        x, w, T = bases.sine_dvr(n, lo, hi, m)
        L = hi - lo
        ev = np.linalg.eigvalsh(T)
        ref = (np.arange(1, n + 1) * np.pi / L) ** 2 / (2 * m)
        np.testing.assert_allclose(ev, ref, rtol=1e-12)
        assert np.all(np.diff(x) > 0) and x[0] > lo and x[-1] < hi
        np.testing.assert_allclose(np.diff(x), L / (n + 1), rtol=1e-12)
        np.testing.assert_allclose(T, T.T, atol=0)


def test_ho_dvr_levels_fig1_setup():
    # Fig. 1 setup, H = (-d^2/dx^2 + x^2)/2: levels n + 1/2 (closed form).
    # With a different m and omega: omega (n + 1/2) for V = m omega^2 x^2 / 2.
    # (x^2 at the nodes differs from the FBR x^2 only in the top basis
    # function, so the lower half of the spectrum is exact.)
    for n, m, om in [(100, 1.0, 1.0), (24, 2.0, 0.5)]:
        x, w, T = bases.ho_dvr(n, m, om)
        ev = np.linalg.eigvalsh(T + np.diag(0.5 * m * om * om * x * x))
        ref = om * (np.arange(n) + 0.5)
        np.testing.assert_allclose(ev[:n // 2], ref[:n // 2], rtol=1e-11, atol=1e-12)
        if n == 100:
            # the first 42 states of Fig. 1
            np.testing.assert_allclose(ev[:42], ref[:42], rtol=1e-12)


def test_ho_dvr_nodes_weights_vs_gauss_hermite():
    # The HO DVR for m = omega = 1 is the Gauss-Hermite quadrature: nodes are
    # the roots of H_n and sqrt-weights turn grid values into coefficients:
    # w_i = W_i exp(x_i^2) with W_i the Gauss-Hermite weights (numpy builds
    # them by a different route).
    n = 24
    x, w, T = bases.ho_dvr(n)
    gx, gw = np.polynomial.hermite.hermgauss(n)
    np.testing.assert_allclose(x, gx, rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(w, gw * np.exp(gx * gx), rtol=1e-10)


def test_sine_dvr_morse_levels():
    # Textbook Morse levels E_n = w(n+1/2) - [w(n+1/2)]^2/(4 De),
    # w = a sqrt(2 De / m): catches a wrong mass or potential in the DVR.
    De, a, m = 0.1, 1.0, 1836.0
    x, w, T = bases.sine_dvr(96, 0.5, 6.0, m)
    V = models.coupled_morse(x[:, None], De, a, 2.0, 0.0)
    ev = np.linalg.eigvalsh(T + np.diag(V))
    om = a * np.sqrt(2 * De / m)
    nn = np.arange(6) + 0.5
    ref = om * nn - (om * nn) ** 2 / (4 * De)
    np.testing.assert_allclose(ev[:6], ref, rtol=1e-8)


def test_henon_heiles_saddle():
    # 2D Henon-Heiles: saddle at (0, 1/lam) with V = 1/(6 lam^2), zero
    # gradient (catches a wrong sign or power in the cubic terms).
    lam = 0.111803
    q = np.array([0.0, 1.0 / lam])
    assert abs(models.henon_heiles(q, lam) - 1 / (6 * lam ** 2)) < 1e-9
    for qs in ([0.0, 1 / lam], [np.sqrt(3) / (2 * lam), -1 / (2 * lam)]):
        qs = np.array(qs)
        g = []
        for k in range(2):
            e = np.zeros(2); e[k] = 1e-5
            g.append((models.henon_heiles(qs + e, lam) - models.henon_heiles(qs - e, lam)) / 2e-5)
        np.testing.assert_allclose(g, 0, atol=1e-6)
        assert abs(models.henon_heiles(qs, lam) - 1 / (6 * lam ** 2)) < 1e-9


def test_gaussian_packet_moments():
    # The packet is fixed by its moments: unit norm, <x> = q0, variance s^2,
    # and <p> = p0 (from the DFT of the grid values; a real Hamiltonian's C(t)
    # cannot tell p0 from -p0, so the sign is pinned here).
    x = np.linspace(-20.0, 20.0, 4096, endpoint=False)
    dx = x[1] - x[0]
    k = 2 * np.pi * np.fft.fftfreq(len(x), d=dx)
    for q0, p0, s in ((0.3, 2.5, 0.7), (-1.0, -4.0, 1.3), (2.0, 0.0, 0.5 ** 0.5)):
        g = models.gaussian_1d(x, q0, p0, s)
        rho = np.abs(g) ** 2 * dx
        assert abs(rho.sum() - 1.0) < 1e-12
        assert abs((x * rho).sum() - q0) < 1e-12
        assert abs(((x - q0) ** 2 * rho).sum() - s * s) < 1e-12
        F = np.abs(np.fft.fft(g)) ** 2
        assert abs((k * F).sum() / F.sum() - p0) < 1e-10


# ------------------------------------------------------------ pruned H.a

def _dense_H(dims, Ts, vfull):
    """Brute force H = sum_k 1 (x) .. T_k .. (x) 1 + diag(V) by Kronecker
    products (row-major: mode 0 is the slowest index)."""
    N = int(np.prod(dims))
    H = np.diag(vfull).astype(np.float64)
    for k in range(len(dims)):
        mats = [np.eye(d) for d in dims]
        mats[k] = Ts[k]
        M = mats[0]
        for mm in mats[1:]:
            M = np.kron(M, mm)
        H += M
    assert H.shape == (N, N)
    return H


@pytest.mark.parametrize("dims,frac,seed", [((6, 5), 0.5, 1), ((4, 5, 3), 0.4, 2),
                                            ((3, 2, 4, 3), 0.6, 3), ((9,), 0.7, 4),
                                            ((4, 5, 3), 1.0, 5)])
def test_pruned_apply_equals_PHP(dims, frac, seed):
    # y = P_A H P_A a exactly for a DVR (diagonal V), and A = full gives the
    # unpruned H (Sec. 2.2.2 / appendix).  Catches a transposed T, a wrong
    # stride or digit, or a dropped mode.
    rng = np.random.default_rng(seed)
    Ts = []
    for d in dims:
        M = rng.standard_normal((d, d))
        Ts.append(M)                      # non-symmetric: catches T vs T^T
    N = int(np.prod(dims))
    vfull = rng.standard_normal(N)
    A = W.random_active_set(dims, frac, seed)
    psi = W.random_psi(len(A), seed + 10)
    y = pruned.apply_H(A, psi, dims, Ts, vfull[A])
    H = _dense_H(dims, Ts, vfull)
    ref = H[np.ix_(A, A)] @ psi
    np.testing.assert_allclose(y, ref, rtol=1e-12, atol=1e-12)


class member_form:
    """Run the oracle's pruned products in their member-by-member form (the
    one large lattices take) instead of the whole-lattice form."""

    def __enter__(self):
        self.old = pruned.WHOLE_LATTICE_LIMIT
        pruned.WHOLE_LATTICE_LIMIT = 0

    def __exit__(self, *a):
        pruned.WHOLE_LATTICE_LIMIT = self.old


@pytest.mark.parametrize("dims,frac,seed", [((6, 5), 0.5, 1), ((4, 5, 3), 0.4, 2),
                                            ((3, 4, 2, 3), 0.3, 3), ((7,), 0.6, 4),
                                            ((4, 5, 3), 1.0, 5)])
def test_pruned_apply_member_form_equals_PHP(dims, frac, seed):
    # the same pin on the member-by-member form of the pruned product
    with member_form():
        test_pruned_apply_equals_PHP(dims, frac, seed)


def test_pruned_apply_forms_agree():
    # the whole-lattice and the member-by-member forms add the same terms (an
    # absent member contributes an exact zero): equal to rounding
    dims = (5, 6, 4)
    rng = np.random.default_rng(21)
    Ts = [rng.standard_normal((d, d)) for d in dims]
    A = W.random_active_set(dims, 0.35, 21)
    psi = W.random_psi(len(A), 22)
    v = rng.standard_normal(len(A))
    y1 = pruned.apply_H(A, psi, dims, Ts, v)
    with member_form():
        y2 = pruned.apply_H(A, psi, dims, Ts, v)
    np.testing.assert_allclose(y1, y2, rtol=1e-13, atol=1e-13)


def test_pruned_apply_at_sample_equals_full():
    dims = (5, 4, 6)
    rng = np.random.default_rng(11)
    Ts = [rng.standard_normal((d, d)) for d in dims]
    A = W.random_active_set(dims, 0.5, 11)
    psi = W.random_psi(len(A), 12)
    v = rng.standard_normal(len(A))
    y = pruned.apply_H(A, psi, dims, Ts, v)
    pos = np.array([0, 3, len(A) - 1, len(A) // 2])
    np.testing.assert_allclose(pruned.apply_H_at(A, psi, dims, Ts, v[pos], pos), y[pos],
                               rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("dims", [(4, 4, 4), (3, 5, 4)])
def test_lattice_helpers_match_library_constructions(dims):
    # Row-major lattice bookkeeping against numpy's own constructions:
    # strides and digits (ravel_multi_index / indices by another route), V on
    # the full lattice against meshgrid(indexing="ij"), and the product packet
    # against a chain of Kronecker products.  Equal mode sizes make a reversed
    # mode order give wrong numbers rather than an index error; an asymmetric
    # V and distinct factors make it visible.
    N = int(np.prod(dims))
    full = np.arange(N, dtype=np.int64)
    st = pruned.strides_of(dims)
    for e in itertools.product(*[range(d) for d in dims]):
        assert sum(i * s for i, s in zip(e, st)) == np.ravel_multi_index(e, dims)
    np.testing.assert_array_equal(pruned.digits(full, dims),
                                  np.indices(dims).reshape(len(dims), -1))
    rng = np.random.default_rng(21)
    grids = [np.sort(rng.uniform(-1, 1, d)) for d in dims]
    vf = lambda q: q[..., 0] + 10 * q[..., 1] ** 2 + 100 * q[..., 2] ** 3
    mesh = np.stack(np.meshgrid(*grids, indexing="ij"), axis=-1)
    np.testing.assert_allclose(pruned.potential_diag(full, dims, grids, vf),
                               vf(mesh).ravel(), rtol=1e-15, atol=1e-15)
    facs = [rng.standard_normal(d) + 1j * rng.standard_normal(d) for d in dims]
    dense = np.kron(np.kron(facs[0], facs[1]), facs[2])
    np.testing.assert_allclose(pruned.product_on(full, dims, facs), dense, rtol=1e-15)
    A = W.random_active_set(dims, 0.5, 22)
    np.testing.assert_allclose(pruned.product_on(A, dims, facs), dense[A], rtol=1e-15)


def test_pruned_apply_empty():
    y = pruned.apply_H(np.zeros(0, np.int64), np.zeros(0, complex), (3, 4),
                       [np.eye(3), np.eye(4)], np.zeros(0))
    assert y.shape == (0,)


# ------------------------------------------------------------------ prune

def _brute_prune(A, psi, axes, theta):
    """Every lattice point L is tested directly against the rule of Sec. 2.5:
    L is kept iff L itself or one of its +-1 axis neighbours is an active
    point with |a| >= theta."""
    Aset = {int(i): k for k, i in enumerate(A)}
    big = {int(i) for k, i in enumerate(A) if abs(complex(psi[k])) ** 2 >= theta * theta}
    out, coef = [], []
    for L in range(int(np.prod(axes))):
        dig = np.unravel_index(L, axes)
        keep = L in big
        for a in range(len(axes)):
            for s in (-1, 1):
                d = list(dig); d[a] += s
                if 0 <= d[a] < axes[a] and int(np.ravel_multi_index(d, axes)) in big:
                    keep = True
        if keep:
            out.append(L)
            coef.append(psi[Aset[L]] if L in Aset else 0)
    return np.array(out, dtype=np.int64), np.array(coef, dtype=complex)


@pytest.mark.parametrize("axes,seed", [((7, 6), 0), ((4, 3, 5), 1), ((2, 2, 2, 3), 2), ((11,), 3)])
def test_prune_bruteforce(axes, seed):
    rng = np.random.default_rng(seed)
    A = W.random_active_set(axes, 0.5, seed)
    theta = 0.3
    psi = (rng.uniform(0, 0.6, len(A)) * np.exp(2j * np.pi * rng.random(len(A))))
    # exact ties |a| = theta (real, representable) must be kept
    psi[::5] = theta
    An, pn = pruned.prune(A, psi, axes, theta)
    Ab, pb = _brute_prune(A, psi, axes, theta)
    np.testing.assert_array_equal(An, Ab)
    np.testing.assert_array_equal(pn, pb)


def test_prune_edges_and_empty():
    # one significant point in a corner: only in-lattice neighbours are added
    An, pn = pruned.prune(np.array([0]), np.array([1.0 + 0j]), (3, 4), 0.5)
    np.testing.assert_array_equal(An, [0, 1, 4])
    np.testing.assert_array_equal(pn, [1, 0, 0])
    An, pn = pruned.prune(np.array([0, 5]), np.array([0.1, 0.2 + 0j]), (3, 4), 0.5)
    assert len(An) == 0 and len(pn) == 0


def _brute_prune_ball(A, psi, axes, theta, radius, rel_excl=0.0):
    """The neighbour rules of Sec. 3.1 written as distances on the lattice: a
    point L is kept iff some significant active point P has
    max_a |L_a - P_a| <= 1 and sum_a (L_a - P_a)^2 <= r^2, with r = 1,
    sqrt(2) or 2 ("phase-space ball radius").  Relative exclusion (Sec. 2.5):
    when at most rel_excl * |A| members of A would leave, none leave."""
    r2 = {pruned.RADIUS_1: 1, pruned.RADIUS_SQRT2: 2, pruned.RADIUS_2: 4}[radius]
    big = [np.array(np.unravel_index(int(i), axes)) for k, i in enumerate(A)
           if abs(complex(psi[k])) ** 2 >= theta * theta]
    keep = set()
    for L in range(int(np.prod(axes))):
        dig = np.array(np.unravel_index(L, axes))
        for P in big:
            d = np.abs(dig - P)
            if d.max() <= 1 and int((d * d).sum()) <= r2:
                keep.add(L)
                break
    leaving = [int(i) for i in A if int(i) not in keep]
    if rel_excl > 0 and len(leaving) <= rel_excl * len(A):
        keep |= {int(i) for i in A}
    Aset = {int(i): k for k, i in enumerate(A)}
    out = sorted(keep)
    coef = [psi[Aset[L]] if L in Aset else 0 for L in out]
    return np.array(out, dtype=np.int64), np.array(coef, dtype=complex)


def test_neighbour_counts_match_the_paper():
    # Sec. 3.1 counts for an interior point on k lattice axes: 2k neighbours
    # for ball radius 1, 2k^2 for radius sqrt(2), 3^k - 1 for radius 2
    # (catches a missing sign, a missing diagonal pair or a wrong box).
    for k in range(1, 5):
        axes = (5,) * k
        centre = np.array([int(np.ravel_multi_index((2,) * k, axes))])
        for rule, count in [(pruned.RADIUS_1, 2 * k), (pruned.RADIUS_SQRT2, 2 * k * k),
                            (pruned.RADIUS_2, 3 ** k - 1)]:
            assert len(pruned.adapt_set(centre, axes, rule)) == count + 1


@pytest.mark.parametrize("rule", [2, 3])
@pytest.mark.parametrize("axes,seed", [((7, 6), 0), ((4, 3, 5), 1), ((2, 3, 2, 3), 2)])
def test_prune_ball_rules_bruteforce(axes, seed, rule):
    rng = np.random.default_rng(seed + 40)
    A = W.random_active_set(axes, 0.4, seed + 40)
    theta = 0.45
    psi = rng.uniform(0, 0.6, len(A)) * np.exp(2j * np.pi * rng.random(len(A)))
    An, pn = pruned.prune(A, psi, axes, theta, rule)
    Ab, pb = _brute_prune_ball(A, psi, axes, theta, rule)
    np.testing.assert_array_equal(An, Ab)
    np.testing.assert_array_equal(pn, pb)


def test_prune_relative_exclusion_bruteforce():
    # exclusion happens only when more than rel_excl * |A| members would
    # leave; at exactly that many they stay (Sec. 2.5 excludes only above the fraction).
    axes = (6, 5)
    rng = np.random.default_rng(77)
    A = W.random_active_set(axes, 0.6, 77)
    psi = rng.uniform(0, 0.6, len(A)) * np.exp(2j * np.pi * rng.random(len(A)))
    theta = 0.5
    A0, _ = pruned.prune(A, psi, axes, theta)
    n_out = len(np.setdiff1d(A, A0))
    assert 0 < n_out < len(A)
    for rho in (0.0, (n_out - 0.5) / len(A), n_out / len(A), 0.99):
        An, pn = pruned.prune(A, psi, axes, theta, pruned.RADIUS_1, rho)
        Ab, pb = _brute_prune_ball(A, psi, axes, theta, pruned.RADIUS_1, rho)
        np.testing.assert_array_equal(An, Ab)
        np.testing.assert_array_equal(pn, pb)
        assert (len(np.setdiff1d(A, An)) == 0) == (n_out <= rho * len(A))


# -------------------------------------------------------------------- SIL

def test_sil_full_krylov_is_exact_exponential():
    # K = dim: the Krylov space is the whole space and SIL is exp(-iH dt)
    # (catches a wrong sign of i, a wrong e_1 column, bad re-orthogonalisation).
    rng = np.random.default_rng(7)
    n = 12
    M = rng.standard_normal((n, n)); H = (M + M.T) / 2
    psi = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    for dt in (0.05, 0.7):
        out, info = sil.sil_step(psi, lambda v: H @ v, n, dt, return_info=True)
        ref = scipy.linalg.expm(-1j * H * dt) @ psi
        np.testing.assert_allclose(out, ref, rtol=1e-11, atol=1e-11)


def test_rk4_is_fourth_order():
    # against the exact exponential: the one-step error falls as dt^5 and the
    # error over a fixed time as dt^4 (catches a wrong stage weight or sign).
    rng = np.random.default_rng(9)
    n = 12
    M = rng.standard_normal((n, n)); H = (M + M.T) / 2
    psi = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    errs = []
    for dt in (0.02, 0.01):
        a = psi.copy()
        for _ in range(int(round(0.4 / dt))):
            a = sil.rk4_step(a, lambda v: H @ v, dt)
        errs.append(np.linalg.norm(a - scipy.linalg.expm(-1j * H * 0.4) @ psi))
    assert 14.0 < errs[0] / errs[1] < 18.0
    one = [np.linalg.norm(sil.rk4_step(psi, lambda v: H @ v, dt)
                          - scipy.linalg.expm(-1j * H * dt) @ psi) for dt in (0.02, 0.01)]
    assert 28.0 < one[0] / one[1] < 36.0


def test_sil_error_control_meets_tolerance():
    # error-controlled order: the step stops early and its error against the
    # exact exponential stays at the level of the requested tolerance, while
    # tol = 0 keeps the full order (catches an estimate taken at the wrong index)
    rng = np.random.default_rng(10)
    n = 60
    M = rng.standard_normal((n, n)); H = (M + M.T) / 2
    psi = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    psi /= np.linalg.norm(psi)
    ref = scipy.linalg.expm(-1j * H * 0.05) @ psi
    for tol in (1e-6, 1e-10):
        out, info = sil.sil_step(psi, lambda v: H @ v, 30, 0.05, return_info=True, tol=tol)
        assert info["K"] < 30
        assert np.linalg.norm(out - ref) < 10 * tol
    _, info = sil.sil_step(psi, lambda v: H @ v, 30, 0.05, return_info=True)
    assert info["K"] == 30


def test_sil_conserves_norm_and_energy():
    rng = np.random.default_rng(8)
    n = 40
    M = rng.standard_normal((n, n)); H = (M + M.T) / 2
    psi = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    out = sil.sil_step(psi, lambda v: H @ v, 6, 0.1)
    assert abs(np.linalg.norm(out) - np.linalg.norm(psi)) < 1e-12 * np.linalg.norm(psi)
    e0 = np.vdot(psi, H @ psi).real / np.vdot(psi, psi).real
    e1 = np.vdot(out, H @ out).real / np.vdot(out, out).real
    assert abs(e1 - e0) < 1e-12 * max(1, abs(e0))


def test_sil_breakdown_invariant_subspace():
    # psi in a 3-dim invariant subspace: Lanczos stops at 3 vectors and is exact
    rng = np.random.default_rng(9)
    n = 10
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = np.arange(n, dtype=float)
    H = Q @ np.diag(lam) @ Q.T
    psi = Q[:, :3] @ np.array([1.0, 2.0, 0.5])
    out, info = sil.sil_step(psi, lambda v: H @ v, 8, 0.3, return_info=True)
    assert info["K"] == 3
    np.testing.assert_allclose(out, scipy.linalg.expm(-1j * H * 0.3) @ psi, atol=1e-12)


# ------------------------------------------------------- whole propagation

def _dense_problem_H(prob):
    dims = prob.dims
    full = np.arange(int(np.prod(dims)), dtype=np.int64)
    return _dense_H(dims, prob.Ts, prob.vdiag(full))


@pytest.mark.parametrize("p0", [(0.0, 0.0), (0.0, 6.0)])
def test_theta0_is_unpruned_exact_dynamics(p0):
    # theta = 0: the active set is the full lattice at all times and the pruned
    # run is the exact direct-product propagation (Sec. 3.1: at 100 % basis
    # all methods agree).  K = dim makes SIL exact, so the run must equal
    # exp(-i H t) a(0) by dense exponential.  The moving packet (p0 != 0) has
    # complex coefficients, so C(t) also checks the conjugated bra of Eq. acorr.
    cfg = W.scaled(W.MORSE2D, n=6)
    prob = propagate.problem_from_config(cfg)
    N = 36
    r = propagate.run(prob, cfg["q0"], p0, cfg["width"], 0.0, N, 10.0, 5)
    assert all(o["n_active"] == N for o in r["obs"])
    H = _dense_problem_H(prob)
    a0 = pruned.product_on(np.arange(N), prob.dims, r["factors"])
    ref = scipy.linalg.expm(-1j * H * 50.0) @ a0
    np.testing.assert_allclose(r["a"], ref, rtol=1e-10, atol=1e-11)
    # C(t) at every step
    for s, o in enumerate(r["obs"]):
        c = np.vdot(a0, scipy.linalg.expm(-1j * H * 10.0 * s) @ a0)
        assert abs(o["C"] - c) < 1e-10


def test_autocorrelation_2t_identity():
    # Eq. acorr: for a real initial packet in a real DVR, C(2t) = sum_I a_I(t)^2.
    cfg = W.scaled(W.MORSE2D, n=6)
    prob = propagate.problem_from_config(cfg)
    r = propagate.run(prob, cfg["q0"], (0.0, 0.0), cfg["width"], 0.0, 36, 10.0, 6)
    # re-run keeping the states
    A, a, f = propagate.initial_state(prob, cfg["q0"], (0.0, 0.0), cfg["width"], 0.0)
    states = [a]
    for _ in range(3):
        a = sil.sil_step(a, lambda v: prob.apply(A, v), 36, 10.0)
        states.append(a)
    for s in range(4):
        assert abs(r["obs"][2 * s]["C"] - np.sum(states[s] ** 2)) < 1e-11


def test_double_well_autocorrelation_2t_identity():
    # Eq. acorr on the paper's own double well (Sec. 3.1, real packet, real
    # FGH DVR, theta = 0): C(2t) = sum_I a_I(t)^2, at the full grid of 13365
    # points (catches a wrong potential sign or a complex-conjugation slip).
    cfg = W.DWELL2D
    prob = propagate.problem_from_config(cfg)
    r = propagate.run(prob, cfg["q0"], cfg["p0"], cfg["width"], 0.0, cfg["K"], cfg["dt"], 6)
    A, a, f = propagate.initial_state(prob, cfg["q0"], cfg["p0"], cfg["width"], 0.0)
    assert len(A) == 165 * 81
    states = [a]
    for _ in range(3):
        a = sil.sil_step(a, lambda v: prob.apply(A, v), cfg["K"], cfg["dt"])
        states.append(a)
    for s in range(4):
        assert abs(r["obs"][2 * s]["C"] - np.sum(states[s] ** 2)) < 1e-10


def test_hh_lambda0_coherent_state_closed_form():
    # lambda = 0: the HH chain is a sum of HO, the packet at q0 = 2 with
    # standard deviation 1/sqrt 2 is a coherent state, and
    # C(t) = prod_k exp(-it/2) exp(-(q0^2/2)(1 - exp(-it))).
    cfg = W.scaled(W.HH4D, D=2, lam=0.0)
    prob = propagate.problem_from_config(cfg)
    q0 = (2.0, 2.0)
    # K = 16 makes the Krylov error negligible (the DVR is exact to 1e-15 for
    # this packet); K = 10, the workload's order, stays within 1e-9 over 40
    # steps (its per-step truncation error is about 1e-11).
    for K, tol in ((16, 1e-13), (10, 1e-9)):
        r = propagate.run(prob, q0, (0.0, 0.0), cfg["width"], 0.0, K, 0.1, 40)
        for s, o in enumerate(r["obs"]):
            t = 0.1 * s
            ref = np.prod([np.exp(-0.5j * t) * np.exp(-(q * q / 2) * (1 - np.exp(-1j * t)))
                           for q in q0])
            assert abs(o["C"] - ref) < tol, (K, s, o["C"], ref)
            # coherent-state energy: sum_k (q0_k^2 + 1) / 2, conserved
            assert abs(o["E"] - sum((q * q + 1) / 2 for q in q0)) < 1e-10


def test_observables_are_scale_invariant_and_count_wasted():
    # E is the Rayleigh quotient <a|H|a> / <a|a> (independent of the scale of
    # a), norm2 = <a|a>, and the wasted count is the number of active
    # coefficients below theta (brute-force count on a pruned state).
    cfg = W.scaled(W.MORSE2D, n=16)
    prob = propagate.problem_from_config(cfg)
    A, a, f = propagate.initial_state(prob, cfg["q0"], cfg["p0"], cfg["width"], 1e-3)
    a = sil.sil_step(a, lambda v: prob.apply(A, v), 8, 10.0)
    o1 = propagate.observables(prob, A, a, f, 1e-3)
    o2 = propagate.observables(prob, A, 2.0 * a, f, 1e-3)
    H = _dense_problem_H(prob)[np.ix_(A, A)]
    assert abs(o1["E"] - np.vdot(a, H @ a).real / np.vdot(a, a).real) < 1e-14
    assert abs(o2["E"] - o1["E"]) < 1e-14 and abs(o2["norm2"] - 4 * o1["norm2"]) < 1e-13
    assert abs(o1["norm2"] - sum(abs(complex(v)) ** 2 for v in a)) < 1e-13
    assert o1["n_wasted"] == sum(1 for v in a if abs(complex(v)) < 1e-3) > 0
    assert o1["n_active"] == len(A)


def test_initial_state_chunked_equals_full_prune():
    cfg = W.MORSE2D
    prob = propagate.problem_from_config(cfg)
    A, a, f = propagate.initial_state(prob, cfg["q0"], cfg["p0"], cfg["width"], 1e-6, chunk=100)
    full = np.arange(32 * 32)
    Af, af = pruned.prune(full, pruned.product_on(full, prob.dims, f), prob.dims, 1e-6)
    np.testing.assert_array_equal(A, Af)
    np.testing.assert_array_equal(a, af)
    assert abs(np.sum(np.abs(pruned.product_on(full, prob.dims, f)) ** 2) - 1) < 1e-13


@pytest.mark.parametrize("radius", [1, 2])
def test_run_sets_are_adaption_fixed_points(radius):
    # After every adaption (Sec. 2.5) the members of S = {|a| >= theta} keep
    # their coefficients and the added neighbours are below theta (zero or
    # carried), so the significant set of the adapted state is S again and the
    # active set must be exactly S plus its neighbours under the run's rule.
    # Checked on the recorded state of every step of a pruned run.
    cfg = W.scaled(W.MORSE2D, n=16)
    prob = propagate.problem_from_config(cfg)
    theta = 1e-4
    A, a, f = propagate.initial_state(prob, cfg["q0"], cfg["p0"], cfg["width"], theta, radius)
    state = (A, a, f)
    for step in range(6):
        A, a, _ = state
        np.testing.assert_array_equal(
            A, pruned.adapt_set(A[pruned.significant(a, theta)], prob.axes, radius))
        r = propagate.run(prob, cfg["q0"], cfg["p0"], cfg["width"], theta, 8, 10.0, 3,
                          radius=radius, state=state)
        assert r["obs"][-1]["n_active"] == len(r["A"])
        state = (r["A"], r["a"], f)
    assert 0 < len(state[0]) < 16 * 16


def test_pruned_infidelity_decreases_with_theta():
    # Sec. 3.1 (Fig. 2/3 trend): a smaller threshold gives a larger basis and
    # a smaller autocorrelation error against the unpruned run.
    cfg = W.scaled(W.MORSE2D, n=16)
    prob = propagate.problem_from_config(cfg)
    args = (cfg["q0"], cfg["p0"], cfg["width"])
    exact = propagate.run(prob, *args, 0.0, 8, 10.0, 30)
    ce = np.array([o["C"] for o in exact["obs"]])
    errs, sizes = [], []
    for th in (1e-2, 1e-3, 1e-4, 1e-5):
        r = propagate.run(prob, *args, th, 8, 10.0, 30)
        c = np.array([o["C"] for o in r["obs"]])
        errs.append(np.linalg.norm(c - ce))
        sizes.append(np.mean([o["n_active"] for o in r["obs"]]))
    assert all(np.diff(errs) < 0), errs
    assert all(np.diff(sizes) > 0), sizes


# ------------------------------------------------------ phase-space bases

def test_pw_orthonormal_and_similar():
    # Sec. 2.4: W = Phi S^(-1/2) is orthonormal, and the pW Hamiltonian is a
    # similarity transform of the DVR one (same eigenvalues, DVR accuracy).
    x, w, T, W = bases.pw_basis(16, 0.5, 6.0, 1836.0, 4, 4)
    np.testing.assert_allclose(W.T @ W, np.eye(16), atol=1e-12)
    V = np.diag(models.coupled_morse(x[:, None], 0.1, 1.0, 2.0, 0.0))
    H = T + V
    np.testing.assert_allclose(np.linalg.eigvalsh(W.T @ H @ W), np.linalg.eigvalsh(H),
                               rtol=1e-10, atol=1e-14)


def _moments(x, w, T, mass, col):
    """Norm, position centroid and <p^2> of a function given by its DVR
    coefficients col_j = sqrt(w_j) f(x_j): quadrature for the first two,
    the DVR kinetic matrix (<p^2> = 2 m <f|T|f>) for the third."""
    nrm = np.vdot(col, col).real
    xc = np.sum(x * np.abs(col) ** 2) / nrm
    p2 = 2.0 * mass * np.vdot(col, T @ col).real / nrm
    return nrm, xc, p2


@pytest.mark.parametrize("dvr", ["sine", "fgh"])
def test_pw_functions_closed_form_moments(dvr):
    # Eq. sG_def on the doubly dense lattice (Dx Dp = pi, alpha = Dp / 2 Dx):
    # in momentum space phi_ab is two Gaussians of variance alpha at +-p_b plus
    # a cross term proportional to cos(2 p_b s); the shift s = sqrt(pi / 8 alpha)
    # makes 2 p_b s = (2b + 1) pi / 2, so the cross term vanishes and, exactly,
    #   ||phi|| = 1,  <p^2> = p_b^2 + alpha,
    #   <x> - x_a = -(-1)^b (p_b / 2 alpha) exp(-p_b^2 / 2 alpha).
    # Checked by DVR quadrature and the DVR kinetic matrix for functions away
    # from the box edges and the DVR's top momentum (catches a wrong alpha,
    # Dp, shift or its sign, normalisation, or centre).
    n, lo, hi, m, nx, np_ = 96, 0.0, 12.0, 2.0, 12, 8
    x, w, T = (bases.fgh_dvr if dvr == "fgh" else bases.sine_dvr)(n, lo, hi, m)
    Phi = bases.pw_functions(x, w, lo, hi, nx, np_)
    dx = (hi - lo) / nx
    dp = np.pi / dx
    alpha = dp / (2 * dx)
    for a in range(2, nx - 2):
        xa = lo + (a + 0.5) * dx
        for b in range(np_ - 2):
            pb = (b + 0.5) * dp
            nrm, xc, p2 = _moments(x, w, T, m, Phi[:, a * np_ + b])
            assert abs(nrm - 1.0) < 1e-8, (a, b, nrm)
            assert abs(p2 - (pb * pb + alpha)) < 1e-6 * (pb * pb + alpha), (a, b, p2)
            shift = -((-1) ** b) * pb / (2 * alpha) * np.exp(-pb * pb / (2 * alpha))
            assert abs(xc - xa - shift) < 1e-8, (a, b, xc - xa, shift)


def test_pw_is_loewdin_orthogonalisation():
    # Sec. 2.3-2.4: W is the symmetric (Loewdin) orthogonalisation of Phi.  Polar
    # decomposition: W orthogonal and W^T Phi symmetric positive definite fix W
    # uniquely (catches Gram-Schmidt / QR, a transposed U or S^(+1/2)).
    for dvr, (n, lo, hi, nx, np_) in (("sine", (16, 0.5, 6.0, 4, 4)),
                                      ("fgh", (165, -0.5, 3.7, 15, 11))):
        x, w, T, Wm = bases.pw_basis(n, lo, hi, 200.0, nx, np_, dvr)
        Phi = bases.pw_functions(x, w, lo, hi, nx, np_)
        np.testing.assert_allclose(Wm.T @ Wm, np.eye(n), atol=1e-10)
        M = Wm.T @ Phi
        np.testing.assert_allclose(M, M.T, atol=1e-10)
        assert np.linalg.eigvalsh((M + M.T) / 2).min() > 0


@pytest.mark.parametrize("dvr", ["sine", "fgh"])
def test_pvb_functions_closed_form_moments(dvr):
    # Sec. 2.2 von Neumann lattice (Dx Dp = 2 pi, alpha = Dp / 2 Dx, momenta
    # centred on zero): each projected Gaussian has, exactly, ||g|| = 1,
    # <x> = x_a, <p^2> = p_b^2 + alpha and <p> = p_b.  <p> is taken from the
    # discrete Fourier transform of the grid values (a route independent of the
    # DVR); the others as for pW.  Interior functions only.
    n, lo, hi, m, nx, np_ = 96, 0.0, 12.0, 2.0, 12, 8
    x, w, T, G, B = bases.pvb_basis(n, lo, hi, m, nx, np_, dvr)
    dx = (hi - lo) / nx
    dp = 2 * np.pi / dx
    alpha = dp / (2 * dx)
    k = 2 * np.pi * np.fft.fftfreq(n, d=x[1] - x[0])
    for a in range(2, nx - 2):
        xa = lo + (a + 0.5) * dx
        for b in range(1, np_ - 1):
            pb = -np_ * dp / 2 + (b + 0.5) * dp
            col = G[:, a * np_ + b]
            nrm, xc, p2 = _moments(x, w, T, m, col)
            assert abs(nrm - 1.0) < 1e-8, (a, b, nrm)
            assert abs(xc - xa) < 1e-8, (a, b, xc, xa)
            assert abs(p2 - (pb * pb + alpha)) < 1e-7 * (pb * pb + alpha), (a, b, p2)
            F = np.abs(np.fft.fft(col / np.sqrt(w))) ** 2
            assert abs(np.sum(k * F) / np.sum(F) - pb) < 1e-6 * dp, (a, b)


def test_pvb_biorthogonal():
    # Eq. pvb_def: <b_n|g_m> = delta_nm, i.e. B^dagger G = 1 (brute force),
    # and the generalised problem S_b^-1 (B^dag H B) has the DVR eigenvalues.
    x, w, T, G, B = bases.pvb_basis(16, 0.5, 6.0, 1836.0, 4, 4)
    np.testing.assert_allclose(B.conj().T @ G, np.eye(16), atol=1e-10)
    H = T + np.diag(models.coupled_morse(x[:, None], 0.1, 1.0, 2.0, 0.0))
    Hb = B.conj().T @ H @ B
    Sb = B.conj().T @ B
    ev = np.sort(np.linalg.eigvals(np.linalg.solve(Sb, Hb)).real)
    np.testing.assert_allclose(ev, np.linalg.eigvalsh(H), rtol=1e-8, atol=1e-12)


@pytest.mark.parametrize("dims,seed", [((5, 4, 6), 1), ((6, 7), 2), ((3, 4, 2, 3), 3)])
def test_sop_sequential_member_form(dims, seed):
    # the same pin on the member-by-member form of each factor's pass
    with member_form():
        test_sop_sequential_equals_dense_truncated_products(dims, seed)


@pytest.mark.parametrize("dims,seed", [((5, 4, 6), 1), ((6, 7), 2), ((3, 4, 2, 3), 3)])
def test_sop_sequential_equals_dense_truncated_products(dims, seed):
    # Sec. 2.2.2: each factor is applied along its mode with the result
    # truncated to A, last mode first.  Dense reference: P_A K_k P_A ... with
    # K_k the Kronecker embedding of the factor (non-symmetric factors catch
    # transposes; three-factor terms check the order).
    rng = np.random.default_rng(seed)
    D = len(dims)
    A = W.random_active_set(dims, 0.5, seed)
    a = W.random_psi(len(A), seed + 1)
    N = int(np.prod(dims))
    P = np.zeros((N, len(A)))
    P[A, np.arange(len(A))] = 1.0

    def K(k, h):
        mats = [np.eye(d) for d in dims]
        mats[k] = h
        M = mats[0]
        for m in mats[1:]:
            M = np.kron(M, m)
        return M

    terms = []
    for t in range(4):
        modes = sorted(rng.choice(D, size=min(D, t % 3 + 1), replace=False))
        terms.append((float(rng.uniform(-1, 1)),
                      {int(k): rng.standard_normal((dims[k], dims[k])) for k in modes}))
    terms.append((0.7, {}))
    y = pruned.apply_H_sop(A, a, dims, terms)
    ref = np.zeros(len(A), dtype=complex)
    for c, facs in terms:
        x = a.copy()
        for k in sorted(facs, reverse=True):
            x = P.T @ K(k, facs[k]) @ P @ x
        ref += c * x
    np.testing.assert_allclose(y, ref, rtol=1e-12, atol=1e-12)


def test_pw_full_basis_equals_transformed_dvr():
    # With A = the full lattice the pruned sequential products are exact
    # Kronecker products, so the pW H.a equals (x W^T) H^chi (x W) a.
    cfg = W.scaled(W.MORSE3D, D=2)
    prob = propagate.pw_problem_from_config(cfg, n=16, nx=4, np_=4)
    dv = propagate.problem_from_config(W.scaled(W.MORSE2D, n=16))
    full = np.arange(256)
    a = W.random_psi(256, 5)
    Wm = prob.Ws[0]
    WW = np.kron(Wm, Wm)
    ref = WW.T @ dv.apply(full, WW @ a)
    np.testing.assert_allclose(prob.apply(full, a), ref, rtol=1e-11, atol=1e-13)


def test_pw_theta0_matches_dvr_dynamics():
    # Sec. 3.1: at 100 % basis the phase-space bases give the DVR result:
    # the autocorrelation of a theta = 0 pW run equals the DVR run's.
    cfg = W.scaled(W.MORSE3D, D=2)
    prob = propagate.pw_problem_from_config(cfg, n=16, nx=4, np_=4)
    dv = propagate.problem_from_config(W.scaled(W.MORSE2D, n=16))
    q0, p0, wd = (2.2, 2.35), (0.0, 0.0), (0.2, 0.2)
    r1 = propagate.run(prob, q0, p0, wd, 0.0, 12, 10.0, 6)
    r2 = propagate.run(dv, q0, p0, wd, 0.0, 12, 10.0, 6)
    for o1, o2 in zip(r1["obs"], r2["obs"]):
        assert abs(o1["C"] - o2["C"]) < 1e-10
        assert abs(o1["E"] - o2["E"]) < 1e-10 * abs(o2["E"])


def test_pw_on_fgh_theta0_matches_fgh_dynamics():
    # Sec. 3.1 builds the projected Weylets on the FGH grid; at 100 % basis
    # they reproduce the FGH DVR dynamics of the double well (small grids).
    cfg = W.scaled(W.DWELL2D, n=(20, 12))
    pcfg = W.scaled(W.DWELL2D_PW, n=(20, 12), nx_lattice=(5, 4), np_lattice=(4, 3))
    dv = propagate.problem_from_config(cfg)
    pw = propagate.problem_from_config(pcfg)
    args = (cfg["q0"], cfg["p0"], cfg["width"], 0.0, cfg["K"], cfg["dt"], 8)
    r1, r2 = propagate.run(pw, *args), propagate.run(dv, *args)
    assert r1["obs"][0]["n_active"] == 240
    for o1, o2 in zip(r1["obs"], r2["obs"]):
        assert abs(o1["C"] - o2["C"]) < 1e-10
        assert abs(o1["E"] - o2["E"]) < 1e-10 * abs(o2["E"])


# ------------------------------------------------------------------- pvB

def test_pvb_cg_solves_overlap():
    from oracle import pvb
    cfg = W.scaled(W.MORSE3D, D=2, basis="pvb")
    prob = pvb.PVBProblem(cfg, n=16, nx=4, np_=4)
    A = W.random_active_set(prob.dims, 0.4, 3)
    y = W.random_psi(len(A), 4)
    x = prob.solve_S(A, y)
    # dense S_AA by brute force
    SS = np.kron(prob.Ss[0], prob.Ss[1])[np.ix_(A, A)]
    np.testing.assert_allclose(SS @ x, y, rtol=1e-10, atol=1e-10)
    np.testing.assert_allclose(prob.S_AA(A, x), SS @ x, rtol=1e-12, atol=1e-12)


def test_pvb_on_fgh_theta0_matches_fgh_dynamics():
    # Sec. 3.1 builds pvB on the FGH grid; at 100 % basis it reproduces the FGH
    # DVR dynamics of the double well (small grids, per-mode sizes).
    from oracle import pvb
    cfg = W.scaled(W.DWELL2D, n=(20, 12))
    pcfg = W.scaled(W.DWELL2D_PVB, n=(20, 12), nx_lattice=(5, 4), np_lattice=(4, 3))
    prob = pvb.PVBProblem(pcfg)
    dv = propagate.problem_from_config(cfg)
    args = (cfg["q0"], cfg["p0"], cfg["width"], 0.0, cfg["K"], cfg["dt"], 5)
    r1, r2 = pvb.run(prob, *args), propagate.run(dv, *args)
    for o1, o2 in zip(r1["obs"], r2["obs"]):
        assert abs(o1["C"] - o2["C"]) < 1e-9
        assert abs(o1["E"] - o2["E"]) < 1e-9 * abs(o2["E"])


def test_pvb_theta0_matches_dvr_dynamics():
    # Sec. 3.1: with 100 % of the basis pvB gives the DVR (FGH) result: the
    # autocorrelation and energy of a theta = 0 pvB run equal the DVR run's.
    from oracle import pvb
    cfg = W.scaled(W.MORSE3D, D=2, basis="pvb")
    prob = pvb.PVBProblem(cfg, n=16, nx=4, np_=4)
    dv = propagate.problem_from_config(W.scaled(W.MORSE2D, n=16))
    q0, p0, wd = (2.2, 2.35), (0.0, 0.0), (0.2, 0.2)
    r1 = pvb.run(prob, q0, p0, wd, 0.0, 12, 10.0, 5)
    r2 = propagate.run(dv, q0, p0, wd, 0.0, 12, 10.0, 5)
    for o1, o2 in zip(r1["obs"], r2["obs"]):
        assert abs(o1["C"] - o2["C"]) < 1e-9, (o1["C"], o2["C"])
        assert abs(o1["norm2"] - o2["norm2"]) < 1e-9
        assert abs(o1["E"] - o2["E"]) < 1e-9 * abs(o2["E"])


# ---------------------------------------------------------------- adjoint

def test_adjoint_frozen_replay_equals_dense_products():
    # The frozen-set map: psi_{n+1} = R_n exp(-i H_{A_n A_n} dt) psi_n with R_n
    # carrying coefficients from A_n to A_{n+1} (kept where the point stays,
    # zero where it is new), and C = sum_{I in A_N} conj(a0_I) psi_N,I.  With
    # K >= |A_n| the SIL step is the exact exponential, so the replay must equal
    # dense products of principal-submatrix exponentials and 0/1 carry matrices
    # (catches a carry taken in the wrong direction, a set used one step off,
    # or a bra on the wrong set).
    from oracle import adjoint
    cfg = W.scaled(W.HH4D, D=2, n=8, dt=0.3)
    params = np.array([0.111803, 1.0, 1.2, 1.4, 1.1])
    prob = propagate.problem_from_config(cfg, omegas=params[1:3], lam=params[0])
    H = _dense_problem_H(prob)
    sets = [W.random_active_set(prob.dims, 0.7, s) for s in range(1, 6)]
    a_init = W.random_psi(len(sets[0]), 3)
    AN, aN = adjoint.run_frozen(prob, sets[0], a_init, sets, 64, cfg["dt"])
    a = a_init.copy()
    for A, An in zip(sets[:-1], sets[1:]):
        a = scipy.linalg.expm(-1j * H[np.ix_(A, A)] * cfg["dt"]) @ a
        R = (An[:, None] == A[None, :]).astype(float)
        a = R @ a
    np.testing.assert_array_equal(AN, sets[-1])
    np.testing.assert_allclose(aN, a, rtol=1e-11, atol=1e-12)

    f = prob.factors(params[3:5], cfg["p0"], cfg["width"])
    P, C = adjoint.survival(cfg, params, sets, K=64)
    b = pruned.product_on(sets[0], prob.dims, f)
    for A, An in zip(sets[:-1], sets[1:]):
        b = (An[:, None] == A[None, :]).astype(float) @ (
            scipy.linalg.expm(-1j * H[np.ix_(A, A)] * cfg["dt"]) @ b)
    Cref = np.vdot(pruned.product_on(sets[-1], prob.dims, f), b)
    assert abs(C - Cref) < 1e-12 and abs(P - abs(Cref) ** 2) < 1e-12


def test_adjoint_finite_differences_equal_analytic_gradient():
    # On the full lattice P(theta) = |a0^T exp(-i H T) a0|^2 (a0 real, unit).
    # Analytic gradient by a different route: for a potential parameter the
    # derivative of exp(-i H T) is the Daleckii-Krein formula in the eigenbasis
    # of H, Q (Gamma o (Q^T dH Q)) Q^T with the divided differences
    # Gamma_mn = -i T exp(-i (E_m + E_n) T / 2) sinc((E_m - E_n) T / 2); for a
    # packet centre q0_k the derivative of the normalised Gaussian factor,
    # df = dv/|v| - v (v.dv)/|v|^3 with dv = v (x - q0) / (2 s^2).  H is linear
    # in lambda and quadratic in omega_k, so dH comes from the model itself.
    # The oracle's central differences (h = 1e-4) must match to O(h^2)
    # (catches a sign, a parameter-slot mix-up or a one-sided difference).
    from oracle import adjoint
    cfg = W.scaled(W.HH4D, D=2, n=16, K=16, dt=0.1, nsteps=10)
    params = np.array([0.111803, 1.0, 1.3, 1.2, 0.8])
    D = 2
    prob = propagate.problem_from_config(cfg, omegas=params[1:3], lam=params[0])
    full = np.arange(int(np.prod(prob.dims)), dtype=np.int64)
    sets = [full] * (cfg["nsteps"] + 1)
    Ttot = cfg["dt"] * cfg["nsteps"]
    H = _dense_problem_H(prob)
    E, Q = np.linalg.eigh(H)
    U = (Q * np.exp(-1j * E * Ttot)) @ Q.T
    Gam = -1j * Ttot * np.exp(-0.5j * np.add.outer(E, E) * Ttot) \
        * np.sinc(np.subtract.outer(E, E) * Ttot / (2 * np.pi))
    f = prob.factors(params[3:5], cfg["p0"], cfg["width"])
    a0 = pruned.product_on(full, prob.dims, f)
    C = np.vdot(a0, U @ a0)

    def vd(lam, om):
        return propagate.problem_from_config(cfg, omegas=om, lam=lam).vdiag(full)

    om = params[1:3]
    dHs = [vd(1.0, om) - vd(0.0, om)]
    for k in range(D):
        om0 = om.copy(); om0[k] = 0.0
        dHs.append(2.0 * (vd(params[0], om) - vd(params[0], om0)) / om[k])
    grad = []
    for dh in dHs:
        dU = Q @ (Gam * (Q.T @ (dh[:, None] * Q))) @ Q.T
        grad.append(2.0 * np.real(np.conj(C) * np.vdot(a0, dU @ a0)))
    s = cfg["width"][0]
    for k in range(D):
        x = prob.grids[k]
        v = np.sqrt(prob.weights[k]) * models.gaussian_1d(x, params[3 + k], 0.0, s).real
        dv = v * (x - params[3 + k]) / (2 * s * s)
        nv = np.linalg.norm(v)
        df = dv / nv - v * (v @ dv) / nv ** 3
        fk = list(f); fk[k] = df
        da0 = pruned.product_on(full, prob.dims, fk)
        dC = np.vdot(da0, U @ a0) + np.vdot(a0, U @ da0)
        grad.append(2.0 * np.real(np.conj(C) * dC))
    P, Cor = adjoint.survival(cfg, params, sets)
    assert abs(Cor - C) < 1e-10 and abs(P - abs(C) ** 2) < 1e-10
    g = adjoint.fd_gradient(cfg, params, sets, h=1e-4)
    np.testing.assert_allclose(g, grad, rtol=1e-6, atol=1e-7)
    assert np.min(np.abs(grad)) > 1e-3          # every slot carries a signal
