"""GPU parity of the pruned H.psi (Sec. 2.2.2 / Appendix) against the FP64
oracle, element by element, through the C ABI.

Tolerances: FP64 |y_gpu - y| <= 1e-13 * s_I, FP32 |y_gpu - y| <= 4e-6 * s_I,
where s_I is the same sum taken with |T|, |V| and |psi| (a rounding bound:
at most ~130 terms of unit roundoff 1.1e-16 resp. 6e-8)."""
import numpy as np
import pytest

import workloads as W
from gpu_helpers import fgh_problem, ho_problem, lib, rel_bound, state_with, vdiag_of

pytestmark = pytest.mark.gpu

TOL = {0: 1e-13, 1: 4e-6}


def _run(dims, A, seed, prec, nterms=3, problem=ho_problem, tol=None):
    import torch
    from oracle import pruned
    pq = lib()
    b, Ts, pot = problem(dims, seed, nterms)
    psi = W.random_psi(len(A), seed + 1)
    dt = np.complex128 if prec == pq.FP64 else np.complex64
    psi = psi.astype(dt)
    s = state_with(b, A, psi, prec)
    assert s.size() == len(A)
    idx, p2 = s.read()
    np.testing.assert_array_equal(idx, A)
    np.testing.assert_array_equal(p2, psi)
    tdt = torch.complex128 if prec == pq.FP64 else torch.complex64
    x = torch.from_numpy(psi).to("cuda")
    y = torch.empty_like(x)
    vhv = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
    s.apply_H(x, y, vhv=vhv)
    torch.cuda.synchronize()
    got = y.cpu().numpy().astype(np.complex128)
    vd = vdiag_of(pot, A, dims)
    ref = pruned.apply_H(A, psi.astype(np.complex128), dims, Ts, vd)
    bound = rel_bound(Ts, A, psi, dims, vd)
    err = np.abs(got - ref)
    tl = TOL[prec] if tol is None else tol[prec]
    assert np.all(err <= tl * bound + 1e-300), (err / np.maximum(bound, 1e-300)).max()
    # <x, Hx> of the same call: the FP64 sum of the products of what was
    # written, and the oracle's value within the elementwise bound
    p64 = psi.astype(np.complex128)
    v = complex(*vhv.cpu().numpy())
    scale = float(np.sum(np.abs(p64) * np.abs(got))) + 1e-300
    assert abs(v - np.vdot(p64, got)) <= 1e-12 * scale
    assert abs(v - np.vdot(p64, ref)) <= tl * float(np.sum(np.abs(p64) * bound)) + 1e-12 * scale
    # host-buffer entry point gives the same numbers
    got_h = s.apply_H_host(psi)
    np.testing.assert_array_equal(got_h, y.cpu().numpy())
    return s


CASES = [
    ((8, 9), 0.6),            # 2D: one plane
    ((6, 7, 5), 0.5),         # 3D: one outer mode
    ((5, 4, 6, 7), 0.4),      # 4D, ragged, two outer modes
    ((3, 4, 2, 3, 5), 0.7),   # 5D
    ((5, 64), 0.5),           # last mode 64 wide (two lanes per warp column)
    ((64, 3, 5), 0.3),        # an outer mode 64 long
    ((17,), 0.8),             # 1D (virtual leading mode)
    ((33, 40), 1.0),          # full lattice (unpruned)
    # register-blocked kernels (fibre lengths 16 / 24 / 32)
    ((24, 24), 0.5),
    ((32, 32), 0.6),
    ((16, 16, 16), 0.4),
    ((24, 24, 24), 0.3),
    ((16, 24, 16, 16), 0.5),
    ((32, 7, 32), 0.5),       # generic inner tile, register outer pass
    ((24, 24), 1.0),
    # compact fibre kernels (other fibre lengths, last mode <= 32)
    ((9, 12, 20), 0.4),
    ((40, 6, 28, 11), 0.3),
    ((5, 30), 0.7),
    # FP32 slab passes: a full 24^3 cube (more points than the staging buffer
    # holds), ragged 6D (cube + pair + single pass), 5D (cube + pair), odd
    # sizes in every tile mode
    ((24, 24, 24), 1.0),
    ((4, 5, 3, 6, 4, 5), 0.5),
    ((3, 5, 7, 9, 11), 0.6),
    ((2, 3, 24, 24, 24), 0.97),
    ((7, 3, 32, 2, 13), 0.5),
    # a 33-64-point mode next to the last one (compact inner pass), and an
    # outer mode of that length
    ((40, 12), 0.6),
    ((3, 48, 16), 0.5),
    ((36, 5, 20), 0.4),
]


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("dims,frac", CASES)
def test_apply_random_sets(dims, frac, prec):
    A = W.random_active_set(dims, frac, seed=len(dims) * 7 + int(frac * 10))
    _run(dims, A, 5, prec)


@pytest.mark.parametrize("prec", [0, 1])
def test_apply_ellipsoid_4d(prec):
    dims = (24, 24, 24, 24)
    A = W.ellipsoid_active_set(dims, (9, 8, 10, 7))
    _run(dims, A, 9, prec, nterms=6)


@pytest.mark.parametrize("prec", [0, 1])
def test_apply_ellipsoid_6d(prec):
    # a 6D ball of 1.1e5 points on 10^6: ragged fibres in every mode
    dims = (10,) * 6
    A = W.ellipsoid_active_set(dims, (4.6, 4.1, 4.9, 4.3, 4.4, 4.8))
    _run(dims, A, 11, prec, nterms=8)


@pytest.mark.parametrize("prec", [0, 1])
def test_apply_empty_and_single(prec):
    import torch
    pq = lib()
    dims = (6, 5, 4)
    b, Ts, pot = ho_problem(dims, 3)
    s = state_with(b, np.zeros(0, np.int64), None, prec)
    assert s.size() == 0
    tdt = torch.complex128 if prec == pq.FP64 else torch.complex64
    x = torch.zeros(1, dtype=tdt, device="cuda")
    y = torch.zeros(1, dtype=tdt, device="cuda")
    s.apply_H(x, y)
    torch.cuda.synchronize()
    _run(dims, np.array([37]), 4, prec)


def test_apply_hh6d_initial_state_sampled():
    """Full-size 6D Henon-Heiles workload (24^6 lattice), FP32 H.psi in the
    launch configuration the benchmark times, checked on a sample of outputs
    the oracle computes one by one."""
    import torch
    from oracle import pruned, propagate
    pq = lib()
    cfg = W.HH6D
    b = pq.build_model(cfg)
    s = pq.State(b, cfg["q0"], cfg["p0"], cfg["width"], cfg["theta"], precision=pq.FP32MIX)
    A, psi = s.read()
    assert len(A) > 1_000_000
    x = torch.from_numpy(psi).to("cuda")
    y = torch.empty_like(x)
    s.apply_H(x, y)
    torch.cuda.synchronize()
    got = y.cpu().numpy().astype(np.complex128)
    prob = propagate.problem_from_config(cfg)
    rng = np.random.default_rng(0)
    pos = np.unique(np.concatenate([rng.integers(0, len(A), 4000), [0, len(A) - 1]]))
    vd = prob.vdiag(A[pos])
    ref = pruned.apply_H_at(A, psi.astype(np.complex128), prob.dims, prob.Ts, vd, pos)
    scale = pruned.apply_H_at(A, np.abs(psi).astype(np.complex128), prob.dims,
                              [np.abs(T) for T in prob.Ts], np.abs(vd), pos).real
    err = np.abs(got[pos] - ref)
    assert np.all(err <= 4e-6 * scale + 1e-30), (err / scale).max()


# Sets covering at least half the lattice: in FP32 these take the dense-tile
# passes (batched contractions over zero-filled tiles; the set size on the
# device selects them): inner + two pairs (6D), inner + pair (4D), inner +
# pair + single mode (5D), pair modes that are not multiples of 4 (no pair
# pass), inner + single mode (3D); full lattices and lattices with holes.
DENSE = [(4, 8, 4, 8, 8, 8), (8, 12, 16, 24), (8, 4, 8, 12, 16), (3, 8, 5, 8, 8, 8), (24, 24, 8)]


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("frac", [1.0, 0.9, 0.55])
@pytest.mark.parametrize("dims", DENSE)
def test_apply_dense_sets(dims, frac, prec):
    if frac == 1.0:
        A = np.arange(int(np.prod(dims)), dtype=np.int64)
    else:
        A = W.random_active_set(dims, frac, seed=len(dims) + int(100 * frac))
    _run(dims, A, 13, prec, nterms=5)


@pytest.mark.parametrize("dims", [(8, 12, 16, 24), (4, 8, 4, 8, 8, 8)])
def test_apply_dense_set_from_packet(dims):
    """A state whose active set comes from its packet (no host-side set
    size: both H.psi paths are launched and the device-side size selects),
    with a packet wide enough that the set covers more than half the lattice:
    FP32 H.psi against the oracle on that set."""
    import torch
    from oracle import pruned
    pq = lib()
    b, Ts, pot = ho_problem(dims, 17, 4)
    D = len(dims)
    s = pq.State(b, [0.0] * D, [0.0] * D, [4.0] * D, 1e-9, precision=pq.FP32MIX)
    A, psi = s.read()
    assert 2 * len(A) >= int(np.prod(dims))
    x = torch.from_numpy(psi).to("cuda")
    y = torch.empty_like(x)
    s.apply_H(x, y)
    torch.cuda.synchronize()
    got = y.cpu().numpy().astype(np.complex128)
    vd = vdiag_of(pot, A, dims)
    p64 = psi.astype(np.complex128)
    ref = pruned.apply_H(A, p64, dims, Ts, vd)
    bound = rel_bound(Ts, A, p64, dims, vd)
    err = np.abs(got - ref)
    assert np.all(err <= TOL[1] * bound + 1e-300), (err / np.maximum(bound, 1e-300)).max()


@pytest.mark.parametrize("dims", [(4, 8, 4, 8, 8, 8), (8, 12, 16, 24)])
def test_apply_dense_set_unaligned_vectors(dims):
    """Input and output views starting 8 bytes past a 16-byte boundary (the
    dense-tile passes take 16-byte copies only where the address allows):
    the same result as aligned vectors, element for element."""
    import torch
    pq = lib()
    b, Ts, pot = ho_problem(dims, 23, 3)
    A = np.arange(int(np.prod(dims)), dtype=np.int64)
    psi = W.random_psi(len(A), 29).astype(np.complex64)
    s = state_with(b, A, psi, pq.FP32MIX)
    x = torch.from_numpy(psi).to("cuda")
    y = torch.empty_like(x)
    s.apply_H(x, y)
    xb = torch.zeros(len(A) + 1, dtype=torch.complex64, device="cuda")
    yb = torch.zeros(len(A) + 1, dtype=torch.complex64, device="cuda")
    xu, yu = xb[1:], yb[1:]
    xu.copy_(x)
    assert xu.data_ptr() % 16 == 8 and yu.data_ptr() % 16 == 8
    s.apply_H(xu, yu)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(yu.cpu().numpy(), y.cpu().numpy())


def test_apply_hh6d_full_lattice_sampled():
    """The 6D Henon-Heiles Hamiltonian on the whole 24^6 lattice (the set the
    propagation reaches after about 100 steps), FP32, in the launch
    configuration the benchmark's late window times; sampled outputs against
    the oracle one by one."""
    import torch
    from oracle import pruned, propagate
    pq = lib()
    cfg = W.HH6D
    b = pq.build_model(cfg)
    nfull = 24 ** 6
    A = np.arange(nfull, dtype=np.int64)
    psi = W.random_psi(nfull, 21).astype(np.complex64)
    s = state_with(b, A, psi, pq.FP32MIX)
    x = torch.from_numpy(psi).to("cuda")
    y = torch.empty_like(x)
    s.apply_H(x, y)
    torch.cuda.synchronize()
    prob = propagate.problem_from_config(cfg)
    rng = np.random.default_rng(1)
    pos = np.unique(np.concatenate([rng.integers(0, nfull, 4000), [0, nfull - 1]]))
    got = y[torch.from_numpy(pos).to("cuda")].cpu().numpy().astype(np.complex128)
    vd = prob.vdiag(A[pos])
    p64 = psi.astype(np.complex128)
    ref = pruned.apply_H_at(A, p64, prob.dims, prob.Ts, vd, pos)
    scale = pruned.apply_H_at(A, np.abs(p64), prob.dims, [np.abs(T) for T in prob.Ts],
                              np.abs(vd), pos).real
    err = np.abs(got - ref)
    assert np.all(err <= 4e-6 * scale + 1e-30), (err / scale).max()


# Lattices with a mode longer than 64 (FGH DVR, point-parallel pass): up to
# 246 terms per output, so the FP32 bound is taken at 1e-5 of the rounding scale.
BIG = [((165, 81), 0.3), ((70, 9), 0.5), ((100, 3, 5), 0.4), ((9, 130), 0.5), ((5, 4, 66), 0.6)]


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("dims,frac", BIG)
def test_apply_long_modes(dims, frac, prec):
    A = W.random_active_set(dims, frac, seed=len(dims) * 3 + int(frac * 10))
    _run(dims, A, 7, prec, problem=fgh_problem, tol={0: 1e-13, 1: 1e-5})


@pytest.mark.parametrize("prec", [0, 1])
def test_apply_tabulated_potential(prec):
    # a diagonal potential given as a table over the lattice (not SoP),
    # added to the SoP part: parity with the oracle on a random set
    import torch
    from oracle import pruned
    pq = lib()
    dims = (7, 6, 5)
    b, Ts, pot = ho_problem(dims, 11)
    rng = np.random.default_rng(12)
    Vg = rng.uniform(-1, 1, int(np.prod(dims)))
    b.set_potential_grid(Vg.reshape(dims))
    A = W.random_active_set(dims, 0.5, seed=13)
    psi = W.random_psi(len(A), 14).astype(np.complex128 if prec == 0 else np.complex64)
    s = state_with(b, A, psi, prec)
    x = torch.from_numpy(psi).to("cuda")
    y = torch.empty_like(x)
    s.apply_H(x, y)
    torch.cuda.synchronize()
    vd = vdiag_of(pot, A, dims) + Vg[A]
    ref = pruned.apply_H(A, psi.astype(np.complex128), dims, Ts, vd)
    bound = rel_bound(Ts, A, psi, dims, vd)
    err = np.abs(y.cpu().numpy().astype(np.complex128) - ref)
    assert np.all(err <= TOL[prec] * bound + 1e-300), (err / np.maximum(bound, 1e-300)).max()


def test_tabulated_coupling_reproduces_sop_run():
    # the 2D Morse coupling 0.005 q1 q2 moved from the SoP form into a table:
    # the propagation (FP64) gives the oracle's active sets and C(t)
    from oracle import propagate
    pq = lib()
    cfg = W.MORSE2D
    n = 20
    prob = propagate.problem_from_config(cfg)
    r = propagate.run(prob, cfg["q0"], cfg["p0"], cfg["width"], cfg["theta"], cfg["K"], cfg["dt"], n)
    b = pq.Basis(pq.modes_of(cfg))
    g = [b.grid(k)[0] for k in range(2)]
    b.set_sop(pq.coupled_morse_terms(g, cfg["morse_D"], cfg["morse_a"], cfg["morse_qe"], 0.0))
    b.set_potential_grid(cfg["coupling"] * np.outer(g[0], g[1]))
    s = pq.State(b, cfg["q0"], cfg["p0"], cfg["width"], cfg["theta"], precision=pq.FP64)
    s.propagate(cfg["K"], cfg["dt"], cfg["theta"], n)
    o = s.observables()
    np.testing.assert_array_equal(o["n_active"], [v["n_active"] for v in r["obs"]])
    assert np.max(np.abs(o["C"] - np.array([v["C"] for v in r["obs"]]))) < 1e-10
