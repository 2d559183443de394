"""GPU propagation (SIL -> adaption -> observables, Sec. 2.5 and Sec. 3.1)
against the FP64 oracle.

FP64 path: identical active sets after every step, C(t) within 1e-10,
wavefunction relative L2 error <= 1e-10 at the end.  FP32-mix path:
|dC(t)| <= 1e-5 and norm drift <= 1e-6 against the FP64 oracle."""
import numpy as np
import pytest
import scipy.linalg

import workloads as W
from gpu_helpers import lib

pytestmark = pytest.mark.gpu


def _oracle(cfg, nsteps, theta=None, K=None):
    from oracle import propagate
    prob = propagate.problem_from_config(cfg)
    th = cfg["theta"] if theta is None else theta
    r = propagate.run(prob, cfg["q0"], cfg["p0"], cfg["width"], th, K or cfg["K"], cfg["dt"],
                      nsteps, record_sets=True)
    return prob, r


def _gpu(cfg, nsteps, prec, theta=None, K=None, reorth=1):
    pq = lib()
    b = pq.build_model(cfg)
    th = cfg["theta"] if theta is None else theta
    s = pq.State(b, cfg["q0"], cfg["p0"], cfg["width"], th, precision=prec)
    s.propagate(K or cfg["K"], cfg["dt"], th, nsteps, reorth=reorth)
    return s, s.observables()


def _series(r, key):
    return np.array([o[key] for o in r["obs"]])


def test_morse2d_fp64_full_run():
    cfg = W.MORSE2D
    n = cfg["nsteps"]
    prob, r = _oracle(cfg, n)
    s, o = _gpu(cfg, n, lib().FP64)
    np.testing.assert_array_equal(o["n_active"], _series(r, "n_active"))
    np.testing.assert_array_equal(o["n_wasted"], _series(r, "n_wasted"))
    assert np.max(np.abs(o["C"] - _series(r, "C"))) < 1e-10
    assert np.max(np.abs(o["norm2"] - _series(r, "norm2"))) < 1e-10
    E = _series(r, "E")
    assert np.max(np.abs(o["energy"] - E)) < 1e-10 * np.abs(E).max()
    A, psi = s.read()
    np.testing.assert_array_equal(A, r["A"])
    assert np.linalg.norm(psi - r["a"]) <= 1e-10 * np.linalg.norm(r["a"])


@pytest.mark.parametrize("reorth", [1, 0])
def test_hh4d_fp64_steps(reorth):
    cfg = W.HH4D
    n = 10
    prob, r = _oracle(cfg, n)
    s, o = _gpu(cfg, n, lib().FP64, reorth=reorth)
    np.testing.assert_array_equal(o["n_active"], _series(r, "n_active"))
    A, psi = s.read()
    np.testing.assert_array_equal(A, r["A"])
    assert np.linalg.norm(psi - r["a"]) <= 1e-10 * np.linalg.norm(r["a"])
    assert np.max(np.abs(o["C"] - _series(r, "C"))) < 1e-10


def test_hh4d_fp32mix_steps():
    cfg = W.HH4D
    n = 10
    prob, r = _oracle(cfg, n)
    s, o = _gpu(cfg, n, lib().FP32MIX)
    assert np.max(np.abs(o["C"] - _series(r, "C"))) <= 1e-5
    assert np.max(np.abs(o["norm2"] - _series(r, "norm2"))) <= 1e-6
    # the active sets may differ only where FP32 moves a coefficient across
    # the threshold: compare sizes loosely, observables strictly (above)
    na = _series(r, "n_active")
    assert np.all(np.abs(o["n_active"] - na) <= 1e-3 * na + 5)


def test_theta0_full_krylov_is_exact():
    """theta = 0 and K = lattice size: SIL is the exact exponential, so the
    GPU run must equal exp(-iHt) a(0) from a dense eigendecomposition."""
    from oracle import propagate, pruned
    pq = lib()
    cfg = W.scaled(W.MORSE2D, n=5)
    N = 25
    s, o = _gpu(cfg, 4, pq.FP64, theta=0.0, K=N)
    prob = propagate.problem_from_config(cfg)
    full = np.arange(N)
    H = np.zeros((N, N))
    for j in range(N):
        e = np.zeros(N, complex)
        e[j] = 1
        H[:, j] = prob.apply(full, e).real
    A, a, f = propagate.initial_state(prob, cfg["q0"], cfg["p0"], cfg["width"], 0.0)
    for step in range(5):
        ref = scipy.linalg.expm(-1j * H * cfg["dt"] * step) @ a
        assert abs(o["C"][step] - np.vdot(a, ref)) < 1e-12
        assert o["n_active"][step] == N
    _, psi = s.read()
    np.testing.assert_allclose(psi, scipy.linalg.expm(-1j * H * cfg["dt"] * 4) @ a, atol=1e-12)


def test_energy_and_norm_conserved_unpruned():
    pq = lib()
    cfg = W.scaled(W.HH4D, D=2, q0=(2.0, 2.0), p0=(0.0, 0.0), width=(0.5 ** 0.5,) * 2)
    s, o = _gpu(cfg, 30, pq.FP64, theta=0.0)
    assert np.max(np.abs(o["norm2"] - o["norm2"][0])) < 1e-12
    assert np.max(np.abs(o["energy"] - o["energy"][0])) < 1e-11 * abs(o["energy"][0])


@pytest.mark.parametrize("rule,rho", [(2, 0.0), (3, 0.0), (1, 0.05)])
def test_morse2d_fp64_neighbour_rules(rule, rho):
    # the adaption variants of Sec. 3.1 / Sec. 2.5 inside the propagation:
    # identical active sets every step, C(t) within 1e-10
    from oracle import propagate
    pq = lib()
    cfg = W.MORSE2D
    n = 40
    prob = propagate.problem_from_config(cfg)
    r = propagate.run(prob, cfg["q0"], cfg["p0"], cfg["width"], cfg["theta"], cfg["K"],
                      cfg["dt"], n, radius=rule, rel_excl=rho)
    b = pq.build_model(cfg)
    s = pq.State(b, cfg["q0"], cfg["p0"], cfg["width"], cfg["theta"], precision=pq.FP64,
                 radius=rule)
    s.propagate(cfg["K"], cfg["dt"], cfg["theta"], n, radius=rule, rel_excl=rho)
    o = s.observables()
    np.testing.assert_array_equal(o["n_active"], _series(r, "n_active"))
    assert np.max(np.abs(o["C"] - _series(r, "C"))) < 1e-10
    A, psi = s.read()
    np.testing.assert_array_equal(A, r["A"])


@pytest.mark.parametrize("prec", [0, 1])
def test_double_well_steps(prec):
    # the paper's double well (Sec. 3.1) on its FGH grids of 165 x 81 points:
    # FP64 identical active sets and C(t) within 1e-10 of the oracle; FP32-mix
    # C(t) within 1e-5
    pq = lib()
    cfg = W.DWELL2D
    n = 150
    prob, r = _oracle(cfg, n)
    s, o = _gpu(cfg, n, prec)
    if prec == pq.FP64:
        np.testing.assert_array_equal(o["n_active"], _series(r, "n_active"))
        assert np.max(np.abs(o["C"] - _series(r, "C"))) < 1e-10
        A, psi = s.read()
        np.testing.assert_array_equal(A, r["A"])
        assert np.linalg.norm(psi - r["a"]) <= 1e-10 * np.linalg.norm(r["a"])
    else:
        assert np.max(np.abs(o["C"] - _series(r, "C"))) < 1e-5


@pytest.mark.parametrize("name,dt,n,prec", [("morse2d", 2.0, 20, 0), ("hh4d", 0.01, 10, 0),
                                            ("hh4d", 0.01, 10, 1)])
def test_rk4_matches_oracle(name, dt, n, prec):
    # the fourth-order Runge-Kutta stepper (not in the paper; the alternative
    # integrator): FP64 identical active sets and C(t) within 1e-10 of the
    # oracle's RK4, FP32-mix within 1e-5
    from oracle import propagate
    pq = lib()
    cfg = W.CONFIGS[name]
    prob = propagate.problem_from_config(cfg)
    r = propagate.run(prob, cfg["q0"], cfg["p0"], cfg["width"], cfg["theta"], cfg["K"], dt, n,
                      integrator="rk4")
    b = pq.build_model(cfg)
    s = pq.State(b, cfg["q0"], cfg["p0"], cfg["width"], cfg["theta"], precision=prec)
    s.propagate(cfg["K"], dt, cfg["theta"], n, integrator=pq.RK4)
    o = s.observables()
    C = _series(r, "C")
    if prec == 0:
        np.testing.assert_array_equal(o["n_active"], _series(r, "n_active"))
        assert np.max(np.abs(o["C"] - C)) < 1e-10
        E = _series(r, "E")
        assert np.max(np.abs(o["energy"] - E)) < 1e-10 * np.abs(E).max()
        A, psi = s.read()
        np.testing.assert_array_equal(A, r["A"])
    else:
        assert np.max(np.abs(o["C"] - C)) < 1e-5


@pytest.mark.parametrize("tol", [1e-8, 1e-12])
def test_sil_error_control_matches_oracle(tol):
    # error-controlled SIL order (K = 16 at most): identical active sets and
    # C(t) within 1e-10 of the oracle's error-controlled SIL (FP64)
    from oracle import propagate
    pq = lib()
    cfg = W.HH4D
    n = 10
    prob = propagate.problem_from_config(cfg)
    r = propagate.run(prob, cfg["q0"], cfg["p0"], cfg["width"], cfg["theta"], 16, cfg["dt"], n,
                      sil_tol=tol)
    b = pq.build_model(cfg)
    s = pq.State(b, cfg["q0"], cfg["p0"], cfg["width"], cfg["theta"], precision=pq.FP64)
    s.propagate(16, cfg["dt"], cfg["theta"], n, sil_tol=tol)
    o = s.observables()
    np.testing.assert_array_equal(o["n_active"], _series(r, "n_active"))
    assert np.max(np.abs(o["C"] - _series(r, "C"))) < 1e-10


def test_sil_error_control_fp32():
    # error-controlled order on the FP32-mix path: C(t) within 1e-5 of the oracle
    from oracle import propagate
    pq = lib()
    cfg = W.HH4D
    n = 10
    prob = propagate.problem_from_config(cfg)
    r = propagate.run(prob, cfg["q0"], cfg["p0"], cfg["width"], cfg["theta"], 16, cfg["dt"], n,
                      sil_tol=1e-8)
    b = pq.build_model(cfg)
    s = pq.State(b, cfg["q0"], cfg["p0"], cfg["width"], cfg["theta"], precision=pq.FP32MIX)
    s.propagate(16, cfg["dt"], cfg["theta"], n, sil_tol=1e-8)
    o = s.observables()
    assert np.max(np.abs(o["C"] - _series(r, "C"))) < 1e-5
