"""GPU adaption (Sec. 2.5: threshold + nearest-neighbour add) and initial
packet against the oracle: bit-exact active sets and coefficients."""
import numpy as np
import pytest

import workloads as W
from gpu_helpers import ho_problem, lib, state_with

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("dims", [(7, 6), (4, 3, 5), (24, 24, 24), (5, 64), (9,), (3, 4, 2, 5, 3)])
def test_prune_matches_oracle(dims, prec):
    from oracle import pruned
    pq = lib()
    rng = np.random.default_rng(len(dims))
    A = W.random_active_set(dims, 0.5, seed=sum(dims))
    theta = 0.3
    mag = rng.uniform(0, 0.6, len(A))
    psi = mag * np.exp(2j * np.pi * rng.random(len(A)))
    psi[::7] = theta            # exact ties are kept
    psi[1::11] = 0.3 * (1 + 2e-16) if prec == 0 else np.float32(0.3) * (1 + 1e-7)
    dt = np.complex128 if prec == pq.FP64 else np.complex64
    psi = psi.astype(dt)
    b, _, _ = ho_problem(dims, 1)
    s = state_with(b, A, psi, prec)
    s.prune(theta)
    An, pn = s.read()
    Ar, pr = pruned.prune(A, psi, dims, theta)
    np.testing.assert_array_equal(An, Ar)
    np.testing.assert_array_equal(pn, pr.astype(dt))


@pytest.mark.parametrize("prec", [0, 1])
def test_prune_everything_below(prec):
    pq = lib()
    dims = (5, 6)
    b, _, _ = ho_problem(dims, 1)
    A = np.arange(30)
    s = state_with(b, A, np.full(30, 1e-3), prec)
    s.prune(0.5)
    assert s.size() == 0
    s.prune(0.5)                # pruning an empty set stays empty
    assert s.size() == 0


@pytest.mark.parametrize("name", ["morse2d", "hh4d"])
def test_initial_packet_matches_oracle(name):
    from oracle import propagate
    pq = lib()
    cfg = W.CONFIGS[name]
    b, prob = pq.build_model(cfg), propagate.problem_from_config(cfg)
    A, a, f = propagate.initial_state(prob, cfg["q0"], cfg["p0"], cfg["width"], cfg["theta"])
    for prec in (pq.FP64, pq.FP32MIX):
        s = pq.State(b, cfg["q0"], cfg["p0"], cfg["width"], cfg["theta"], precision=prec)
        Ag, ag = s.read()
        np.testing.assert_array_equal(Ag, A)
        tol = 1e-13 if prec == pq.FP64 else 1e-7
        np.testing.assert_allclose(ag, a, rtol=tol, atol=tol * np.abs(a).max())
        o = s.observables()
        C0 = np.vdot(a, a)     # C(0) = sum over A of |a0|^2 (< 1 after the prune)
        assert abs(o["C"][0] - C0) < (1e-13 if prec == pq.FP64 else 1e-6)
        assert o["n_active"][0] == len(A)


def test_capacity_overflow_reported():
    pq = lib()
    cfg = W.HH4D
    b = pq.build_model(cfg)
    with pytest.raises(pq.PQError) as e:
        pq.State(b, cfg["q0"], cfg["p0"], cfg["width"], cfg["theta"], capacity=1000)
    assert e.value.status == pq.ECAPACITY


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("rule", [2, 3])
@pytest.mark.parametrize("dims", [(7, 6), (4, 3, 5), (9,), (3, 4, 2, 5, 3), (24, 24, 24)])
def test_prune_ball_rules_match_oracle(dims, rule, prec):
    # neighbour radius sqrt(2) and 2 of Sec. 3.1: bit-exact sets and values
    from oracle import pruned
    pq = lib()
    rng = np.random.default_rng(len(dims) + 10 * rule)
    A = W.random_active_set(dims, 0.3, seed=sum(dims) + rule)
    theta = 0.5
    psi = rng.uniform(0, 0.6, len(A)) * np.exp(2j * np.pi * rng.random(len(A)))
    dt = np.complex128 if prec == pq.FP64 else np.complex64
    psi = psi.astype(dt)
    b, _, _ = ho_problem(dims, 1)
    s = state_with(b, A, psi, prec)
    s.prune(theta, radius=rule)
    An, pn = s.read()
    Ar, pr = pruned.prune(A, psi, dims, theta, rule)
    np.testing.assert_array_equal(An, Ar)
    np.testing.assert_array_equal(pn, pr.astype(dt))


@pytest.mark.parametrize("prec", [0, 1])
def test_prune_relative_exclusion_matches_oracle(prec):
    # Sec. 2.5: functions leave only when more than rel_excl * |A| would leave
    from oracle import pruned
    pq = lib()
    dims = (12, 10, 9)
    rng = np.random.default_rng(5)
    A = W.random_active_set(dims, 0.5, seed=5)
    psi = (rng.uniform(0, 0.6, len(A)) * np.exp(2j * np.pi * rng.random(len(A))))
    dt = np.complex128 if prec == pq.FP64 else np.complex64
    psi = psi.astype(dt)
    theta = 0.55
    A0, _ = pruned.prune(A, psi, dims, theta)
    n_out = len(np.setdiff1d(A, A0))
    assert 0 < n_out < len(A)
    b, _, _ = ho_problem(dims, 1)
    for rho in (n_out / len(A) - 1e-9, n_out / len(A), 0.9):
        s = state_with(b, A, psi, prec)
        s.prune(theta, radius=1, rel_excl=rho)
        An, pn = s.read()
        Ar, pr = pruned.prune(A, psi, dims, theta, 1, rho)
        np.testing.assert_array_equal(An, Ar)
        np.testing.assert_array_equal(pn, pr.astype(dt))


def test_neighbour_rule_errors():
    pq = lib()
    dims = (5, 6)
    b, _, _ = ho_problem(dims, 1)
    s = state_with(b, np.arange(30), np.full(30, 1.0), 0)
    for bad in (0, 4):
        with pytest.raises(pq.PQError) as e:
            s.prune(0.5, radius=bad)
        assert e.value.status == pq.EINVAL
    with pytest.raises(pq.PQError) as e:
        s.prune(0.5, rel_excl=-1.0)
    assert e.value.status == pq.EINVAL


def test_initial_packet_radius_sqrt2_matches_oracle():
    from oracle import propagate
    pq = lib()
    cfg = W.MORSE2D
    b, prob = pq.build_model(cfg), propagate.problem_from_config(cfg)
    A, a, f = propagate.initial_state(prob, cfg["q0"], cfg["p0"], cfg["width"], cfg["theta"],
                                      radius=2)
    s = pq.State(b, cfg["q0"], cfg["p0"], cfg["width"], cfg["theta"], precision=pq.FP64,
                 radius=2)
    Ag, ag = s.read()
    np.testing.assert_array_equal(Ag, A)
    np.testing.assert_allclose(ag, a, rtol=1e-13, atol=1e-13 * np.abs(a).max())
