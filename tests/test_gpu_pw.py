"""GPU parity of the projected-Weylet path (Sec. 2.4; pruned sequential
transform of Sec. 2.2.2 with dense 1D factors; adaption on the phase-space
lattice with two axes per mode) against the FP64 oracle.

H.psi tolerances: FP64 |y - y_ref| <= 1e-12 s_I, FP32 <= 2e-5 s_I with s_I
the same sequential products taken with |h| and |psi| (each term is up to two
64-long passes: about 130 roundings of 1.1e-16 resp. 6e-8)."""
import numpy as np
import pytest

import workloads as W
from gpu_helpers import lib

pytestmark = pytest.mark.gpu


def _pw_cfg(D, n, nx, np_):
    return W.scaled(W.MORSE3D, D=D, n=n, nx_lattice=nx, np_lattice=np_,
                    q0=W.morse3d_centres()[:D], p0=(0.0,) * D, width=(0.2,) * D)


def _state_with(b, A, psi, prec):
    pq = lib()
    s = pq.State(b, [0.0] * b.D, [0.0] * b.D, [1.0] * b.D, 1e30, precision=prec)
    s.load(A, psi)
    return s


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("D,n,nx,np_,frac", [(2, 16, 4, 4, 0.5), (3, 16, 4, 4, 0.3),
                                             (2, 64, 8, 8, 0.4), (1, 16, 4, 4, 0.8),
                                             (3, 64, 8, 8, 0.15), (3, 24, 4, 6, 0.5)])
def test_pw_apply_random_sets(D, n, nx, np_, frac, prec):
    import torch
    from oracle import propagate, pruned
    pq = lib()
    cfg = _pw_cfg(D, n, nx, np_)
    b = pq.build_model(cfg)
    prob = propagate.problem_from_config(cfg)
    dims = (n,) * D
    A = W.random_active_set(dims, frac, seed=D * 10 + n)
    psi = W.random_psi(len(A), 3).astype(np.complex128 if prec == 0 else np.complex64)
    s = _state_with(b, A, psi, prec)
    x = torch.from_numpy(psi).to("cuda")
    y = torch.empty_like(x)
    s.apply_H(x, y)
    torch.cuda.synchronize()
    got = y.cpu().numpy().astype(np.complex128)
    ref = prob.apply(A, psi.astype(np.complex128))
    absterms = [(abs(c), {k: np.abs(h) for k, h in f.items()}) for c, f in prob.terms]
    bound = pruned.apply_H_sop(A, np.abs(psi).astype(np.complex128), dims, absterms).real
    tol = 1e-12 if prec == 0 else 2e-5
    err = np.abs(got - ref)
    assert np.all(err <= tol * bound + 1e-300), (err / np.maximum(bound, 1e-300)).max()


@pytest.mark.parametrize("prec", [0, 1])
def test_pw_prune_phase_space_axes(prec):
    from oracle import pruned
    pq = lib()
    cfg = _pw_cfg(2, 64, 8, 8)
    b = pq.build_model(cfg)
    dims = (64, 64)
    axes = (8, 8, 8, 8)
    rng = np.random.default_rng(4)
    A = W.random_active_set(dims, 0.3, seed=5)
    psi = rng.uniform(0, 0.6, len(A)) * np.exp(2j * np.pi * rng.random(len(A)))
    psi[::9] = 0.3
    psi = psi.astype(np.complex128 if prec == 0 else np.complex64)
    s = _state_with(b, A, psi, prec)
    s.prune(0.3)
    An, pn = s.read()
    Ar, pr = pruned.prune(A, psi, axes, 0.3)
    np.testing.assert_array_equal(An, Ar)
    np.testing.assert_array_equal(pn, pr.astype(pn.dtype))


def test_pw_initial_state_morse3d():
    """The 3D coupled Morse workload in projected Weylets (64^3 lattice)."""
    from oracle import propagate
    pq = lib()
    cfg = W.scaled(W.MORSE3D, q0=W.morse3d_centres())
    b = pq.build_model(cfg)
    prob = propagate.problem_from_config(cfg)
    A, a, f = propagate.initial_state(prob, cfg["q0"], cfg["p0"], cfg["width"], cfg["theta"])
    s = pq.State(b, cfg["q0"], cfg["p0"], cfg["width"], cfg["theta"], precision=pq.FP64)
    Ag, ag = s.read()
    np.testing.assert_array_equal(Ag, A)
    np.testing.assert_allclose(ag, a, rtol=1e-12, atol=1e-12 * np.abs(a).max())


@pytest.mark.parametrize("name,D,n,nx,np_,nsteps", [("small", 2, 16, 4, 4, 8),
                                                   ("morse3d", 3, 64, 8, 8, 3)])
def test_pw_propagation_fp64(name, D, n, nx, np_, nsteps):
    from oracle import propagate
    pq = lib()
    cfg = _pw_cfg(D, n, nx, np_)
    b = pq.build_model(cfg)
    prob = propagate.problem_from_config(cfg)
    r = propagate.run(prob, cfg["q0"], cfg["p0"], cfg["width"], cfg["theta"], cfg["K"], cfg["dt"],
                      nsteps)
    s = pq.State(b, cfg["q0"], cfg["p0"], cfg["width"], cfg["theta"], precision=pq.FP64)
    s.propagate(cfg["K"], cfg["dt"], cfg["theta"], nsteps)
    o = s.observables()
    np.testing.assert_array_equal(o["n_active"], [x["n_active"] for x in r["obs"]])
    A, psi = s.read()
    np.testing.assert_array_equal(A, r["A"])
    assert np.linalg.norm(psi - r["a"]) <= 1e-10 * np.linalg.norm(r["a"])
    assert np.max(np.abs(o["C"] - np.array([x["C"] for x in r["obs"]]))) < 1e-10


def test_pw_double_well_propagation_fp64():
    # the double well of Sec. 3.1 in projected Weylets on its FGH grids
    # (165 and 81 functions per mode: point-parallel passes): identical active
    # sets on the (15 x 11) x (9 x 9) phase-space lattice, C(t) within 1e-10
    from oracle import propagate
    pq = lib()
    cfg = W.DWELL2D_PW
    n = 30
    b = pq.build_model(cfg)
    prob = propagate.problem_from_config(cfg)
    r = propagate.run(prob, cfg["q0"], cfg["p0"], cfg["width"], cfg["theta"], cfg["K"], cfg["dt"], n)
    s = pq.State(b, cfg["q0"], cfg["p0"], cfg["width"], cfg["theta"], precision=pq.FP64)
    s.propagate(cfg["K"], cfg["dt"], cfg["theta"], n)
    o = s.observables()
    np.testing.assert_array_equal(o["n_active"], [x["n_active"] for x in r["obs"]])
    A, psi = s.read()
    np.testing.assert_array_equal(A, r["A"])
    assert np.linalg.norm(psi - r["a"]) <= 1e-10 * np.linalg.norm(r["a"])
    assert np.max(np.abs(o["C"] - np.array([x["C"] for x in r["obs"]]))) < 1e-10


def _mixed_problem():
    """Mode 0 in projected Weylets (16 = 4 x 4 on a sine DVR), mode 1 a plain
    sine DVR (16 points): the library basis and the oracle's problem."""
    from oracle import bases, propagate
    pq = lib()
    cfg = W.MORSE3D
    n, lo, hi, m = 16, cfg["xmin"], cfg["xmax"], cfg["mass"]
    b = pq.Basis([dict(kind=pq.PW, n=n, xmin=lo, xmax=hi, mass=m, nx_lattice=4, np_lattice=4),
                  dict(kind=pq.SINE_DVR, n=n, xmin=lo, xmax=hi, mass=m)])
    grids = [b.grid(k)[0] for k in range(2)]
    b.set_sop(pq.coupled_morse_terms(grids, cfg["morse_D"], cfg["morse_a"], cfg["morse_qe"],
                                     cfg["coupling"]))
    x, w, T, Wm = bases.pw_basis(n, lo, hi, m, 4, 4)
    terms = propagate.morse_sop_terms([x, x], cfg["morse_D"], cfg["morse_a"], cfg["morse_qe"],
                                      cfg["coupling"])
    prob = propagate.PWProblem([x, x], [w, w], [T, T], [Wm, np.eye(n)], [(4, 4), (n,)], terms)
    return b, prob


@pytest.mark.parametrize("prec", [0, 1])
def test_mixed_pw_and_dvr_modes(prec):
    # a pW mode next to a DVR mode (SoP factors of the DVR mode used as they
    # are): H.psi parity on a random set, then 5 propagation steps with
    # identical active sets on the mixed lattice (axes 4, 4, 16)
    import torch
    from oracle import propagate, pruned
    pq = lib()
    b, prob = _mixed_problem()
    dims = (16, 16)
    A = W.random_active_set(dims, 0.5, seed=21)
    psi = W.random_psi(len(A), 22).astype(np.complex128 if prec == 0 else np.complex64)
    s = _state_with(b, A, psi, prec)
    x = torch.from_numpy(psi).to("cuda")
    y = torch.empty_like(x)
    s.apply_H(x, y)
    torch.cuda.synchronize()
    ref = prob.apply(A, psi.astype(np.complex128))
    absterms = [(abs(c), {k: np.abs(h) for k, h in f.items()}) for c, f in prob.terms]
    bound = pruned.apply_H_sop(A, np.abs(psi).astype(np.complex128), dims, absterms).real
    tol = 1e-12 if prec == 0 else 2e-5
    assert np.all(np.abs(y.cpu().numpy() - ref) <= tol * bound + 1e-300)
    if prec == 0:
        q0, p0, wd = (2.2, 2.35), (0.0, 0.0), (0.2, 0.2)
        r = propagate.run(prob, q0, p0, wd, 1e-6, 10, 10.0, 5)
        s2 = pq.State(b, q0, p0, wd, 1e-6, precision=pq.FP64)
        s2.propagate(10, 10.0, 1e-6, 5)
        o = s2.observables()
        np.testing.assert_array_equal(o["n_active"], [v["n_active"] for v in r["obs"]])
        assert np.max(np.abs(o["C"] - np.array([v["C"] for v in r["obs"]]))) < 1e-10


@pytest.mark.parametrize("prec", [0, 1])
def test_pw_double_well_apply(prec):
    # the point-parallel generic passes (165- and 81-function modes) on a
    # random subset of the double-well pW lattice
    import torch
    from oracle import propagate, pruned
    pq = lib()
    cfg = W.DWELL2D_PW
    b = pq.build_model(cfg)
    prob = propagate.problem_from_config(cfg)
    dims = prob.dims
    A = W.random_active_set(dims, 0.2, seed=31)
    psi = W.random_psi(len(A), 32).astype(np.complex128 if prec == 0 else np.complex64)
    s = _state_with(b, A, psi, prec)
    x = torch.from_numpy(psi).to("cuda")
    y = torch.empty_like(x)
    s.apply_H(x, y)
    torch.cuda.synchronize()
    ref = prob.apply(A, psi.astype(np.complex128))
    absterms = [(abs(c), {k: np.abs(h) for k, h in f.items()}) for c, f in prob.terms]
    bound = pruned.apply_H_sop(A, np.abs(psi).astype(np.complex128), dims, absterms).real
    tol = 1e-12 if prec == 0 else 5e-5
    err = np.abs(y.cpu().numpy() - ref)
    assert np.all(err <= tol * bound + 1e-300), (err / np.maximum(bound, 1e-300)).max()


def test_pw_rk4_small():
    # RK4 through the generic pW passes (FP64) against the oracle's RK4
    from oracle import propagate
    pq = lib()
    cfg = _pw_cfg(2, 16, 4, 4)
    b = pq.build_model(cfg)
    prob = propagate.problem_from_config(cfg)
    n, dt = 8, 2.0
    r = propagate.run(prob, cfg["q0"], cfg["p0"], cfg["width"], cfg["theta"], cfg["K"], dt, n,
                      integrator="rk4")
    s = pq.State(b, cfg["q0"], cfg["p0"], cfg["width"], cfg["theta"], precision=pq.FP64)
    s.propagate(cfg["K"], dt, cfg["theta"], n, integrator=pq.RK4)
    o = s.observables()
    np.testing.assert_array_equal(o["n_active"], [v["n_active"] for v in r["obs"]])
    assert np.max(np.abs(o["C"] - np.array([v["C"] for v in r["obs"]]))) < 1e-10
