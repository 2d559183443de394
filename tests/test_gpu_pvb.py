"""GPU parity of the pvB path (Sec. 2.2: biorthogonal projected von Neumann
basis; H_AA on the full grid, S_AA^-1 by conjugate gradients, Lanczos in the
S inner product) against the FP64 oracle (oracle/pvb.py)."""
import numpy as np
import pytest

import workloads as W
from gpu_helpers import lib

pytestmark = pytest.mark.gpu


def _cfg(D, n, nx, np_):
    return W.scaled(W.MORSE3D, basis="pvb", D=D, n=n, nx_lattice=nx, np_lattice=np_,
                    q0=W.morse3d_centres()[:D], p0=(0.0,) * D, width=(0.2,) * D)


def _abs_problem(prob):
    """The same full-grid chain with |B|, |T| and |V|: applied to |a| it bounds
    every product's magnitude (the rounding scale of each output)."""
    import copy
    q = copy.copy(prob)
    q.Bs = [np.abs(B) for B in prob.Bs]
    q.Ts = [np.abs(T) for T in prob.Ts]
    q.V = np.abs(prob.V)
    return q


def _assert_elementwise(got, ref, prob, A, a, tol):
    """|got - ref| <= tol * (the rounding scale of each element): 9 chained
    sums of up to 64 terms per output (B along 3 modes, T along 3 modes + V,
    B^dagger along 3 modes)."""
    bound = _abs_problem(prob).H_AA(A, np.abs(a).astype(np.complex128)).real
    err = np.abs(got - ref)
    assert np.all(err <= tol * bound + 1e-300), (err / np.maximum(bound, 1e-300)).max()


def _state_with(b, A, psi, prec):
    pq = lib()
    s = pq.State(b, [2.2] * b.D, [0.0] * b.D, [0.2] * b.D, 1e30, precision=prec)
    s.load(A, psi)
    return s


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("D,n,nx,np_,frac", [(2, 16, 4, 4, 0.5), (3, 16, 4, 4, 0.3), (1, 16, 4, 4, 0.8)])
def test_pvb_H_AA_random_sets(D, n, nx, np_, frac, prec):
    import torch
    from oracle import pvb
    pq = lib()
    cfg = _cfg(D, n, nx, np_)
    b = pq.build_model(cfg)
    prob = pvb.PVBProblem(cfg)
    A = W.random_active_set(prob.dims, frac, seed=D * 7 + n)
    psi = W.random_psi(len(A), 2).astype(np.complex128 if prec == 0 else np.complex64)
    s = _state_with(b, A, psi, prec)
    x = torch.from_numpy(psi).to("cuda")
    y = torch.empty_like(x)
    s.apply_H(x, y)
    torch.cuda.synchronize()
    got = y.cpu().numpy().astype(np.complex128)
    ref = prob.H_AA(A, psi.astype(np.complex128))
    _assert_elementwise(got, ref, prob, A, psi, 1e-12 if prec == 0 else 2e-5)


@pytest.mark.parametrize("prec", [0, 1])
def test_pvb_propagation_small(prec):
    from oracle import pvb
    pq = lib()
    cfg = _cfg(2, 16, 4, 4)
    b = pq.build_model(cfg)
    prob = pvb.PVBProblem(cfg)
    nsteps = 4
    r = pvb.run(prob, cfg["q0"], cfg["p0"], cfg["width"], cfg["theta"], cfg["K"], cfg["dt"], nsteps)
    s = pq.State(b, cfg["q0"], cfg["p0"], cfg["width"], cfg["theta"], precision=prec)
    s.propagate(cfg["K"], cfg["dt"], cfg["theta"], nsteps)
    o = s.observables()
    C = np.array([x["C"] for x in r["obs"]])
    n2 = np.array([x["norm2"] for x in r["obs"]])
    if prec == 0:
        np.testing.assert_array_equal(o["n_active"], [x["n_active"] for x in r["obs"]])
        A, a = s.read()
        np.testing.assert_array_equal(A, r["A"])
        assert np.linalg.norm(a - r["a"]) <= 1e-9 * np.linalg.norm(r["a"])
        assert np.max(np.abs(o["C"] - C)) < 1e-10
        assert np.max(np.abs(o["norm2"] - n2)) < 1e-10
    else:
        assert np.max(np.abs(o["C"] - C)) <= 1e-5
        assert np.max(np.abs(o["norm2"] - n2)) <= 1e-5


def test_pvb_morse3d_initial_state_and_H():
    """The 3D coupled Morse workload in pvB (64^3 grid, 8 x 8 lattices)."""
    import torch
    from oracle import pvb, pruned
    pq = lib()
    cfg = W.scaled(W.MORSE3D, basis="pvb", q0=W.morse3d_centres())
    b = pq.build_model(cfg)
    prob = pvb.PVBProblem(cfg)
    fa = prob.factors(cfg["q0"], cfg["p0"], cfg["width"], "G")
    full = np.arange(64 ** 3)
    a_full = pruned.product_on(full, prob.dims, fa)
    A = pruned.adapt_set(full[pruned.significant(a_full, cfg["theta"])], prob.axes)
    a = pruned.product_on(A, prob.dims, fa)
    s = pq.State(b, cfg["q0"], cfg["p0"], cfg["width"], cfg["theta"], precision=pq.FP64)
    Ag, ag = s.read()
    np.testing.assert_array_equal(Ag, A)
    np.testing.assert_allclose(ag, a, rtol=1e-11, atol=1e-11 * np.abs(a).max())
    x = torch.from_numpy(ag).to("cuda")
    y = torch.empty_like(x)
    s.apply_H(x, y)
    torch.cuda.synchronize()
    ref = prob.H_AA(A, a)
    _assert_elementwise(y.cpu().numpy(), ref, prob, A, a, 1e-12)
    o = s.observables()
    fb = prob.factors(cfg["q0"], cfg["p0"], cfg["width"], "B")
    C0 = np.vdot(pruned.product_on(A, prob.dims, fb), a)
    assert abs(o["C"][0] - C0) < 1e-11


def test_pvb_double_well():
    """The double well of Sec. 3.1 in pvB on its FGH grids (165- and
    81-function modes: the long-mode full-grid transforms): H_AA of the initial
    state and three propagation steps against the oracle (FP64)."""
    import torch
    from oracle import pvb
    pq = lib()
    cfg = W.DWELL2D_PVB
    b = pq.build_model(cfg)
    prob = pvb.PVBProblem(cfg)
    nsteps = 3
    r = pvb.run(prob, cfg["q0"], cfg["p0"], cfg["width"], cfg["theta"], cfg["K"], cfg["dt"], nsteps)
    s = pq.State(b, cfg["q0"], cfg["p0"], cfg["width"], cfg["theta"], precision=pq.FP64)
    A0, a0 = s.read()
    x = torch.from_numpy(a0).to("cuda")
    y = torch.empty_like(x)
    s.apply_H(x, y)
    torch.cuda.synchronize()
    ref = prob.H_AA(A0, a0)
    _assert_elementwise(y.cpu().numpy(), ref, prob, A0, a0, 1e-12)
    s.propagate(cfg["K"], cfg["dt"], cfg["theta"], nsteps)
    o = s.observables()
    np.testing.assert_array_equal(o["n_active"], [x["n_active"] for x in r["obs"]])
    A, a = s.read()
    np.testing.assert_array_equal(A, r["A"])
    assert np.linalg.norm(a - r["a"]) <= 1e-9 * np.linalg.norm(r["a"])
    assert np.max(np.abs(o["C"] - np.array([x["C"] for x in r["obs"]]))) < 1e-10
