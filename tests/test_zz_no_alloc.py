"""pq_observe_noalloc: the observables of the current state computed with a
fixed device scratch array instead of allocated scratch, for callers that
must not let the library allocate device memory (a framework allocator that
owns the budget, or step loops that must not synchronise on cudaMalloc /
cudaFree).  Checked through the C ABI against the observables the existing
entry point (pq_observables_get) records for the same state, on two calls in
a row with different states, sizes and precisions.  This file is collected
last so that a stop at the first failure has already run every other test."""
import numpy as np
import pytest

import workloads as W
from gpu_helpers import lib

pytestmark = pytest.mark.gpu


def _state(cfg, prec, nsteps):
    pq = lib()
    b = pq.build_model(cfg)
    s = pq.State(b, cfg["q0"], cfg["p0"], cfg["width"], cfg["theta"], precision=prec)
    s.propagate(cfg["K"], cfg["dt"], cfg["theta"], nsteps)
    return b, s


def _check(s, theta, tol):
    o = s.observables()                # newest record = the current state
    got = s.observe_noalloc(theta)
    assert abs(got["C"] - o["C"][-1]) <= tol
    assert abs(got["norm2"] - o["norm2"][-1]) <= tol
    assert got["n_wasted"] == o["n_wasted"][-1]


def test_observe_noalloc_two_calls_in_a_row():
    pq = lib()
    b1, s1 = _state(W.MORSE2D, pq.FP64, 3)
    b2, s2 = _state(W.HH4D, pq.FP32MIX, 2)
    # FP64 sums in another order: 1e-13; FP32 coefficients summed in FP64 vs
    # double-float: 1e-6 (the FP32 tolerance of the propagation tests)
    _check(s1, W.MORSE2D["theta"], 1e-13)
    _check(s2, W.HH4D["theta"], 1e-6)
    # the same state again after a larger one: stale scratch must not leak in
    _check(s1, W.MORSE2D["theta"], 1e-13)


def test_observe_noalloc_empty_state():
    pq = lib()
    b = pq.build_model(W.MORSE2D)
    s = pq.State(b, W.MORSE2D["q0"], W.MORSE2D["p0"], W.MORSE2D["width"], W.MORSE2D["theta"])
    s.load(np.zeros(0, np.int64))
    got = s.observe_noalloc(1e-6)
    assert got["C"] == 0 and got["norm2"] == 0 and got["n_wasted"] == 0


def test_observe_noalloc_refuses_pvb_states():
    """A pvB state's C and norm take the bra factors B^dagger f and
    a^dagger S_AA a (Sec. 2.2); the fixed-scratch reduction does not form them,
    so the call refuses such a state instead of returning DVR-form sums."""
    pq = lib()
    cfg = W.scaled(W.MORSE3D, basis="pvb", D=2, n=16, nx_lattice=4, np_lattice=4,
                   q0=W.morse3d_centres()[:2], p0=(0.0,) * 2, width=(0.2,) * 2)
    b = pq.build_model(cfg)
    s = pq.State(b, cfg["q0"], cfg["p0"], cfg["width"], cfg["theta"], precision=pq.FP64)
    with pytest.raises(pq.PQError) as e:
        s.observe_noalloc(cfg["theta"])
    assert e.value.status == pq.ENOTSUP
    # the refusal leaves the state usable
    assert s.observables()["norm2"][-1] > 0
