"""Adjoint gradient of the survival probability on the GPU (pq_survival_grad)
against central finite differences (h = 1e-4) of the FP64 oracle with the
sets of active functions frozen, relative error <= 1e-4 (norm-wise, and per
component against the largest component)."""
import numpy as np
import pytest

import workloads as W
from gpu_helpers import lib

pytestmark = pytest.mark.gpu


def _reduced(nsteps=6):
    # 4D Henon-Heiles with 12 HO-DVR points per mode, short horizon so that
    # P stays O(0.1) and the finite differences are well conditioned
    return W.scaled(W.HH4D, n=12, nsteps=nsteps)


def _gpu_grad(cfg, prec, ckpt):
    pq = lib()
    b = pq.build_model(cfg)
    s = pq.State(b, cfg["q0"], cfg["p0"], cfg["width"], cfg["theta"], precision=prec)
    grids = [b.grid(k)[0] for k in range(cfg["D"])]
    return s.survival_grad(cfg["K"], cfg["dt"], cfg["theta"], cfg["nsteps"], ckpt,
                           pq.henon_heiles_param_derivs(grids, cfg["lam"]))


_FD_CACHE = {}


def _oracle_fd(cfg):
    key = (cfg["n"], cfg["nsteps"])
    if key not in _FD_CACHE:
        _FD_CACHE[key] = _oracle_fd_compute(cfg)
    return _FD_CACHE[key]


def _oracle_fd_compute(cfg):
    from oracle import adjoint, propagate
    prob = propagate.problem_from_config(cfg)
    r = propagate.run(prob, cfg["q0"], cfg["p0"], cfg["width"], cfg["theta"], cfg["K"], cfg["dt"],
                      cfg["nsteps"], record_sets=True)
    params = [cfg["lam"]] + [1.0] * cfg["D"] + list(cfg["q0"])
    P, C = adjoint.survival(cfg, params, r["sets"])
    return P, adjoint.fd_gradient(cfg, params, r["sets"], h=1e-4)


@pytest.mark.parametrize("prec,ckpt", [(0, 2), (0, 100), (1, 3)])
def test_adjoint_vs_oracle_fd(prec, ckpt):
    cfg = _reduced()
    P_ref, g_ref = _oracle_fd(cfg)
    P, g = _gpu_grad(cfg, prec, ckpt)
    assert abs(P - P_ref) <= (1e-12 if prec == 0 else 1e-6) * max(P_ref, 1e-300)
    scale = np.abs(g_ref).max()
    assert np.linalg.norm(g - g_ref) <= 1e-4 * np.linalg.norm(g_ref), (g, g_ref)
    assert np.all(np.abs(g - g_ref) <= 1e-4 * scale), (g, g_ref)


def _golden_adjoint():
    import json
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "series_adjoint4d.json")
    with open(path) as f:
        return json.load(f)


@pytest.mark.parametrize("prec", [0, 1])
def test_adjoint_full_config(prec):
    """The adjoint workload as specified (4D Henon-Heiles, 24 points per mode,
    T = 20 in 200 steps, checkpoints every 25 steps) against the FP64 oracle's
    frozen-set finite differences stored by tests/golden/make_series.py.  The
    reference is the Richardson combination of the central differences at
    h = 1e-4 and h/2 (truncation error O(h^4)): relative error <= 1e-4,
    norm-wise and per component against the largest.  Against the plain
    h = 1e-4 difference the gradient agrees within that difference's own
    truncation error (estimated from h and h/2) plus 1e-4.  prec 1 is the
    FP32-mix forward run (its own sets and checkpoints) with the FP64 reverse
    sweep."""
    g = _golden_adjoint()
    cfg = W.ADJOINT4D
    assert g["nsteps"] == cfg["nsteps"]
    ref = np.array(g["grad"])
    P, grad = _gpu_grad(cfg, prec, cfg["ckpt_every"])
    assert abs(P - g["P"]) <= (1e-10 if prec == 0 else 1e-4) * g["P"]
    assert np.linalg.norm(grad - ref) <= 1e-4 * np.linalg.norm(ref), (grad, ref)
    assert np.all(np.abs(grad - ref) <= 1e-4 * np.abs(ref).max()), (grad, ref)
    gh, gh2 = np.array(g["grad_h"]), np.array(g["grad_h2"])
    trunc = 4.0 / 3.0 * np.abs(gh - gh2)
    assert np.all(np.abs(grad - gh) <= trunc + 1e-4 * np.abs(ref).max()), (grad, gh, trunc)


def test_adjoint_checkpoint_interval_is_exact():
    """FP64: the recomputation replays the forward run exactly, so the
    gradient does not depend on the checkpoint interval."""
    cfg = W.ADJOINT4D
    P64, g64 = _gpu_grad(cfg, 0, cfg["ckpt_every"])
    P64b, g64b = _gpu_grad(cfg, 0, 2 * cfg["ckpt_every"])
    assert P64 > 0 and P64b == P64
    np.testing.assert_allclose(g64b, g64, rtol=1e-12, atol=1e-15)


def test_autograd_function():
    import torch
    from paper_1606_04004_gb300.autograd import survival_probability
    pq = lib()
    cfg = _reduced(4)
    theta = torch.tensor([cfg["lam"]] + [1.0] * 4 + list(cfg["q0"]), dtype=torch.float64,
                         requires_grad=True)
    P = survival_probability(theta, cfg, pq.FP64, 2)
    P.backward()
    _, g = _gpu_grad(cfg, 0, 2)
    np.testing.assert_allclose(theta.grad.numpy(), g, rtol=1e-12, atol=0)


def test_adjoint_fp32_after_propagation_matches_fresh_state():
    """An FP32-mix state that was propagated before gives the same P and
    gradient as a fresh one: the gradient's run restarts from the packet, and
    the norm keeping of the earlier propagation does not carry over."""
    pq = lib()
    cfg = _reduced(4)
    b = pq.build_model(cfg)
    grids = [b.grid(k)[0] for k in range(cfg["D"])]
    derivs = pq.henon_heiles_param_derivs(grids, cfg["lam"])
    res = []
    for warm in (0, 30):
        s = pq.State(b, cfg["q0"], cfg["p0"], cfg["width"], cfg["theta"], precision=pq.FP32MIX)
        if warm:
            s.propagate(cfg["K"], cfg["dt"], cfg["theta"], warm)
        res.append(s.survival_grad(cfg["K"], cfg["dt"], cfg["theta"], cfg["nsteps"], 2, derivs))
        s.free()
    assert res[0][0] == res[1][0]
    np.testing.assert_array_equal(res[0][1], res[1][1])
