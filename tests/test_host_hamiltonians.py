"""CPU checks of the library's host-side Hamiltonian set-up
(``paper_1606_04004_gb300.hamiltonians``): the sum-of-products terms it hands
to ``pq_set_sop``, summed over the full grid, must equal the oracle's
potentials written as plain functions of the coordinates, and the
parameter-derivative terms of the survival gradient must equal the
derivatives of those functions.  No GPU is needed."""
import numpy as np
import pytest

import workloads as W
from oracle import bases, models


def _hmod():
    try:
        from paper_1606_04004_gb300 import hamiltonians
    except ImportError as e:   # the library must be built first
        pytest.fail(f"library not built: {e}")
    return hamiltonians


def _sum_on_grid(terms, grids):
    """Sum of the potential terms (kinetic factors skipped) as a dense array
    over the direct-product grid, row-major."""
    dims = tuple(len(g) for g in grids)
    V = np.zeros(dims)
    nkin = 0
    for coef, facs in terms:
        if any(isinstance(f, str) for f in facs):
            assert sum(isinstance(f, str) for f in facs) == 1 and all(
                f is None for f in facs if not isinstance(f, str))
            nkin += 1
            continue
        t = np.full(dims, float(coef))
        for k, f in enumerate(facs):
            if f is None:
                continue
            shape = [1] * len(dims)
            shape[k] = dims[k]
            t = t * np.asarray(f, dtype=np.float64).reshape(shape)
        V += t
    return V, nkin


def _mesh(grids):
    return np.stack(np.meshgrid(*grids, indexing="ij"), axis=-1)


def test_henon_heiles_terms_equal_the_potential():
    H = _hmod()
    x, _, _ = bases.ho_dvr(9)
    grids = [x, 0.9 * x, 1.1 * x]
    om = np.array([1.0, 0.7, 1.3])
    V, nkin = _sum_on_grid(H.henon_heiles_terms(grids, 0.111803, om), grids)
    assert nkin == 3
    np.testing.assert_allclose(V, models.henon_heiles(_mesh(grids), 0.111803, om),
                               rtol=1e-13, atol=1e-13)


def test_coupled_morse_terms_equal_the_potential():
    H = _hmod()
    x, _, _ = bases.sine_dvr(7, 0.5, 6.0, 1836.0)
    grids = [x, x[::-1] * 0.9 + 0.3, x + 0.1]
    V, nkin = _sum_on_grid(H.coupled_morse_terms(grids, 0.1, 1.0, 2.0, 0.005), grids)
    assert nkin == 3
    np.testing.assert_allclose(V, models.coupled_morse(_mesh(grids), 0.1, 1.0, 2.0, 0.005),
                               rtol=1e-13, atol=1e-15)


def test_double_well_terms_equal_the_printed_model():
    H = _hmod()
    cfg = W.DWELL2D
    grids = [bases.fgh_dvr(cfg["n"][k], cfg["xmin"][k], cfg["xmax"][k], cfg["mass"])[0]
             for k in range(2)]
    V, nkin = _sum_on_grid(H.double_well_terms(grids, *cfg["dw_coef"]), grids)
    assert nkin == 2
    np.testing.assert_allclose(V, models.double_well(_mesh(grids), *cfg["dw_coef"]),
                               rtol=1e-13, atol=1e-12)


def test_henon_heiles_parameter_derivatives():
    # dV/dlambda and dV/domega_k against central differences of the oracle's
    # potential (exact up to rounding: V is linear in lambda, quadratic in
    # omega_k); the centre parameters come last, one per mode.
    H = _hmod()
    x, _, _ = bases.ho_dvr(8)
    grids = [x, 1.2 * x, 0.8 * x]
    lam, om = 0.111803, np.array([1.0, 0.6, 1.4])
    q = _mesh(grids)
    params = H.henon_heiles_param_derivs(grids, lam, om)
    assert [p[0] for p in params] == ["potential"] * 4 + ["centre"] * 3
    assert [p[1] for p in params[4:]] == [0, 1, 2]
    h = 1e-3
    ref = [(models.henon_heiles(q, lam + h, om) - models.henon_heiles(q, lam - h, om)) / (2 * h)]
    for k in range(3):
        op, omm = om.copy(), om.copy()
        op[k] += h
        omm[k] -= h
        ref.append((models.henon_heiles(q, lam, op) - models.henon_heiles(q, lam, omm)) / (2 * h))
    for (kind, terms), r in zip(params[:4], ref):
        V, nkin = _sum_on_grid(terms, grids)
        assert nkin == 0
        np.testing.assert_allclose(V, r, rtol=1e-9, atol=1e-9)


def test_modes_of_every_workload():
    # mode descriptors: one per mode, the workload's sizes and boxes
    H = _hmod()
    import paper_1606_04004_gb300 as pq
    for name, cfg in W.CONFIGS.items():
        modes = H.modes_of(cfg)
        assert len(modes) == cfg["D"], name
        for k, m in enumerate(modes):
            n = cfg["n"][k] if isinstance(cfg["n"], tuple) else cfg["n"]
            assert m["n"] == n, name
            kind = {"sine": pq.SINE_DVR, "ho": pq.HO_DVR, "fgh": pq.FGH_DVR,
                    "pw": pq.PW, "pvb": pq.PVB}[cfg["basis"]]
            assert m["kind"] == kind, name
            if cfg["basis"] in ("pw", "pvb"):
                nx = cfg["nx_lattice"][k] if isinstance(cfg["nx_lattice"], tuple) else cfg["nx_lattice"]
                npl = cfg["np_lattice"][k] if isinstance(cfg["np_lattice"], tuple) else cfg["np_lattice"]
                assert (m["nx_lattice"], m["np_lattice"]) == (nx, npl) and nx * npl == n, name
