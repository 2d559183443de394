"""The stored per-step series (tests/golden/series_*.json) are the FP64
oracle's: the first steps of each are recomputed here by the script that wrote
them (tests/golden/make_series.py, oracle only) and must agree with the file.
The series pin the GPU propagation over the workloads' stated run lengths
(tests/test_gpu_series.py)."""
import json
import os

import numpy as np
import pytest

import workloads as W

HERE = os.path.join(os.path.dirname(__file__), "golden")


def _load(name):
    with open(os.path.join(HERE, f"series_{name}.json")) as f:
        return json.load(f)


def _script():
    import importlib.util
    spec = importlib.util.spec_from_file_location("make_series", os.path.join(HERE, "make_series.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _same_steps(got, ref, k):
    for a, b in zip(got[:k], ref[:k]):
        assert a["n_active"] == b["n_active"] and a["n_wasted"] == b["n_wasted"]
        assert a["set_sha256"] == b["set_sha256"]
        np.testing.assert_allclose(a["C"], b["C"], rtol=0, atol=1e-13)
        assert abs(a["norm2"] - b["norm2"]) <= 1e-13
        assert abs(a["E"] - b["E"]) <= 1e-12 * abs(b["E"])


@pytest.mark.parametrize("name,k", [("hh4d", 4), ("morse3d_pw", 2)])
def test_series_file_is_the_oracle_run(name, k):
    rec = _load(name)
    mk = _script()
    cfg = mk.config_of(name)
    assert rec["nsteps"] == cfg["nsteps"], "the series must cover the workload's stated length"
    body = mk.run_dvr(cfg, k) if name != "morse3d_pw" else mk.run_pw(cfg, k)
    _same_steps(body["steps"], rec["steps"], k + 1)


def test_adjoint_record_is_the_oracle_run():
    rec = _load("adjoint4d")
    mk = _script()
    cfg = W.ADJOINT4D
    assert rec["nsteps"] == cfg["nsteps"] and rec["h"] == 1e-4
    assert rec["params"] == [cfg["lam"]] + [1.0] * cfg["D"] + list(cfg["q0"])
    body = mk.run_dvr(cfg, 3)
    _same_steps(body["steps"], rec["steps"], 4)
    # the stored reference is the Richardson combination of the central
    # differences at h and h/2 that the record also holds
    g, g1, g2 = (np.array(rec[k]) for k in ("grad", "grad_h", "grad_h2"))
    assert np.all(np.isfinite(g)) and 0 < rec["P"] < 1
    np.testing.assert_allclose(g, (4.0 * g2 - g1) / 3.0, rtol=1e-13, atol=1e-15)


def test_pvb_and_hh6d_records_cover_their_stated_lengths():
    # recomputing these takes an hour or more (full-grid conjugate gradients, a
    # 24^6 lattice); their provenance is the same script, checked above on the
    # other workloads.  The lengths asserted here: pvB 60 steps, hh6d 20 (the
    # window the hh6d benchmark times, steps 3-23, up to step 20).
    pvb = _load("morse3d_pvb")
    assert pvb["nsteps"] >= 60 and len(pvb["steps"]) == pvb["nsteps"] + 1
    hh6 = _load("hh6d")
    assert hh6["nsteps"] >= 20 and len(hh6["steps"]) == hh6["nsteps"] + 1
