"""The workload records and the oracle against values the paper prints
(tests/golden/paper_printed_values.json, typed in from the text)."""
import json
import os

import numpy as np

import workloads as W
from oracle import models, pruned

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden",
                                   "paper_printed_values.json")))


def test_double_well_record_is_the_printed_model():
    g = GOLD["double_well"]
    cfg = W.DWELL2D
    # -1/(2 m) (d2/dx2 + d2/dy2) with the printed prefactor 1/(2 x 200)
    assert abs(1.0 / (2.0 * cfg["mass"]) - g["kinetic_prefactor"]) < 1e-15
    assert cfg["mass"] == g["mass"]
    p = g["potential"]
    assert tuple(cfg["dw_coef"]) == (p["c_x"], p["c_y"], p["c_xxy"])
    # the oracle's potential at a few points against the printed formula
    for x, y in [(1.0, 2.0), (2.0, 2.0), (1.5, 1.7), (2.1, 2.05), (-0.3, 2.8)]:
        ref = (p["c_x"] * (x - p["x_roots"][0]) ** 2 * (x - p["x_roots"][1]) ** 2
               + p["c_y"] * (y - p["y_min"]) ** 2 + p["c_xxy"] * x * x * y)
        assert abs(models.double_well(np.array([x, y]), *cfg["dw_coef"]) - ref) < 1e-12
    assert tuple(cfg["q0"]) == tuple(g["packet_centre"])
    # exp(-(q - q0)^2 / d) = exp(-(q - q0)^2 / (4 w^2)) with w the width
    for w, d in zip(cfg["width"], g["packet_exponent_denominators"]):
        assert abs(4.0 * w * w - d) < 1e-15
    assert abs(cfg["dt"] * cfg["nsteps"] - g["t_end"]) < 1e-9
    assert (cfg["xmin"][0], cfg["xmax"][0]) == tuple(g["x_range"])
    assert (cfg["xmin"][1], cfg["xmax"][1]) == tuple(g["y_range"])
    pw = W.DWELL2D_PW
    assert (pw["nx_lattice"][0], pw["np_lattice"][0]) == tuple(g["lattice_x"])
    assert (pw["nx_lattice"][1], pw["np_lattice"][1]) == tuple(g["lattice_y"])
    assert int(np.prod(cfg["n"])) == g["basis_size"]
    assert cfg["n"] == (g["lattice_x"][0] * g["lattice_x"][1], g["lattice_y"][0] * g["lattice_y"][1])


def test_neighbour_counts_in_phase_space():
    # a D-dimensional phase-space lattice has k = 2D axes: 2k = 4D, 2k^2 = 8D^2,
    # 3^k - 1 = 3^(2D) - 1 (the paper's 3^(2D) - 1 for radius 2)
    for D in (1, 2):
        axes = (5,) * (2 * D)
        c = np.array([int(np.ravel_multi_index((2,) * (2 * D), axes))])
        assert len(pruned.adapt_set(c, axes, pruned.RADIUS_2)) - 1 == 3 ** (2 * D) - 1
        assert len(pruned.adapt_set(c, axes, pruned.RADIUS_1)) - 1 == 2 * (2 * D)


def _printed(total, me):
    """The total as the paper prints it, ~m x 10^e (digits truncated)."""
    m, e = me
    return int(total // 10 ** e) == m


def test_printed_basis_sizes_are_consistent():
    # the per-mode sizes of Table I multiply (times the two electronic states)
    # to the printed total of about 322 x 10^6; the NO2 basis (two radial FGH
    # modes of 13 x 13 and an angular 10 x 10) to about 285 x 10^4
    py = GOLD["pyrazine_basis"]
    n = [a * b for a, b in zip(py["nx"], py["np"])]
    total = int(np.prod(n)) * py["electronic_states"]
    assert _printed(total, py["total_printed_mantissa_exponent"])
    no2 = GOLD["no2_basis"]
    r = no2["radial_nx_np"][0] * no2["radial_nx_np"][1]
    t = r ** no2["radial_coordinates"] * no2["angular_nx_np"][0] * no2["angular_nx_np"][1]
    assert _printed(t, no2["total_printed_mantissa_exponent"])


def test_hh6d_workload_is_pyrazine_sized():
    # the 6D throughput workload stands in for the 6D pyrazine benchmark: six
    # modes and a direct-product lattice within a factor 1.5 of pyrazine's
    # per-electronic-state basis (24^6 = 1.91e8 against 1.61e8)
    py = GOLD["pyrazine_basis"]
    per_state = int(np.prod([a * b for a, b in zip(py["nx"], py["np"])]))
    cfg = W.HH6D
    assert cfg["D"] == len(py["modes"])
    ratio = cfg["n"] ** cfg["D"] / per_state
    assert 1 / 1.5 < ratio < 1.5
