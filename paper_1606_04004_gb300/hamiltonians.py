"""Sum-of-products forms of the model Hamiltonians, tabulated on the
library's DVR grids (host set-up; Sec. 2.2.2 SoP form, Sec. 2.5: for a pruned DVR
the potential is a sum of products of diagonal factors).

Kinetic energy: one term per mode with the mode's kinetic factor.
Henon-Heiles chain: sum_k 1/2 omega_k^2 q_k^2 + lam sum_{k<D} (q_k^2 q_{k+1} - q_{k+1}^3 / 3).
Coupled Morse:      sum_k De (1 - exp(-a (q_k - qe)))^2 + c sum_{i<j} q_i q_j.
Double well (Sec. 3.1, Eq. ex_dwell): c1 (x-1)^2 (x-2)^2 + c2 (y-2)^2 + c3 x^2 y.
"""
from __future__ import annotations

import numpy as np


def kinetic_terms(D):
    return [(1.0, ["T" if k == m else None for k in range(D)]) for m in range(D)]


def henon_heiles_terms(grids, lam, omegas=None):
    D = len(grids)
    om = np.ones(D) if omegas is None else np.asarray(omegas, dtype=np.float64)
    terms = kinetic_terms(D)
    for k in range(D):
        f = [None] * D
        f[k] = grids[k] ** 2
        terms.append((0.5 * om[k] ** 2, f))
    for k in range(D - 1):
        f = [None] * D
        f[k] = grids[k] ** 2
        f[k + 1] = grids[k + 1]
        terms.append((lam, f))
        g = [None] * D
        g[k + 1] = grids[k + 1] ** 3
        terms.append((-lam / 3.0, g))
    return terms


def coupled_morse_terms(grids, De, a, qe, coupling):
    D = len(grids)
    terms = kinetic_terms(D)
    for k in range(D):
        f = [None] * D
        f[k] = De * (1.0 - np.exp(-a * (grids[k] - qe))) ** 2
        terms.append((1.0, f))
    for i in range(D):
        for j in range(i + 1, D):
            f = [None] * D
            f[i] = grids[i]
            f[j] = grids[j]
            terms.append((coupling, f))
    return terms


def double_well_terms(grids, c1, c2, c3):
    x, y = grids
    terms = kinetic_terms(2)
    terms.append((c1, [(x - 1.0) ** 2 * (x - 2.0) ** 2, None]))
    terms.append((c2, [None, (y - 2.0) ** 2]))
    terms.append((c3, [x * x, y]))
    return terms


def modes_of(cfg):
    """Mode descriptors of a workload record (see ``workloads``)."""
    from . import SINE_DVR, HO_DVR, PW, PVB, FGH_DVR
    if cfg["basis"] == "fgh":
        return [dict(kind=FGH_DVR, n=cfg["n"][k], xmin=cfg["xmin"][k], xmax=cfg["xmax"][k],
                     mass=cfg["mass"]) for k in range(cfg["D"])]
    if cfg["basis"] in ("pw", "pvb") and cfg.get("dvr") == "fgh":
        kind = PW if cfg["basis"] == "pw" else PVB
        return [dict(kind=kind, n=cfg["n"][k], xmin=cfg["xmin"][k], xmax=cfg["xmax"][k],
                     mass=cfg["mass"], nx_lattice=cfg["nx_lattice"][k],
                     np_lattice=cfg["np_lattice"][k], dvr=FGH_DVR) for k in range(cfg["D"])]
    if cfg["basis"] in ("pw", "pvb"):
        kind = PW if cfg["basis"] == "pw" else PVB
        return [dict(kind=kind, n=cfg["n"], xmin=cfg["xmin"], xmax=cfg["xmax"], mass=cfg["mass"],
                     nx_lattice=cfg["nx_lattice"], np_lattice=cfg["np_lattice"])] * cfg["D"]
    if cfg["basis"] == "sine":
        return [dict(kind=SINE_DVR, n=cfg["n"], xmin=cfg["xmin"], xmax=cfg["xmax"],
                     mass=cfg["mass"])] * cfg["D"]
    if cfg["basis"] == "ho":
        return [dict(kind=HO_DVR, n=cfg["n"], mass=cfg.get("mass", 1.0),
                     omega=cfg.get("omega", 1.0))] * cfg["D"]
    raise ValueError(cfg["basis"])


def build_model(cfg, omegas=None, lam=None):
    """Basis with the workload's SoP Hamiltonian set."""
    from . import Basis
    b = Basis(modes_of(cfg))
    grids = [b.grid(k)[0] for k in range(b.D)]
    if "dw_coef" in cfg:
        terms = double_well_terms(grids, *cfg["dw_coef"])
    elif cfg["basis"] in ("sine", "pw", "pvb"):
        terms = coupled_morse_terms(grids, cfg["morse_D"], cfg["morse_a"], cfg["morse_qe"],
                                    cfg["coupling"])
    else:
        terms = henon_heiles_terms(grids, cfg["lam"] if lam is None else lam, omegas)
    b.set_sop(terms)
    return b


def henon_heiles_param_derivs(grids, lam, omegas=None):
    """Parameters of the Henon-Heiles workload for the survival gradient, in
    the order (lambda, omega_1..omega_D, q0_1..q0_D): dH/dlambda =
    sum_k (q_k^2 q_{k+1} - q_{k+1}^3/3), dH/domega_k = omega_k q_k^2, and the
    packet centres."""
    D = len(grids)
    om = np.ones(D) if omegas is None else np.asarray(omegas, dtype=np.float64)
    dlam = []
    for k in range(D - 1):
        f = [None] * D
        f[k] = grids[k] ** 2
        f[k + 1] = grids[k + 1]
        dlam.append((1.0, f))
        g = [None] * D
        g[k + 1] = grids[k + 1] ** 3
        dlam.append((-1.0 / 3.0, g))
    params = [("potential", dlam)]
    for k in range(D):
        f = [None] * D
        f[k] = grids[k] ** 2
        params.append(("potential", [(float(om[k]), f)]))
    params += [("centre", k) for k in range(D)]
    return params
