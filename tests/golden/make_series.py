"""Writes the expected per-step series of the workloads' pruned propagations
(tests/golden/series_<name>.json) from the FP64 oracle alone.

Nothing here touches the CUDA library: every stored number comes from
``oracle/`` (the propagation of Sec. 3.1 with the adaption of Sec. 2.5 after
every step) on the seeded inputs of ``workloads``.  Per recorded step the file
holds |A|, the count of coefficients below the threshold, C(t) (Eq. acorr),
||psi||^2 and E, and the SHA-256 of the active set (sorted int64 linear
indices, little-endian) so that a test can demand identical sets.  At the end
it holds a deterministic sample of the final coefficients (every stride-th
member of A) with their linear indices, and ||psi_final||.

The adjoint record (``adjoint4d``) holds the oracle's frozen-set central
finite-difference gradients of P = |C(T)|^2 at h = 1e-4 and h/2 for the nine
parameters (lambda, omega_1..4, q0_1..4), the sets frozen at those of the
unperturbed run, and their Richardson combination (4 g(h/2) - g(h)) / 3, whose
truncation error is O(h^4) instead of O(h^2): at T = 20 the third derivative of
P in lambda makes the plain h = 1e-4 difference err by 2e-3 relative.

Usage:  python tests/golden/make_series.py NAME [NSTEPS] [--workers N]
NAME is one of hh4d, hh6d, morse3d_pw, morse3d_pvb, adjoint4d.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import multiprocessing as mp
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

N_SAMPLE = 4096


def set_digest(A) -> str:
    return hashlib.sha256(np.ascontiguousarray(np.asarray(A, dtype="<i8")).tobytes()).hexdigest()


def sample(A, a):
    A = np.asarray(A, dtype=np.int64)
    stride = max(1, len(A) // N_SAMPLE)
    pos = np.arange(0, len(A), stride)[:N_SAMPLE]
    return dict(stride=int(stride), key=[int(v) for v in A[pos]],
                re=[float(v) for v in a[pos].real], im=[float(v) for v in a[pos].imag],
                norm=float(np.linalg.norm(a)))


def _record(obs, digests):
    return [dict(n_active=int(o["n_active"]), n_wasted=int(o.get("n_wasted", -1)),
                 C=[float(o["C"].real), float(o["C"].imag)], norm2=float(o["norm2"]),
                 E=float(o["E"]), set_sha256=d) for o, d in zip(obs, digests)]


def run_dvr(cfg, nsteps):
    from oracle import propagate
    prob = propagate.problem_from_config(cfg)
    r = propagate.run(prob, cfg["q0"], cfg["p0"], cfg["width"], cfg["theta"], cfg["K"], cfg["dt"],
                      nsteps, record_sets=True)
    return dict(steps=_record(r["obs"], [set_digest(A) for A in r["sets"]]),
                final=sample(r["A"], r["a"]))


def run_pw(cfg, nsteps):
    from oracle import propagate
    prob = propagate.problem_from_config(cfg)
    r = propagate.run(prob, cfg["q0"], cfg["p0"], cfg["width"], cfg["theta"], cfg["K"], cfg["dt"],
                      nsteps, record_sets=True)
    return dict(steps=_record(r["obs"], [set_digest(A) for A in r["sets"]]),
                final=sample(r["A"], r["a"]))


def run_pvb(cfg, nsteps):
    from oracle import pruned, pvb
    prob = pvb.PVBProblem(cfg)
    # the oracle's pvB run, step by step, so that each set is digested
    fa = prob.factors(cfg["q0"], cfg["p0"], cfg["width"], "G")
    fb = prob.factors(cfg["q0"], cfg["p0"], cfg["width"], "B")
    full = np.arange(int(np.prod(prob.dims)), dtype=np.int64)
    S0 = full[pruned.significant(pruned.product_on(full, prob.dims, fa), cfg["theta"])]
    A = pruned.adapt_set(S0, prob.axes, cfg["radius"])
    a = pruned.product_on(A, prob.dims, fa)

    def obs(A, a):
        c = pruned.product_on(A, prob.dims, fb)
        n2 = float(np.vdot(a, prob.S_AA(A, a)).real)
        E = float(np.vdot(a, prob.H_AA(A, a)).real) / n2 if n2 > 0 else 0.0
        return dict(C=complex(np.vdot(c, a)), norm2=n2, E=E, n_active=len(A),
                    n_wasted=int(np.count_nonzero(~pruned.significant(a, cfg["theta"]))))

    out, dig = [obs(A, a)], [set_digest(A)]
    for _ in range(nsteps):
        a = pvb.sil_step_S(prob, A, a, cfg["K"], cfg["dt"])
        A, a = pruned.prune(A, a, prob.axes, cfg["theta"], cfg["radius"])
        out.append(obs(A, a))
        dig.append(set_digest(A))
    return dict(steps=_record(out, dig), final=sample(A, a))


def _fd_one(args):
    cfg, params, sets, i, h = args
    from oracle import adjoint
    p1, p2 = np.array(params, float), np.array(params, float)
    p1[i] += h
    p2[i] -= h
    return (adjoint.survival(cfg, p1, sets)[0] - adjoint.survival(cfg, p2, sets)[0]) / (2 * h)


def run_adjoint(cfg, nsteps, workers):
    from oracle import adjoint, propagate
    prob = propagate.problem_from_config(cfg)
    r = propagate.run(prob, cfg["q0"], cfg["p0"], cfg["width"], cfg["theta"], cfg["K"], cfg["dt"],
                      nsteps, record_sets=True)
    sets = r["sets"]
    params = [cfg["lam"]] + [1.0] * cfg["D"] + list(cfg["q0"])
    P, C = adjoint.survival(cfg, params, sets)
    h = 1e-4
    npar = len(params)
    jobs = [(cfg, params, sets, i, hh) for hh in (h, h / 2) for i in range(npar)]
    with mp.get_context("spawn").Pool(workers) as pool:
        g = pool.map(_fd_one, jobs)
    g1, g2 = np.array(g[:npar]), np.array(g[npar:])
    rich = (4.0 * g2 - g1) / 3.0
    return dict(params=params, h=h, P=float(P), C=[float(C.real), float(C.imag)],
                grad=[float(v) for v in rich], grad_h=[float(v) for v in g1],
                grad_h2=[float(v) for v in g2],
                steps=_record(r["obs"], [set_digest(A) for A in sets]))


def config_of(name):
    if name == "morse3d_pw":
        return W.scaled(W.MORSE3D, q0=W.morse3d_centres(W.MORSE3D["seed"]))
    if name == "morse3d_pvb":
        return W.scaled(W.MORSE3D, basis="pvb", q0=W.morse3d_centres(W.MORSE3D["seed"]))
    return W.CONFIGS[name]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("name")
    ap.add_argument("nsteps", type=int, nargs="?")
    ap.add_argument("--workers", type=int, default=4)
    args = ap.parse_args()
    cfg = config_of(args.name)
    nsteps = args.nsteps if args.nsteps is not None else cfg["nsteps"]
    t0 = time.time()
    if args.name == "adjoint4d":
        body = run_adjoint(cfg, nsteps, args.workers)
    elif args.name == "morse3d_pvb":
        body = run_pvb(cfg, nsteps)
    elif args.name == "morse3d_pw":
        body = run_pw(cfg, nsteps)
    else:
        body = run_dvr(cfg, nsteps)
    rec = dict(workload=args.name, nsteps=nsteps,
               generator="tests/golden/make_series.py (FP64 oracle only)",
               oracle_seconds=round(time.time() - t0, 1), **body)
    path = os.path.join(HERE, f"series_{args.name}.json")
    with open(path, "w") as f:
        json.dump(rec, f, separators=(",", ":"))
    print(f"{path}: {nsteps} steps in {time.time() - t0:.0f} s")


if __name__ == "__main__":
    main()
