"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and bench.py.

This module holds plain parameter records and random-number draws only: it
contains none of the method's arithmetic (no basis construction, no
Hamiltonian, no propagation, no prune rule).  Both the CUDA library and the
oracle consume what it returns, each through its own code.

Workloads (parameters in atomic units unless stated):

* ``morse2d`` -- 2D coupled Morse, sine-DVR 32 points per mode on the box
  [0.5, 6] bohr, m = 1836, D = 0.1, a = 1, coupling 0.005 q1 q2, Gaussian
  packet at (2.3, 2.3) with position standard deviation 0.2, SIL order 8,
  dt = 10, 200 steps, threshold 1e-6, FP64.
* ``hh4d`` -- 4D Henon-Heiles chain, lambda = 0.111803, HO-DVR 24 points per
  mode (hbar = m = omega = 1), coherent packet at q_k = 2 (standard deviation
  1/sqrt 2), SIL order 10, dt = 0.1, 1000 steps, threshold 1e-7.
* ``hh6d`` -- the same chain in 6D (24^6 = 1.91e8 lattice points), threshold
  1e-6, 500 steps; the throughput workload.
* ``morse3d`` -- 3D coupled Morse (pairwise 0.005 q_i q_j), 64-point sine-DVR
  per mode, phase-space lattices of 8 x 8 per mode, seed-drawn packet centres,
  SIL order 10, dt = 2 (not stated for this workload: at dt = 10 the order-10
  step on this grid errs by 2e-5 and amplifies rounding differences about
  1000-fold per 100 time units; at dt = 2 it errs by 5e-11 and does not),
  400 steps, threshold 1e-6.
* ``adjoint4d`` -- the hh4d model, T = 20, checkpoint every 25 steps.
* ``dwell2d`` -- the two-dimensional double well of Sec. 3.1 as printed there
  (mass 200, potential coefficients 6.4, 37.5 and 10, packet centre (2.1, 2.05)
  with exponents 1/0.04 and 1/0.02, final time 24.6) on FGH grids of 165
  points on [-0.5, 3.7) and 81 points on [1.0, 2.9); SIL order 10, dt = 0.01
  (not given in the paper; at dt = 0.05 the order-10 step error is 5e-5),
  2460 steps.
* ``dwell2d_pw`` / ``dwell2d_pvb`` -- the same double well in projected
  Weylets / in the biorthogonal projected von Neumann basis, built on those FGH
  grids (Sec. 3.1): phase-space lattices 15 x 11 (x) and 9 x 9 (y).
"""
from __future__ import annotations

import numpy as np

MORSE2D = dict(
    name="morse2d", D=2, basis="sine", n=32, xmin=0.5, xmax=6.0, mass=1836.0,
    morse_D=0.1, morse_a=1.0, morse_qe=2.0, coupling=0.005,
    q0=(2.3, 2.3), p0=(0.0, 0.0), width=(0.2, 0.2),
    K=8, dt=10.0, nsteps=200, theta=1e-6, radius=1,
)

HH4D = dict(
    name="hh4d", D=4, basis="ho", n=24, mass=1.0, omega=1.0, lam=0.111803,
    q0=(2.0,) * 4, p0=(0.0,) * 4, width=(0.5 ** 0.5,) * 4,
    K=10, dt=0.1, nsteps=1000, theta=1e-7, radius=1,
)

HH6D = dict(
    name="hh6d", D=6, basis="ho", n=24, mass=1.0, omega=1.0, lam=0.111803,
    q0=(2.0,) * 6, p0=(0.0,) * 6, width=(0.5 ** 0.5,) * 6,
    K=10, dt=0.1, nsteps=500, theta=1e-6, radius=1,
)

MORSE3D = dict(
    name="morse3d", D=3, basis="pw", n=64, xmin=0.5, xmax=6.0, mass=1836.0,
    morse_D=0.1, morse_a=1.0, morse_qe=2.0, coupling=0.005,
    nx_lattice=8, np_lattice=8, width=(0.2,) * 3, p0=(0.0,) * 3,
    K=10, dt=2.0, nsteps=400, theta=1e-6, radius=1, seed=1606,
)

ADJOINT4D = dict(HH4D, name="adjoint4d", nsteps=200, ckpt_every=25)

DWELL2D = dict(
    name="dwell2d", D=2, basis="fgh", n=(165, 81), xmin=(-0.5, 1.0), xmax=(3.7, 2.9),
    mass=200.0, dw_coef=(6.4, 37.5, 10.0),
    q0=(2.1, 2.05), p0=(0.0, 0.0), width=(0.1, 0.005 ** 0.5),
    K=10, dt=0.01, nsteps=2460, theta=1e-5, radius=1,
)

DWELL2D_PW = dict(DWELL2D, name="dwell2d_pw", basis="pw", dvr="fgh",
                  nx_lattice=(15, 9), np_lattice=(11, 9))

DWELL2D_PVB = dict(DWELL2D_PW, name="dwell2d_pvb", basis="pvb")

CONFIGS = {c["name"]: c for c in (MORSE2D, HH4D, HH6D, MORSE3D, ADJOINT4D, DWELL2D, DWELL2D_PW,
                                    DWELL2D_PVB)}


def morse3d_centres(seed: int = 1606) -> tuple:
    """Packet centres of the 3D Morse workload: q0_k ~ U[2.1, 2.5] (PCG64)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return tuple(float(v) for v in rng.uniform(2.1, 2.5, size=3))


def scaled(cfg: dict, **over) -> dict:
    """A copy of a workload record with some fields replaced (smaller cases)."""
    out = dict(cfg)
    out.update(over)
    return out


def random_psi(n: int, seed: int, dtype=np.complex128) -> np.ndarray:
    """Complex standard-normal coefficients (PCG64), one per active point."""
    rng = np.random.Generator(np.random.PCG64(seed))
    v = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    return v.astype(dtype)


def random_active_set(dims, frac: float, seed: int) -> np.ndarray:
    """Sorted int64 linear indices (row-major, last mode fastest) of a random
    subset of the direct-product lattice, each point kept with probability
    ``frac``."""
    rng = np.random.Generator(np.random.PCG64(seed))
    total = int(np.prod(dims))
    keep = rng.random(total) < frac
    return np.flatnonzero(keep).astype(np.int64)


def ellipsoid_active_set(dims, radii, centre=None) -> np.ndarray:
    """Sorted int64 linear indices of the lattice points inside the ellipsoid
    sum_k ((i_k - c_k) / r_k)^2 <= 1 (the shape a Gaussian packet's active set
    takes); ``centre`` defaults to the lattice centre.  Built one value of the
    first digit at a time so that 6D lattices fit in host memory."""
    dims = tuple(int(d) for d in dims)
    if centre is None:
        centre = [(d - 1) / 2.0 for d in dims]
    rest = np.zeros(dims[1:], dtype=np.float64) if len(dims) > 1 else np.zeros(())
    for k, d in enumerate(dims[1:], start=1):
        shape = [1] * (len(dims) - 1)
        shape[k - 1] = d
        rest = rest + (((np.arange(d) - centre[k]) / radii[k]) ** 2).reshape(shape)
    rest = rest.ravel()
    stride0 = rest.size
    out = []
    for i0 in range(dims[0]):
        lim = 1.0 - ((i0 - centre[0]) / radii[0]) ** 2
        if lim < 0:
            continue
        out.append(np.flatnonzero(rest <= lim).astype(np.int64) + i0 * stride0)
    return np.concatenate(out) if out else np.zeros(0, np.int64)
