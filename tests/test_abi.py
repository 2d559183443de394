"""CPU checks of the C ABI: the library loads, exports every function that
include/prunedq.h declares, and its host-side basis construction (no GPU
needed) agrees with the oracle's independent construction."""
import os
import re

import numpy as np
import pytest

import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _lib():
    try:
        import paper_1606_04004_gb300 as pq
    except ImportError as e:   # the library must be built first
        pytest.fail(f"library not built: {e}")
    return pq


def declared_functions():
    txt = open(os.path.join(ROOT, "include", "prunedq.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(pq_[A-Za-z0-9_]+)\s*\(", txt)))


def test_header_symbols_exported():
    import ctypes
    pq = _lib()
    lib = ctypes.CDLL(pq.lib_path())
    names = declared_functions()
    assert "pq_apply_H" in names and "pq_propagate" in names
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(pq.EXPORTS)


def test_host_bases_match_oracle():
    from oracle import bases
    pq = _lib()
    b = pq.Basis(pq.modes_of(W.HH4D))
    x, w, T = bases.ho_dvr(24)
    xl, wl = b.grid(0)
    np.testing.assert_allclose(xl, x, atol=1e-13)
    np.testing.assert_allclose(wl, w, rtol=1e-12)
    np.testing.assert_allclose(b.kinetic(0), T, atol=1e-12)
    b = pq.Basis(pq.modes_of(W.MORSE2D))
    x, w, T = bases.sine_dvr(32, 0.5, 6.0, 1836.0)
    xl, wl = b.grid(1)
    np.testing.assert_allclose(xl, x, atol=1e-14)
    np.testing.assert_allclose(wl, w, rtol=1e-14)
    np.testing.assert_allclose(b.kinetic(1), T, atol=1e-14 * abs(T).max())
    b = pq.Basis(pq.modes_of(W.DWELL2D))
    for k in range(2):
        cfg = W.DWELL2D
        x, w, T = bases.fgh_dvr(cfg["n"][k], cfg["xmin"][k], cfg["xmax"][k], cfg["mass"])
        xl, wl = b.grid(k)
        np.testing.assert_allclose(xl, x, atol=1e-14)
        np.testing.assert_allclose(wl, w, rtol=1e-14)
        np.testing.assert_allclose(b.kinetic(k), T, atol=1e-12 * abs(T).max())


def test_pw_on_fgh_matches_oracle():
    # projected Weylets on the FGH grids of the double well (165 and 81 points)
    from oracle import bases
    pq = _lib()
    cfg = W.DWELL2D_PW
    b = pq.Basis(pq.modes_of(cfg))
    for k in range(2):
        x, w, T, Wm = bases.pw_basis(cfg["n"][k], cfg["xmin"][k], cfg["xmax"][k], cfg["mass"],
                                     cfg["nx_lattice"][k], cfg["np_lattice"][k], dvr="fgh")
        np.testing.assert_allclose(b.grid(k)[0], x, atol=1e-14)
        Wl = b.transform(k)
        np.testing.assert_allclose(Wl, Wm, atol=1e-10)


def test_pvb_on_fgh_matches_oracle():
    from oracle import bases
    pq = _lib()
    cfg = W.DWELL2D_PVB
    b = pq.Basis(pq.modes_of(cfg))
    for k in range(2):
        x, w, T, G, B = bases.pvb_basis(cfg["n"][k], cfg["xmin"][k], cfg["xmax"][k], cfg["mass"],
                                        cfg["nx_lattice"][k], cfg["np_lattice"][k], dvr="fgh")
        np.testing.assert_allclose(b.grid(k)[0], x, atol=1e-14)
        np.testing.assert_allclose(b.kinetic(k), T, atol=1e-12 * abs(T).max())
    with pytest.raises(pq.PQError) as e:
        pq.Basis([dict(kind=pq.PVB, n=258, xmin=0.5, xmax=6.0, mass=1.0, nx_lattice=43,
                       np_lattice=6)])
    assert e.value.status == pq.EINVAL


def test_set_allocator_arguments():
    import ctypes
    pq = _lib()
    lib = ctypes.CDLL(pq.lib_path())
    alloc = pq.ALLOC_FN(lambda n, st, ctx: None)
    # one function without the other
    assert lib.pq_set_allocator(alloc, pq.FREE_FN(), None) == pq.EINVAL
    # set and restore while no state exists (host-only basis objects do not count)
    b = pq.Basis(pq.modes_of(W.MORSE2D))
    pq.set_allocator(lambda n, st, ctx: None, lambda p, st, ctx: None)
    pq.set_allocator()
    del b


def test_tabulated_potential_errors():
    pq = _lib()
    b = pq.Basis(pq.modes_of(W.MORSE2D))
    with pytest.raises(pq.PQError) as e:
        b.set_potential_grid(np.zeros(31 * 32))
    assert e.value.status == pq.EINVAL
    with pytest.raises(pq.PQError) as e:
        b.set_potential_grid(np.full(32 * 32, np.nan))
    assert e.value.status == pq.EINVAL
    b.set_potential_grid(np.zeros((32, 32)))
    b.set_potential_grid(None)
    cfg = W.scaled(W.MORSE3D, D=2, n=16, nx_lattice=4, np_lattice=4)
    bw = pq.Basis(pq.modes_of(cfg))
    with pytest.raises(pq.PQError) as e:
        bw.set_potential_grid(np.zeros(16 * 16))
    assert e.value.status == pq.ENOTSUP


def test_argument_errors():
    pq = _lib()
    with pytest.raises(pq.PQError) as e:
        pq.Basis([dict(kind=pq.SINE_DVR, n=1, xmin=0, xmax=1, mass=1)])
    assert e.value.status == pq.EINVAL
    with pytest.raises(pq.PQError) as e:
        pq.Basis([dict(kind=pq.HO_DVR, n=257)])
    assert e.value.status == pq.EINVAL
    with pytest.raises(pq.PQError) as e:   # 64^6 > 2^32
        pq.Basis([dict(kind=pq.HO_DVR, n=64)] * 6)
    assert e.value.status == pq.EINVAL
    with pytest.raises(pq.PQError) as e:   # pvB mixed with another basis
        pq.Basis([dict(kind=pq.PVB, n=16, xmin=0.5, xmax=6.0, mass=1.0, nx_lattice=4, np_lattice=4),
                  dict(kind=pq.HO_DVR, n=8)])
    assert e.value.status == pq.ENOTSUP
    b = pq.Basis(pq.modes_of(W.scaled(W.HH4D, D=2)))
    with pytest.raises(pq.PQError) as e:   # kinetic times a diagonal factor
        b.set_sop([(1.0, ["T", np.ones(24)])])
    assert e.value.status == pq.ENOTSUP
    with pytest.raises(pq.PQError) as e:
        b.set_sop([(float("nan"), [None, None])])
    assert e.value.status == pq.EINVAL


def test_host_pw_basis_matches_oracle():
    # the library's projected-Weylet construction (its own Jacobi solver) and
    # the oracle's (LAPACK) agree: same W = Phi S^(-1/2), a unique matrix
    pq = _lib()
    from oracle import bases, propagate
    cfg = W.scaled(W.MORSE3D, D=2, n=16, nx_lattice=4, np_lattice=4)
    b = pq.Basis(pq.modes_of(cfg))
    x, w, T, Wo = bases.pw_basis(16, 0.5, 6.0, 1836.0, 4, 4)
    xl, wl = b.grid(0)
    np.testing.assert_allclose(xl, x, atol=1e-14)
    np.testing.assert_allclose(b.transform(0), Wo, atol=1e-12)
    np.testing.assert_allclose(b.transform(1), Wo, atol=1e-12)
    with pytest.raises(pq.PQError) as e:   # lattice does not match the DVR size
        pq.Basis([dict(kind=pq.PW, n=16, xmin=0.5, xmax=6.0, mass=1.0, nx_lattice=4, np_lattice=3)])
    assert e.value.status == pq.EINVAL
    b.set_sop(pq.coupled_morse_terms([xl, xl], 0.1, 1.0, 2.0, 0.005))


def test_missing_library_fails_loudly(tmp_path):
    # no CPU fallback: with the shared library absent the package refuses to
    # import (checked in a child process so this one keeps its library)
    import subprocess
    import sys
    code = ("import paper_1606_04004_gb300\n")
    env = dict(os.environ, PQ_LIBRARY=str(tmp_path / "absent" / "libprunedq.so"))
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=120)
    assert r.returncode != 0
    assert "ImportError" in r.stderr and "is missing" in r.stderr
