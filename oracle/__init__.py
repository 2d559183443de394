"""Plain, slow FP64 CPU oracle of the pruned time-dependent dynamics of
Larsson, Hartke and Tannor, "Efficient molecular quantum dynamics in coordinate
and phase space using pruned bases" (arXiv:1606.04004).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import or run this package.  It shares no
code with the CUDA library (``paper_1606_04004_gb300``) and never imports it;
the only common module is ``workloads`` (seeded inputs, no method arithmetic).

Everything is numpy float64 / complex128.  Library primitives used as single
steps: ``numpy.linalg.eigh`` (symmetric eigendecomposition), ``numpy.unique``
and ``numpy.searchsorted`` (sorting / lookup), matrix products.

Modules
-------
bases      1D primitive bases: sine DVR, HO (Gauss-Hermite) DVR; von Neumann
           and momentum-symmetrised Gaussians projected on a DVR (pvB, pW).
models     potentials written as plain functions of the coordinates and the
           initial Gaussian packet.
pruned     the pruned H.a on an active set, the adaption (prune + add) set
           function, observables.
sil        short-iterative Lanczos step with full re-orthogonalisation.
propagate  the whole run: initial prune, then SIL -> prune -> observables.

Parity status: every function here is pinned by a ``-m "not gpu"`` test
against closed forms, brute force or a dense reference (see tests/).
"""
