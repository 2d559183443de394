"""Plain, slow FP64 CPU oracle of the pruned time-dependent dynamics of
Larsson, Hartke and Tannor, "Efficient molecular quantum dynamics in coordinate
and phase space using pruned bases" (arXiv:1606.04004).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import or run this package.  It shares no
code with the CUDA library (``paper_1606_04004_gb300``) and never imports it;
the only common module is ``workloads`` (seeded inputs, no method arithmetic).

Everything is numpy float64 / complex128.  Library primitives used as single
steps: ``numpy.linalg.eigh`` (symmetric eigendecomposition), ``numpy.fft.fft`` (FGH kinetic matrix), ``numpy.unique``
and ``numpy.searchsorted`` (sorting / lookup), matrix products.

Modules
-------
bases      1D primitive bases: sine, HO (Gauss-Hermite) and FGH DVRs; von
           Neumann and momentum-symmetrised Gaussians projected on a DVR (pvB, pW).
models     potentials written as plain functions of the coordinates (including
           the paper's double well) and the initial Gaussian packet.
pruned     the pruned H.a on an active set, the adaption (prune + add) set
           function with its neighbour rules and relative exclusion, observables.
sil        short-iterative Lanczos step with full re-orthogonalisation (fixed or
           error-controlled order) and the RK4 step.
propagate  the whole run: initial prune, then step -> prune -> observables.
pvb        pvB dynamics: H_AA on the full grid, CG on S_AA, Lanczos in the S
           inner product.
adjoint    frozen-set replay, survival probability, finite differences.

Parity status: every function here is pinned by a ``-m "not gpu"`` test
against closed forms, brute force or a dense reference (see tests/).
"""
