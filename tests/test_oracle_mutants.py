"""Planted mistakes in the oracle, on the CPU.

Each mutant rewrites one expression of one oracle function -- a dropped term
or factor, a wrong sign, index or offset, a transposed operand, a missing
conjugate -- installs the rewritten function for the duration of one test
(``monkeypatch``), and requires that at least one of the named pins fails with
an assertion.  A mutant that no pin catches is a hole in the pins, so this file
is what backs the claim that the pins would see a plausible slip anywhere in
the oracle.  Nothing here touches a GPU or the CUDA library.

The snippet each mutant replaces must occur exactly once in the function's
source, so an edit of the oracle that removes it fails here loudly instead of
leaving a stale mutant that changes nothing.
"""
import importlib
import inspect
import textwrap

import pytest

import test_golden as G
import test_oracle_pins as P


def _install(monkeypatch, modname, qualname, old, new):
    """Recompile ``modname.qualname`` with ``old`` replaced by ``new`` in the
    module's own namespace and patch it in place."""
    mod = importlib.import_module(modname)
    owner = mod
    parts = qualname.split(".")
    for part in parts[:-1]:
        owner = getattr(owner, part)
    fn = getattr(owner, parts[-1])
    src = textwrap.dedent(inspect.getsource(fn))
    assert src.count(old) == 1, f"{qualname}: snippet occurs {src.count(old)} times"
    code = compile(src.replace(old, new), f"<mutant of {modname}.{qualname}>", "exec")
    ns = {}
    exec(code, mod.__dict__, ns)
    monkeypatch.setattr(owner, parts[-1], ns[parts[-1]])


# (id, module, function, snippet, replacement, pins that must catch it)
MUTANTS = [
    # ------------------------------------------------------------ bases
    ("sine_dvr_spacing", "oracle.bases", "sine_dvr",
     "x = xmin + j * L / (n + 1)", "x = xmin + j * L / n",
     [P.test_sine_dvr_free_particle_levels]),
    ("sine_dvr_kinetic_half", "oracle.bases", "sine_dvr",
     "ek = (j * np.pi / L) ** 2 / (2.0 * mass)", "ek = (j * np.pi / L) ** 2 / mass",
     [P.test_sine_dvr_free_particle_levels, P.test_sine_dvr_morse_levels]),
    ("sine_dvr_U_norm", "oracle.bases", "sine_dvr",
     "U = np.sqrt(2.0 / (n + 1))", "U = np.sqrt(1.0 / (n + 1))",
     [P.test_sine_dvr_free_particle_levels]),
    ("fgh_grid_offset", "oracle.bases", "fgh_dvr",
     "x = xmin + j * L / n", "x = xmin + (j + 0.5) * L / n",
     [P.test_fgh_free_particle_spectrum]),
    ("fgh_momentum_spacing", "oracle.bases", "fgh_dvr",
     "k = 2.0 * np.pi * l / L", "k = np.pi * l / L",
     [P.test_fgh_free_particle_spectrum, P.test_fgh_is_circulant_and_gives_ho_levels]),
    ("fgh_missing_conjugate", "oracle.bases", "fgh_dvr",
     "F.conj().T @ np.diag", "F.T @ np.diag",
     [P.test_fgh_free_particle_spectrum, P.test_fgh_is_circulant_and_gives_ho_levels]),
    ("ho_zero_point", "oracle.bases", "ho_dvr",
     "mass * omega * (kk + 0.5)", "mass * omega * (kk + 1.0)",
     [P.test_ho_dvr_levels_fig1_setup]),
    ("ho_p2_offdiagonal_sign", "oracle.bases", "ho_dvr",
     "off = -0.5 * mass * omega", "off = 0.5 * mass * omega",
     [P.test_ho_dvr_levels_fig1_setup]),
    ("ho_x_matrix_factor", "oracle.bases", "ho_dvr",
     "np.sqrt((k + 1) / (2.0 * mass * omega))", "np.sqrt((k + 1) / (mass * omega))",
     [P.test_ho_dvr_nodes_weights_vs_gauss_hermite, P.test_ho_dvr_levels_fig1_setup]),
    ("ho_weights_not_squared", "oracle.bases", "ho_dvr",
     "w = (U[0, :] / phi0) ** 2", "w = U[0, :] / phi0",
     [P.test_ho_dvr_nodes_weights_vs_gauss_hermite]),
    ("pw_shift_sign", "oracle.bases", "pw_functions",
     "(x - xa[a] - shift)", "(x - xa[a] + shift)",
     [lambda: P.test_pw_functions_closed_form_moments("sine")]),
    ("pw_von_neumann_density", "oracle.bases", "pw_functions",
     "dp = np.pi / dx", "dp = 2.0 * np.pi / dx",
     [lambda: P.test_pw_functions_closed_form_moments("sine")]),
    ("pw_alpha", "oracle.bases", "pw_functions",
     "alpha = dp / (2.0 * dx)", "alpha = dp / dx",
     [lambda: P.test_pw_functions_closed_form_moments("fgh")]),
    ("pw_momentum_offset", "oracle.bases", "pw_functions",
     "pb = (np.arange(np_) + 0.5) * dp", "pb = (np.arange(np_) + 1.0) * dp",
     [lambda: P.test_pw_functions_closed_form_moments("sine")]),
    ("pw_centre_offset", "oracle.bases", "pw_functions",
     "xa = xmin + (np.arange(nx) + 0.5) * dx", "xa = xmin + np.arange(nx) * dx",
     [lambda: P.test_pw_functions_closed_form_moments("sine")]),
    ("pw_gram_schmidt", "oracle.bases", "pw_basis",
     "W = Phi @ (U @ np.diag(lam ** -0.5) @ U.T)", "W = np.linalg.qr(Phi)[0]",
     [P.test_pw_is_loewdin_orthogonalisation]),
    ("pvb_momenta_not_centred", "oracle.bases", "pvb_basis",
     "pb = -pmax + (np.arange(np_) + 0.5) * dp", "pb = (np.arange(np_) + 0.5) * dp",
     [lambda: P.test_pvb_functions_closed_form_moments("sine")]),
    ("pvb_momentum_sign", "oracle.bases", "pvb_basis",
     "+ 1j * pb[b] * (x - xa[a])", "- 1j * pb[b] * (x - xa[a])",
     [lambda: P.test_pvb_functions_closed_form_moments("fgh")]),
    ("pvb_lattice_density", "oracle.bases", "pvb_basis",
     "dp = 2.0 * np.pi / dx", "dp = np.pi / dx",
     [lambda: P.test_pvb_functions_closed_form_moments("sine")]),
    ("pvb_biorthogonal_no_conjugate", "oracle.bases", "pvb_basis",
     "B = np.linalg.inv(G).conj().T", "B = np.linalg.inv(G).T",
     [P.test_pvb_biorthogonal]),
    ("sine_dvr_weight", "oracle.bases", "sine_dvr",
     "w = np.full(n, L / (n + 1))", "w = np.full(n, L / n)",
     [lambda: P.test_pvb_functions_closed_form_moments("sine")]),
    ("fgh_weight", "oracle.bases", "fgh_dvr",
     "w = np.full(n, L / n)", "w = np.full(n, L / (n + 1))",
     [P.test_fgh_free_particle_spectrum]),
    ("ho_sign_convention_dropped", "oracle.bases", "ho_dvr",
     "U = U * np.sign(U[0, :])[None, :]", "U = U",
     [P.test_hh_lambda0_coherent_state_closed_form]),
    ("pvb_alpha", "oracle.bases", "pvb_basis",
     "alpha = dp / (2.0 * dx)", "alpha = dp / dx",
     [lambda: P.test_pvb_functions_closed_form_moments("sine")]),
    # ----------------------------------------------------------- models
    ("hh_harmonic_half_dropped", "oracle.models", "henon_heiles",
     "v = 0.5 * np.sum((om * q) ** 2, axis=-1)", "v = np.sum((om * q) ** 2, axis=-1)",
     [P.test_henon_heiles_saddle]),
    ("morse_coupling_sign", "oracle.models", "coupled_morse",
     "v = v + coupling * q[..., i] * q[..., j]", "v = v - coupling * q[..., i] * q[..., j]",
     [P.test_pw_theta0_matches_dvr_dynamics]),
    ("hh_cubic_sign", "oracle.models", "henon_heiles",
     "(a * a * b - b ** 3 / 3.0)", "(a * a * b + b ** 3 / 3.0)",
     [P.test_henon_heiles_saddle]),
    ("morse_exponent_sign", "oracle.models", "coupled_morse",
     "np.exp(-a * (q - qe))", "np.exp(a * (q - qe))",
     [P.test_sine_dvr_morse_levels]),
    ("double_well_coupling", "oracle.models", "double_well",
     "c3 * x * x * y", "c3 * x * y * y",
     [G.test_double_well_record_is_the_printed_model]),
    ("gaussian_width", "oracle.models", "gaussian_1d",
     "/ (4.0 * s2)", "/ (2.0 * s2)",
     [P.test_hh_lambda0_coherent_state_closed_form, P.test_gaussian_packet_moments]),
    ("gaussian_momentum_sign", "oracle.models", "gaussian_1d",
     "+ 1j * p0 * (x - q0)", "- 1j * p0 * (x - q0)",
     [P.test_gaussian_packet_moments]),
    # ----------------------------------------------------------- pruned
    ("digits_column_major", "oracle.pruned", "digits",
     "np.unravel_index(np.asarray(A, dtype=np.int64), dims)",
     "np.unravel_index(np.asarray(A, dtype=np.int64), dims, order=\"F\")",
     [lambda: P.test_lattice_helpers_match_library_constructions((4, 4, 4))]),
    ("potential_modes_reversed", "oracle.pruned", "potential_diag",
     "np.asarray(grids[k])[dg[k]]", "np.asarray(grids[k])[dg[len(dims) - 1 - k]]",
     [lambda: P.test_lattice_helpers_match_library_constructions((4, 4, 4))]),
    ("product_modes_reversed", "oracle.pruned", "product_on",
     "np.asarray(factors[k])[dg[k]]", "np.asarray(factors[k])[dg[len(dims) - 1 - k]]",
     [lambda: P.test_lattice_helpers_match_library_constructions((4, 4, 4))]),
    ("lookup_without_key_check", "oracle.pruned", "lookup",
     "found = (pos < len(A)) & (A[pos_c] == keys)", "found = (pos < len(A))",
     [P.test_pruned_apply_at_sample_equals_full]),
    ("adapt_offset_sign_dropped", "oracle.pruned", "adapt_set",
     "delta += d * st[a]", "delta += st[a]",
     [lambda: P.test_prune_bruteforce((4, 3, 5), 1)]),
    ("strides_wrong_extent", "oracle.pruned", "strides_of",
     "s[k] = s[k + 1] * int(dims[k + 1])", "s[k] = s[k + 1] * int(dims[k])",
     [lambda: P.test_pruned_apply_member_form_equals_PHP((4, 5, 3), 0.4, 2)]),
    ("apply_T_transposed", "oracle.pruned", "apply_H",
     "T[ik[found], j]", "T[j, ik[found]]",
     [lambda: P.test_pruned_apply_member_form_equals_PHP((6, 5), 0.5, 1)]),
    ("apply_mode_dropped", "oracle.pruned", "apply_H",
     "for kappa, n in enumerate(dims):", "for kappa, n in list(enumerate(dims))[1:]:",
     [lambda: P.test_pruned_apply_member_form_equals_PHP((6, 5), 0.5, 1)]),
    ("apply_potential_dropped", "oracle.pruned", "apply_H",
     "y = np.asarray(vdiag, dtype=np.float64) * psi", "y = 0.0 * psi",
     [lambda: P.test_pruned_apply_equals_PHP((6, 5), 0.5, 1)]),
    ("apply_whole_mode_dropped", "oracle.pruned", "apply_H",
     "for k in range(len(dims)):", "for k in range(1, len(dims)):",
     [lambda: P.test_pruned_apply_equals_PHP((6, 5), 0.5, 1)]),
    ("along_transposed", "oracle.pruned", "_along",
     "axes=([1], [kappa])", "axes=([0], [kappa])",
     [lambda: P.test_pruned_apply_equals_PHP((6, 5), 0.5, 1)]),
    ("embed_off_set", "oracle.pruned", "_embed",
     "full[A] = x", "full[np.sort((A + 1) % full.size)] = x",
     [lambda: P.test_pruned_apply_equals_PHP((6, 5), 0.5, 1)]),
    ("mode_apply_whole_transposed", "oracle.pruned", "mode_apply",
     "return _along(h, _embed(A, x, dims), kappa)",
     "return _along(np.asarray(h).T, _embed(A, x, dims), kappa)",
     [lambda: P.test_sop_sequential_equals_dense_truncated_products((6, 7), 2)]),
    ("apply_at_T_transposed", "oracle.pruned", "apply_H_at",
     "T[ik[found], j]", "T[j, ik[found]]",
     [P.test_pruned_apply_at_sample_equals_full]),
    ("mode_apply_transposed", "oracle.pruned", "mode_apply",
     "h[ik[found], j]", "h[j, ik[found]]",
     [lambda: P.test_sop_sequential_member_form((6, 7), 2)]),
    ("sop_mode_order", "oracle.pruned", "apply_H_sop",
     "sorted(facs, reverse=True)", "sorted(facs)",
     [lambda: P.test_sop_sequential_equals_dense_truncated_products((5, 4, 6), 1)]),
    ("sop_coefficient_dropped", "oracle.pruned", "apply_H_sop",
     "y += coef * x", "y += x",
     [lambda: P.test_sop_sequential_equals_dense_truncated_products((5, 4, 6), 1)]),
    ("neighbour_sqrt2_as_radius1", "oracle.pruned", "neighbour_offsets",
     "RADIUS_SQRT2: 2,", "RADIUS_SQRT2: 1,",
     [P.test_neighbour_counts_match_the_paper]),
    ("neighbour_radius2_as_sqrt2", "oracle.pruned", "neighbour_offsets",
     "RADIUS_2: k}", "RADIUS_2: 2}",
     [P.test_neighbour_counts_match_the_paper]),
    ("significant_strict", "oracle.pruned", "significant",
     "mag2 >= np.float64(theta)", "mag2 > np.float64(theta)",
     [lambda: P.test_prune_bruteforce((7, 6), 0)]),
    ("adapt_no_upper_clip", "oracle.pruned", "adapt_set",
     "ok &= (nd >= 0) & (nd < axes[a])", "ok &= (nd >= 0)",
     [P.test_prune_edges_and_empty, lambda: P.test_prune_bruteforce((7, 6), 0)]),
    ("rel_excl_strict", "oracle.pruned", "prune",
     "if n_out <= rel_excl * len(A):", "if n_out < rel_excl * len(A):",
     [P.test_prune_relative_exclusion_bruteforce]),
    ("prune_new_members_not_zero", "oracle.pruned", "prune",
     "out[found] = psi[pos[found]]", "out[:] = psi[pos]",
     [lambda: P.test_prune_bruteforce((4, 3, 5), 1)]),
    ("packet_not_normalised", "oracle.pruned", "packet_factors",
     "out.append(v / np.linalg.norm(v))", "out.append(v)",
     [P.test_initial_state_chunked_equals_full_prune]),
    ("autocorrelation_no_conjugate", "oracle.pruned", "autocorrelation",
     "np.vdot(a0_on_A,", "np.dot(a0_on_A,",
     [lambda: P.test_theta0_is_unpruned_exact_dynamics((0.0, 6.0))]),
    # -------------------------------------------------------------- sil
    ("sil_exponent_sign", "oracle.sil", "tridiag_exp_e1",
     "np.exp(-1j * lam * dt)", "np.exp(1j * lam * dt)",
     [P.test_sil_full_krylov_is_exact_exponential]),
    ("sil_e1_row_vs_column", "oracle.sil", "tridiag_exp_e1",
     "* Z[0, :])", "* Z[:, 0])",
     [P.test_sil_full_krylov_is_exact_exponential]),
    ("sil_norm_dropped", "oracle.sil", "sil_step",
     "out = beta0 * sum(", "out = sum(",
     [P.test_sil_conserves_norm_and_energy]),
    ("sil_tol_estimate_index", "oracle.sil", "sil_step",
     "ck = tridiag_exp_e1(alpha, beta, dt)[k]", "ck = tridiag_exp_e1(alpha, beta, dt)[0]",
     [P.test_sil_error_control_meets_tolerance]),
    ("sil_no_orthogonalisation", "oracle.sil", "sil_step",
     "for _ in range(2):", "for _ in range(0):",
     [P.test_sil_full_krylov_is_exact_exponential]),
    ("rk4_stage_weights", "oracle.sil", "rk4_step",
     "(k1 + 2.0 * k2 + 2.0 * k3 + k4)", "(k1 + 2.0 * k2 + k3 + 2.0 * k4)",
     [P.test_rk4_is_fourth_order]),
    ("rk4_stage_input", "oracle.sil", "rk4_step",
     "k3 = -1j * apply(a + 0.5 * dt * k2)", "k3 = -1j * apply(a + 0.5 * dt * k1)",
     [P.test_rk4_is_fourth_order]),
    # -------------------------------------------------------- propagate
    ("initial_state_no_neighbours", "oracle.propagate", "initial_state",
     "A = pruned.adapt_set(np.concatenate(S), prob.axes, radius)", "A = np.concatenate(S)",
     [P.test_initial_state_chunked_equals_full_prune]),
    ("energy_not_normalised", "oracle.propagate", "observables",
     "E = float(np.real(np.vdot(psi, Hpsi))) / nrm2", "E = float(np.real(np.vdot(psi, Hpsi)))",
     [P.test_observables_are_scale_invariant_and_count_wasted]),
    ("wasted_uses_zero_threshold", "oracle.propagate", "observables",
     "~pruned.significant(psi, theta)", "~pruned.significant(psi, 0.0)",
     [P.test_observables_are_scale_invariant_and_count_wasted]),
    ("run_prunes_at_another_threshold", "oracle.propagate", "run",
     "A, a = pruned.prune(A, a, prob.axes, theta, radius, rel_excl)",
     "A, a = pruned.prune(A, a, prob.axes, 10 * theta, radius, rel_excl)",
     [lambda: P.test_run_sets_are_adaption_fixed_points(2)]),
    ("run_ignores_neighbour_rule", "oracle.propagate", "run",
     "A, a = pruned.prune(A, a, prob.axes, theta, radius, rel_excl)",
     "A, a = pruned.prune(A, a, prob.axes, theta, 1, rel_excl)",
     [lambda: P.test_run_sets_are_adaption_fixed_points(2)]),
    ("initial_state_ignores_neighbour_rule", "oracle.propagate", "initial_state",
     "A = pruned.adapt_set(np.concatenate(S), prob.axes, radius)",
     "A = pruned.adapt_set(np.concatenate(S), prob.axes, 1)",
     [lambda: P.test_run_sets_are_adaption_fixed_points(2)]),
    ("pw_congruence_transposed", "oracle.propagate", "PWProblem.__init__",
     "tf[k] = self.Ws[k].T @ h @ self.Ws[k]", "tf[k] = self.Ws[k] @ h @ self.Ws[k].T",
     [P.test_pw_full_basis_equals_transformed_dvr]),
    ("pw_packet_untransformed", "oracle.propagate", "PWProblem.factors",
     "self.Ws[k].T @ f[k]", "self.Ws[k] @ f[k]",
     [P.test_pw_theta0_matches_dvr_dynamics]),
    ("dwell_pw_coupling_modes", "oracle.propagate", "dwell_pw_problem",
     "(c3, {0: x * x, 1: y})", "(c3, {0: x, 1: y * y})",
     [P.test_pw_on_fgh_theta0_matches_fgh_dynamics]),
    ("morse_sop_coupling_factor", "oracle.propagate", "morse_sop_terms",
     "terms.append((coupling, {i: grids[i], j: grids[j]}))",
     "terms.append((2.0 * coupling, {i: grids[i], j: grids[j]}))",
     [P.test_pw_theta0_matches_dvr_dynamics]),
    # -------------------------------------------------------------- pvb
    ("pvb_lanczos_euclidean_norm", "oracle.pvb", "sil_step_S",
     "b = np.sqrt(max(np.vdot(w, prob.S_AA(A, w)).real, 0.0))", "b = np.linalg.norm(w)",
     [P.test_pvb_theta0_matches_dvr_dynamics]),
    ("pvb_start_euclidean_norm", "oracle.pvb", "sil_step_S",
     "beta0 = np.sqrt(max(np.vdot(a, Sa).real, 0.0))", "beta0 = np.linalg.norm(a)",
     [P.test_pvb_theta0_matches_dvr_dynamics]),
    ("pvb_norm_without_overlap", "oracle.pvb", "run",
     "n2 = float(np.vdot(a, prob.S_AA(A, a)).real)", "n2 = float(np.vdot(a, a).real)",
     [P.test_pvb_theta0_matches_dvr_dynamics]),
    ("pvb_H_no_conjugate", "oracle.pvb", "PVBProblem.H_AA",
     "self.Bs[k].conj().T", "self.Bs[k].T",
     [P.test_pvb_theta0_matches_dvr_dynamics]),
    ("pvb_overlap_transposed", "oracle.pvb", "PVBProblem.__init__",
     "self.Ss = [B.conj().T @ B for B in self.Bs]", "self.Ss = [B @ B.conj().T for B in self.Bs]",
     [P.test_pvb_theta0_matches_dvr_dynamics]),
    ("pvb_cg_residual_sign", "oracle.pvb", "PVBProblem.solve_S",
     "r = r - al * Sp", "r = r + al * Sp",
     [P.test_pvb_cg_solves_overlap]),
    ("pvb_bra_uses_G", "oracle.pvb", "PVBProblem.factors",
     'Ms = self.Gs if which == "G" else self.Bs', "Ms = self.Gs",
     [P.test_pvb_theta0_matches_dvr_dynamics]),
    ("pvb_lanczos_euclidean_product", "oracle.pvb", "sil_step_S",
     "c = [np.vdot(v, Sw) for v in V]", "c = [np.vdot(v, w) for v in V]",
     [P.test_pvb_theta0_matches_dvr_dynamics]),
    # ---------------------------------------------------------- adjoint
    ("adjoint_carry_conjugated", "oracle.adjoint", "run_frozen",
     "b[found] = a[pos[found]]", "b[found] = a[pos[found]].conj()",
     [P.test_adjoint_frozen_replay_equals_dense_products]),
    ("sil_beta_squared", "oracle.sil", "sil_step",
     "b = np.linalg.norm(w)", "b = np.linalg.norm(w) ** 2",
     [P.test_sil_full_krylov_is_exact_exponential]),
    ("adjoint_set_one_step_off", "oracle.adjoint", "run_frozen",
     "An = np.asarray(sets[n + 1], dtype=np.int64)", "An = np.asarray(sets[n], dtype=np.int64)",
     [P.test_adjoint_frozen_replay_equals_dense_products]),
    ("adjoint_one_sided_difference", "oracle.adjoint", "fd_gradient",
     "p2[i] -= h", "p2[i] -= 0.0",
     [P.test_adjoint_finite_differences_equal_analytic_gradient]),
    ("adjoint_parameter_slots", "oracle.adjoint", "survival",
     "params[1 + D:1 + 2 * D]", "params[D:2 * D]",
     [P.test_adjoint_finite_differences_equal_analytic_gradient]),
]


@pytest.mark.parametrize("mutant", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_planted_mistake(mutant, monkeypatch):
    name, modname, qualname, old, new, pins = mutant
    _install(monkeypatch, modname, qualname, old, new)
    caught = 0
    for pin in pins:
        try:
            pin()
        except AssertionError:
            caught += 1
    assert caught > 0, f"no pin caught the planted mistake {name}"


def test_every_oracle_module_has_mutants():
    mods = {m[1] for m in MUTANTS}
    assert mods == {"oracle." + m for m in ("bases", "models", "pruned", "sil", "propagate",
                                            "pvb", "adjoint")}
