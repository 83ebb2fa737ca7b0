"""Planted mistakes in the oracle, on the CPU, to show that its pins can fail.

Each mutant changes one expression of one oracle function: a dropped factor
or term, a flipped sign or transform direction, a wrong or transposed index,
a missing conjugate, a skipped step.  It is made from the function's own
source by an exact text substitution and installed in the oracle module for
the length of one test; the pins of test_oracle_pins.py named beside it must
then fail (an assertion, or the breakdown the mistake provokes).  A
substitution whose text no longer occurs in the oracle fails here loudly, so
an edit of the oracle cannot leave a pin silently untested.

Edits that leave the method's results unchanged are not mistakes and are
not listed: a constant phase of a projector column (beta D beta^H is the
same), the sign of the residual (W spans the same space), which side of the
Gram and subspace products is conjugated before they are symmetrised, and
the sphere's boundary comparison (no plane wave lies within 1e-9 Ha of the
cutoff, which the oracle checks).
"""
import __future__
import inspect
import textwrap

import numpy as np
import pytest

import test_oracle_pins as pins
from oracle import pw_oracle as O

# (name, oracle function, text, replacement, pins that must fail)
MUTANTS = [
    # plane-wave sphere, grid and kinetic energy (Sec. II-A)
    ("kinetic_without_half", "kinetic", "return 0.5 * np.sum(g * g, axis=1)", "return np.sum(g * g, axis=1)",
     [("test_sphere_brute_force", ("Si", 4.0)), "test_free_electron_shells"]),
    ("grid_without_factor", "grid_size_1d", "target = factor * math.sqrt", "target = math.sqrt",
     ["test_grid_rule"]),
    ("sphere_box_too_small", "sphere", "L / TWO_PI)) + 1 for L in Ls]", "L / TWO_PI)) - 1 for L in Ls]",
     [("test_sphere_brute_force", ("Si", 10.0)), "test_sphere_counts_and_volume"]),
    ("sphere_order_xy", "sphere", 'indexing="ij"', 'indexing="xy"',
     [("test_sphere_brute_force", ("C", 8.0))]),
    ("cell_grid_from_first_axis", "make_cell", "tuple(grid_size_1d(ecut, Ls[i]) for i in range(3))",
     "tuple(grid_size_1d(ecut, Ls[0]) for i in range(3))",
     ["test_grid_rule"]),
    # local potential and its grid Fourier coefficients
    ("vloc_width_halved", "vloc_grid", "(2.0 * sigma * sigma)", "(sigma * sigma)",
     ["test_vloc_direct_image_sum", "test_vloc_cell_average"]),
    ("vloc_no_images", "vloc_grid", "n = np.arange(-nimg, nimg + 1)", "n = np.arange(0, 1)",
     ["test_vloc_direct_image_sum", "test_vloc_cell_average"]),
    ("vloc_wrong_axis", "vloc_grid", "d = r[None, :] - tau[:, ax][:, None]",
     "d = r[None, :] - tau[:, 0][:, None]",
     ["test_vloc_direct_image_sum", "test_grid_shift_and_permutation_invariance"]),
    ("vloc_wrong_atom", "vloc_grid", "V += depth[a] * np.einsum", "V += depth[0] * np.einsum",
     ["test_vloc_direct_image_sum", "test_vloc_cell_average"]),
    ("vloc_fourier_unscaled", "vloc_fourier", "np.fft.fftn(V) / V.size", "np.fft.fftn(V)",
     ["test_vloc_fourier_brute_force", "test_constant_potential_shift"]),
    ("vloc_fourier_direction", "vloc_fourier", "np.fft.fftn(V) / V.size", "np.fft.ifftn(V)",
     ["test_vloc_fourier_brute_force", "test_hermiticity_and_dense_agreement"]),
    # projectors (Sec. III-A)
    ("projector_phase_sign", "projectors", "phase = np.exp(-1j * (G @ tau[a]))",
     "phase = np.exp(1j * (G @ tau[a]))",
     ["test_grid_shift_and_permutation_invariance"]),
    ("projector_p_norm", "projectors", "16.0 * math.pi ** 1.5 * rp ** 5", "8.0 * math.pi ** 1.5 * rp ** 5",
     ["test_projector_normalisation"]),
    ("projector_radial_width", "projectors", "np.exp(-0.5 * g2 * rp * rp)", "np.exp(-g2 * rp * rp)",
     ["test_projector_normalisation"]),
    ("projector_p_axis", "projectors", "(-1j) * G[:, k]", "(-1j) * G[:, 0]",
     ["test_projector_normalisation"]),
    ("projector_no_volume", "projectors", "rp * rp) / math.sqrt(omega)", "rp * rp)",
     ["test_projector_normalisation", "test_hermiticity_and_dense_agreement"]),
    # FFT between the sphere and the grid (Sec. II-B)
    ("real_space_unscaled", "to_real_space", "np.fft.ifftn(grid, axes=(0, 1, 2)) * (N[0] * N[1] * N[2])",
     "np.fft.ifftn(grid, axes=(0, 1, 2))",
     ["test_fft_convention_brute_force", "test_parseval_and_roundtrip", "test_density_sum_rule"]),
    ("real_space_negated_index", "to_real_space", "idx = tuple((cell.m[:, k] % N[k])",
     "idx = tuple((-cell.m[:, k] % N[k])",
     ["test_fft_convention_brute_force", "test_parseval_and_roundtrip"]),
    ("to_sphere_direction", "to_sphere", "F = np.fft.fftn(f, axes=(0, 1, 2)) / (N[0] * N[1] * N[2])",
     "F = np.fft.ifftn(f, axes=(0, 1, 2))",
     ["test_fft_convention_brute_force", "test_parseval_and_roundtrip"]),
    ("to_sphere_axes_swapped", "to_sphere", "idx = tuple((cell.m[:, k] % N[k])",
     "idx = tuple((cell.m[:, 2 - k] % N[k])",
     ["test_parseval_and_roundtrip", "test_hermiticity_and_dense_agreement"]),
    # the three terms of H
    ("local_term_dropped", "apply_local", "cell.V[..., None] * psi_r", "0.0 * psi_r",
     ["test_hermiticity_and_dense_agreement", "test_supercell_folding"]),
    ("nonlocal_missing_conjugate", "apply_nonlocal", "B = cell.beta.conj().T @ c", "B = cell.beta.T @ c",
     ["test_hermiticity_and_dense_agreement", "test_lobpcg_step_drops_p_on_breakdown"]),
    ("nonlocal_sign", "apply_nonlocal", "return cell.beta @ (cell.D[:, None] * B)",
     "return -cell.beta @ (cell.D[:, None] * B)",
     ["test_hermiticity_and_dense_agreement", "test_supercell_folding"]),
    ("kinetic_term_dropped", "apply_H", "cell.kin[:, None] * c + ", "",
     ["test_hermiticity_and_dense_agreement", "test_supercell_folding"]),
    ("dense_local_transposed", "dense_H", "dm = cell.m[:, None, :] - cell.m[None, :, :]",
     "dm = cell.m[None, :, :] - cell.m[:, None, :]",
     ["test_hermiticity_and_dense_agreement", "test_grid_shift_and_permutation_invariance"]),
    ("cell_projector_weights_transposed", "make_cell", "D = np.asarray(dkb, float).reshape(-1)",
     "D = np.asarray(dkb, float).T.reshape(-1)",
     ["test_grid_shift_and_permutation_invariance", "test_supercell_folding"]),
    ("dense_nonlocal_missing_conjugate", "dense_H", "@ cell.beta.conj().T", "@ cell.beta.T",
     ["test_hermiticity_and_dense_agreement", "test_rank_one_secular_equation"]),
    # preconditioner
    ("tpa_coefficient", "tpa", "p / (p + 16.0 * x ** 4)", "p / (p + 8.0 * x ** 4)",
     ["test_tpa_closed_form", "test_lobpcg_step_drops_p_on_breakdown"]),
    ("tpa_argument_inverted", "precondition", "tpa(cell.kin[:, None] / ek[None, :])",
     "tpa(cell.kin[:, None] * ek[None, :])",
     ["test_lobpcg_step_drops_p_on_breakdown", "test_lobpcg_step_direction_update"]),
    ("band_kinetic_weights", "band_kinetic", "w = np.abs(X) ** 2", "w = np.abs(X)",
     ["test_lobpcg_step_drops_p_on_breakdown", "test_lobpcg_step_direction_update"]),
    # Rayleigh-Ritz (Sec. III-D)
    ("rr_subspace_matrix_unscaled", "rayleigh_ritz", "As = d[:, None] * A * d[None, :]", "As = A",
     ["test_rayleigh_ritz_breakdown_and_solution", "test_lobpcg_step_keeps_p_when_it_is_independent"]),
    ("rr_coefficients_unscaled", "rayleigh_ritz", "C = d[:, None] * sla.solve_triangular", "C = sla.solve_triangular",
     ["test_rayleigh_ritz_breakdown_and_solution", "test_lobpcg_step_drops_p_on_breakdown"]),
    ("rr_highest_pairs", "rayleigh_ritz", "theta, Y = sla.eigh(At)", "theta, Y = sla.eigh(-At)\n    theta = -theta",
     ["test_rayleigh_ritz_breakdown_and_solution", "test_lobpcg_step_keeps_p_when_it_is_independent"]),
    ("rr_back_substitution_untransposed", "rayleigh_ritz",
     "sla.solve_triangular(L.conj().T, Y[:, :nb], lower=False)", "sla.solve_triangular(L, Y[:, :nb], lower=True)",
     ["test_rayleigh_ritz_breakdown_and_solution", "test_lobpcg_step_drops_p_on_breakdown"]),
    ("rr_scaling_inverted", "rayleigh_ritz", "d = 1.0 / np.sqrt(np.real(np.diag(G)))",
     "d = np.sqrt(np.real(np.diag(G)))",
     ["test_free_electron_shells"]),
    ("rr_no_pivot_test", "rayleigh_ritz", "if piv.min() <= piv_tol * np.real(np.diag(Gs)).max():", "if False:",
     ["test_rayleigh_ritz_pivot_threshold"]),
    # the LOBPCG step (Knyazev's method)
    ("init_not_rotated", "lobpcg_init", "X=X0 @ C, HX=HX0 @ C", "X=X0[:, :nb], HX=HX0[:, :nb]",
     ["test_lobpcg_init_is_the_ritz_block_of_the_start"]),
    ("init_values_reversed", "lobpcg_init", "lam, C = rayleigh_ritz(X0, HX0, nb)",
     "lam, C = rayleigh_ritz(X0, HX0, nb)\n    lam = lam[::-1].copy()",
     ["test_lobpcg_init_is_the_ritz_block_of_the_start"]),
    ("residual_sign", "residual", "R = st.HX - st.X * st.lam[None, :]", "R = st.HX + st.X * st.lam[None, :]",
     ["test_lobpcg_step_drops_p_on_breakdown", "test_lobpcg_step_keeps_p_when_it_is_independent"]),
    ("step_preconditions_HX", "lobpcg_step", "W = precondition(cell, st.X, R)[:, act]",
     "W = precondition(cell, st.X, st.HX)[:, act]",
     ["test_lobpcg_step_drops_p_on_breakdown", "test_lobpcg_step_direction_update"]),
    ("step_active_set_inverted", "lobpcg_step", "act = (rn > tol_lock)", "act = (rn <= tol_lock)",
     ["test_lobpcg_step_drops_p_on_breakdown", "test_lobpcg_step_keeps_p_when_it_is_independent"]),
    ("step_direction_is_new_block", "lobpcg_step", "P = S[:, nb:] @ C[nb:]\n    HP = HS[:, nb:] @ C[nb:]",
     "P = S @ C\n    HP = HS @ C",
     ["test_lobpcg_step_direction_update"]),
    ("step_hx_from_basis", "lobpcg_step", "HX = HS @ C", "HX = S @ C",
     ["test_lobpcg_step_direction_update"]),
    ("step_retry_drops_w", "lobpcg_step", "k = nb + int(act.sum())", "k = nb",
     ["test_lobpcg_step_drops_p_on_breakdown"]),
    ("dense_eigs_real_part", "dense_eigs", "return sla.eigh(H)\n", "return sla.eigh(H.real)\n",
     ["test_dense_eigs_against_cyclic_jacobi"]),
    ("dense_eigs_off_by_one", "dense_eigs", "subset_by_index=[0, nb - 1]", "subset_by_index=[1, nb]",
     ["test_lobpcg_vs_dense_and_bounds"]),
    ("convergence_on_smallest_residual", "eigsolve", "if rn.max() <= tol:", "if rn.min() <= tol:",
     ["test_free_electron_shells"]),
    # density and the SCF outer loop (Sec. II-A)
    ("density_not_squared", "density", "np.abs(psi) ** 2", "np.abs(psi)",
     ["test_density_sum_rule", "test_scf_reduces_to_fixed_potential_and_counts_electrons"]),
    ("density_ignores_occupations", "density", "w = np.ones(X.shape[1]) if occ is None else occ",
     "w = np.ones(X.shape[1])",
     ["test_scf_reduces_to_fixed_potential_and_counts_electrons"]),
    ("electron_density_no_volume", "electron_density", " / float(np.prod(cell.Ls))", "",
     ["test_scf_reduces_to_fixed_potential_and_counts_electrons"]),
    ("hartree_two_pi", "hartree_potential", "vt[nz] = 4.0 * math.pi", "vt[nz] = 2.0 * math.pi",
     ["test_hartree_single_mode_closed_form", "test_hartree_sine_mode_sign"]),
    ("hartree_direction", "hartree_potential", "np.fft.ifftn(vt) * n.size", "np.fft.fftn(vt)",
     ["test_hartree_sine_mode_sign"]),
    ("hartree_unsigned_frequencies", "grid_gvectors", "np.fft.fftfreq(Ns[a]) * Ns[a]", "np.arange(Ns[a])",
     ["test_hartree_single_mode_closed_form", "test_hartree_sine_mode_sign"]),
    ("exchange_coefficient", "slater_exchange", "/ math.pi)", "/ (4.0 * math.pi))",
     ["test_slater_exchange_uniform_gas"]),
    ("mixing_weights_swapped", "scf", "n_in = (1.0 - mix) * n_in + mix * n_out",
     "n_in = mix * n_in + (1.0 - mix) * n_out",
     ["test_scf_linear_mixing_is_a_geometric_series"]),
    ("scf_bare_potential", "scf", "w, X = dense_eigs(cell, nocc)", "w, X = dense_eigs(cell0, nocc)",
     ["test_scf_mixing_converges_to_a_fixed_point"]),
    ("scf_hxc_sign", "scf", "V = cell0.V + hxc_scale", "V = cell0.V - hxc_scale",
     ["test_scf_mixing_converges_to_a_fixed_point"]),
]


def _mutant(fname, old, new):
    src = textwrap.dedent(inspect.getsource(getattr(O, fname)))
    assert src.count(old) == 1, f"{fname}: the mutated text must occur exactly once"
    ns = dict(vars(O))
    code = compile(src.replace(old, new), f"<mutant of {fname}>", "exec",
                   flags=__future__.annotations.compiler_flag, dont_inherit=True)
    exec(code, ns)
    return ns[fname]


def _run(pin):
    name, args = (pin, ()) if isinstance(pin, str) else pin
    getattr(pins, name)(*args)


@pytest.mark.parametrize("name,fname,old,new,catch", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_planted_mistake(name, fname, old, new, catch, monkeypatch):
    monkeypatch.setattr(O, fname, _mutant(fname, old, new))
    with np.errstate(all="ignore"):
        for pin in catch:
            with pytest.raises((AssertionError, pytest.fail.Exception, O.CholeskyBreakdown,
                                np.linalg.LinAlgError)):
                _run(pin)


def test_unmutated_oracle_passes_the_same_pins():
    # the catching pins pass on the oracle as written (a mutant that fails
    # them is the only difference)
    seen = set()
    for *_, catch in MUTANTS:
        for pin in catch:
            key = pin if isinstance(pin, str) else (pin[0], pin[1])
            if key in seen:
                continue
            seen.add(key)
            _run(pin)
