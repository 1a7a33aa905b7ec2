"""Planted mistakes in the oracle, on the CPU: every case changes one spot of one oracle function (a
dropped term, a wrong sign, a transposed operand, a misread constant or index) and runs the pin
that must catch it.  The pin has to fail; a mistake that no pin notices would mean the oracle is
not pinned against that kind of error.

The changed function is rebuilt from its own source with the edit applied and swapped in for the
duration of the test only (pytest's monkeypatch restores it).  Nothing here touches the CUDA path.
"""
import inspect
import textwrap

import pytest

from oracle import geometry, gmres, layer, near, offsurface, reparam, sh, surfactant, timestep, wigner

import test_oracle_geometry as PG
import test_oracle_layer as PL
import test_oracle_offsurface as PO
import test_oracle_reparam as PR
import test_oracle_sh as PS
import test_oracle_surfactant as PF
import test_oracle_timestep as PT
import test_oracle_wigner as PW


def plant(monkeypatch, module, name, edits):
    """Replace module.name by a copy of its source with the (old, new) text edits applied."""
    src = textwrap.dedent(inspect.getsource(getattr(module, name)))
    for old, new in edits:
        assert src.count(old) == 1, (name, old)
        src = src.replace(old, new)
    ns = dict(module.__dict__)
    code = compile("from __future__ import annotations\n" + src, f"<planted {module.__name__}.{name}>", "exec")
    exec(code, ns)
    monkeypatch.setattr(module, name, ns[name])


# (id, module, function or class, [(old, new), ...], pin, pin arguments)
CASES = [
    # Legendre basis and transforms (Sec. 1.1, Sec. 2.1, App. A)
    ("condon_shortley_phase_dropped", sh, "legendre_normalised",
     [("P[m, m] = -c * s * P[m - 1, m - 1]", "P[m, m] = c * s * P[m - 1, m - 1]")],
     PS.test_legendre_recursion_matches_library_harmonics, ()),
    ("legendre_recursion_sign", sh, "legendre_normalised",
     [("b = -math.sqrt(", "b = math.sqrt(")],
     PS.test_legendre_recursion_matches_library_harmonics, ()),
    ("dtheta_cot_term_sign", sh, "legendre_dtheta",
     [("dP[n, m] = alpha * up + m * cot * P[n, m]", "dP[n, m] = alpha * up - m * cot * P[n, m]")],
     PS.test_theta_derivatives_against_finite_differences, ()),
    ("second_derivative_cot_sign", sh, "legendre_dtheta",
     [("d2P[n, m] = -cot * dP[n, m]", "d2P[n, m] = cot * dP[n, m]")],
     PS.test_laplace_beltrami_eigen_relation, ()),
    ("analysis_weight_printed_pi_over_p", sh, "analyze",
     [("(np.pi / (p_grid + 1)) * np.sum(", "(np.pi / p_grid) * np.sum(")],
     PS.test_area_of_unit_sphere_by_regular_rule, ()),
    ("analysis_without_conjugate", sh, "analyze",
     [("e = np.exp(-1j * m * phi)", "e = np.exp(1j * m * phi)")],
     PS.test_round_trip_and_zero_padding, (9,)),
    ("packed_imaginary_part_sign", sh, "to_complex",
     [("+ 1j * coef[n * (n + 1) - m]", "- 1j * coef[n * (n + 1) - m]")],
     PS.test_round_trip_and_zero_padding, (9,)),
    ("synthesis_negative_m_dropped", sh, "_synth_from_tables",
     [("out += term.real if m == 0 else 2.0 * term.real", "out += term.real")],
     PS.test_round_trip_and_zero_padding, (9,)),
    ("phi_grid_of_2p_points", sh, "gauss_grid",
     [("phi = np.pi * np.arange(2 * p + 2) / (p + 1)", "phi = np.pi * np.arange(2 * p) / p")],
     PS.test_discrete_orthogonality_needs_2p_plus_2_points_and_pi_over_p_plus_1, ()),
    # Wigner rotation (App. B)
    ("wigner_generator_sign", wigner, "_generator",
     [("return 0.5 * (Jm - Jp)", "return 0.5 * (Jp - Jm)")],
     PW.test_rotated_expansion_is_function_at_rotated_points, ()),
    ("rotation_alpha_phase_sign", wigner, "rotate",
     [("full[n + m] = c[n, m] * np.exp(1j * m * alpha)", "full[n + m] = c[n, m] * np.exp(-1j * m * alpha)")],
     PW.test_rotated_expansion_is_function_at_rotated_points, ()),
    ("rotation_small_d_transposed", wigner, "rotate",
     [("dd = small_d(n, beta).T", "dd = small_d(n, beta)")],
     PW.test_rotated_expansion_is_function_at_rotated_points, ()),
    ("rotation_gamma_phase_sign", wigner, "rotate",
     [("np.exp(1j * mp * gamma)", "np.exp(-1j * mp * gamma)")],
     PW.test_rotated_expansion_is_function_at_rotated_points, ()),
    # geometry and force (Table 2, Sec. 1)
    ("normal_inward", geometry, "forms",
     [("n = np.cross(xt, xp, axis=0) / W", "n = np.cross(xp, xt, axis=0) / W")],
     PG.test_sphere_forms_normal_and_curvature, ()),
    ("curvature_labels_swapped", geometry, "forms",
     [("K = (E * N - 2.0 * F * M + G * L) / (2.0 * W * W)", "K = (L * N - M * M) / (W * W)")],
     PG.test_sphere_forms_normal_and_curvature, ()),
    ("mean_curvature_operands_swapped", geometry, "forms",
     [("(E * N - 2.0 * F * M + G * L)", "(E * L - 2.0 * F * M + G * N)")],
     PG.test_sphere_forms_normal_and_curvature, ()),
    ("force_sign_as_printed", geometry, "interfacial_force",
     [('f = -2.0 * sig * g["K"] * g["n"] - grad', 'f = 2.0 * sig * g["K"] * g["n"] - grad')],
     PG.test_clean_sphere_force_is_outward_two_sigma_over_r, ()),
    ("marangoni_sign", geometry, "interfacial_force",
     [('f = -2.0 * sig * g["K"] * g["n"] - grad', 'f = -2.0 * sig * g["K"] * g["n"] + grad')],
     PG.test_marangoni_term_points_down_the_tension_gradient_sign_reading, ()),
    ("surface_gradient_metric_swapped", geometry, "interfacial_force",
     [('grad = ((G * sp - F * st) * g["xp"] + (E * st - F * sp) * g["xt"])',
       'grad = ((E * sp - F * st) * g["xp"] + (G * st - F * sp) * g["xt"])')],
     PG.test_marangoni_term_points_down_the_tension_gradient_sign_reading, ()),
    ("surface_gradient_cross_metric_sign", geometry, "interfacial_force",
     [('grad = ((G * sp - F * st) * g["xp"] + (E * st - F * sp) * g["xt"])',
       'grad = ((G * sp + F * st) * g["xp"] + (E * st - F * sp) * g["xt"])')],
     PG.test_interfacial_force_carries_no_net_force_or_torque, ()),
    ("equation_of_state_sign", geometry, "sigma_of_gamma",
     [("return 1.0 - elasticity * gamma", "return 1.0 + elasticity * gamma")],
     PG.test_clean_sphere_force_is_outward_two_sigma_over_r, ()),
    ("volume_without_one_third", geometry, "volume",
     [("float(np.sum(w[:, None] * integrand)) / 3.0", "float(np.sum(w[:, None] * integrand))")],
     PG.test_ellipsoid_volume_and_mean_radius, ()),
    # kernels and the singular rule (Eq. main_eq, Thm 1)
    ("stokeslet_dyadic_term_dropped", layer, "stokeslet",
     [("return f / r + xh * (xf / (r2 * r))", "return f / r")],
     PL.test_single_layer_of_constant_on_sphere_radius_a, ()),
    ("stresslet_sign", layer, "stresslet",
     [("return -6.0 * xh *", "return 6.0 * xh *")],
     PL.test_single_layer_of_normal_vanishes_and_double_layer_identity_on_deformed_drop, ()),
    ("stresslet_wrong_contraction", layer, "stresslet",
     [("np.sum(u * xh, axis=0) * np.sum(xh * n, axis=0)", "np.sum(u * n, axis=0) * np.sum(xh * xh, axis=0)")],
     PL.test_single_layer_of_normal_vanishes_and_double_layer_identity_on_deformed_drop, ()),
    ("singular_weight_divides_by_sin_twice", layer, "singular_weights",
     [("* P, axis=0)", "* P, axis=0) / np.sin(theta)")],
     PL.test_singular_rule_is_exact_for_laplace_on_unit_sphere, ()),
    ("singular_weight_printed_pi_over_p", layer, "singular_weights",
     [("(np.pi / (pq + 1)) * w", "(np.pi / pq) * w")],
     PL.test_singular_rule_is_exact_for_laplace_on_unit_sphere, ()),
    ("legendre_p_recursion_index", layer, "legendre_p",
     [("- n * P[n - 1]) / (n + 1)", "- (n + 1) * P[n - 1]) / (n + 1)")],
     PL.test_singular_rule_is_exact_for_laplace_on_unit_sphere, ()),
    ("target_rotation_small_d_transposed", layer, "rotate_batch",
     [("dd = wigner.small_d(n, beta).T", "dd = wigner.small_d(n, beta)")],
     PG.test_rotated_geometry_matches_direct_evaluation_at_rotated_points, ()),
    ("target_rotation_negative_m_phase", layer, "rotate_batch",
     [("((-1) ** m) * np.conj(c[:, n, m])", "np.conj(c[:, n, m])")],
     PG.test_rotated_geometry_matches_direct_evaluation_at_rotated_points, ()),
    ("rotated_area_density_without_sin", layer, "SelfQuadrature",
     [("* W / np.sin(self.thq)[None, :, None]", "* W")],
     PL.test_single_layer_of_constant_on_sphere_radius_a, ()),
    # regular, upsampled and near-singular rules, system (Sec. 2.1, 2.3, Eq. main_eq)
    ("regular_weight_printed_pi_over_p", layer, "DropGrid",
     [("self.wJ = ((np.pi / (P + 1))", "self.wJ = ((np.pi / P)")],
     PL.test_regular_rule_reproduces_translating_sphere_field_far_away, ()),
    ("regions_use_swapped_grids", layer, "Drops",
     [("((0, self.std[j], std_rho[j]), (1, self.ups[j], up_rho[j]))",
       "((0, self.ups[j], up_rho[j]), (1, self.std[j], std_rho[j]))")],
     PL.test_two_drops_near_contact_closed_forms_through_all_regions, ()),
    ("double_layer_lambda_of_target_drop", layer, "Drops",
     [("if j == i or weights[j] == 0.0:", "if j == i or weights[i] == 0.0:"),
      ("v[:, sel] += weights[j] * regular_sum(", "v[:, sel] += weights[i] * regular_sum("),
      ("v[:, sel] += weights[j] * near.near_values(", "v[:, sel] += weights[i] * near.near_values(")],
     PL.test_force_free_drop_of_matched_viscosity_is_invisible, ()),
    ("system_double_layer_sign", layer, "Drops",
     [("(self.lam[i] + 1.0) * ul[i] - d[i]", "(self.lam[i] + 1.0) * ul[i] + d[i]")],
     PL.test_solution_of_rigid_rotation_is_the_flow_for_any_viscosity_ratio, ()),
    ("far_field_without_factor_two", layer, "Drops",
     [("out.append(2.0 * uinf + s[i])", "out.append(uinf + s[i])")],
     PL.test_force_free_drop_of_matched_viscosity_is_invisible, ()),
    ("near_anchor_without_jump", near, "near_value_at",
     [("anchor = anchor - 4.0 * np.pi * u_star", "anchor = anchor")],
     PL.test_two_drops_near_contact_closed_forms_through_all_regions, ()),
    ("near_check_points_inside", near, "near_value_at",
     [("pts = xs[:, None] + e[:, None] * nodes[None, 1:]", "pts = xs[:, None] - e[:, None] * nodes[None, 1:]")],
     PL.test_two_drops_near_contact_closed_forms_through_all_regions, ()),
    ("newton_step_uphill", near, "newton_closest",
     [("step = -np.linalg.solve(", "step = np.linalg.solve(")],
     PL.test_newton_closest_point_is_the_nearest_surface_point, ()),
    ("closest_point_left_at_the_seed", near, "near_value_at",
     [("th, ph, xs = newton_closest(xr, p, x0)", "th, ph, xs = newton_closest(xr, p, x0, max_it=0)")],
     PL.test_near_singular_values_converge_to_brute_force_on_a_deformed_drop, ()),
    ("newton_hessian_without_curvature", near, "newton_closest",
     [('[[d["t"] @ d["t"] + r @ d["tt"],', '[[d["t"] @ d["t"] - r @ d["tt"],')],
     PL.test_newton_closest_point_is_the_nearest_surface_point, ()),
    # off-surface evaluation (Sec. 1 with the rules of Sec. 2.1-2.3)
    ("offsurface_double_layer_sign", offsurface, "velocity_at",
     [('layer_at(drops, pts, f_list, "S") + layer_at(', 'layer_at(drops, pts, f_list, "S") - layer_at(')],
     PO.test_velocity_is_continuous_across_the_interface, ()),
    ("offsurface_without_half", offsurface, "velocity_at",
     [("u = 0.5 * (layer_at(", "u = (layer_at(")],
     PO.test_velocity_is_continuous_across_the_interface, ()),
    ("offsurface_upsampled_region_on_the_standard_grid", offsurface, "raw_layer_at",
     [("for r, grid in ((0, drops.std[j]), (1, drops.ups[j])):", "for r, grid in ((0, drops.std[j]), (1, drops.std[j])):")],
     PO.test_layers_converge_to_brute_force_on_two_deformed_drops, ()),
    ("offsurface_inside_side_flipped", offsurface, "classify_points",
     [("codes[s:s + 256] = np.where(side <= 0.0, INSIDE, c)", "codes[s:s + 256] = np.where(side >= 0.0, INSIDE, c)")],
     PO.test_inside_points_are_rejected, ()),
    # GMRES (Sec. 6) and the drop update (Sec. 3)
    ("givens_rotation_sign", gmres, "gmres",
     [("H[i + 1, k] = -sn[i] * H[i, k] + cs[i] * H[i + 1, k]", "H[i + 1, k] = sn[i] * H[i, k] + cs[i] * H[i + 1, k]")],
     PL.test_gmres_iterate_minimises_the_residual_over_the_krylov_space, ()),
    ("triangular_solve_transposed", gmres, "gmres",
     [("y = np.linalg.solve(np.triu(H[:k_used, :k_used]), g[:k_used])",
       "y = np.linalg.solve(np.triu(H[:k_used, :k_used]).T, g[:k_used])")],
     PL.test_gmres_iterate_minimises_the_residual_over_the_krylov_space, ()),
    ("gram_schmidt_sign", gmres, "gmres",
     [("w = w - H[i, k] * V[i]", "w = w + H[i, k] * V[i]")],
     PL.test_gmres_matches_direct_solve, ()),
    ("forward_euler_instead_of_midpoint", timestep, "midpoint_step",
     [("return [x + dt * u for x, u in zip(xs, u1)]", "return [x + dt * u for x, u in zip(xs, u0)]")],
     PT.test_volume_change_per_step_is_third_order, ()),
    ("midpoint_at_full_step", timestep, "midpoint_step",
     [("xh = [x + 0.5 * dt * u", "xh = [x + dt * u")],
     PT.test_volume_change_per_step_is_third_order, ()),
    # surfactant transport and the coupled step (Eq. surfactant0, Sec. 3, Alg. 1)
    ("stretching_sign_as_printed", surfactant, "f_explicit_grid",
     [("stretch = 2.0 * S.K * G * un", "stretch = -2.0 * S.K * G * un")],
     PF.test_stretching_term_of_an_expanding_sphere, ()),
    ("convection_without_moving_frame_term", surfactant, "f_explicit_grid",
     [("return -conv + frame + stretch", "return -conv + stretch")],
     PF.test_rigid_motion_leaves_any_concentration_unchanged, ()),
    ("laplacian_without_christoffel_term", surfactant, "Surface",
     [('self.gtt * (s["tt"] - dot(self.d["tt"], gs))', 'self.gtt * s["tt"]')],
     PF.test_surface_operators_of_the_position_vector_on_a_deformed_drop, ()),
    ("inverse_metric_cross_term_sign", surfactant, "Surface",
     [("self.E / W2, -self.F / W2, self.G / W2", "self.E / W2, self.F / W2, self.G / W2")],
     PF.test_surface_operators_of_the_position_vector_on_a_deformed_drop, ()),
    ("inverse_metric_diagonal_swapped", surfactant, "Surface",
     [("self.E / W2, -self.F / W2, self.G / W2", "self.G / W2, -self.F / W2, self.E / W2")],
     PF.test_laplace_beltrami_on_a_sphere_of_radius_r, ()),
    ("normal_derivative_operand_order", surfactant, "Surface",
     [('ct = np.cross(d["tt"], self.xp, axis=0)', 'ct = np.cross(self.xp, d["tt"], axis=0)')],
     PF.test_rigid_motion_leaves_any_concentration_unchanged, ()),
    ("imex2_diffusion_at_the_old_level", surfactant, "imex2_full",
     [("f_implicit(xh, gh, p, pe)", "f_implicit(xh, g0, p, pe)")],
     PF.test_imex2_step_of_pure_diffusion_on_a_resting_sphere, ()),
    ("imex2_half_stage_with_full_step", surfactant, "imex2_half",
     [("g0 + 0.5 * dt * k0", "g0 + dt * k0")],
     PF.test_expanding_sphere_keeps_gamma_r_squared_to_second_order, ()),
    ("drop_update_from_the_half_point_as_printed", surfactant, "coupled_step",
     [("x1 = [x + dt * u for x, u in zip(xs, uh)]", "x1 = [x + dt * u for x, u in zip(xh, uh)]")],
     PF.test_expanding_sphere_keeps_gamma_r_squared_to_second_order, ()),
    ("step_size_rule_without_square_root", surfactant, "next_dt",
     [("dt * math.sqrt(0.9 * tol / err)", "dt * (0.9 * tol / err)")],
     PF.test_adaptive_run_keeps_every_accepted_step_below_tolerance, ()),
    # angle reparametrisation (Sec. 4, Alg. 2)
    ("mode_norms_without_negative_orders", reparam, "mode_norms",
     [("out[n, P - n: P] = a[n, 1: n + 1][::-1]", "out[n, P - n: P] = 0.0")],
     PR.test_mode_norms_satisfy_parseval_on_the_unit_sphere, ()),
    ("cutoff_with_the_largest_order_per_degree", reparam, "adaptive_cutoff",
     [("per_n = np.sum(mode_norms(xcoef, P), axis=1)", "per_n = np.max(mode_norms(xcoef, P), axis=1)")],
     PR.test_adaptive_cutoff_on_a_designed_spectrum, ()),
    ("angle_velocity_cross_term_sign", reparam, "angle_velocity",
     [("return (A22 * b1 - A12 * b2) / det, (-A12 * b1 + A11 * b2) / det",
       "return (A22 * b1 + A12 * b2) / det, (A12 * b1 + A11 * b2) / det")],
     PR.test_angle_velocity_moves_the_point_with_the_tangential_velocity, ()),
    ("pseudo_velocity_up_the_gradient", reparam, "reparametrize",
     [("al_t, al_p = angle_velocity(e, -gvec)", "al_t, al_p = angle_velocity(e, gvec)")],
     PR.test_distorted_sphere_returns_to_its_one_mode_parametrisation, ()),
    ("surfactant_at_the_grid_angles", reparam, "reparametrize",
     [("gg = sh.evaluate(g0, P, th, ph)", "gg = sh.evaluate(g0, P, T, F)")],
     PR.test_concentration_linear_in_the_position_is_carried_exactly, ()),
]


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_planted_mistake_fails_its_pin(monkeypatch, case):
    # each pin also runs on the oracle as it stands, as a test of its own module
    _, module, name, edits, pin, args = case
    plant(monkeypatch, module, name, edits)
    with pytest.raises(AssertionError):
        pin(*args)
