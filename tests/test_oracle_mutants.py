"""The oracle's pins catch plausible mistakes in the oracle (CPU only).

Each case below plants one mistake in a copy of ``oracle/magnus_oracle.c`` -- a wrong sign, index,
weight, factor order or dropped term of the kind a restatement of the paper could contain -- builds
the copy with gcc in a temporary folder, points the oracle's Python wrapper at it, and runs the pins
named beside the case: at least one of them must fail.  The unmodified copy, built the same way,
passes all of them (the control case), so a failure is the planted mistake's doing.  The oracle's
own source and library are never touched.
"""
import concurrent.futures as cf
import gc
import os
import subprocess

import pytest

import oracle
import test_oracle_adjoint as adj
import test_oracle_pins as pins

# (name, text in magnus_oracle.c, replacement, pins that must catch it)
MUTANTS = [
    # Leja points (Sec. 3)
    ("leja_second_point", "xi[1] = -2.0;", "xi[1] = 0.0;",
     [pins.test_leja_first_points_closed_form]),
    ("leja_tie_to_smaller_x", "if (cl[g] >= best - 1e-10 && cx[g] > pick) pick = cx[g];",
     "if (cl[g] >= best - 1e-10 && (pick == -INFINITY || cx[g] < pick)) pick = cx[g];",
     [pins.test_leja_first_points_closed_form]),
    ("leja_bisection_direction", "if (slope > 0.0) lo = mid; else hi = mid;",
     "if (slope > 0.0) hi = mid; else lo = mid;",
     [pins.test_leja_first_points_closed_form]),
    # divided differences, Opitz matrix (Sec. 3)
    ("dd_subdiagonal_sign", "if (j > 0) A[j * n + j - 1] = -I * rho;", "if (j > 0) A[j * n + j - 1] = I * rho;",
     [pins.test_divided_differences_interpolate_and_approximate]),
    ("dd_squaring_dropped", "for (int r = 0; r < q; r++) {", "for (int r = 0; r < 0; r++) {",
     [pins.test_divided_differences_interpolate_and_approximate]),
    ("dd_taylor_factorial", "P[e] = Q[e] / (double)k;", "P[e] = Q[e] / (double)(k + 1);",
     [pins.test_divided_differences_interpolate_and_approximate]),
    # spin-chain builders (Sec. 4, Kronecker order)
    ("spin_order_lsb_first", "return (int64_t)1 << (nspins - j);", "return (int64_t)1 << (j - 1);",
     [lambda: pins.test_xxz_and_field_csr_match_kronecker(5)]),
    ("spin_z_sign", "? -1.0 : 1.0; }", "? 1.0 : -1.0; }",
     [lambda: pins.test_xxz_and_field_csr_match_kronecker(5)]),
    ("xxz_flip_factor_two", "cval[cnt] = J[i - 1] * (1.0 - zz);", "cval[cnt] = J[i - 1];",
     [lambda: pins.test_xxz_and_field_csr_match_kronecker(5)]),
    ("xxz_anisotropy_dropped", "diag += delta * J[i - 1] * spin_z", "diag += J[i - 1] * spin_z",
     [lambda: pins.test_xxz_and_field_csr_match_kronecker(5)]),
    ("longrange_exponent", "1.0 / pow((double)(j - i), alpha);", "1.0 / pow((double)(j - i), 1.0);",
     [lambda: pins.test_longrange_dense_matches_kronecker(4)]),
    ("field_dense_value", "H[x * D + (x ^ spin_bit(nspins, i))] = 1.0;", "H[x * D + (x ^ spin_bit(nspins, i))] = 2.0;",
     [lambda: pins.test_longrange_dense_matches_kronecker(4)]),
    ("longrange_pairs_twice", "for (int j = i + 1; j <= nspins; j++) {", "for (int j = 1; j <= nspins; j++) if (j != i) {",
     [lambda: pins.test_longrange_dense_matches_kronecker(4)]),
    # term products, Gershgorin enclosure, drive coefficients
    ("csr_value_conjugated", "acc += t->val[e] * x[t->col[e]];", "acc += conj(t->val[e]) * x[t->col[e]];",
     [pins.test_apply_term_complex_hermitian_csr]),
    ("csr_column_ignored", "acc += t->val[e] * x[t->col[e]];", "acc += t->val[e] * x[i];",
     [pins.test_apply_term_and_gershgorin]),
    ("gershgorin_half_radius", "else R += cabs(t->val[e]);", "else R += 0.5 * cabs(t->val[e]);",
     [pins.test_apply_term_and_gershgorin]),
    ("drive_cos_sin_swapped", "f += c->ac[m] * cos(c->om[m] * t) + c->as[m] * sin(c->om[m] * t);",
     "f += c->ac[m] * sin(c->om[m] * t) + c->as[m] * cos(c->om[m] * t);",
     [pins.test_apply_term_and_gershgorin]),
    ("gershgorin_dense_centre_modulus", "if (j == i) c += creal(t->val[i * D + j]);",
     "if (j == i) c += cabs(t->val[i * D + j]);",
     [pins.test_lanczos_interval_dense_complex_and_small_dim, pins.test_csr_and_dense_storage_agree]),
    ("weyl_sum_ignores_sign", "lo += (x1 < x2) ? x1 : x2;", "lo += x1;",
     [lambda: adj.test_adjoint_gradient_matches_central_differences("M2")]),  # the costate has beta < 0
    ("m4_enclosure_radius_dropped", "lo -= kappa * r;\n    hi += kappa * r;", "lo -= 0.0 * r;\n    hi += 0.0 * r;",
     [lambda: pins.test_commutator_enclosure_contains_the_generator_spectrum("M4")]),
    ("m6_enclosure_radius_dropped", "    lo -= r;\n    hi += r;\n  }\n  *a = lo;", "  }\n  *a = lo;",
     [lambda: pins.test_commutator_enclosure_contains_the_generator_spectrum("M6")]),
    # Lanczos enclosure (the tighter spectral estimate)
    ("lanczos_three_term_dropped", "w[i] -= a * v1[i] + be[j] * v0[i];", "w[i] -= a * v1[i];",
     [lambda: pins.test_lanczos_interval_encloses_spectrum_and_is_tighter(6)]),
    ("lanczos_alpha_imaginary_part", "a += creal(conj(v1[i]) * w[i]);", "a += cimag(conj(v1[i]) * w[i]);",
     [lambda: pins.test_lanczos_interval_encloses_spectrum_and_is_tighter(6)]),
    ("sturm_count_sign", "if (q < 0.0) cnt++;", "if (q > 0.0) cnt++;",
     [lambda: pins.test_lanczos_interval_encloses_spectrum_and_is_tighter(6)]),
    ("ritz_second_largest", "tmax = tridiag_eig(al, be, mj, mj - 1);", "tmax = tridiag_eig(al, be, mj, mj > 1 ? mj - 2 : 0);",
     [lambda: pins.test_lanczos_interval_encloses_spectrum_and_is_tighter(6)]),
    ("lanczos_not_intersected", "if (a < t->a) a = t->a;\n  if (b > t->b) b = t->b;",
     "if (a > t->a) a = t->a;\n  if (b < t->b) b = t->b;",
     [lambda: pins.test_lanczos_interval_encloses_spectrum_and_is_tighter(6)]),
    ("ritz_residual_dropped", "double a = tmin - rmin - 0.01 * W, b = tmax + rmax + 0.01 * W;",
     "double a = tmin - 0.01 * W, b = tmax + 0.01 * W;", [pins.test_lanczos_residuals_on_three_eigenvalues]),
    ("ritz_margin_dropped", "double a = tmin - rmin - 0.01 * W, b = tmax + rmax + 0.01 * W;",
     "double a = tmin - rmin, b = tmax + rmax;", [pins.test_lanczos_residuals_on_three_eigenvalues]),
    ("inverse_iteration_sign", "d[i] = (x[i] - be[i] * d[i - 1]) / piv;", "d[i] = (x[i] + be[i] * d[i - 1]) / piv;",
     [pins.test_lanczos_residuals_on_three_eigenvalues]),
    # Newton-form Leja recurrence (Sec. 3)
    ("newton_shift_sign", "w[i] = (Kw[i] - c * w[i]) / gamma", "w[i] = (Kw[i] + c * w[i]) / gamma",
     [pins.test_expv_matches_scipy_expm_multiply]),
    ("newton_node_index", "- p->xi[j - 1] * w[i];", "- p->xi[j] * w[i];",
     [pins.test_expv_matches_scipy_expm_multiply]),
    ("newton_phase_sign", "cexp(-I * c / s);\n  int rc = ORC_OK;", "cexp(I * c / s);\n  int rc = ORC_OK;",
     [pins.test_expv_matches_scipy_expm_multiply]),
    ("newton_no_substeps", "int s = (int)ceil(gamma / p->rho_max);\n  if (s < 1) s = 1;\n  const double rho",
     "int s = 1;\n  const double rho", [lambda: pins.test_expv_matches_eigh_dim1024((3.0, -1.5))]),
    ("substep_phase_not_split", "cexp(-I * c / s);\n  int rc = ORC_OK;", "cexp(-I * c);\n  int rc = ORC_OK;",
     [lambda: pins.test_expv_matches_eigh_dim1024((3.0, -1.5))]),
    # Magnus integrators (Sec. 2)
    ("m4_commutator_sign", "- I * kappa * (y[i] - g->t2[i]);", "+ I * kappa * (y[i] - g->t2[i]);",
     [pins.test_order_four_against_independent_integrator]),
    ("m4_commutator_weight", "g->h * g->h / 12.0;\n  apply_combo", "g->h * g->h / 6.0;\n  apply_combo",
     [pins.test_order_four_against_independent_integrator]),
    ("cf4_factor_order", "const double right[2] = {a2, a1}, left[2] = {a1, a2};",
     "const double right[2] = {a1, a2}, left[2] = {a2, a1};",
     [pins.test_order_four_against_independent_integrator]),
    ("gauss_node", "const double c4[2] = {0.5 - r3 / 6.0, 0.5 + r3 / 6.0};",
     "const double c4[2] = {0.5 - r3 / 6.0, 0.5 + r3 / 3.0};",
     [lambda: pins.test_commuting_terms_give_gauss_quadrature("CF4")]),
    ("cf43_weight", "al3[3][3] = {\n      {37.0 / 240.0 - 10.0 * r15 / 261.0",
     "al3[3][3] = {\n      {37.0 / 240.0 - 10.0 * r15 / 216.0",
     [lambda: pins.test_commuting_terms_give_gauss_quadrature("CF4_3")]),
    ("m2_left_point", "const double one = 1.0, half = 0.5;", "const double one = 1.0, half = 0.0;",
     [pins.test_order_two_of_the_midpoint_method]),
    ("m6_printed_b3_weight", "y[i] = I * (ux[i] + vx[i] / 12.0", "y[i] = I * (ux[i] + vx[i] / 2.0",
     [lambda: pins.test_commuting_terms_give_gauss_quadrature("M6")]),
    ("m6_commutator_sign", "(uvx[i] - vux[i]) / 240.0", "(vux[i] - uvx[i]) / 240.0",
     [pins.test_order_six_against_independent_integrator]),
    ("exponent_without_step", "g->beta[k] = h * s;", "g->beta[k] = s;",
     [lambda: pins.test_time_independent_is_exact("CF4")]),
    ("m6_b2_weight", "else if (j == 2) coef[k] = r15 / 3.0 * g->h", "else if (j == 2) coef[k] = r15 / 2.0 * g->h",
     [pins.test_order_six_against_independent_integrator]),
    ("m6_v_weight", "y[i] -= (b1wx[i] - wb1x[i]) / 60.0;", "y[i] -= (b1wx[i] - wb1x[i]) / 30.0;",
     [pins.test_order_six_against_independent_integrator]),
    ("m6_w_weight", "y[i] += 2.0 * b3[i];", "y[i] += b3[i];",
     [pins.test_order_six_against_independent_integrator]),
    ("m6_u_b3_sign", "y[i] += -20.0 * b1[i] - b3[i];", "y[i] += -20.0 * b1[i] + b3[i];",
     [pins.test_order_six_with_two_driven_terms]),
    # augmented block matrix and adjoint gradient
    ("frechet_block_sign", "(ka[i] + g.u1[i] - c * wa[i])", "(ka[i] - g.u1[i] - c * wa[i])",
     [lambda: adj.test_frechet_matches_daleckii_krein((0.03, 0.02))]),
    ("costate_direction", "negb[k] = -betas[e * MAX_TERMS + k];", "negb[k] = betas[e * MAX_TERMS + k];",
     [lambda: adj.test_adjoint_gradient_matches_central_differences("M2")]),
    ("adjoint_weight_derivative", "dbeta[e * ng + 1 + m] = h * sc;", "dbeta[e * ng + 1 + m] = sc;",
     [lambda: adj.test_adjoint_gradient_matches_central_differences("M2")]),
    ("adjoint_constant_derivative", "dbeta[e * ng] = h * s0;", "dbeta[e * ng] = s0;",
     [lambda: adj.test_adjoint_gradient_matches_central_differences("M2")]),
    ("fidelity_gradient_unconjugated", "grad[q] = 2.0 * creal(conj(z) * dz[q]);", "grad[q] = 2.0 * creal(z * dz[q]);",
     [lambda: adj.test_adjoint_gradient_matches_central_differences("M2")]),
    ("frechet_node_index", "- p->xi[j - 1] * wb[i];", "- p->xi[j] * wb[i];",
     [lambda: adj.test_frechet_matches_daleckii_krein((0.03, 0.02))]),
    ("frechet_scalar_block_sign", "a[i] = ph * (a[i] - I * g.u1[i]);", "a[i] = ph * (a[i] + I * g.u1[i]);",
     [adj.test_frechet_of_a_scalar_generator]),
    ("adjoint_cf43_stage_order", "w[q][j] = al[2 - q][j];", "w[q][j] = al[q][j];",
     [lambda: adj.test_adjoint_gradient_matches_central_differences("CF4_3")]),
    ("adjoint_cf4_stage_order", "w[0][0] = a2; w[0][1] = a1;   /* right factor, applied first */\n    w[1][0] = a1; w[1][1] = a2;",
     "w[0][0] = a1; w[0][1] = a2;   /* right factor, applied first */\n    w[1][0] = a2; w[1][1] = a1;",
     [lambda: adj.test_adjoint_gradient_matches_central_differences("CF4")]),
    ("overlap_unconjugated", "z += conj(phi[i]) * states[nexp * D + i];", "z += phi[i] * states[nexp * D + i];",
     [lambda: adj.test_adjoint_gradient_matches_central_differences("M2")]),
]


def _compile(src_text, folder):
    os.makedirs(folder, exist_ok=True)
    src = os.path.join(folder, "magnus_oracle.c")
    with open(src, "w") as f:
        f.write(src_text)
    with open(os.path.join(os.path.dirname(oracle._SRC), "magnus_oracle.h")) as f:
        hdr = f.read()
    with open(os.path.join(folder, "magnus_oracle.h"), "w") as f:
        f.write(hdr)
    lib = os.path.join(folder, "libmutant.so")
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", lib, src, "-lm"])
    return lib


@pytest.fixture(scope="module")
def builds(tmp_path_factory):
    """Every mutant (and the unmodified control) compiled once, in parallel."""
    with open(oracle._SRC) as f:
        original = f.read()
    root = tmp_path_factory.mktemp("oracle_mutants")
    jobs = {"control": original}
    for name, old, new, _ in MUTANTS:
        assert original.count(old) == 1, (name, original.count(old))
        jobs[name] = original.replace(old, new)
    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        futs = {name: ex.submit(_compile, text, str(root / name)) for name, text in jobs.items()}
        return {name: fut.result() for name, fut in futs.items()}


def _run_pins(monkeypatch, lib_path, pin_list):
    """Run the pins with the wrapper bound to ``lib_path``; return the pins that failed."""
    failed = []
    with monkeypatch.context() as m:
        m.setattr(oracle, "_lib", oracle.load(lib_path))
        for pin in pin_list:
            try:
                pin()
            except (AssertionError, oracle.OracleError):
                failed.append(pin)
        gc.collect()  # free the problems made by this library while it is still bound
    return failed


def test_control_copy_passes_every_pin(builds, monkeypatch):
    every = []
    for _, _, _, pin_list in MUTANTS:
        every += [p for p in pin_list if p not in every]
    # the lambdas are distinct objects; run each case's pins once
    assert _run_pins(monkeypatch, builds["control"], every) == []


@pytest.mark.parametrize("name", [m[0] for m in MUTANTS])
def test_planted_mistake_is_caught(name, builds, monkeypatch):
    pin_list = next(m[3] for m in MUTANTS if m[0] == name)
    failed = _run_pins(monkeypatch, builds[name], pin_list)
    assert failed, f"no pin caught the planted mistake {name}"
