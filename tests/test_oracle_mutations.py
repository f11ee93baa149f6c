"""Planted mistakes in the oracle, on the CPU: each mutant of scivr_oracle.c (one
plausible slip: a dropped term, a wrong sign, factor or index) is compiled into its own
shared object and the pin that should catch it is run against that build in a child
process (SCIVR_ORACLE_LIB).  Every mutant must fail its pin, and the unmodified source
compiled the same way must pass all of them.  Nothing here runs on a GPU."""
import os
import subprocess
import sys

import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "scivr_oracle.c")

P = "tests/test_oracle_propagation.py::"
S = "tests/test_oracle_spectrum.py::"
H = "tests/test_oracle_hk.py::"
E = "tests/test_oracle_pes.py::"
N = "tests/test_oracle_mlp.py::"
CA = "tests/test_oracle_cartesian.py::"

# name: ([(exact source text, replacement), ...], [pins that must fail])
MUTANTS = {
    "kick with the wrong sign": (
        [("for (int a = 0; a < F; ++a) p[a] -= tau * g[a];", "for (int a = 0; a < F; ++a) p[a] += tau * g[a];")],
        [P + "test_harmonic_amplitude_closed_form"]),
    "kinetic action of the drift dropped": (
        [("    *S += tau * kin;", "    (void)kin;")],
        [P + "test_action_is_a_generating_function"]),
    "wrong triple-jump weight": (
        [("double w0 = -cbrt2 / (2.0 - cbrt2);", "double w0 = -cbrt2 / (2.0 + cbrt2);")],
        [P + "test_fourth_order_convergence_of_the_flow"]),
    "monodromy kick halved": (
        [("M[a * n + col] -= tau * hm;", "M[a * n + col] -= 0.5 * tau * hm;")],
        [P + "test_monodromy_matches_finite_differences"]),
    "overlap phase factor": (
        [("im += 0.5 * (p1[i] + p2[i]) * dq;", "im += (p1[i] + p2[i]) * dq;")],
        [E + "test_overlap_vs_quadrature"]),
    "overlap width factor": (
        [("re += -0.25 * gamma[i] * dq * dq", "re += -0.5 * gamma[i] * dq * dq")],
        [E + "test_overlap_vs_quadrature"]),
    "prefactor phase not halved": (
        [("double phase = cimag(lo) + S + 0.5 * theta;", "double phase = cimag(lo) + S + theta;")],
        [P + "test_harmonic_amplitude_closed_form"]),
    "width ordering of the prefactor matrix": (
        [("double re = ga / gb * Mqq + gb / ga * Mpp;", "double re = gb / ga * Mqq + ga / gb * Mpp;")],
        [P + "test_prefactor_matrix_is_the_analytic_block_of_the_monodromy"]),
    "unwrapping without the reference rotation": (
        [("double d = arg_new - arg_old + ref_step;", "double d = arg_new - arg_old;"),
         ("return theta + d - ref_step;", "return theta + d;")],
        [P + "test_phase_unwrapping_when_arg_det_A_turns_more_than_pi_per_step"]),
    "stability quantity |det M - 1|": (
        [("fabs(detM * detM - 1.0)", "fabs(detM - 1.0)")],
        [P + "test_stability_quantity_is_det_squared_minus_one"]),
    "spectrum normalisation missing dt": (
        [("dt * dt / (OR_TWO_PI * T * (double)n_good)", "dt / (OR_TWO_PI * T * (double)n_good)")],
        [S + "test_spectra_obey_the_sum_rule"]),
    "Husimi position width": (
        [("qj[i] = q_eq[i] + or_normal(seed, j, i) / sqrt(gamma[i]);",
          "qj[i] = q_eq[i] + or_normal(seed, j, i) / sqrt(2.0 * gamma[i]);")],
        [S + "test_husimi_moments_and_normality"]),
    "sampling weight exponent": (
        [("w[j] = exp(-2.0 * creal(lo));", "w[j] = exp(-creal(lo));")],
        [S + "test_weights_are_inverse_husimi_density"]),
    "HK weight of each state's own density": (
        [("double complex lo00 = x == 0 ? lo0 : or_log_overlap(F, prm->gamma, prm->p_eq,\n"
          "                                                                        prm->q_eq, p0, q0);",
          "double complex lo00 = lo0;")],
        [H + "test_reference_states_share_trajectories_sampled_around_the_first"]),
    "HK prefactor modulus dropped": (
        [("double complex Ct = sqrt(cabs(detA)) * cexp(0.5 * I * theta);",
          "double complex Ct = cexp(0.5 * I * theta);")],
        [H + "test_widths_unequal_to_the_frequency_exercise_the_prefactor_modulus"]),
    "Morse curvature": (
        [("H[i * F + i] += 2.0 * Dm * am * am * u * (2.0 * u - 1.0);",
          "H[i * F + i] += 2.0 * Dm * am * am * u * (u - 1.0);")],
        [E + "test_gradient_and_hessian_match_finite_differences"]),
    "coupling Hessian halved": (
        [("H[idx[s] * F + idx[t]] += prod;", "H[idx[s] * F + idx[t]] += 0.5 * prod;")],
        [E + "test_gradient_and_hessian_match_finite_differences"]),
    "activation's second derivative": (
        [("*f2 = s * (1.0 - s) * (2.0 + z * (1.0 - 2.0 * s));", "*f2 = s * (1.0 - s) * (1.0 + z * (1.0 - 2.0 * s));")],
        [N + "test_mlp_gradient_and_hessian_vs_finite_differences"]),
    "pivot swap without the sign change": (
        [("            det = -det;\n        }\n        double akk = A[k * n + k];",
          "        }\n        double akk = A[k * n + k];")],
        [E + "test_real_determinant_vs_lapack"]),
    "complex pivot swap without the sign change": (
        [("            det = -det;\n        }\n        double complex akk = A[k * n + k];",
          "        }\n        double complex akk = A[k * n + k];")],
        [E + "test_complex_determinant_vs_lapack"]),
    "monodromy drift with the wrong sign": (
        [("M[(F + a) * n + col] += tau * M[a * n + col];", "M[(F + a) * n + col] -= tau * M[a * n + col];")],
        [P + "test_monodromy_matches_finite_differences"]),
    "coupling gradient halved": (
        [("g[idx[s]] += prod;", "g[idx[s]] += 0.5 * prod;")],
        [E + "test_gradient_and_hessian_match_finite_differences"]),
    "time-to-energy transform with the wrong sign": (
        [("tw[c] = cos(ang) + I * sin(ang);", "tw[c] = cos(ang) - I * sin(ang);")],
        [S + "test_dirichlet_closed_form"]),
    "HK transform without the half weight at t = 0": (
        [("double complex acc = 0.5 * C[0];", "double complex acc = C[0];")],
        [H + "test_one_sided_transform_is_the_dirichlet_kernel"]),
    "nine Philox rounds": (
        [("for (int r = 0; r < 10; ++r) {", "for (int r = 0; r < 9; ++r) {")],
        [S + "test_philox_known_answers"]),
    "Box-Muller radius": (
        [("double r = sqrt(-2.0 * log(u1));", "double r = sqrt(-log(u1));")],
        [S + "test_husimi_moments_and_normality"]),
    "bad trajectories kept in the time-averaged sum": (
        [("                if (!good[j]) continue;\n                double complex X = 0.0;",
          "                double complex X = 0.0;")],
        [S + "test_bad_trajectories_are_excluded_and_n_good_normalises"]),
    "sampling weights left out of the time-averaged sum": (
        [("acc += w[j] * (creal(X) * creal(X) + cimag(X) * cimag(X));",
          "acc += (creal(X) * creal(X) + cimag(X) * cimag(X));")],
        [S + "test_parseval_on_the_dft_grid"]),
    "bad trajectories kept in the survival amplitude": (
        [("            if (good[j]) acc += amp[j * amp_ld + c];", "            acc += amp[j * amp_ld + c];")],
        [H + "test_one_sided_transform_is_the_dirichlet_kernel"]),
    "every reference state given the first one's overlap": (
        [("double complex lo = or_log_overlap(F, prm->gamma, prm->p_eq + x * F,\n"
          "                                                   prm->q_eq + x * F, p, q);",
          "double complex lo = or_log_overlap(F, prm->gamma, prm->p_eq,\n"
          "                                                   prm->q_eq, p, q);")],
        [H + "test_reference_states_share_trajectories_sampled_around_the_first"]),
    "Cartesian bend gradient with the wrong sign": (
        [("const double gi = c->k_bend * dc * dcy[i];", "const double gi = -c->k_bend * dc * dcy[i];")],
        [CA + "test_cartesian_derivatives_match_finite_differences"]),
    "Cartesian bond Hessian without its transverse part": (
        [("f1 * ((d == f ? 1.0 : 0.0) - w[d] * w[f] / ww) / r", "0.0 * f1")],
        [CA + "test_cartesian_derivatives_match_finite_differences"]),   # zero at the minimum: FD off it
    "normal modes of the Hessian without mass weighting": (
        [("A[i * 9 + j] = Hx[i * 9 + j] / sqrt(c->mass[i / 3] * c->mass[j / 3]);", "A[i * 9 + j] = Hx[i * 9 + j];")],
        [CA + "test_normal_mode_frequencies_match_the_wilson_gf_closed_form"]),
    "mode matrix not divided by the square root of the mass": (
        [("c->Lm[i * 3 + m] = sgn * Vm[i * 9 + col] / sqrt(c->mass[i / 3]);", "c->Lm[i * 3 + m] = sgn * Vm[i * 9 + col];")],
        [CA + "test_mode_matrix_is_mass_orthonormal_and_free_of_rigid_motions"]),
    "Jacobi rotation of the columns with the wrong sign": (
        [("A[k * 9 + p] = cs * akp - sn * akq;", "A[k * 9 + p] = cs * akp + sn * akq;")],
        [CA + "test_normal_mode_frequencies_match_the_wilson_gf_closed_form"]),
    "gradient-matching term of the training gradient halved": (
        [("u[i] = 2.0 * beta * e / (double)n;", "u[i] = beta * e / (double)n;")],
        [N + "test_training_gradient_vs_finite_differences"]),
}


def _build(workdir, name, pairs):
    src = open(SRC).read()
    for old, new in pairs:
        assert src.count(old) == 1, (name, old)
        src = src.replace(old, new)
    os.makedirs(workdir, exist_ok=True)
    c = os.path.join(workdir, "mutant.c")
    with open(c, "w") as f:
        f.write(src)
    so = os.path.join(workdir, "libmutant.so")
    subprocess.run(["gcc", *oracle._CFLAGS, c, "-o", so, "-lm"], check=True)
    return so


def _run_pins(lib, pins):
    # one OpenMP thread per child: the children run side by side
    env = dict(os.environ, SCIVR_ORACLE_LIB=lib, OMP_NUM_THREADS="1")
    return subprocess.run([sys.executable, "-m", "pytest", *pins, "-x", "-q", "-p", "no:cacheprovider"],
                          cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)


CONTROL = "unmodified source"


@pytest.fixture(scope="module")
def outcomes(tmp_path_factory):
    """Build every mutant (and the unmodified source) and run its pins, in parallel."""
    from concurrent.futures import ThreadPoolExecutor
    base = tmp_path_factory.mktemp("mutants")
    jobs = {name: (pairs, pins) for name, (pairs, pins) in MUTANTS.items()}
    jobs[CONTROL] = ([], sorted({p for _, ps in MUTANTS.values() for p in ps}))

    def one(item):
        k, (name, (pairs, pins)) = item
        return name, _run_pins(_build(os.path.join(base, str(k)), name, pairs), pins)

    with ThreadPoolExecutor(max_workers=max(1, min(8, os.cpu_count() or 1))) as ex:
        return dict(ex.map(one, enumerate(sorted(jobs.items()))))


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(outcomes, name):
    out = outcomes[name]
    assert out.returncode == 1, (name, out.returncode, out.stdout[-1500:], out.stderr[-1500:])
    assert " failed" in out.stdout, out.stdout[-1500:]


def test_unmodified_source_passes_every_pin(outcomes):
    out = outcomes[CONTROL]
    assert out.returncode == 0, (out.stdout[-2000:], out.stderr[-1500:])
