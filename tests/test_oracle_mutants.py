"""Planted mistakes: each case copies the oracle, plants one plausible mistake
in the copy (a dropped term, a flipped sign, a wrong factor or index) and
checks that the pins meant to catch it fail on the copy. The oracle's test
infrastructure checking itself, on the CPU; the CUDA path is not involved.
Each planted text must occur exactly once in the current oracle source, so an
edit of the oracle that moves a line makes the case fail loudly instead of
silently testing nothing."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
C = "oracle/wl_oracle.c"
T = "tests/test_oracle.py::"

# (name, file, original text, planted text, pins that must fail)
CASES = [
    ("limiter_without_inner_median", C, "median3(phi, c, median3(10.0 * c - 9.0 * uu, c, d))",
     "median3(phi, c, d)", [T + "test_limited_advection_of_a_square_wave_makes_no_new_extrema"]),
    ("first_moment_sign", C, "0.25 - 0.25 * r * r", "0.25 + 0.25 * r * r",
     [T + "test_kernel_moments_match_quadrature"]),
    ("blend_gradient_sign", C, "* 0.5 * (up - dn);", "* 0.5 * (dn - up);",
     [T + "test_bdim_blend_closed_form_for_linear_f"]),
    ("exit_mass_correction_sign", C, "double corr = -q / (double)np;", "double corr = q / (double)np;",
     [T + "test_exit_condition_zeroes_net_flux_and_keeps_uniform_flow"]),
    ("coarse_face_coefficient_factor", C, "lv_lin(C, i, j, k)] = 0.5 * s;", "lv_lin(C, i, j, k)] = 0.25 * s;",
     [T + "test_multigrid_convergence_is_grid_independent"]),
    ("pcg_beta_inverted", C, "double beta = rho2 / rho;", "double beta = rho / rho2;",
     [T + "test_multigrid_matches_dense_solve", T + "test_multigrid_convergence_is_grid_independent"]),
    ("cfl_viscous_term", C, "cfl / (m + 5.0 * g->nu)", "cfl / (m + 0.5 * g->nu)",
     [T + "test_cfl_closed_form_on_uniform_field"]),
    ("pressure_force_sign", C, "F[a] -= pk * nrm[a];", "F[a] += pk * nrm[a];",
     [T + "test_pressure_force_invariants"]),
    ("adjoint_exit_plane_index_3d", C, "*index = (size_t)idx[1] + (size_t)g->n[1] * idx[2];",
     "*index = (size_t)idx[1] - (size_t)g->n[1] * idx[2];",
     ["tests/test_oracle_adjoint.py::test_conv_diff_vjp_matches_central_differences[sphere3d_exit]"]),
    ("viscous_transpose_z_index", C, "su_loc(g, a, i + A[0], j + A[1], k + A[2], &kind, &at);",
     "su_loc(g, a, i + A[0], j + A[1], k - A[2], &kind, &at);",
     ["tests/test_oracle_sampled.py::test_viscous_force_transpose_is_its_linear_part_3d"]),
    ("adjoint_blend_periodic_wrap", C, "P[ax] = ((P[ax] % N) + N) % N; M[ax]", "P[ax] = ((P[ax] % N) - N) % N; M[ax]",
     ["tests/test_oracle_adjoint.py::test_step_vjp_matches_central_differences[sphere3d_exit]"]),
    ("adjoint_exit_scaling", C, "ueGb[p] += -w * dt * Ubar * e;", "ueGb[p] += -w * dt / Ubar * e;",
     ["tests/test_oracle_adjoint.py::test_step_vjp_matches_central_differences[sphere3d_exit]"]),
    ("field_cotangent_upper_clamp", C, "else if (P[ax] > N - 1) P[ax] = N - 1;", "else if (P[ax] > N + 1) P[ax] = N - 1;",
     ["tests/test_oracle_adjoint.py::test_field_cotangents_match_central_differences[wall_circle]"]),
    ("stepping_clock", "oracle/__init__.py", "self.t += dt", "self.t -= dt",
     [T + "test_sim_moves_a_body_on_its_own_clock"]),
    ("network_loss_sign", "oracle/net.py", "L = float(np.sum((y - t) ** 2) / den)",
     "L = float(np.sum((y + t) ** 2) / den)",
     ["tests/test_oracle_net.py::test_backward_loss_of_an_identity_network_is_its_closed_form"]),
]


@pytest.mark.parametrize("name,path,old,new,pins", CASES, ids=[c[0] for c in CASES])
def test_pins_fail_on_a_planted_mistake(tmp_path, name, path, old, new, pins):
    for sub in ("oracle", "synth", "tests"):
        shutil.copytree(os.path.join(ROOT, sub), tmp_path / sub,
                        ignore=shutil.ignore_patterns("__pycache__", "*.so", "*.tmp"))
    f = tmp_path / path
    src = f.read_text()
    assert src.count(old) == 1, f"{name}: the planted text must occur once in {path}"
    f.write_text(src.replace(old, new))
    env = dict(os.environ, OMP_NUM_THREADS="2")
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-p", "no:cacheprovider", *pins],
                       cwd=tmp_path, env=env, capture_output=True, text=True, timeout=600)
    # exit status 1: tests ran and some failed (not a collection or usage error)
    assert r.returncode == 1 and " failed" in r.stdout, (name, r.returncode, r.stdout[-1500:])
