"""Planted mistakes in the oracle are caught by its pins (CPU only).

Each mutant is a copy of ``oracle/sop_oracle.c`` with one plausible mistake
(a dropped term, a wrong sign, index or convention, a transposed operand),
compiled to a temporary library.  The test swaps it in and checks that at
least one of the listed pins fails.  The real oracle source is never edited.
"""
import os
import subprocess
import tempfile

import pytest

import oracle
import oracle_pins as pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "sop_oracle.c")

# (name, text to replace, replacement, pins expected to catch it)
MUTANTS = [
    ("kinetic_sign", "double ang = -tau * p2 / (2.0 * mass * hbar);",
     "double ang = tau * p2 / (2.0 * mass * hbar);", [pins.pin_free_schrodinger_exact]),
    ("kinetic_mass_factor", "double ang = -tau * p2 / (2.0 * mass * hbar);",
     "double ang = -tau * p2 / (mass * hbar);", [pins.pin_free_schrodinger_exact]),
    ("nyquist_sign", "int64_t kap = (2 * k < n) ? k : k - n;",
     "int64_t kap = (2 * k <= n) ? k : k - n;", [pins.pin_free_dirac_exact]),
    ("inverse_drops_1_over_n", "const double s = 1.0 / (double)N;",
     "const double s = 1.0;", [pins.pin_fftn_library, pins.pin_free_schrodinger_exact]),
    ("twiddle_index", "int64_t e = ((int64_t)q * (k + m * s)) % n;",
     "int64_t e = ((int64_t)q * k) % n;", [pins.pin_fft_brute_force]),
    ("full_instead_of_half_V", "schr_real_space(psi, V, ndim, dims, h, charge, hbar, tau, 0.5, E);\n        orc_fftn",
     "schr_real_space(psi, V, ndim, dims, h, charge, hbar, tau, 1.0, E);\n        orc_fftn",
     [pins.pin_coherent_state_second_order, pins.pin_constant_potential_phase]),
    ("field_sign", "W -= charge * lattice_x(dims[a], h[a], idx[a]) * E[a];",
     "W += charge * lattice_x(dims[a], h[a], idx[a]) * E[a];", [pins.pin_field_kick_plane_wave]),
    ("velocity_gauge_sign", "if (A) p -= charge * A[a];", "if (A) p += charge * A[a];",
     [pins.pin_velocity_gauge_plane_waves, pins.pin_velocity_gauge_lattice_shift]),
    ("velocity_gauge_drops_A", "if (A) p -= charge * A[a];", "(void)A;",
     [pins.pin_velocity_gauge_plane_waves, pins.pin_velocity_gauge_lattice_shift]),
    ("dirac1d_u_sign", "u[i][j] = (i == j ? dp : 0.0) + dm * sgn * ba;",
     "u[i][j] = (i == j ? dp : 0.0) - dm * sgn * ba;",
     [pins.pin_dirac1d_u_diagonalises, pins.pin_dirac1d_free_exact]),
    ("dirac1d_mixing_sign", "R[i][j] = (i == j ? cos(theta) : 0.0) + I * sin(theta) * al[i][j];",
     "R[i][j] = (i == j ? cos(theta) : 0.0) - I * sin(theta) * al[i][j];",
     [pins.pin_dirac1d_equals_2d_pair, pins.pin_dirac1d_uniform_A_second_order]),
    ("dirac1d_beta_sign", "be[1][0] = 0; be[1][1] = -1;", "be[1][0] = 0; be[1][1] = 1;",
     [pins.pin_dirac1d_u_diagonalises, pins.pin_dirac1d_free_exact]),
    ("dirac1d_energy_u_not_h", "dirac1d_h(p[0], mass, c, H);", "dirac1d_u(p[0], mass, c, H);",
     [pins.pin_dirac1d_energy]),
    ("alpha3_sign", "alpha[2][0][2] = 1; alpha[2][1][3] = -1;", "alpha[2][0][2] = -1; alpha[2][1][3] = 1;",
     [pins.pin_free_dirac_exact_3d, pins.pin_dirac_uniform_A_second_order_3d]),
    ("profile_column_index", "const cplx(*Rj)[4] = (const cplx(*)[4])R[j % nx];",
     "const cplx(*Rj)[4] = (const cplx(*)[4])R[(j + 1) % nx];", [pins.pin_dirac_profile_two_steps_numpy]),
    ("profile_step_index", "dirac_mixing(field + (n * nx + i) * ndim,", "dirac_mixing(field + i * ndim,",
     [pins.pin_dirac_profile_two_steps_numpy]),
    ("lattice_origin", "return -0.5 * (double)n * h + (double)j * h;",
     "return -0.5 * (double)n * h + (double)(j + 1) * h;", [pins.pin_field_kick_plane_wave]),
    ("dirac_u_not_adjoint", "for (int k = 0; k < 4; ++k) s += conj(u[k][i]) * w[k];",
     "for (int k = 0; k < 4; ++k) s += u[i][k] * w[k];",
     [pins.pin_dirac_kinetic_expm, pins.pin_free_dirac_exact]),
    ("alpha2_sign", "alpha[1][0][3] = -I;", "alpha[1][0][3] = I;", [pins.pin_dirac_algebra]),
    ("alpha_transposed", "alpha[1][0][3] = -I; alpha[1][1][2] = I; alpha[1][2][1] = -I; alpha[1][3][0] = I;",
     "alpha[1][0][3] = I; alpha[1][1][2] = -I; alpha[1][2][1] = I; alpha[1][3][0] = -I;",
     [pins.pin_dirac_algebra, pins.pin_dirac_kinetic_expm]),
    ("d_minus_sign", "const double dm = sqrt(0.5 - 0.5 / root);",
     "const double dm = sqrt(0.5 + 0.5 / root);", [pins.pin_dirac_u_diagonalises]),
    ("dirac_energy_c_power", "const double E = sqrt(mass * mass * c * c * c * c + p2 * c * c);",
     "const double E = sqrt(mass * mass * c * c * c * c + p2 * c);",
     [pins.pin_dirac_kinetic_expm, pins.pin_dirac_velocity]),
    ("mixing_charge_sign", "const double theta = delta * charge * c * Aabs / hbar;",
     "const double theta = -delta * charge * c * Aabs / hbar;",
     [pins.pin_dirac_mixing_expm, pins.pin_dirac_uniform_A_second_order]),
    ("energy_drops_parseval_factor", "return dV * kv.s + (dV / (double)N) * kt.s;",
     "return dV * kv.s + dV * kt.s;", [pins.pin_schrodinger_energy, pins.pin_dirac_energy]),
    ("dirac_V_full_step", "double ang = -0.5 * tau * (V ? V[j] : 0.0) / hbar;",
     "double ang = -tau * (V ? V[j] : 0.0) / hbar;", [pins.pin_dirac_constant_potential_phase]),
]


def _build_mutant(name, old, new, tmp):
    src = open(SRC).read()
    assert src.count(old) >= 1, f"mutation site for {name} not found"
    path_c = os.path.join(tmp, f"{name}.c")
    path_so = os.path.join(tmp, f"lib{name}.so")
    with open(path_c, "w") as f:
        f.write(src.replace(old, new))
    subprocess.run(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-ffp-contract=off",
                    path_c, "-o", path_so, "-lm"], check=True)
    return path_so


@pytest.mark.parametrize("name,old,new,catchers", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_is_caught(orc, name, old, new, catchers):
    with tempfile.TemporaryDirectory() as tmp:
        so = _build_mutant(name, old, new, tmp)
        caught = []
        with oracle._swap_library(so):
            for pin in catchers:
                try:
                    pin(orc)
                except AssertionError:
                    caught.append(pin.__name__)
        assert caught, f"mutant {name} passed every pin in {[p.__name__ for p in catchers]}"
    # the real oracle is back in place and still passes the same pins
    for pin in catchers:
        pin(orc)
