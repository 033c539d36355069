"""The pins catch plausible mistakes: each case plants one in a copy of the
oracle's source (on the CPU), builds it, and runs the pin that must fail."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "lbm_oracle.c")

MUTATIONS = [
    ("force sign", "F[i] = -s->G * p0 * acc[i];", "F[i] = s->G * p0 * acc[i];",
     "tests/test_oracle_force.py::test_force_on_monomials_gives_isotropic_moments"),
    ("streaming direction", "size_t dst = cell_index(s, wrap(x + s->c[b][0], s->nx),",
     "size_t dst = cell_index(s, wrap(x - s->c[b][0], s->nx),",
     "tests/test_oracle_collision.py::test_streaming_is_the_shift_permutation"),
    ("dropped u.u term of feq", " - uu / (2.0 * s->cs2));", ");",
     "tests/test_oracle_collision.py::test_feq_moments"),
    ("Guo prefactor", "double pref = 1.0 - 1.0 / (2.0 * s->tau);", "double pref = 1.0 - 1.0 / s->tau;",
     "tests/test_oracle_collision.py::test_guo_forcing_moments"),
    ("E8 weight", "s->sq[1] = 2; s->w[1] = 4.0 / 45.0;", "s->sq[1] = 2; s->w[1] = 4.0 / 44.0;",
     "tests/test_oracle_tables.py::test_force_stencil_matches_exact_isotropy_solution"),
    ("transposed MRT inverse", "fout[b] += s->Minv[b][k] * mpost[k];", "fout[b] += s->Minv[k][b] * mpost[k];",
     "tests/test_oracle_collision.py::test_mrt_with_uniform_rates_is_bgk"),
    ("half-force velocity", "u[i] = (j[i] + 0.5 * F[i]) / rho;", "u[i] = (j[i] + F[i]) / rho;",
     "tests/test_oracle_collision.py::test_guo_forcing_moments"),
    ("exact-difference half increment", "uv[i] = up[i] + F[i] / rho;", "uv[i] = up[i] + 0.5 * F[i] / rho;",
     "tests/test_oracle_collision.py::test_exact_difference_forcing_moments"),
    ("exact-difference relaxes to the shifted state", "fout[b] = fin[b] - (fin[b] - e0) / s->tau + (e1 - e0);",
     "fout[b] = fin[b] - (fin[b] - e1) / s->tau + (e1 - e0);",
     "tests/test_oracle_collision.py::test_exact_difference_forcing_moments"),
    ("wall passes populations through", "for (int b = 0; b < s->Q; ++b) fout[b] = fin[s->opp[b]];",
     "for (int b = 0; b < s->Q; ++b) fout[b] = fin[b];",
     "tests/test_oracle_wall.py::test_wall_channel_shear_wave_decays_with_no_slip"),
    ("wall reflects specularly", "if (s->c[k][0] == -s->c[b][0] && s->c[k][1] == -s->c[b][1]",
     "if (s->c[k][0] == s->c[b][0] && s->c[k][1] == -s->c[b][1]",
     "tests/test_oracle_wall.py::test_wall_channel_shear_wave_decays_with_no_slip"),
    ("wall psi from the populations it holds",
     "s->psi[n] = is_solid(s, (n / s->nx) % s->ny) ? s->psi_w : or_psi_of_rho(s, r);",
     "s->psi[n] = or_psi_of_rho(s, r);",
     "tests/test_oracle_wall.py::test_wall_force_is_one_sided"),
    ("wall one row too thick", "static int is_solid(const or_sim* s, int y) { return y < s->wall_rows; }",
     "static int is_solid(const or_sim* s, int y) { return y <= s->wall_rows; }",
     "tests/test_oracle_wall.py::test_wall_force_is_one_sided"),
    ("init width W in place of W/2", "0.5 * (rho_l + rho_g) - 0.5 * (rho_l - rho_g) * tanh(2.0 * (r - R) / W);",
     "0.5 * (rho_l + rho_g) - 0.5 * (rho_l - rho_g) * tanh((r - R) / W);",
     "tests/test_oracle_init.py::test_droplet_initial_state_is_the_tanh_profile"),
    ("init centre at (n - 1)/2", "double d = (double)i - (double)(n / 2);",
     "double d = (double)i - 0.5 * (double)(n - 1);",
     "tests/test_oracle_init.py::test_droplet_initial_state_is_the_tanh_profile"),
    ("flat slab width W in place of W/2", "tanh(2.0 * (r - 0.25 * L) / W);", "tanh((r - 0.25 * L) / W);",
     "tests/test_oracle_init.py::test_flat_initial_state_is_the_tanh_slab"),
    ("MRT s_e and s_eps swapped", "double r[9] = { st, s_e, s_eps, st, s_q, st, s_q, st, st };",
     "double r[9] = { st, s_eps, s_e, st, s_q, st, s_q, st, st };",
     "tests/test_oracle_mrt.py::test_each_moment_relaxes_at_its_own_rate"),
    ("MRT s_q missing from the D3Q19 m moments", "st, s_eps, st, s_eps, st, st, st, s_q, s_q, s_q };",
     "st, s_eps, st, s_eps, st, st, st, s_eps, s_eps, s_eps };",
     "tests/test_oracle_mrt.py::test_each_moment_relaxes_at_its_own_rate"),
    ("MRT D3Q19 m_x polynomial sign", "case 16: return (y * y - z * z) * x;", "case 16: return (y * y + z * z) * x;",
     "tests/test_oracle_mrt.py::test_each_moment_relaxes_at_its_own_rate"),
    ("thickness band edge", "if (r >= 1.05 * rg && r <= 0.95 * rl) thick += 1.0;",
     "if (r >= 1.05 * rg && r <= 0.9 * rl) thick += 1.0;",
     "tests/test_oracle_init.py::test_thickness_counts_band_nodes_of_a_flat_slab"),
    ("thickness counted from one", "double thick = 0.0;", "double thick = 1.0;",
     "tests/test_oracle_init.py::test_thickness_counts_band_nodes_of_a_flat_slab"),
    ("thickness along the wrong axis", "double r = s->rho[cell_index(s, x, s->ny / 2, s->nz / 2)];",
     "double r = s->rho[cell_index(s, s->nx / 2, x % s->ny, s->nz / 2)];",
     "tests/test_oracle_init.py::test_thickness_counts_band_nodes_of_a_flat_slab"),
]


@pytest.mark.parametrize("name,old,new,pin", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_pin_catches_planted_mistake(tmp_path, name, old, new, pin):
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor for {name} not unique"
    mutated = tmp_path / "mutated.c"
    mutated.write_text(src.replace(old, new))
    lib = tmp_path / "libmutated.so"
    subprocess.run(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
                    "-o", str(lib), str(mutated), "-lm"], check=True)
    env = dict(os.environ, LBM_ORACLE_LIB=str(lib))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", pin],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"pin {pin} did not catch: {name}"
