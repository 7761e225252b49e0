"""The oracle's pins catch plausible mistakes (CPU only).

Each case plants one mistake in a copy of the C oracle (a dropped term, a
wrong sign, a transposed operand or index, a wrong weight or factor),
compiles it, and runs the pins that should catch it in a subprocess that
loads the mutated library (LBPM_ORACLE_LIB). The case passes when at least
one of those pins fails. The pins named are closed forms, values the paper
prints, invariants, or the independent dense implementation on tiny inputs.
The NumPy oracles of shell aggregation and image preparation get the same
treatment: the subprocess puts a mutated copy of the module in place of the
original before the pins import it.

Left out on purpose, because they change nothing: relaxing a conserved
moment (rho, j), whose equilibrium equals the moment itself, and flipping
the direction of a shift over a symmetric ball of offsets.
"""
import os
import shutil
import subprocess
import sys

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(ROOT, "oracle", "lbpm_oracle.c")

PHYS = "tests/test_oracle_physics.py::"
OPS = "tests/test_oracle_ops.py::"
LAT = "tests/test_oracle_lattice.py::"
DYN = "tests/test_oracle_dynamics.py::"
MEAS = "tests/test_oracle_measures.py::"
PBC = "tests/test_oracle_pressure_bc.py::"
IDX = "tests/test_oracle_index.py::"
RES = "tests/test_oracle_reservoirs.py::"

# (name, text in the oracle, planted replacement, pins expected to catch it)
MUTANTS = [
    ("interfacial term of m9 dropped",
     "+ 0.5 * ac * (2.0 * nx * nx - ny * ny - nz * nz)", "",
     [PHYS + "test_flat_interface_normal_stress_balance"]),
    ("sign of the interfacial term of m1",
     "meq[1] = -11.0 * rho + 19.0 * jj - ac;", "meq[1] = -11.0 * rho + 19.0 * jj + ac;",
     [PHYS + "test_flat_interface_normal_stress_balance"]),
    ("sign of the interfacial term of m11",
     "+ 0.5 * ac * (ny * ny - nz * nz);", "+ 0.5 * ac * (nz * nz - ny * ny);",
     [PHYS + "test_flat_interface_normal_stress_balance"]),
    ("transposed normal in m13",
     "meq[13] = jx * jy / RHO0 + 0.5 * ac * nx * ny;", "meq[13] = jx * jy / RHO0 + 0.5 * ac * nx * nz;",
     [PHYS + "test_laplace_law_cylinders_other_planes"]),
    ("sign of m2's equilibrium",
     "meq[2] = 3.0 * rho - 5.5 * jj;", "meq[2] = 3.0 * rho + 5.5 * jj;",
     [OPS + "test_collision_fixed_point_at_equilibrium"]),
    ("edge weight of D3Q19",
     "for (int q = 7; q < Q19; ++q) T19[q] = 1.0 / 36.0;", "for (int q = 7; q < Q19; ++q) T19[q] = 1.0 / 30.0;",
     [LAT + "test_weights_match_paper"]),
    ("sign of one lattice velocity",
     "{1, 1, 0},   {-1, -1, 0},", "{1, 1, 0},   {-1, 1, 0},",
     [LAT + "test_velocity_groups_match_paper"]),
    ("forcing term without its factor 1/c_s^2",
     "fout[q] = f[q] + acc + 3.0 * T19[q] * xf;", "fout[q] = f[q] + acc + T19[q] * xf;",
     [OPS + "test_collision_conserves_mass_and_adds_force"]),
    ("relaxation rate of the odd moments",
     "8.0 * (2.0 - s_nu) / (8.0 - s_nu)", "(2.0 - s_nu)",
     [OPS + "test_collision_relaxes_toward_equilibrium_with_dhumieres_rates"]),
    ("sign of the recoloring term of B",
     "B[q] = W7[q] * Nb * (1.0 + 4.5 * ux - beta * fb * nx);", "B[q] = W7[q] * Nb * (1.0 + 4.5 * ux + beta * fb * nx);",
     [OPS + "test_recolor_beta_terms_cancel_in_total"]),
    ("velocity factor of the recoloring (D3Q19's 3 for D3Q7's 4.5)",
     "A[q] = W7[q] * Na * (1.0 + 4.5 * ux + beta * fa * nx);", "A[q] = W7[q] * Na * (1.0 + 3.0 * ux + beta * fa * nx);",
     [OPS + "test_recolor_beta_terms_cancel_in_total", PHYS + "test_flat_interface_tanh_profile"]),
    ("phase normalised by Na",
     "o->phi[n] = Nt > 0.0 ? (Na - Nb) / Nt : 0.0;", "o->phi[n] = Nt > 0.0 ? (Na - Nb) / Na : 0.0;",
     [OPS + "test_gradient_exact_on_polynomials"]),
    ("viscosity mixing with the phases swapped",
     "0.5 * (1.0 + o->phi[n]);", "0.5 * (1.0 - o->phi[n]);",
     [DYN + "test_brute_force_dense_random_state_anisotropic_box"]),
    ("bounce-back into the same direction",
     "else o->fn[n * Q19 + opposite(q)] = fpost[q];", "else o->fn[n * Q19 + q] = fpost[q];",
     [DYN + "test_rest_state_is_steady"]),
    ("component streamed into the opposite slot",
     "o->An[(long long)t * Q7 + q] = Apost[q];", "o->An[(long long)t * Q7 + opposite(q)] = Apost[q];",
     [DYN + "test_rest_state_is_steady"]),
    ("reported velocity without the half force",
     "u[a] = (j[a] + 0.5 * o->F[a]) / RHO0;", "u[a] = j[a] / RHO0;",
     [MEAS + "test_uniform_flow_of_pure_a"]),
    ("interfacial tension alpha instead of 6 alpha",
     "/ (6.0 * o->alpha);", "/ o->alpha;",
     [MEAS + "test_uniform_flow_of_pure_a"]),
    ("viscosities of the two fluids swapped",
     "const double mu_a = RHO0 * (o->tau_a - 0.5) / 3.0, mu_b = RHO0 * (o->tau_b - 0.5) / 3.0;",
     "const double mu_a = RHO0 * (o->tau_b - 0.5) / 3.0, mu_b = RHO0 * (o->tau_a - 0.5) / 3.0;",
     [MEAS + "test_two_phases_on_alternating_sites"]),
    ("phase volume fraction over the pore sites",
     "ca = ((cnt_a / V) * mu_a * ua + (cnt_b / V) * mu_b * ub)",
     "ca = ((cnt_a / (double)N) * mu_a * ua + (cnt_b / (double)N) * mu_b * ub)",
     [MEAS + "test_uniform_flow_of_pure_a"]),
    ("flux of A weighted by Nb/N",
     "qa[a] += xa * u[a];", "qa[a] += xb * u[a];",
     [MEAS + "test_uniform_mixture_splits_by_component_fraction"]),
    ("Darcy flux over the pore sites instead of the volume",
     "out[12 + a] = q[a] / V;", "out[12 + a] = q[a] / (double)N;",
     [MEAS + "test_uniform_flow_of_pure_a"]),
    ("reservoir slabs one layer thin",
     "if (z < RESERVOIR_DEPTH) side = 1;", "if (z < RESERVOIR_DEPTH - 1) side = 1;",
     [RES + "test_slab_sites_hold_the_reset_state_after_every_step"]),
    ("inlet slab filled with B as well",
     "B[n * Q7 + q] = side == 1 ? 0.0 : W7[q];", "B[n * Q7 + q] = W7[q];",
     [RES + "test_slab_sites_hold_the_reset_state_after_every_step"]),
    ("outlet density in both slabs",
     "const double rho = side == 1 ? o->rho_in : o->rho_out;", "const double rho = o->rho_out;",
     [RES + "test_slab_sites_hold_the_reset_state_after_every_step"]),
    ("inlet slab one layer thin, seen in the steady state",
     "if (z < RESERVOIR_DEPTH) side = 1;", "if (z < RESERVOIR_DEPTH - 1) side = 1;",
     [RES + "test_equal_reservoirs_reach_rest_and_a_linear_component_profile"]),
    ("inlet slab filled with B as well, seen in the steady state",
     "B[n * Q7 + q] = side == 1 ? 0.0 : W7[q];", "B[n * Q7 + q] = W7[q];",
     [RES + "test_equal_reservoirs_reach_rest_and_a_linear_component_profile"]),
    ("outlet slab filled with A as well",
     "A[n * Q7 + q] = side == 1 ? W7[q] : 0.0;", "A[n * Q7 + q] = W7[q];",
     [RES + "test_equal_reservoirs_reach_rest_and_a_linear_component_profile"]),
    ("initial phases of A and B swapped",
     "const double Na = 0.5 * (1.0 + p), Nb = 0.5 * (1.0 - p);",
     "const double Na = 0.5 * (1.0 - p), Nb = 0.5 * (1.0 + p);",
     [RES + "test_injection_raises_saturation_and_advances_the_front"]),
    ("periodic flag of x applied to every axis",
     "if (!o->periodic[a]) return 0;", "if (!o->periodic[0]) return 0;",
     [IDX + "test_index_matches_brute_force"]),
    ("neighbour table laid out site-major",
     "o->nbr[(long long)(q - 1) * N + s] = t;", "o->nbr[(long long)s * 18 + (q - 1)] = t;",
     [IDX + "test_index_matches_brute_force"]),
    ("affinity of solid voxels lost",
     "o->phis[v] = affinity ? (double)affinity[v] : 0.0;", "o->phis[v] = 0.0;",
     [OPS + "test_gradient_sees_affinity_of_solid_neighbour"]),
    ("Zou-He normal and edge weights swapped",
     "(tang ? 1.0 / 6.0 : 1.0 / 3.0)", "(tang ? 1.0 / 3.0 : 1.0 / 6.0)",
     [PBC + "test_face_sites_hold_the_face_density_and_no_tangential_momentum"]),
    ("sign of the tangential-momentum correction",
     "- XI[q][0] * Nt[0] - XI[q][1] * Nt[1];", "+ XI[q][0] * Nt[0] + XI[q][1] * Nt[1];",
     [PBC + "test_face_sites_hold_the_face_density_and_no_tangential_momentum"]),
    ("tangential momentum without its 1/2",
     "Nt[0] *= 0.5;\n        Nt[1] *= 0.5;", "",
     [PBC + "test_face_sites_hold_the_face_density_and_no_tangential_momentum"]),
    ("face velocity with the leaving populations once",
     "const double un = 1.0 - (s0 + 2.0 * sout) / rho;", "const double un = 1.0 - (s0 + sout) / rho;",
     [PBC + "test_face_sites_hold_the_face_density_and_no_tangential_momentum"]),
    ("entering component population with the face velocity's sign flipped",
     "const double eq = W7[qin] * rho * (1.0 + 4.5 * XI[qin][2] * uz);",
     "const double eq = W7[qin] * rho * (1.0 - 4.5 * XI[qin][2] * uz);",
     [PBC + "test_entering_component_population_keeps_the_face_density"]),
    ("entering component population at density 1 instead of the face density",
     "const double eq = W7[qin] * rho * (1.0 + 4.5 * XI[qin][2] * uz);",
     "const double eq = W7[qin] * (1.0 + 4.5 * XI[qin][2] * uz);",
     [PBC + "test_entering_component_population_keeps_the_face_density"]),
    ("flux inlet density with n_in + Q",
     "rho_in = K / ((double)n_in - o->flux_in);", "rho_in = K / ((double)n_in + o->flux_in);",
     [PBC + "test_flux_inlet_carries_exactly_the_prescribed_flux"]),
    ("flux inlet sum with the leaving populations once",
     "else if (XI[q][2] < 0) K += 2.0 * g[q];", "else if (XI[q][2] < 0) K += g[q];",
     [PBC + "test_flux_inlet_carries_exactly_the_prescribed_flux"]),
    ("instability flagged at any negative component density",
     "if (Na < -1e-2 || Nb < -1e-2 || Nt <= 0.0 || rho <= 0.0) status |= 2;",
     "if (Na < 0.0 || Nb < 0.0 || Nt <= 0.0 || rho <= 0.0) status |= 2;",
     [MEAS + "test_instability_flags"]),
]


@pytest.fixture(scope="module")
def source():
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    with open(SRC) as fh:
        return fh.read()


@pytest.mark.parametrize("name,old,new,pins", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_fails_a_pin(source, tmp_path, name, old, new, pins):
    assert source.count(old) == 1, f"the text to mutate is not unique: {old!r}"
    c = tmp_path / "mutant.c"
    so = tmp_path / "libmutant.so"
    c.write_text(source.replace(old, new))
    r = subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", str(c), "-o", str(so), "-lm"],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    env = dict(os.environ, LBPM_ORACLE_LIB=str(so))
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider", "-m", "not gpu",
                        *pins], capture_output=True, text=True, cwd=ROOT, env=env)
    # exit code 1: tests ran and at least one failed; 0 would mean the pins
    # missed the mistake, anything else that they did not run
    assert r.returncode == 1, f"{name}: pins {pins} did not catch it\n{r.stdout[-2000:]}"


# (module, name, text, planted replacement, pins expected to catch it)
PY_MUTANTS = [
    ("morph", "sign of the shift delta",
     "-np.tanh(beta * (Phi - delta))", "-np.tanh(beta * (Phi + delta))",
     "tests/test_oracle_morph.py::test_one_voxel_of_dilation_adds_one_plane"),
    ("morph", "distance scaled by beta instead of 1/beta",
     "np.abs(np.arctanh(phi[band])) / beta", "np.abs(np.arctanh(phi[band])) * beta",
     "tests/test_oracle_morph.py::test_flat_equilibrium_interface_moves_by_delta"),
    ("morph", "far field by squared distance",
     "np.sqrt(o[0] ** 2 + o[1] ** 2 + o[2] ** 2) +", "(o[0] ** 2 + o[1] ** 2 + o[2] ** 2) +",
     "tests/test_oracle_morph.py::test_flat_equilibrium_interface_moves_by_delta"),
    ("morph", "sign of the far-field distance",
     "np.where(phi > 0, -best, best)", "np.where(phi > 0, best, -best)",
     "tests/test_oracle_morph.py::test_relaxed_drop_grows_by_a_shell"),
    ("morph", "band of the exact distance too narrow",
     "np.tanh(3.0 * beta)", "np.tanh(1.0 * beta)",
     "tests/test_oracle_morph.py::test_relaxed_drop_grows_by_a_shell"),
    ("morph", "re-initialised densities swapped",
     "na, nb = 0.5 * N * (1 + phin), 0.5 * N * (1 - phin)", "na, nb = 0.5 * N * (1 - phin), 0.5 * N * (1 + phin)",
     "tests/test_oracle_morph.py::test_flat_equilibrium_interface_moves_by_delta"),
    ("morph", "site density not kept",
     "na, nb = 0.5 * N * (1 + phin), 0.5 * N * (1 - phin)", "na, nb = 0.5 * (1 + phin), 0.5 * (1 - phin)",
     "tests/test_oracle_morph.py::test_flat_equilibrium_interface_moves_by_delta"),
    ("prepare", "open ball (distance < radius)",
     "x * x + y * y + z * z <= radius * radius", "x * x + y * y + z * z < radius * radius",
     "tests/test_oracle_prepare.py::test_ball_sizes_are_lattice_point_counts"),
    ("prepare", "inlet layers tested against the inlet face",
     "new = np.where((layer != 0) & (outlet_face == 0), 0, new)",
     "new = np.where((layer != 0) & (inlet_face == 0), 0, new)",
     "tests/test_oracle_prepare.py::test_mixing_layer_by_hand"),
    ("prepare", "one outlet layer too few",
     "if a >= L - n_mix:", "if a > L - n_mix:",
     "tests/test_oracle_prepare.py::test_mixing_layer_by_hand"),
    ("prepare", "pore voxels relabelled too",
     "out[(lab != 0) & near] = new_label", "out[near] = new_label",
     "tests/test_oracle_prepare.py::test_relabel_matches_scipy_distance_transform"),
]

_BOOT = """
import sys, types
sys.path.insert(0, {root!r})
import oracle
src = open({path!r}).read()
mod = types.ModuleType("oracle.{name}")
mod.__file__ = {path!r}
mod.__package__ = "oracle"
exec(compile(src, {path!r}, "exec"), mod.__dict__)
sys.modules["oracle.{name}"] = mod
setattr(oracle, "{name}", mod)
import pytest
sys.exit(pytest.main(["-q", "-x", "-p", "no:cacheprovider", {pins!r}]))
"""


@pytest.mark.parametrize("module,name,old,new,pins", PY_MUTANTS, ids=[m[1] for m in PY_MUTANTS])
def test_planted_mistake_in_a_numpy_oracle_fails_a_pin(tmp_path, module, name, old, new, pins):
    with open(os.path.join(ROOT, "oracle", f"{module}.py")) as fh:
        src = fh.read()
    assert src.count(old) == 1, f"the text to mutate is not unique: {old!r}"
    path = tmp_path / f"{module}.py"
    path.write_text(src.replace(old, new))
    boot = _BOOT.format(root=ROOT, path=str(path), name=module, pins=pins)
    r = subprocess.run([sys.executable, "-c", boot], capture_output=True, text=True, cwd=ROOT)
    assert r.returncode == 1, f"{name}: {pins} did not catch it\n{r.stdout[-2000:]}"
