"""The oracle's pins catch plausible mistakes (CPU only).

Each case plants one mistake in a copy of the C oracle (a dropped term, a
wrong sign, a transposed operand or index, a wrong weight or factor),
compiles it, and runs the pins that should catch it in a subprocess that
loads the mutated library (LBPM_ORACLE_LIB). The case passes when at least
one of those pins fails. The pins named are closed forms, values the paper
prints, invariants, or the independent dense implementation on tiny inputs.

Left out on purpose: relaxing a conserved moment (rho, j) is not a mistake
that changes anything, since its equilibrium equals the moment itself.
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
