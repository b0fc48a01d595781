"""Planted mistakes in the oracle, on the CPU: each plausible slip (dropped
term, wrong sign, wrong power, transposed operand, missing factor) compiled
into a mutant of md_oracle.c must make at least one physics pin fail.  This
shows that the pins constrain every part of the FP64 oracle."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "md_oracle.c")

# (name, exact text in md_oracle.c, replacement)
MUTANTS = [
    ("drop_softening", "double r2 = dx * dx + dy * dy + dz * dz + eps2;",
     "double r2 = dx * dx + dy * dy + dz * dz;"),
    ("field_sign", "double dx = xi - xs[3 * j];", "double dx = xs[3 * j] - xi;"),
    ("field_power", "double inv_r3 = 1.0 / (r2 * r);", "double inv_r3 = 1.0 / r2;"),
    ("field_index", "double dz = zi - xs[3 * j + 2];", "double dz = zi - xs[3 * j + 1];"),
    ("potential_power", "ph += qs[j] / r;", "ph += qs[j] / r2;"),
    ("kc_missing_2pi", "return 2.0 * OR_PI * OR_R_E / (lambda_um * 1.0e-6);",
     "return OR_R_E / (lambda_um * 1.0e-6);"),
    ("boris_half_missing", "double h = 0.5 * dt * qm;", "double h = dt * qm;"),
    ("boris_rotation_transposed",
     "double up[3] = {um[0] + (um[1] * tv[2] - um[2] * tv[1]),",
     "double up[3] = {um[0] + (um[2] * tv[1] - um[1] * tv[2]),"),
    ("boris_gamma_dropped", "double tv[3] = {h * b[0] / g, h * b[1] / g, h * b[2] / g};",
     "double tv[3] = {h * b[0], h * b[1], h * b[2]};"),
    ("boris_second_kick_dropped", "u[0] = pl[0] + h * e[0];", "u[0] = pl[0];"),
    ("drift_nonrelativistic", "x[0] += dt * u[0] / g;", "x[0] += dt * u[0];"),
    ("laser_by_phase", "b[1] = amp * sin(t);", "b[1] = amp * cos(t);"),
    ("laser_circular_phase", "double phi_e = 1.5 * OR_PI, phi_b = 0.5 * OR_PI;",
     "double phi_e = 0.5 * OR_PI, phi_b = 0.5 * OR_PI;"),
    ("envelope_gauss_constant", "return exp(-2.0 * log(2.0) * s * s);",
     "return exp(-4.0 * log(2.0) * s * s);"),
    ("sin2_envelope_power", "return s * s;\n    }\n    case OR_ENV_LITERAL_EQ3",
     "return s;\n    }\n    case OR_ENV_LITERAL_EQ3"),
    ("pe_double_count", "pe += 0.5 * q[i] * phi[i];", "pe += q[i] * phi[i];"),
    ("diag_no_half_step_mean", "double um[3] = {0.5 * (u[3 * i] + un[0]),",
     "double um[3] = {(un[0]),"),
    ("eq2_wrong_lambda_power",
     "return sqrt(intensity_wcm2 * lambda_um * lambda_um / 1.366e18);",
     "return sqrt(intensity_wcm2 * lambda_um / 1.366e18);"),
    ("eq1_wrong_power", "return q * q * q;", "return q * q;"),
    ("self_not_excluded", "if ((int64_t)j == self || qs[j] == 0.0) continue;",
     "if (qs[j] == 0.0) continue;"),
]


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_planted_mistake(name, old, new, tmp_path):
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor for {name} not unique"
    mut = tmp_path / "md_oracle_mutant.c"
    mut.write_text(src.replace(old, new))
    so = tmp_path / "libmut.so"
    subprocess.run(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
                    "-std=c11", "-o", str(so), str(mut), "-lm"], check=True)
    env = dict(os.environ, MD_ORACLE_LIB=str(so))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_pins.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"mutant {name} survived the pins:\n{r.stdout[-2000:]}"
