"""Planted mistakes in the oracle, on the CPU: each plausible slip (dropped
term, wrong sign, wrong power, transposed operand, missing factor), compiled
into a mutant of the oracle's C sources or re-executed in its Python layer,
must make at least one pin fail.  The mutants run side by side, each in its
own process and directory.  Not constrained: the l* and Gamma terms of the
ADK prefactor away from n* = 1, where no independent value is at hand."""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ORACLE = os.path.join(ROOT, "oracle")
SOURCES = ["md_oracle.c", "ionize_oracle.c", "mlp_oracle.c", "generate_oracle.c"]

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
    ("min_image_floor", "d[k] -= box * nearbyint(d[k] / box);", "d[k] -= box * floor(d[k] / box);"),
    ("min_image_two_axes", "for (int k = 0; k < 3; ++k) d[k] -= box",
     "for (int k = 0; k < 2; ++k) d[k] -= box"),
    ("min_image_not_in_steps", "if (p->min_image && periodic)", "if (p->min_image && !periodic)"),
    ("min_image_softening", "double rm2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2] + eps2;",
     "double rm2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];"),
    ("wrap_box_not_centred", "x[k] = x[k] - box * floor((x[k] + h) / box);",
     "x[k] = x[k] - box * floor(x[k] / box);"),
    ("mixed_switch_inverted", "if (mode == 2 && t >= t_switch) return;",
     "if (mode == 2 && t < t_switch) return;"),
    ("mixed_switch_at_step_start",
     "or_boundary(&x[3 * i], p->boundary, p->box, t + p->dt, p->t_switch);",
     "or_boundary(&x[3 * i], p->boundary, p->box, t, p->t_switch);"),
    ("diag_time_without_t0",
     "double t = p->t0 + (double)step * p->dt;\n    double a[3], b[3];\n    for",
     "double t = (double)step * p->dt;\n    double a[3], b[3];\n    for"),
    ("ke_neutral_atoms_as_electrons", "if (z[i] < 0) kee += k; else kei += k;",
     "if (z[i] <= 0) kee += k; else kei += k;"),
    ("inactive_records_pushed", "            if (!active[i]) continue;\n            double et",
     "            double et"),
    ("wrap_half_box", "double h = 0.5 * box;", "double h = 0.5 / box;"),
]

# (name, file, exact text, replacement, pin file) for the ionization and
# surrogate oracles
MUTANTS_OTHER = [
    ("philox_multiplier", "ionize_oracle.c", "uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;",
     "uint64_t p1 = (uint64_t)0xCD9E8D55u * c2;", "test_oracle_ionize.py"),
    ("philox_key_bump", "ionize_oracle.c", "k1 += 0xBB67AE85u;", "k1 += 0xBB67AE86u;",
     "test_oracle_ionize.py"),
    ("philox_word_order", "ionize_oracle.c", "uint32_t n2 = hi0 ^ c3 ^ k1;",
     "uint32_t n2 = hi0 ^ c1 ^ k1;", "test_oracle_ionize.py"),
    ("alpha_closed_at_zero", "ionize_oracle.c", "return ((double)w + 1.0) * (1.0 / 4294967296.0);",
     "return ((double)w) * (1.0 / 4294967296.0);", "test_oracle_ionize.py"),
    ("e1_series_sign", "ionize_oracle.c", "return -IO_EULER_GAMMA - log(x) + sum;",
     "return -IO_EULER_GAMMA - log(x) - sum;", "test_oracle_ionize.py"),
    ("adk_field_scale", "ionize_oracle.c",
     "return c2 * ip * pow(2.0 * F0 / F, 2.0 * ns - 1.0)",
     "return c2 * ip * pow(2.0 / F0 / F, 2.0 * ns - 1.0)", "test_oracle_ionize.py"),
    ("adk_exponent", "ionize_oracle.c",
     "return c2 * ip * pow(2.0 * F0 / F, 2.0 * ns - 1.0) * exp(-2.0 * F0 / (3.0 * F));",
     "return c2 * ip * pow(2.0 * F0 / F, 2.0 * ns) * exp(-2.0 * F0 / (3.0 * F));",
     "test_oracle_ionize.py"),
    ("lotz_sqrt_t", "ionize_oracle.c",
     "return v_th * IO_LOTZ_A * q * io_e1(P / T) / (P * sqrt(T));",
     "return v_th * IO_LOTZ_A * q * io_e1(P / T) / (P * T);", "test_oracle_ionize.py"),
    ("moments_no_mean_frame", "ionize_oracle.c",
     "double var = su2 / sw - (mx * mx + my * my + mz * mz);", "double var = su2 / sw;",
     "test_oracle_ionize.py"),
    ("rate_residual_charge", "ionize_oracle.c",
     "double w_ofi = io_adk_rate_au(F, ip, (double)(z + 1)) / IO_TIME_AU;",
     "double w_ofi = io_adk_rate_au(F, ip, (double)z) / IO_TIME_AU;", "test_oracle_ionize.py"),
    ("rate_lotz_wrong_shell", "ionize_oracle.c",
     "io_lotz_rate_cgs(ip_ev[z], te, q_outer[z])", "io_lotz_rate_cgs(ip_ev[z], te, q_outer[0])",
     "test_oracle_ionize.py"),
    ("moments_min_image_dropped", "ionize_oracle.c",
     "if (box > 0.0) d[c] -= box * nearbyint(d[c] / box);", "", "test_oracle_ionize.py"),
    ("decision_le", "ionize_oracle.c", "if (alpha < P) {", "if (alpha > P) {",
     "test_oracle_ionize.py"),
    ("moments_count_neutral_atoms", "ionize_oracle.c",
     "if (!active_s[j] || zs[j] >= 0) continue;\n            double dx",
     "if (!active_s[j] || zs[j] > 0) continue;\n            double dx", "test_oracle_ionize.py"),
    ("counter_step_high_word", "ionize_oracle.c",
     "uint32_t ctr[4] = {(uint32_t)id[i], (uint32_t)step, (uint32_t)((uint64_t)step >> 32), 0u};",
     "uint32_t ctr[4] = {(uint32_t)id[i], (uint32_t)step, 0u, 0u};", "test_oracle_ionize.py"),
    ("key_seed_high_word", "ionize_oracle.c",
     "uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};",
     "uint32_t key[2] = {(uint32_t)seed, 0u};", "test_oracle_ionize.py"),
    ("probability_first_order", "ionize_oracle.c", "double P = -expm1(-nu * dt_ion);",
     "double P = nu * dt_ion;", "test_oracle_ionize.py"),
    ("placement_radius", "ionize_oracle.c", "double ph = 2.0 * IO_PI * u2, r = r_create * cbrt(u3);",
     "double ph = 2.0 * IO_PI * u2, r = r_create * u3;", "test_oracle_ionize.py"),
    ("mlp_dsilu", "mlp_oracle.c", "return s * (1.0 + a * (1.0 - s));", "return s * (1.0 + a * s);",
     "test_oracle_mlp.py"),
    ("mlp_grad_w2_index", "mlp_oracle.c", "grad[OFF_W2 + j * NH + k] += da2[j] * h1[k];",
     "grad[OFF_W2 + k * NH + j] += da2[j] * h1[k];", "test_oracle_mlp.py"),
    ("mlp_loss_scale", "mlp_oracle.c", "dy[zs] = 2.0 * r / n;", "dy[zs] = r / n;",
     "test_oracle_mlp.py"),
    ("mlp_temperature_scale", "mlp_oracle.c",
     "f[3] = (log10(fmax(te, 0.1) / ip_ev) + 0.2) / 3.0;",
     "f[3] = (log10(fmax(te, 0.1) / ip_ev) + 0.2) / 2.0;", "test_oracle_mlp.py"),
    ("detector_no_cone", "md_oracle.c", "if (b0 >= c) hist[0 * (nbins + 1) + bin] += 1;",
     "if (b0 >= 0.0) hist[0 * (nbins + 1) + bin] += 1;", "test_oracle_detectors.py"),
    ("detector_inward", "md_oracle.c", "if (!(rp2 < R2 && rn2 >= R2)) continue;",
     "if (!(rp2 >= R2 && rn2 < R2)) continue;", "test_oracle_detectors.py"),
    ("detector_gamma_not_minus_one", "md_oracle.c",
     "return (uu / (sqrt(1.0 + uu) + 1.0)) * mass * OR_ME_C2_EV;",
     "return sqrt(1.0 + uu) * mass * OR_ME_C2_EV;", "test_oracle_detectors.py"),
    ("detector_no_once", "md_oracle.c", "        crossed[i] = 1;\n", "\n",
     "test_oracle_detectors.py"),
    ("detector_bin_width", "md_oracle.c", "int b = (int)floor(ke * (double)nbins / e_max);",
     "int b = (int)floor(ke * (double)(nbins - 1) / e_max);", "test_oracle_detectors.py"),
    ("detector_centre_sign", "md_oracle.c", "double a0 = x_prev[3 * i] - center[0]",
     "double a0 = x_prev[3 * i] + center[0]", "test_oracle_detectors.py"),
    ("detector_radius_sign", "md_oracle.c", "double rp2 = (a0 * a0 + a1 * a1) + a2 * a2;",
     "double rp2 = (a0 * a0 - a1 * a1) + a2 * a2;", "test_oracle_detectors.py"),
    ("detector_row_offset", "md_oracle.c", "if (-b0 >= c) hist[1 * (nbins + 1) + bin] += 1;",
     "if (-b0 >= c) hist[1 * (nbins - 1) + bin] += 1;", "test_oracle_detectors.py"),
    ("gen_cube_not_centred", "generate_oracle.c",
     "c[k] = ((double)w[k] + 0.5) * (1.0 / 2147483648.0) - 1.0;",
     "c[k] = ((double)w[k] + 0.5) * (1.0 / 4294967296.0);", "test_oracle_generate.py"),
    ("gen_no_rejection", "generate_oracle.c", "if (r2 < 1.0) {", "if (r2 < 3.0) {",
     "test_oracle_generate.py"),
    ("gen_radius_misses_an_axis", "generate_oracle.c", "r2 = r2 + c[2] * c[2];",
     "r2 = r2 + c[1] * c[1];", "test_oracle_generate.py"),
    ("gen_attempts_share_a_counter", "generate_oracle.c",
     "(uint32_t)((uint64_t)rec >> 32), a, GO_TAG_POSITION};",
     "(uint32_t)((uint64_t)rec >> 32), 0u, GO_TAG_POSITION};", "test_oracle_generate.py"),
    ("gen_position_unscaled", "generate_oracle.c", "x[3 * i + c] = center[c] + r0 * s[c];",
     "x[3 * i + c] = center[c] + s[c];", "test_oracle_generate.py"),
    ("gen_sigma_without_sqrt", "generate_oracle.c",
     "sqrt(kt_e_ev / (1.0 * GO_ME_C2_EV))", "(kt_e_ev / (1.0 * GO_ME_C2_EV))",
     "test_oracle_generate.py"),
    ("gen_sigma_without_ion_mass", "generate_oracle.c",
     "sqrt(kt_i_ev / (ion_mass * GO_ME_C2_EV))", "sqrt(kt_i_ev / GO_ME_C2_EV)",
     "test_oracle_generate.py"),
    ("gen_box_muller_cos_twice", "generate_oracle.c", "n[1] = rho * sin(2.0 * GO_PI * v1);",
     "n[1] = rho * cos(2.0 * GO_PI * v1);", "test_oracle_generate.py"),
    ("gen_box_muller_radius", "generate_oracle.c", "double rho = sqrt(-2.0 * log(v0));",
     "double rho = sqrt(-log(v0));", "test_oracle_generate.py"),
    ("gen_momentum_draws_reuse_positions", "generate_oracle.c",
     "(uint32_t)((uint64_t)rec >> 32), 0u, GO_TAG_MOMENTUM};",
     "(uint32_t)((uint64_t)rec >> 32), 0u, GO_TAG_POSITION};", "test_oracle_generate.py"),
    ("gen_electron_charge_sign", "generate_oracle.c",
     "z[i] = k == 0 ? ion_charge : (k == 1 ? -1 : 0);",
     "z[i] = k == 0 ? ion_charge : (k == 1 ? 1 : 0);", "test_oracle_generate.py"),
    ("gen_slots_not_at_rest", "generate_oracle.c",
     "const double sig = k == 0 ? sig_i : (k == 1 ? sig_e : 0.0);",
     "const double sig = k == 0 ? sig_i : sig_e;", "test_oracle_generate.py"),
    ("gen_seed_high_word", "generate_oracle.c",
     "uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};\n    for",
     "uint32_t key[2] = {(uint32_t)seed, 0u};\n    for", "test_oracle_generate.py"),
    ("iedf_inside_wrong_record", "md_oracle.c",
     "hist[or_energy_bin(or_ke_ev(&u[3 * i], mass[i]), e_max_ev, nbins)] += 1;",
     "hist[or_energy_bin(or_ke_ev(&u[3 / (i + 1)], mass[i]), e_max_ev, nbins)] += 1;",
     "test_oracle_detectors.py"),
]


def _run_mutant(tmp_path, fname, old, new, pin_file):
    sources = {f: open(os.path.join(ORACLE, f)).read() for f in SOURCES}
    assert sources[fname].count(old) == 1, f"mutation anchor not unique in {fname}: {old}"
    sources[fname] = sources[fname].replace(old, new)
    paths = []
    for f, txt in sources.items():
        pth = tmp_path / f
        pth.write_text(txt)
        paths.append(str(pth))
    so = tmp_path / "libmut.so"
    subprocess.run(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
                    "-std=c11", "-o", str(so)] + paths + ["-lm"], check=True)
    env = dict(os.environ, MD_ORACLE_LIB=str(so))
    return subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                           os.path.join(ROOT, "tests", pin_file)],
                          cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)


# (name, exact text in oracle/__init__.py, replacement, pin file): slips in the
# oracle's Python layer, which forms each macro's charge and charge-to-mass
# ratio from its weight (Eq. 1) before calling the C code, and which adds the
# laser field to the Coulomb field and places the freed electrons in a pass
MUTANTS_PY = [
    ("macro_charge_unweighted", "np.where(self.active > 0, self.w * self.z, 0.0)",
     "np.where(self.active > 0, 1.0 * self.z, 0.0)", "test_oracle_pins.py"),
    ("charge_to_mass_of_the_macro", "return (self.z / self.mass)",
     "return (self.w * self.z / self.mass)", "test_oracle_pins.py"),
    ("kinetic_energy_unweighted", "wm = (state.w * state.mass)", "wm = (state.mass)",
     "test_oracle_pins.py"),
    ("pass_field_laser_dropped", "amag = np.linalg.norm(e + a[None, :], axis=1)",
     "amag = np.linalg.norm(e, axis=1)", "test_oracle_ionize.py"),
    ("pass_field_laser_subtracted", "amag = np.linalg.norm(e + a[None, :], axis=1)",
     "amag = np.linalg.norm(e - a[None, :], axis=1)", "test_oracle_ionize.py"),
    ("pass_time_without_t0", "t = params.t0 + state.step * params.dt",
     "t = state.step * params.dt", "test_oracle_ionize.py"),
    ("freed_electron_unit_weight", "state.w[slot] = state.w[i]", "state.w[slot] = 1.0",
     "test_oracle_ionize.py"),
    ("freed_electron_ion_mass", "state.mass[slot] = 1.0", "state.mass[slot] = state.mass[i]",
     "test_oracle_ionize.py"),
    ("pass_moments_not_at_the_ions",
     "ne, te = local_moments(state.x[:n_ion], state, r_loc, lambda_um, box=box)",
     "ne, te = local_moments(state.x[:n_ion] * 0.0, state, r_loc, lambda_um, box=box)",
     "test_oracle_ionize.py"),
    ("box_moments_fixed_wavelength",
     "_ptr(state.active), float(r_loc), float(lambda_um), float(box),",
     "_ptr(state.active), float(r_loc), 0.8, float(box),", "test_oracle_ionize.py"),
]

_PY_RUNNER = """
import sys
sys.path.insert(0, {root!r})
import pytest
import oracle
src = open(oracle.__file__).read()
assert src.count({old!r}) == 1, "mutation anchor not unique"
exec(compile(src.replace({old!r}, {new!r}), oracle.__file__, "exec"), oracle.__dict__)
sys.exit(pytest.main(["-x", "-q", "-p", "no:cacheprovider", {pins!r}]))
"""




def _run_py_mutant(tmp_path, old, new, pin_file):
    runner = tmp_path / "run_mutant.py"
    runner.write_text(_PY_RUNNER.format(root=ROOT, old=old, new=new,
                                        pins=os.path.join(ROOT, "tests", pin_file)))
    return subprocess.run([sys.executable, str(runner)], cwd=ROOT, capture_output=True,
                          text=True, timeout=600)


# every mutant by name: (runner, file, anchor, replacement, pin file)
ALL = {}
for _n, _old, _new in MUTANTS:
    ALL[_n] = ("c", "md_oracle.c", _old, _new, "test_oracle_pins.py")
for _n, _f, _old, _new, _pins in MUTANTS_OTHER:
    ALL[_n] = ("c", _f, _old, _new, _pins)
for _n, _old, _new, _pins in MUTANTS_PY:
    ALL[_n] = ("py", None, _old, _new, _pins)
ALL["control_no_mistake"] = ("py", None, MUTANTS_PY[0][1], MUTANTS_PY[0][1],
                             "test_oracle_pins.py")
assert len(ALL) == len(MUTANTS) + len(MUTANTS_OTHER) + len(MUTANTS_PY) + 1, "names collide"


@pytest.fixture(scope="module")
def mutant_runs(request, tmp_path_factory):
    """Runs the selected mutants' pin files side by side (each in its own
    process and directory) and returns {name: CompletedProcess or exception}."""
    wanted = [it.callspec.params["name"] for it in request.session.items
              if getattr(it, "module", None) is not None and it.module.__file__ == __file__
              and hasattr(it, "callspec") and "name" in it.callspec.params]

    # the directories are made here, one by one: mktemp is not thread-safe
    dirs = {name: tmp_path_factory.mktemp(name) for name in wanted}

    def one(name):
        kind, fname, old, new, pins = ALL[name]
        d = dirs[name]
        try:
            if kind == "c":
                return name, _run_mutant(d, fname, old, new, pins)
            return name, _run_py_mutant(d, old, new, pins)
        except Exception as exc:  # reported by the mutant's own test
            return name, exc

    with ThreadPoolExecutor(max_workers=max(2, (os.cpu_count() or 2) // 2)) as ex:
        return dict(ex.map(one, wanted))


def _result(runs, name):
    r = runs[name]
    if isinstance(r, Exception):
        raise r
    return r


@pytest.mark.parametrize("name", [m[0] for m in MUTANTS])
def test_pins_catch_planted_mistake(name, mutant_runs):
    r = _result(mutant_runs, name)
    assert r.returncode != 0, f"mutant {name} survived the pins:\n{r.stdout[-2000:]}"


@pytest.mark.parametrize("name", [m[0] for m in MUTANTS_OTHER])
def test_ionization_and_surrogate_pins_catch_planted_mistake(name, mutant_runs):
    r = _result(mutant_runs, name)
    assert r.returncode != 0, f"mutant {name} survived the pins:\n{r.stdout[-2000:]}"


@pytest.mark.parametrize("name", [m[0] for m in MUTANTS_PY])
def test_pins_catch_planted_mistake_in_python_layer(name, mutant_runs):
    r = _result(mutant_runs, name)
    assert r.returncode not in (0, 5), f"mutant {name} survived the pins:\n{r.stdout[-2000:]}"
    assert "AssertionError" in r.stdout or "assert" in r.stdout, r.stdout[-2000:]


@pytest.mark.parametrize("name", ["control_no_mistake"])
def test_python_layer_runner_passes_without_a_mistake(name, mutant_runs):
    """Control: the same runner with the anchor left as it is passes every pin,
    so a caught mutant fails because of its slip alone."""
    r = _result(mutant_runs, name)
    assert r.returncode == 0, r.stdout[-2000:]
