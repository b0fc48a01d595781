"""Clusters generated on the device (md_init_generate) against the oracle's
generator: the same records, positions bit for bit (rejection from the cube in
FP64, each operation rounded to nearest in the same order), Maxwellian momenta
to a few ulps (the device's log, sin and cos against the host's), and a
context built this way steps exactly like one uploaded from the same records,
with and without ionization."""
import numpy as np
import pytest

import oracle
from paper_1307_3711_gb300 import synth

pytestmark = pytest.mark.gpu

# |u_gpu - u_oracle| / |u_oracle| per component: Box-Muller through log, sqrt,
# sin and cos, each within a few ulps on either side
U_RTOL = 1e-14


@pytest.fixture(scope="module")
def md():
    from paper_1307_3711_gb300 import build
    build.build()
    from paper_1307_3711_gb300 import md as m
    return m


GENS = [
    # Xe3+ ions at rest with 10 eV electrons, off-centre
    dict(r0=synth.nm_to_len(3.0), n_ions=5003, n_electrons=15009, n_slots=0, ion_charge=3,
         ion_mass=synth.MASS_XE, weight=1.0, kt_e_ev=10.0, kt_i_ev=0.0, seed=42,
         center=(0.01, -0.02, 0.005)),
    # neutral Ar atoms with electron slots for ionization, macro weight 2.5
    dict(r0=synth.nm_to_len(2.0, 0.806), n_ions=1500, n_electrons=0, n_slots=12000,
         ion_charge=0, ion_mass=synth.MASS_AR, weight=2.5, kt_e_ev=0.0, kt_i_ev=0.0,
         seed=(7 << 32) + 3, center=(0.0, 0.0, 0.0)),
    # warm ions and electrons, a seed beyond 2^32
    dict(r0=0.05, n_ions=777, n_electrons=1554, n_slots=33, ion_charge=2, ion_mass=500.0,
         weight=1.0, kt_e_ev=200.0, kt_i_ev=50.0, seed=2 ** 40 + 11, center=(0.0, 0.0, 0.0)),
]


def _configs(md, ionize=False):
    cfgs = [md.make_config(a0=0.05, tau=300.0, dt=0.02, softening=synth.nm_to_len(0.1)),
            md.make_config(a0=0.0617, tau=300.0, t0=150.0, dt=0.02, lambda_um=0.806,
                           softening=synth.nm_to_len(0.1, 0.806),
                           rate_model=md.RATES_PLAIN if ionize else 0, ionize_every=1, zmax=8,
                           n_ions=1500, slot_base=1500, seed=5,
                           r_loc=3 * synth.nm_to_len(0.24, 0.806),
                           r_create=synth.nm_to_len(0.24, 0.806), species=synth.ARGON),
            md.make_config(a0=0.01, tau=300.0, dt=0.01, softening=0.002)]
    return cfgs


def test_generated_records_match_the_oracle(md):
    gens = [md.make_generate(**g) for g in GENS]
    with md.Context.generate(_configs(md), gens) as ctx:
        got = [ctx.get_particles(k) for k in range(len(GENS))]
    for g, p in zip(GENS, got):
        ref = oracle.generate_cluster(**g)
        np.testing.assert_array_equal(p.x, ref["x"])
        np.testing.assert_array_equal(p.z, ref["z"])
        np.testing.assert_array_equal(p.mass, ref["mass"])
        np.testing.assert_array_equal(p.w, ref["w"])
        np.testing.assert_array_equal(p.kind, ref["kind"])
        warm = ref["u"] != 0.0
        assert np.array_equal(p.u == 0.0, ~warm)
        if warm.any():
            rel = np.abs(p.u[warm] - ref["u"][warm]) / np.abs(ref["u"][warm])
            assert rel.max() <= U_RTOL, rel.max()


@pytest.mark.parametrize("ionize", [False, True])
def test_generated_context_steps_as_an_uploaded_one(md, ionize):
    """The generated context and an md_init context holding the records read
    back from it give the same bits after 6 steps (ionizing passes included
    for the argon cluster: the next free slot and the liveness flags of the
    generated context are those of an upload)."""
    gens = [md.make_generate(**g) for g in GENS]
    with md.Context.generate(_configs(md, ionize), gens) as ga:
        parts = [ga.get_particles(k) for k in range(len(GENS))]
        ga.step(6)
        after_gen = [ga.get_particles(k) for k in range(len(GENS))]
    with md.Context(_configs(md, ionize), parts) as ua:
        ua.step(6)
        after_up = [ua.get_particles(k) for k in range(len(GENS))]
    for a, b in zip(after_gen, after_up):
        np.testing.assert_array_equal(a.x, b.x)
        np.testing.assert_array_equal(a.u, b.u)
        np.testing.assert_array_equal(a.z, b.z)
        np.testing.assert_array_equal(a.kind, b.kind)
    if ionize:
        ar = after_gen[1]
        assert (ar.z[:1500] > 0).any()          # the pass ionized
        # charge conservation and the dense block of freed electrons
        assert float(np.sum(ar.w * ar.z)) == 0.0
        act = ar.kind[1500:] != md.KIND_INACTIVE
        assert act[:act.sum()].all()
