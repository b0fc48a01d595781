"""Ion energy detectors on the GPU (Sec. III, Fig. 3 diagnostic) against the
oracle's detectors applied to the GPU's own states, step by step (exact
counts), and the Coulomb explosion of a uniform ion sphere seen at 9 R0."""
import math

import numpy as np
import pytest

import oracle
from paper_1307_3711_gb300 import synth

pytestmark = pytest.mark.gpu
KC = oracle.coulomb_constant(0.8)
ME_C2_EV = 510998.95


@pytest.fixture(scope="module")
def md():
    from paper_1307_3711_gb300 import build
    build.build()
    from paper_1307_3711_gb300 import md as m
    return m


def explosion(md, n, seed=5, r0_nm=2.0, eps_nm=0.005):
    r0 = synth.nm_to_len(r0_nm)
    c = synth.make_cluster(seed, n, 0, r0, 1, synth.MASS_40AMU)
    q = c.w * c.z
    tau = math.sqrt(synth.MASS_40AMU * r0 ** 3 / (KC * q.sum()))
    e_max = KC * q.sum() / r0
    cfg = md.make_config(a0=0.0, dt=tau / 40, softening=synth.nm_to_len(eps_nm),
                         envelope=synth.ENV_FLAT)
    return c, r0, e_max, cfg


def state_of(g):
    return oracle.State(g.x, g.u, g.z, g.mass, g.w, (g.kind != 2).astype(np.uint8))


@pytest.mark.parametrize("offset", [(0.0, 0.0, 0.0), (0.3, -0.2, 0.1)])
def test_detector_counts_match_oracle_on_gpu_states(md, offset):
    """Exact counts against the oracle's detectors on the GPU's states, with
    the detector sphere centred on the cluster and off it (centre offset in
    units of R0)."""
    n = 600
    c, r0, e_max, cfg = explosion(md, n)
    nb = 64
    e_max_ev = 0.4 * e_max * ME_C2_EV   # at 2.5 R0 energies reach 0.6 E_max: some overflow
    center = tuple(r0 * v for v in offset)
    det = oracle.Detectors(n, radius=2.5 * r0, cone_deg=30.0, e_max_ev=e_max_ev, nbins=nb,
                           center=center)
    with md.Context([cfg], [md.HostParticles.from_cluster(c)]) as ctx:
        ctx.set_detectors(0, 2.5 * r0, cone_deg=30.0, e_max_ev=e_max_ev, n_bins=nb,
                          center=center)
        g0 = ctx.get_particles(0)
        for _ in range(200):
            ctx.step(1)
            g1 = ctx.get_particles(0)
            det.record(g0.x, g1.x, state_of(g1))
            g0 = g1
        got, inside = ctx.iedf(0)
    assert det.hist[4].sum() > 0.5 * n
    assert det.hist[4][nb] > 0 and all(det.hist[k].sum() > 0 for k in range(4))
    np.testing.assert_array_equal(got, det.hist)
    np.testing.assert_array_equal(inside, det.inside(state_of(g0)))


def test_explosion_seen_at_nine_radii_on_gpu(md):
    """As the oracle pin: the recorded mean energy is that of ions keeping
    their initially enclosed charge, E_i/E_max = (n_below_i/N)(R0/r0_i - 1/9),
    and each 30-degree cone sees (1 - cos 30)/2 of the ions."""
    n = 1200
    c, r0, e_max, cfg = explosion(md, n)
    nb = 400
    s0 = np.linalg.norm(c.x, axis=1) / r0
    with md.Context([cfg], [md.HostParticles.from_cluster(c)]) as ctx:
        ctx.set_detectors(0, 9 * r0, cone_deg=30.0, e_max_ev=e_max * ME_C2_EV, n_bins=nb)
        ctx.step(480)
        got, inside = ctx.iedf(0)
    n_hit = int(got[4].sum())
    assert n_hit > 0.5 * n and n_hit + int(inside.sum()) == n
    assert got[4][nb] == 0
    centers = (np.arange(nb) + 0.5) / nb
    mean_rec = (got[4][:nb] * centers).sum() / n_hit
    n_below = np.argsort(np.argsort(s0))
    pred = (n_below / n) * (1.0 / s0 - 1.0 / 9.0)
    # the recorded ions are the outer ones: compare with the n_hit largest r0
    outer = np.argsort(s0)[-n_hit:]
    assert mean_rec == pytest.approx(pred[outer].mean(), abs=0.006)
    frac = (1 - math.cos(math.radians(30))) / 2
    for k in range(4):
        assert abs(int(got[k].sum()) - frac * n_hit) < 4 * math.sqrt(frac * n_hit)


def test_detector_arguments_and_state(md):
    n = 100
    c, r0, e_max, cfg = explosion(md, n)
    with md.Context([cfg], [md.HostParticles.from_cluster(c)]) as ctx:
        with pytest.raises(md.MDError):
            ctx.iedf(0)
        for bad in (dict(radius=-1.0), dict(radius=1.0, cone_deg=120.0),
                    dict(radius=1.0, n_bins=0), dict(radius=1.0, e_max_ev=0.0)):
            with pytest.raises(md.MDError):
                ctx.set_detectors(0, **bad)
        ctx.set_detectors(0, 2 * r0)
        ctx.step(5)
        ctx.set_detectors(0, None)
        with pytest.raises(md.MDError):
            ctx.iedf(0)


def test_detectors_on_an_ionizing_cluster_match_oracle(md):
    """An Ar cluster ionizing before every step (its ion-only i-blocks pushed
    with the pass's field, the rest by the step kernel) and detectors at
    0.9 R0: every crossing recorded by either push matches the oracle's
    detectors applied to the GPU's own states, step by step."""
    n = 1500
    r0 = synth.nm_to_len(2.5)
    c = synth.make_cluster(8, n, 0, r0, 0, synth.ARGON["mass"], n_electron_slots=8 * n)
    rw = synth.nm_to_len(synth.ARGON["r_w_nm"])
    cfg = md.make_config(a0=0.3, tau=1.0, t0=0.5 * math.pi, dt=0.1,
                         softening=synth.nm_to_len(0.1), envelope=synth.ENV_FLAT, rate_model=1,
                         ionize_every=1, zmax=8, n_ions=n, slot_base=n, seed=31,
                         r_loc=3 * rw, r_create=rw, species=synth.ARGON)
    nb = 50
    radius = 0.9 * r0
    e_max_ev = 2e3
    det = oracle.Detectors(c.n, radius=radius, cone_deg=30.0, e_max_ev=e_max_ev, nbins=nb)
    with md.Context([cfg], [md.HostParticles.from_cluster(c)]) as ctx:
        ctx.set_tuning(128, 4, 512, 0, 1, 0)      # ions 0..1023 pushed with the pass's field
        ctx.set_detectors(0, radius, cone_deg=30.0, e_max_ev=e_max_ev, n_bins=nb)
        g0 = ctx.get_particles(0)
        for _ in range(300):
            ctx.step(1)
            g1 = ctx.get_particles(0)
            det.record(g0.x, g1.x, state_of(g1))
            g0 = g1
        got, inside = ctx.iedf(0)
    crossed = np.flatnonzero(det.crossed)
    print("crossings", crossed.size, "pushed with the pass's field", int(np.sum(crossed < 1024)),
          "charges", np.bincount(g0.z[:n], minlength=9))
    assert np.sum(crossed < 1024) > 5 and np.sum(crossed >= 1024) > 2
    np.testing.assert_array_equal(got, det.hist)
    np.testing.assert_array_equal(inside, det.inside(state_of(g0)))


@pytest.mark.parametrize("packed", [0, 1])
def test_detectors_with_minimum_image_forces_match_oracle(md, packed):
    """The exploding ion sphere in a periodic cube of 6 R0 with minimum-image
    forces (the step kernel's image twin with the detector epilogue, scalar
    and packed): every crossing of 2.5 R0 matches the oracle's detectors
    applied to the GPU's own states, step by step."""
    n = 600
    c, r0, e_max, cfg = explosion(md, n, seed=6)
    cfg.boundary, cfg.box, cfg.min_image = 1, 6.0 * r0, 1
    nb = 32
    e_max_ev = 0.4 * e_max * ME_C2_EV
    det = oracle.Detectors(n, radius=2.5 * r0, cone_deg=30.0, e_max_ev=e_max_ev, nbins=nb)
    with md.Context([cfg], [md.HostParticles.from_cluster(c)]) as ctx:
        if packed:
            ctx.set_tuning(128, 8, 256, 0, 0, 1)
        ctx.set_detectors(0, 2.5 * r0, cone_deg=30.0, e_max_ev=e_max_ev, n_bins=nb)
        g0 = ctx.get_particles(0)
        for _ in range(200):
            ctx.step(1)
            g1 = ctx.get_particles(0)
            det.record(g0.x, g1.x, state_of(g1))
            g0 = g1
        got, inside = ctx.iedf(0)
    assert det.hist[4].sum() > 0.5 * n
    np.testing.assert_array_equal(got, det.hist)
    np.testing.assert_array_equal(inside, det.inside(state_of(g0)))
