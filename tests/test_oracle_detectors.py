"""Pins of the ion energy detectors of the oracle (Sec. III, Fig. 3: ion energy
distributions seen along and across the laser polarization, here read at a
fixed radius): constructed crossings, the relativistic kinetic energy, and the
Coulomb explosion of a uniform ion sphere, whose ions reach the detector
sphere 9 R0 with E = E_max (s^2 - s^3/9), s = r0/R0, in every direction."""
import math

import numpy as np
import pytest

import oracle
from paper_1307_3711_gb300 import synth

KC = oracle.coulomb_constant(0.8)
ME_C2_EV = 510998.95


def one_ion_state(n=1, z=1, mass=1000.0):
    return oracle.State(np.zeros((n, 3)), np.zeros((n, 3)), np.full(n, z, np.int32),
                        np.full(n, mass), np.ones(n))


@pytest.mark.parametrize("direction,expect", [
    ((1, 0, 0), {"+x", "all"}), ((-1, 0, 0), {"-x", "all"}), ((0, 1, 0), {"+y", "all"}),
    ((0, -1, 0), {"-y", "all"}), ((0, 0, 1), {"all"}),
    ((math.cos(math.radians(45)), math.sin(math.radians(45)), 0), {"all"}),
    ((math.cos(math.radians(25)), math.sin(math.radians(25)), 0), {"+x", "all"}),
    ((math.cos(math.radians(25)), 0, -math.sin(math.radians(25))), {"+x", "all"})])
def test_outward_crossing_lands_in_its_cone(direction, expect):
    d = np.array(direction, float)
    st = one_ion_state()
    st.u[0] = 1e-3 * d
    det = oracle.Detectors(1, radius=1.0, cone_deg=30.0, e_max_ev=1e3, nbins=10)
    det.record(0.95 * d[None, :], 1.05 * d[None, :], st)
    got = {oracle.DETECTORS[k] for k in range(5) if det.hist[k].sum()}
    assert got == expect
    assert det.crossed[0] == 1


def test_recorded_once_outward_only_and_ions_only():
    st = one_ion_state(5)
    st.z[:] = [1, 1, -1, 0, 2]
    st.active[3] = 1
    det = oracle.Detectors(5, radius=1.0, nbins=10)
    x0 = np.zeros((5, 3)); x0[:, 0] = [0.99, 1.01, 0.99, 0.99, 0.99]
    x1 = x0.copy(); x1[:, 0] = [1.01, 0.99, 1.01, 1.01, 1.01]
    st.active[4] = 0
    det.record(x0, x1, st)
    # ion 0 out: counted; ion 1 in: not; electron, neutral atom, inactive ion: not
    assert det.hist[4].sum() == 1 and list(det.crossed) == [1, 0, 0, 0, 0]
    xin = x1.copy(); xin[0, 0] = 0.99      # ion 0 back inside, the others stay put
    det.record(x1, xin, st)
    det.record(xin, x1, st)                 # ion 0 out again: already recorded
    assert det.hist[4].sum() == 1


def test_energy_bins_and_relativistic_energy():
    """u = sqrt(3): gamma = 2, E = m c^2 (bin 1 of 4 over [0, 2.5 m c^2));
    u = sqrt(15): gamma = 4, E = 3 m c^2 beyond e_max (overflow bin); a slow
    ion with E = m c^2 (gamma - 1) lands in bin floor(E nbins / e_max)."""
    mass = 1.0
    det = oracle.Detectors(3, radius=1.0, e_max_ev=2.5 * ME_C2_EV, nbins=4)
    st = one_ion_state(3, mass=mass)
    st.u[0] = [math.sqrt(3), 0, 0]
    st.u[1] = [0, math.sqrt(15), 0]
    st.u[2] = [0.3, 0.4, 0.0]                 # gamma - 1 = sqrt(1.25) - 1 = 0.118
    x0 = np.array([[0.9, 0, 0]] * 3)
    x1 = np.array([[1.1, 0, 0]] * 3)
    det.record(x0, x1, st)
    assert det.hist[4].tolist() == [1, 1, 0, 0, 1]
    assert det.hist[0].tolist() == [1, 1, 0, 0, 1]   # all moved along +x


@pytest.mark.parametrize("axis,sign,row", [(0, 1, 0), (0, -1, 1), (1, 1, 2), (1, -1, 3)])
def test_energy_bins_are_equal_widths_of_e_max(axis, sign, row):
    """The IEDF bins split [0, e_max) into nbins equal widths: ions with
    E = (k + 1/2) e_max / nbins, k = 0..nbins-1, fill one bin each of their
    cone's histogram and of the all-directions one, and one at 1.001 e_max goes
    to the overflow bin (E = (gamma - 1) m c^2 set by u).  The detector sphere
    is centred off the origin; the crossing is along the cone's axis."""
    mass, nbins, e_max = synth.MASS_40AMU, 10, 2.0e4
    center = np.array([0.3, -0.2, 0.1])
    energies = np.concatenate([(np.arange(nbins) + 0.5) * e_max / nbins, [1.001 * e_max]])
    n = energies.size
    st = one_ion_state(n, mass=mass)
    g = 1.0 + energies / (mass * ME_C2_EV)
    st.u[:, axis] = sign * np.sqrt(g * g - 1.0)
    d = np.zeros(3)
    d[axis] = sign
    det = oracle.Detectors(n, radius=1.0, e_max_ev=e_max, nbins=nbins, center=center)
    det.record(np.tile(center + 0.9 * d, (n, 1)), np.tile(center + 1.1 * d, (n, 1)), st)
    for k in range(5):
        want = [1] * (nbins + 1) if k in (row, 4) else [0] * (nbins + 1)
        assert det.hist[k].tolist() == want, k
    # the ions not yet recorded are binned at their own energies
    st2 = one_ion_state(n, mass=mass)
    st2.u[:] = st.u
    fresh = oracle.Detectors(n, radius=1.0, e_max_ev=e_max, nbins=nbins, center=center)
    assert fresh.inside(st2).tolist() == [1] * (nbins + 1)
    assert det.inside(st).tolist() == [0] * (nbins + 1)   # all recorded already


def test_only_crossings_from_inside_count():
    """An ion that is already outside the sphere and moves further out (along
    each axis and a diagonal), or one that stays inside, is not recorded; the
    sphere is centred off the origin, so positions are taken relative to it."""
    center = np.array([0.5, 0.4, -0.3])
    dirs = np.array([[1, 0, 0], [0, 1, 0], [0, 0, 1], [0, -1, 0], [1, 1, 1] / np.sqrt(3)])
    n = 2 * len(dirs)
    st = one_ion_state(n)
    st.u[:, 0] = 1e-3
    x0 = np.concatenate([center + 1.05 * dirs, center + 0.5 * dirs])
    x1 = np.concatenate([center + 1.2 * dirs, center + 0.9 * dirs])
    det = oracle.Detectors(n, radius=1.0, nbins=10, center=center)
    det.record(x0, x1, st)
    assert det.hist.sum() == 0 and not det.crossed.any()
    # the same moves seen from a sphere at the origin do cross it
    det0 = oracle.Detectors(n, radius=1.0, nbins=10)
    det0.record(x0 - center, x1 - center, st)
    assert det0.hist[4].sum() == 0
    det0.record(x1 - center, 1.1 * (x1 - center) / np.linalg.norm(x1 - center, axis=1)[:, None], st)
    assert det0.hist[4].sum() == len(dirs)   # the inner ones now cross, the outer ones do not


def test_coulomb_explosion_seen_at_nine_radii():
    """Uniform ion sphere from rest, laser off: an ion starting at s = r0/R0
    keeps its enclosed charge Q s^3 and crosses 9 R0 with
    E = K q Q s^3 (1/(s R0) - 1/(9 R0)) = E_max (s^2 - s^3/9).  The mean
    recorded energy matches that of the recorded ions, and the four 30-degree
    cones each see a fraction (1 - cos 30)/2 of them."""
    n, r0, m, qv = 1200, synth.nm_to_len(2.0), synth.MASS_40AMU, 1
    c = synth.make_cluster(5, n, 0, r0, qv, m)
    q = c.w * c.z
    e_max = KC * qv * q.sum() / r0                   # m_e c^2 units
    tau = math.sqrt(m * r0 ** 3 / (KC * qv * q.sum()))
    st = oracle.State(c.x, c.u, c.z, c.mass, c.w)
    s0 = np.linalg.norm(c.x, axis=1) / r0
    p = oracle.make_params(a0=0.0, dt=tau / 40, eps=0.0, env=oracle.ENV_FLAT)
    nb = 400
    e_max_ev = e_max * ME_C2_EV
    det = oracle.Detectors(n, radius=9 * r0, cone_deg=30.0, e_max_ev=e_max_ev, nbins=nb)
    oracle.md_steps_detected(st, p, 480, det, nthreads=4)   # t = 12 tau
    hit = det.crossed > 0
    assert hit.sum() > 0.5 * n and det.hist[4].sum() == hit.sum()
    centers = (np.arange(nb) + 0.5) / nb
    mean_rec = (det.hist[4][:nb] * centers).sum() / det.hist[4][:nb].sum()
    # each ion keeps the charge of the ions that start inside it (no shell
    # crossing): E_i / E_max = (n_below_i / N) (R0 / r0_i - 1/9); with a
    # continuous density this is s^2 - s^3/9
    n_below = np.argsort(np.argsort(s0))
    pred = (n_below / n) * (1.0 / s0 - 1.0 / 9.0)
    mean_pred = pred[hit].mean()
    assert det.hist[4][nb] == 0                       # nobody beyond E_max
    assert mean_rec == pytest.approx(mean_pred, abs=0.005)
    assert mean_pred == pytest.approx((s0[hit] ** 2 - s0[hit] ** 3 / 9).mean(), abs=0.02)
    frac = (1 - math.cos(math.radians(30))) / 2
    for k in range(4):
        expect = frac * hit.sum()
        assert abs(det.hist[k].sum() - expect) < 4 * math.sqrt(expect), oracle.DETECTORS[k]
    inside = det.inside(st)
    assert inside.sum() == n - hit.sum()
