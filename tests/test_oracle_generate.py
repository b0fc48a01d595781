"""Pins of the oracle's seeded cluster generation (Sec. II: the atoms of a
cluster of radius R0 are placed at random inside the sphere; Eq. 1: one macro
particle of weight w stands for w atoms), on the CPU.

What fixes it, independently of its code: the records' layout, charges,
masses and weights; every position strictly inside the ball; the law of a
uniform ball (radius CDF (r/R0)^3, cos(theta) uniform on [-1, 1], azimuth
uniform, centroid at the centre); a Maxwellian of the stated temperature
(each component normal with variance kT / (m c^2), components independent and
independent of the position); reproducibility and independence across seeds;
records that do not depend on how many follow them."""
import numpy as np
import pytest
from scipy import stats

import oracle

ME_C2_EV = 510998.95
N = 40000
R0 = 0.37
CENTER = (0.2, -0.1, 0.05)


@pytest.fixture(scope="module")
def cl():
    return oracle.generate_cluster(R0, N // 4, 3 * N // 4, n_slots=500, ion_charge=3,
                                   ion_mass=2000.0, weight=2.5, kt_e_ev=10.0, kt_i_ev=40.0,
                                   seed=123456789, center=CENTER)


def test_layout_charges_masses_weights(cl):
    ni, ne, ns = N // 4, 3 * N // 4, 500
    assert len(cl["z"]) == ni + ne + ns
    assert (cl["kind"][:ni] == 0).all() and (cl["kind"][ni:ni + ne] == 1).all()
    assert (cl["kind"][ni + ne:] == 2).all()
    assert (cl["z"][:ni] == 3).all() and (cl["z"][ni:ni + ne] == -1).all()
    assert (cl["z"][ni + ne:] == 0).all()
    assert (cl["mass"][:ni] == 2000.0).all() and (cl["mass"][ni:] == 1.0).all()
    assert (cl["w"] == 2.5).all()
    # charge neutrality of 3+ ions with three electrons each (Eq. 1 weights)
    assert float(np.sum(cl["w"] * cl["z"])) == 0.0
    # inactive slots: at the centre, at rest
    np.testing.assert_array_equal(cl["x"][ni + ne:], np.tile(CENTER, (ns, 1)))
    assert (cl["u"][ni + ne:] == 0.0).all()


def _active(cl):
    return cl["kind"] != 2


def test_every_position_strictly_inside_the_ball(cl):
    d = cl["x"][_active(cl)] - np.array(CENTER)
    r = np.linalg.norm(d, axis=1)
    assert r.max() < R0
    assert r.max() > 0.99 * R0   # and the ball is filled out to its edge


def test_uniform_ball_radius_angles_and_centroid(cl):
    d = cl["x"][_active(cl)] - np.array(CENTER)
    n = len(d)
    r = np.linalg.norm(d, axis=1)
    assert stats.kstest((r / R0) ** 3, "uniform").pvalue > 1e-3
    assert stats.kstest(d[:, 2] / r, stats.uniform(-1, 2).cdf).pvalue > 1e-3
    phi = (np.arctan2(d[:, 1], d[:, 0]) + np.pi) / (2 * np.pi)
    assert stats.kstest(phi, "uniform").pvalue > 1e-3
    # centroid: each component has variance R0^2/5 per point
    assert np.all(np.abs(d.mean(axis=0)) < 4.0 * R0 * np.sqrt(0.2 / n))
    # octants equally populated
    octant = (d[:, 0] > 0) * 4 + (d[:, 1] > 0) * 2 + (d[:, 2] > 0)
    cnt = np.bincount(octant, minlength=8)
    assert stats.chisquare(cnt).pvalue > 1e-3


def test_maxwellian_momenta(cl):
    ni, ne = N // 4, 3 * N // 4
    for sl, kt, m in ((slice(0, ni), 40.0, 2000.0), (slice(ni, ni + ne), 10.0, 1.0)):
        u = cl["u"][sl]
        sig = np.sqrt(kt / (m * ME_C2_EV))
        n = len(u)
        for k in range(3):
            assert stats.kstest(u[:, k] / sig, "norm").pvalue > 1e-3
            assert abs(u[:, k].mean()) < 4.0 * sig / np.sqrt(n)
            assert abs(u[:, k].var() / sig ** 2 - 1.0) < 4.0 * np.sqrt(2.0 / n)
        # kinetic temperature: (m c^2 / 3) <u^2> = kT
        assert m * ME_C2_EV * np.mean(np.sum(u ** 2, axis=1)) / 3.0 == pytest.approx(kt, rel=0.03)
        c = np.corrcoef(u.T)
        assert np.all(np.abs(c[np.triu_indices(3, 1)]) < 4.0 / np.sqrt(n))


def test_momenta_independent_of_positions(cl):
    act = _active(cl)
    d = cl["x"][act] - np.array(CENTER)
    u2 = np.sum(cl["u"][act] ** 2, axis=1) / np.where(cl["kind"][act] == 0, 40.0 / 2000.0, 10.0)
    n = len(d)
    for k in range(3):
        assert abs(np.corrcoef(d[:, k], u2)[0, 1]) < 4.0 / np.sqrt(n)
        assert abs(np.corrcoef(np.abs(d[:, k]), u2)[0, 1]) < 4.0 / np.sqrt(n)
    assert abs(np.corrcoef(np.linalg.norm(d, axis=1), u2)[0, 1]) < 4.0 / np.sqrt(n)


def test_zero_temperature_is_at_rest_and_seeds_differ():
    a = oracle.generate_cluster(1.0, 300, 300, seed=5)
    assert (a["u"] == 0.0).all()
    b = oracle.generate_cluster(1.0, 300, 300, seed=5)
    np.testing.assert_array_equal(a["x"], b["x"])
    c = oracle.generate_cluster(1.0, 300, 300, seed=6)
    assert not np.any(np.all(a["x"] == c["x"], axis=1))
    # a seed that differs only in its high 32 bits draws other positions
    d = oracle.generate_cluster(1.0, 300, 300, seed=5 + (1 << 32))
    assert not np.any(np.all(a["x"] == d["x"], axis=1))
    # no two records share a position
    assert len(np.unique(a["x"], axis=0)) == 600


def test_a_record_does_not_depend_on_the_records_after_it():
    a = oracle.generate_cluster(1.0, 200, 0, kt_i_ev=5.0, ion_mass=50.0, seed=9)
    b = oracle.generate_cluster(1.0, 200, 100, n_slots=50, kt_i_ev=5.0, ion_mass=50.0, seed=9)
    np.testing.assert_array_equal(a["x"], b["x"][:200])
    np.testing.assert_array_equal(a["u"], b["u"][:200])


def test_position_scale_and_centre():
    """The same draws at another radius and centre: x - c scales with r0."""
    a = oracle.generate_cluster(1.0, 500, 0, seed=3)
    b = oracle.generate_cluster(0.25, 500, 0, seed=3, center=(1.0, 2.0, 3.0))
    np.testing.assert_allclose(b["x"] - np.array([1.0, 2.0, 3.0]), 0.25 * a["x"],
                               rtol=0, atol=1e-15)
