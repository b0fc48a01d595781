"""Pins of the ionization oracle (Sec. II, ionization paragraph) against
closed forms, library routines and exact invariants."""
import json
import math
import os

import numpy as np
import pytest
from scipy import constants as sc
from scipy import integrate, special, stats

import oracle
from paper_1307_3711_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
AR = synth.ARGON


def test_philox_known_answers():
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.json")) as f:
        kat = json.load(f)
    for v in kat["vectors"]:
        ctr = [int(x, 16) for x in v["ctr"]]
        key = [int(x, 16) for x in v["key"]]
        out = [int(x, 16) for x in v["out"]]
        assert oracle.philox4x32_10(ctr, key).tolist() == out


def test_philox_uniform_and_decorrelated():
    """Words of consecutive counters are uniform (KS) and a one-bit change of
    the counter flips about half of the output bits."""
    ws = np.array([oracle.philox4x32_10([i, 7, 0, 0], [11, 13]) for i in range(4000)])
    u = ws.astype(np.float64) / 2 ** 32
    for k in range(4):
        assert stats.kstest(u[:, k], "uniform").pvalue > 1e-3
    flips = []
    for i in range(200):
        a = oracle.philox4x32_10([i, 3, 5, 0], [1, 2])
        b = oracle.philox4x32_10([i ^ 1, 3, 5, 0], [1, 2])
        flips.append(sum(bin(int(x) ^ int(y)).count("1") for x, y in zip(a, b)))
    assert np.mean(flips) == pytest.approx(64, abs=2)
    assert oracle.uniform_open0(0) == 2.0 ** -32 and oracle.uniform_open0(2 ** 32 - 1) == 1.0


@pytest.mark.parametrize("x", [1e-8, 1e-3, 0.3, 0.999, 1.0, 1.001, 2.5, 10.0, 50.0, 300.0])
def test_e1_matches_library(x):
    assert oracle.e1(x) == pytest.approx(special.exp1(x), rel=1e-13)


@pytest.mark.parametrize("F", [0.02, 0.05, 0.1, 0.3, 1.0])
def test_adk_reduces_to_landau_hydrogen_rate(F):
    """For hydrogen (Ip = 1/2 a.u., Z = 1: n* = 1, l* = 0) the static ADK
    rate is the exact weak-field tunnelling rate of the ground state,
    w = (4/F) exp(-2/(3F)) (Landau & Lifshitz, QM, Sec. 77)."""
    assert oracle.adk_rate_au(F, 0.5, 1.0) == pytest.approx(4.0 / F * math.exp(-2.0 / (3 * F)),
                                                            rel=1e-12)


@pytest.mark.parametrize("Z", [2, 3, 5])
@pytest.mark.parametrize("f", [0.02, 0.05, 0.1])
def test_adk_for_hydrogen_like_ions_follows_coulomb_scaling(Z, f):
    """A hydrogen-like ion of nuclear charge Z (Ip = Z^2/2, residual charge Z,
    so n* = 1 again) is hydrogen rescaled: lengths 1/Z, energies Z^2, fields
    Z^3, rates Z^2.  Its exact weak-field rate is therefore Landau's rate at
    F / Z^3 times Z^2: w = (4 Z^5 / F) exp(-2 Z^3 / (3F)).  This fixes the
    Ip and F0 = (2 Ip)^{3/2} dependence of the ADK expression away from
    Ip = 1/2 (f = F / Z^3)."""
    F = f * Z ** 3
    landau = Z ** 2 * (4.0 / f) * math.exp(-2.0 / (3.0 * f))
    assert oracle.adk_rate_au(F, Z * Z / 2.0, float(Z)) == pytest.approx(landau, rel=1e-12)
    assert landau == pytest.approx(4.0 * Z ** 5 / F * math.exp(-2.0 * Z ** 3 / (3.0 * F)),
                                   rel=1e-12)


def test_adk_structure():
    """Monotone in the field, vanishing as F -> 0, and suppressed for higher
    potentials at the same field."""
    ip = AR["ip_ev"][0] / 27.211386245988
    f = np.logspace(-3, 0, 40)
    w = np.array([oracle.adk_rate_au(x, ip, 1.0) for x in f])
    assert np.all(np.diff(w) > 0) and w[0] < 1e-100
    assert oracle.adk_rate_au(0.0, ip, 1.0) == 0.0
    ip2 = AR["ip_ev"][1] / 27.211386245988
    assert oracle.adk_rate_au(0.05, ip2, 2.0) < oracle.adk_rate_au(0.05, ip, 1.0)


@pytest.mark.parametrize("P,T,q", [(15.76, 5.0, 6), (15.76, 40.0, 6), (143.46, 30.0, 1),
                                   (59.58, 200.0, 3), (179.84, 150.0, 10), (374.0, 900.0, 3)])
def test_lotz_rate_is_maxwell_average_of_cross_section(P, T, q):
    """<sigma v> of the Lotz cross section sigma = a q ln(E/P)/(E P) over a
    Maxwellian, integrated numerically in SI units, equals the closed form."""
    a = 4.5e-14 * 1e-4 * sc.e ** 2            # m^2 J^2
    Pj, Tj = P * sc.e, T * sc.e

    def integrand(E):  # energy in J
        sigma = a * q * math.log(E / Pj) / (E * Pj)
        v = math.sqrt(2 * E / sc.m_e)
        f = 2 * math.sqrt(E / math.pi) * Tj ** -1.5 * math.exp(-E / Tj)  # Maxwell energy pdf
        return sigma * v * f

    val, _ = integrate.quad(integrand, Pj, Pj + 60 * Tj, limit=400, epsabs=0, epsrel=1e-11)
    assert oracle.lotz_rate_cgs(P, T, q) == pytest.approx(val * 1e6, rel=1e-8)  # m^3 -> cm^3
    assert oracle.lotz_rate_cgs(P, 0.0, q) == 0.0


@pytest.mark.parametrize("species", [synth.ARGON, synth.XENON], ids=["Ar", "Xe"])
def test_species_tables_follow_the_shell_structure(species):
    """The ionization energies rise with the charge state; the outer-subshell
    occupation counts down by one per ionization and restarts at a full
    inner subshell (Ar: 3p^6, 3s^2; Xe: 5p^6, 5s^2, 4d^10)."""
    ip, q = np.array(species["ip_ev"]), np.array(species["q_outer"])
    assert ip.size == q.size and np.all(np.diff(ip) > 0)
    shells = {"Ar": [6, 2], "Xe": [6, 2, 10]}[species["name"]]
    expect = np.concatenate([np.arange(s, 0, -1) for s in shells])[:q.size]
    assert np.array_equal(q, expect)


@pytest.mark.parametrize("z", [0, 7, 8, 9, 15])
def test_rate_total_indexes_the_xenon_table(z):
    """Xe at 790 nm: the rate of Xe^z uses I_p(z), the residual charge z + 1
    and the outer-subshell count q(z) of the table, for every charge state
    up to 15 (ADK and Lotz pinned on their own above)."""
    XE, lam = synth.XENON, 0.79
    omega = 2 * math.pi * sc.c / (lam * 1e-6)
    amag, ne, te = 0.3, 5e22, 400.0
    F = amag * sc.m_e * sc.c * omega / sc.e / sc.physical_constants["atomic unit of electric field"][0]
    ip = XE["ip_ev"][z] / sc.physical_constants["Hartree energy in eV"][0]
    t_au = sc.physical_constants["atomic unit of time"][0]
    nu = (oracle.adk_rate_au(F, ip, z + 1.0) / t_au
          + ne * oracle.lotz_rate_cgs(XE["ip_ev"][z], te, XE["q_outer"][z])) / omega
    assert oracle.rate_total(amag, z, ne, te, XE, lambda_um=lam) == pytest.approx(nu, rel=1e-8)


def test_rate_total_units():
    """nu_total in 1/omega: field a -> E = a m_e c omega / e, ADK in a.u.
    converted with the atomic unit of time; collisions n_e <sigma v>."""
    lam = 0.8e-6
    omega = 2 * math.pi * sc.c / lam
    amag = 0.05
    e_si = amag * sc.m_e * sc.c * omega / sc.e
    F = e_si / (sc.physical_constants["atomic unit of electric field"][0])
    ip = AR["ip_ev"][0] / (sc.physical_constants["Hartree energy in eV"][0])
    t_au = sc.physical_constants["atomic unit of time"][0]
    nu_ofi = oracle.adk_rate_au(F, ip, 1.0) / t_au / omega
    assert oracle.rate_total(amag, 0, 0.0, 0.0, AR) == pytest.approx(nu_ofi, rel=1e-8)
    ne, te = 1e22, 30.0
    nu_ci = ne * oracle.lotz_rate_cgs(AR["ip_ev"][0], te, 6) / omega
    assert oracle.rate_total(amag, 0, ne, te, AR) == pytest.approx(nu_ofi + nu_ci, rel=1e-8)


def test_local_moments_constructed_case():
    """Six electrons at 0.5 r_loc along +-x, +-y, +-z with u = drift +- v
    along the same axis (spread about the mean: <|u - <u>|^2> = v^2):
    ne = 6 w / volume, Te = m c^2 v^2 / 3 in the local mean frame; an ion,
    a neutral atom, an inactive slot and a far electron do not count.  The
    periodic version in a box much larger than r_loc gives the same."""
    r_loc, v, w = 0.01, 0.003, 2.0
    drift = np.array([0.002, -0.001, 0.0005])
    pos = []
    vel = []
    for ax in range(3):
        for s in (1, -1):
            p = np.zeros(3); p[ax] = 0.5 * s * r_loc
            q = drift.copy(); q[ax] += s * v
            pos.append(p); vel.append(q)
    x = np.array(pos + [[0.001, 0, 0], [0, 0.002, 0], [2 * r_loc, 0, 0], [0, 0, -0.003]])
    u = np.array(vel + [[0, 0, 0], [0, 0, 0], [0.5, 0, 0], [0.4, 0, 0]])
    z = np.array([-1] * 6 + [3, 0, -1, 0])
    active = np.array([1] * 6 + [1, 0, 1, 1], np.uint8)
    st = oracle.State(x, u, z, np.ones(10), np.full(10, w), active)
    k = 2 * math.pi / 0.8e-6
    vol_cm3 = 4 / 3 * math.pi * (r_loc / k) ** 3 * 1e6
    for box in (0.0, 1.0):
        ne, te = oracle.local_moments(np.zeros((1, 3)), st, r_loc, box=box)
        assert ne[0] == pytest.approx(6 * w / vol_cm3, rel=1e-12)
        assert te[0] == pytest.approx(510998.95 * v * v / 3, rel=1e-9)
        # at 0.4 micron the same r_loc (in 1/k) is half as long in cm: 8 times the density
        ne4, te4 = oracle.local_moments(np.zeros((1, 3)), st, r_loc, lambda_um=0.4, box=box)
        assert ne4[0] == pytest.approx(8 * 6 * w / vol_cm3, rel=1e-12)
        assert te4[0] == pytest.approx(te[0], rel=1e-12)
    ne, te = oracle.local_moments(np.array([[10.0, 0, 0]]), st, r_loc)
    assert ne[0] == 0 and te[0] == 0


def test_decision_statistics_constant_rate():
    """With a fixed probability per pass, the ionized fraction after one pass
    is binomial(P), independent of the ion id and step."""
    n = 20000
    ids = np.arange(n)
    z = np.zeros(n, np.int32)
    amag = np.full(n, 0.012)
    P = None
    frac = []
    for step in range(3):
        z1, fired, off, prob = oracle.decide(ids, z, amag, np.zeros(n), np.zeros(n), AR, 8,
                                             seed=5, step=step, dt_ion=2.0, r_create=0.001)
        P = prob[0]
        assert np.all(prob == P) and 0.05 < P < 0.95
        frac.append(fired.mean())
        assert np.array_equal(z1, z + fired)
    for f in frac:
        assert abs(f - P) < 4 * math.sqrt(P * (1 - P) / n)
    # the decision is a pure function of (seed, id, step)
    a = oracle.decide(ids[:50], z[:50], amag[:50], np.zeros(50), np.zeros(50), AR, 8, 5, 1, 2.0,
                      0.001)
    b = oracle.decide(ids[:50], z[:50], amag[:50], np.zeros(50), np.zeros(50), AR, 8, 5, 1, 2.0,
                      0.001)
    assert np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])
    # zmax caps the charge
    zc = np.full(5, 8, np.int32)
    z2, f2, _, p2 = oracle.decide(ids[:5], zc, np.full(5, 10.0), np.zeros(5), np.zeros(5), AR, 8,
                                  5, 1, 2.0, 0.001)
    assert np.all(f2 == 0) and np.all(z2 == 8) and np.all(p2 == 0)


def test_survival_after_n_passes_is_exponential():
    """Sec. II: at a constant rate nu each pass ionizes with P = 1 - exp(-nu dt),
    independently of the earlier passes, so the fraction of atoms not yet
    ionized after n passes is exp(-nu n dt) (memoryless decay); nu is the rate
    function's, pinned above.  nu dt = 0.35: a first-order P = nu dt would
    leave (0.65)^n instead."""
    n = 40000
    ids = np.arange(n)
    z = np.zeros(n, np.int32)
    amag = np.full(n, 0.012)
    nu = oracle.rate_total(0.012, 0, 0.0, 0.0, AR)
    dt_ion = 0.35 / nu
    alive = np.ones(n, bool)
    for k in range(6):
        _, fired, _, _ = oracle.decide(ids, z, amag, np.zeros(n), np.zeros(n), AR, 8, seed=12,
                                       step=100 + k, dt_ion=dt_ion, r_create=0.001)
        alive &= fired == 0
        s_exp = math.exp(-nu * dt_ion * (k + 1))
        assert abs(alive.mean() - s_exp) < 4 * math.sqrt(s_exp * (1 - s_exp) / n)


def test_decision_uses_all_64_bits_of_seed_and_step():
    """The Philox key is the whole 64-bit seed and the counter holds the whole
    64-bit step (with the ion index), so seeds or steps that differ only in
    their high 32 bits draw independent numbers."""
    n = 4000
    ids = np.arange(n)
    z = np.zeros(n, np.int32)
    amag = np.full(n, 0.012)
    args = (np.zeros(n), np.zeros(n), AR, 8)

    def fired(seed, step):
        return oracle.decide(ids, z, amag, *args, seed=seed, step=step, dt_ion=2.0,
                             r_create=0.001)[1]

    base = fired(5, 3)
    for seed, step in ((5 + 2 ** 32, 3), (5, 3 + 2 ** 32)):
        other = fired(seed, step)
        # independent Bernoulli draws agree on about P^2 + (1-P)^2 of the ions
        assert 0.05 < (base != other).mean() < 0.95


def test_electron_placement_uniform_in_ball():
    n = 20000
    rc = 0.004
    _, fired, off, _ = oracle.decide(np.arange(n), np.zeros(n, np.int32), np.full(n, 0.2),
                                     np.zeros(n), np.zeros(n), AR, 8, 9, 0, 100.0, rc)
    assert fired.mean() > 0.99
    r = np.linalg.norm(off[fired > 0], axis=1)
    assert r.max() <= rc
    assert stats.kstest(r / rc, lambda s: np.clip(s, 0, 1) ** 3).pvalue > 1e-3
    assert np.abs(off[fired > 0].mean(axis=0)).max() < 0.03 * rc


def test_ionize_pass_conserves_charge_and_uses_slots():
    """Neutral Ar atoms in a strong field: every pass conserves the total
    charge exactly; the electrons freed in a pass fill the next free slots in
    the order of their ions, so the active slots stay one dense block."""
    n_ion, zmax = 300, 8
    c = synth.make_cluster(4, n_ion, 0, synth.nm_to_len(2.0), 0, AR["mass"],
                           n_electron_slots=n_ion * zmax)
    st = oracle.State(c.x, c.u, c.z, c.mass, c.w, c.active)
    p = oracle.make_params(a0=0.3, tau=1.0, dt=0.05, eps=synth.nm_to_len(0.1),
                           env=oracle.ENV_FLAT)
    r_loc = 3 * synth.nm_to_len(AR["r_w_nm"])
    total = []
    for k in range(4):
        st.step = 10 + k
        before = st.copy()
        n_before = int(st.active[n_ion:].sum())
        fired, amag, ne, te = oracle.ionize_pass(st, p, AR, n_ion, n_ion, zmax, seed=3,
                                                 dt_ion=5.0, r_loc=r_loc,
                                                 r_create=synth.nm_to_len(AR["r_w_nm"]))
        total.append(int(np.sum(st.w * st.z * st.active)))
        for rank, i in enumerate(np.nonzero(fired)[0]):
            slot = n_ion + n_before + rank
            assert before.active[slot] == 0
            assert st.active[slot] == 1 and st.z[slot] == -1
            assert np.array_equal(st.u[slot], before.u[i])
            assert np.linalg.norm(st.x[slot] - before.x[i]) <= synth.nm_to_len(AR["r_w_nm"])
        n_el = int(st.active[n_ion:].sum())
        assert st.active[n_ion:n_ion + n_el].all() and not st.active[n_ion + n_el:].any()
    assert total == [0, 0, 0, 0]
    assert st.z[:n_ion].max() >= 2
    assert st.active[n_ion:].sum() == st.z[:n_ion].sum()


def test_ionize_pass_field_is_coulomb_plus_laser_at_t_n():
    """The pass ionizes in the total field at the ion (Sec. II): the softened
    Coulomb field of the others plus the laser field a(t_n), t_n = t0 + n dt.
    Two records along the polarization: a neutral atom at the origin and a
    Z = 2 ion at distance d on +x.  At the atom the two fields are collinear:
    |a0 sin t_n - K Z d / (d^2 + eps^2)^{3/2}| (flat envelope, linear
    polarization); at the ion the neutral atom adds nothing: |a0 sin t_n|."""
    n_ion, zmax = 2, 8
    d, eps, a0, zq = synth.nm_to_len(1.0), synth.nm_to_len(0.1), 1e-3, 2
    x = np.zeros((n_ion + n_ion * zmax, 3))
    x[1, 0] = d
    z = np.zeros(x.shape[0], np.int32)
    z[1] = zq
    active = np.zeros(x.shape[0], np.uint8)
    active[:n_ion] = 1
    st = oracle.State(x, np.zeros_like(x), z, np.full(x.shape[0], AR["mass"]),
                      np.ones(x.shape[0]), active, step=13)
    p = oracle.make_params(a0=a0, tau=1.0, t0=0.7, dt=0.05, eps=eps, env=oracle.ENV_FLAT)
    kc = oracle.coulomb_constant(0.8)
    t_n = 0.7 + 13 * 0.05
    e_c = kc * zq * d / (d * d + eps * eps) ** 1.5
    assert 0.2 < e_c / (a0 * abs(math.sin(t_n))) < 5  # both terms matter
    _, amag, _, _ = oracle.ionize_pass(st, p, AR, n_ion, n_ion, zmax, seed=1, dt_ion=1e-9,
                                       r_loc=d / 4, r_create=d / 4)
    assert amag[0] == pytest.approx(abs(a0 * math.sin(t_n) - e_c), rel=1e-12)
    assert amag[1] == pytest.approx(abs(a0 * math.sin(t_n)), rel=1e-12)


def test_ionize_pass_takes_the_moments_at_each_ion():
    """The pass measures n_e and T_e around each ion (Sec. II): two neutral
    atoms 10 r_loc apart, three electrons within r_loc of the second only,
    with u = (+v, 0, 0), (-v, 0, 0), 0: n_e = 3 w / (4/3 pi r_loc^3) and
    T_e = m c^2 (2 v^2 / 3) / 3 there, nothing at the first atom."""
    n_ion, zmax, w = 2, 8, 1.5
    r_loc, v = 0.01, 0.004
    n = n_ion + n_ion * zmax
    x = np.zeros((n, 3))
    x[1, 0] = 10 * r_loc
    x[2:5] = x[1] + np.array([[0, 0.3 * r_loc, 0], [0, -0.3 * r_loc, 0], [0, 0, 0.5 * r_loc]])
    u = np.zeros((n, 3))
    u[2, 0], u[3, 0] = v, -v
    z = np.zeros(n, np.int32)
    z[2:5] = -1
    mass = np.ones(n)
    mass[:n_ion] = AR["mass"]
    active = np.zeros(n, np.uint8)
    active[:5] = 1
    st = oracle.State(x, u, z, mass, np.full(n, w), active)
    p = oracle.make_params(a0=0.0, tau=1.0, dt=0.05, eps=1e-3, env=oracle.ENV_FLAT)
    _, _, ne, te = oracle.ionize_pass(st, p, AR, n_ion, n_ion, zmax, seed=1, dt_ion=1e-9,
                                      r_loc=r_loc, r_create=1e-4)
    k = 2 * math.pi / 0.8e-6
    vol_cm3 = 4 / 3 * math.pi * (r_loc / k) ** 3 * 1e6
    assert ne[0] == 0.0 and te[0] == 0.0
    assert ne[1] == pytest.approx(3 * w / vol_cm3, rel=1e-12)
    assert te[1] == pytest.approx(510998.95 * (2 * v * v / 3) / 3, rel=1e-9)


def test_ionize_pass_conserves_weighted_charge():
    """Macro atoms of unequal weight (Eq. 1): a freed electron stands for as
    many electrons as its atom has atoms, and has the electron mass, so the
    total charge sum w z stays zero pass after pass."""
    n_ion, zmax = 200, 8
    c = synth.make_cluster(6, n_ion, 0, synth.nm_to_len(2.0), 0, AR["mass"],
                           n_electron_slots=n_ion * zmax)
    c.w[:n_ion] = np.random.default_rng(2).uniform(0.5, 3.0, n_ion)
    st = oracle.State(c.x, c.u, c.z, c.mass, c.w, c.active)
    p = oracle.make_params(a0=0.3, tau=1.0, dt=0.05, eps=synth.nm_to_len(0.1),
                           env=oracle.ENV_FLAT)
    for k in range(3):
        st.step = 20 + k
        oracle.ionize_pass(st, p, AR, n_ion, n_ion, zmax, seed=8, dt_ion=5.0,
                           r_loc=3 * synth.nm_to_len(AR["r_w_nm"]),
                           r_create=synth.nm_to_len(AR["r_w_nm"]))
        q = st.w * st.z * st.active
        assert abs(q.sum()) < 1e-12 * np.abs(q).sum()
    el = np.nonzero(st.active[n_ion:])[0] + n_ion
    assert el.size > n_ion and np.all(st.mass[el] == 1.0)


def test_next_free_slot_follows_the_last_active_slot():
    """A state whose slot region has holes: new electrons go after the last
    active slot, never into a hole."""
    n_ion, zmax = 4, 2
    st = oracle.State(np.zeros((12, 3)), np.zeros((12, 3)), np.zeros(12, np.int32),
                      np.ones(12), np.ones(12), np.zeros(12, np.uint8))
    assert oracle.next_free_slot(st, 4, n_ion, zmax) == 4
    st.active[[4, 7]] = 1
    assert oracle.next_free_slot(st, 4, n_ion, zmax) == 8


def test_local_moments_with_minimum_image():
    """Minimum-image moments: an electron just across a face is within r_loc
    of an ion near the opposite face through its image; the moments are
    invariant under a periodic translation of the whole system; a system
    within half the box has exactly its open moments."""
    box, r_loc = 1.0, 0.05
    x = np.array([[0.49, 0.0, 0.0], [-0.48, 0.01, 0.0], [0.47, 0.0, 0.02]])
    u = np.array([[0.0, 0.0, 0.0], [0.01, 0.0, 0.0], [-0.02, 0.003, 0.0]])
    st = oracle.State(x, u, [1, -1, -1], [7e4, 1.0, 1.0], [1.0, 1.0, 1.0])
    ne_b, te_b = oracle.local_moments(x[:1], st, r_loc, box=box)
    ne_o, te_o = oracle.local_moments(x[:1], st, r_loc)
    assert ne_b[0] == pytest.approx(2 * ne_o[0]) and te_b[0] > 0.0 and te_o[0] == 0.0
    rng = np.random.default_rng(5)
    n = 400
    xr = rng.uniform(-0.5, 0.5, size=(n, 3))
    ur = rng.normal(size=(n, 3)) * 0.01
    z = np.where(np.arange(n) < 100, 2, -1)
    st = oracle.State(xr, ur, z, np.where(z > 0, 7e4, 1.0), np.ones(n))
    ne0, te0 = oracle.local_moments(xr[:100], st, 0.2, box=box)
    xs = xr + np.array([0.3, -0.45, 0.2])
    xs -= box * np.floor((xs + 0.5 * box) / box)
    st2 = oracle.State(xs, ur, z, st.mass, st.w)
    ne1, te1 = oracle.local_moments(xs[:100], st2, 0.2, box=box)
    np.testing.assert_allclose(ne1, ne0, rtol=1e-12)
    np.testing.assert_allclose(te1, te0, rtol=1e-9, atol=1e-12)
    xc = rng.uniform(-0.2, 0.2, size=(n, 3))
    st3 = oracle.State(xc, ur, z, st.mass, st.w)
    a = oracle.local_moments(xc[:100], st3, 0.2, box=box)
    b = oracle.local_moments(xc[:100], st3, 0.2)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
