"""Seeded synthetic inputs: cluster geometries, charges, masses and thermal
velocities for the workloads of the laser-cluster MD hot path.

This module holds no arithmetic of the method itself (no field, no push, no
rates): it only draws particle records and converts the workload's SI numbers
(nm, fs, eV) into the paper's dimensionless units (Sec. II: length in 1/k, time
in 1/omega, energy in m_e c^2).  Both the CUDA path and the FP64 oracle receive
the same arrays from here.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# physical constants used only for unit conversion of workload parameters
C_LIGHT = 299792458.0            # m/s
AMU_IN_ME = 1822.888486209       # atomic mass unit / electron mass
ME_C2_EV = 510998.95             # electron rest energy in eV

MASS_AR = 39.948 * AMU_IN_ME     # argon ion mass in m_e
MASS_XE = 131.293 * AMU_IN_ME    # xenon ion mass in m_e
MASS_40AMU = 40.0 * AMU_IN_ME

# Wigner-Seitz radii quoted in Sec. II (angstrom): D, Ne, Ar, Xe
R_W_ANGSTROM = {"D": 1.70, "Ne": 2.02, "Ar": 2.40, "Xe": 2.73}

ENV_GAUSS, ENV_SIN2, ENV_LITERAL_EQ3, ENV_FLAT = 0, 1, 2, 3

# Argon ionization data used as input by the ionization runs: ionization
# energies of Ar^z -> Ar^(z+1), z = 0..7 (eV, NIST Atomic Spectra Database,
# rounded), and the number of electrons in the outermost occupied subshell of
# Ar^z (3p^6 ... 3p^1, then 3s^2, 3s^1).
ARGON = {
    "name": "Ar",
    "ip_ev": [15.7596, 27.62967, 40.735, 59.58, 74.84, 91.290, 124.41, 143.4567],
    "q_outer": [6.0, 5.0, 4.0, 3.0, 2.0, 1.0, 2.0, 1.0],
    "mass": MASS_AR,
    "r_w_nm": 0.240,
}

# Xenon ionization data for the Xe runs (Sec. III, the Xe_2600 case, whose
# collisional rates the paper takes from the Lotz formula): ionization energies
# of Xe^z -> Xe^(z+1), z = 0..15 (eV, NIST Atomic Spectra Database, rounded),
# and the electrons in the outermost occupied subshell of Xe^z (5p^6 ... 5p^1,
# then 5s^2, 5s^1, then 4d^10 ... 4d^3).
XENON = {
    "name": "Xe",
    "ip_ev": [12.1298, 20.975, 31.05, 42.20, 54.1, 66.703, 91.6, 105.978,
              179.84, 202.0, 229.02, 255.0, 281.0, 314.0, 343.0, 374.0],
    "q_outer": [6.0, 5.0, 4.0, 3.0, 2.0, 1.0, 2.0, 1.0,
                10.0, 9.0, 8.0, 7.0, 6.0, 5.0, 4.0, 3.0],
    "mass": MASS_XE,
    "r_w_nm": R_W_ANGSTROM["Xe"] / 10.0,
}


def nm_to_len(nm: float, lambda_um: float = 0.8) -> float:
    """Length in nm -> units of 1/k (k = 2 pi / lambda)."""
    return nm * 1e-9 * 2.0 * math.pi / (lambda_um * 1e-6)


def fs_to_time(fs: float, lambda_um: float = 0.8) -> float:
    """Time in fs -> units of 1/omega."""
    return fs * 1e-15 * 2.0 * math.pi * C_LIGHT / (lambda_um * 1e-6)


def sin2_length_from_fwhm(fwhm: float) -> float:
    """Total length T of a sin^2 field envelope whose intensity (sin^4) has the
    given FWHM: sin^4(pi t/T) = 1/2 at pi t/T = asin(2^-1/4)."""
    return math.pi * fwhm / (math.pi - 2.0 * math.asin(2.0 ** -0.25))


def thermal_sigma_u(kT_ev: float, mass_me: float) -> float:
    """Per-component spread of u for a (non-relativistic) Maxwellian."""
    return math.sqrt(kT_ev / (mass_me * ME_C2_EV))


def uniform_sphere(rng: np.random.Generator, n: int, r0: float) -> np.ndarray:
    """n points uniform in the ball of radius r0 centred at the origin
    (Sec. II: atoms placed at random inside the cluster)."""
    v = rng.normal(size=(n, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    r = r0 * rng.random(n) ** (1.0 / 3.0)
    return v * r[:, None]


@dataclass
class Cluster:
    """Particle records of one cluster, in paper units."""
    x: np.ndarray        # [n,3] float64
    u: np.ndarray        # [n,3] float64
    z: np.ndarray        # [n] int32 charge number (-1 electron, 0 neutral/inactive)
    mass: np.ndarray     # [n] float64, m_e
    w: np.ndarray        # [n] float64 macro weight
    active: np.ndarray   # [n] uint8
    n_ions: int = 0
    n_electrons: int = 0

    @property
    def n(self) -> int:
        return int(self.x.shape[0])


def make_cluster(seed: int, n_ions: int, n_electrons: int, r0: float,
                 ion_charge: int, ion_mass: float, kT_e_ev: float = 0.0,
                 kT_i_ev: float = 0.0, weight: float = 1.0,
                 n_electron_slots: int = 0) -> Cluster:
    """Ions first, then electrons, then ``n_electron_slots`` inactive electron
    slots (zero charge, parked at the origin)."""
    rng = np.random.default_rng(seed)
    xi = uniform_sphere(rng, n_ions, r0)
    xe = uniform_sphere(rng, n_electrons, r0)
    ui = rng.normal(size=(n_ions, 3)) * thermal_sigma_u(kT_i_ev, ion_mass) if kT_i_ev > 0 \
        else np.zeros((n_ions, 3))
    ue = rng.normal(size=(n_electrons, 3)) * thermal_sigma_u(kT_e_ev, 1.0) if kT_e_ev > 0 \
        else np.zeros((n_electrons, 3))
    ns = n_electron_slots
    x = np.concatenate([xi, xe, np.zeros((ns, 3))])
    u = np.concatenate([ui, ue, np.zeros((ns, 3))])
    z = np.concatenate([np.full(n_ions, ion_charge, np.int32), np.full(n_electrons, -1, np.int32),
                        np.zeros(ns, np.int32)])
    mass = np.concatenate([np.full(n_ions, ion_mass), np.ones(n_electrons), np.ones(ns)])
    w = np.full(n_ions + n_electrons + ns, float(weight))
    active = np.concatenate([np.ones(n_ions + n_electrons, np.uint8), np.zeros(ns, np.uint8)])
    return Cluster(x, u, z, mass, w, active, n_ions, n_electrons)


@dataclass
class Workload:
    """One cluster run: physics parameters in paper units + the particles."""
    name: str
    cluster: Cluster
    a0: float
    pol: int
    env: int
    tau: float           # FWHM (gauss) or total length T (sin2), 1/omega
    eps: float
    dt: float
    nsteps: int
    t0: float = 0.0
    lambda_um: float = 0.8
    boundary: int = 0
    box: float = 0.0
    t_switch: float = 0.0
    extra: dict = field(default_factory=dict)


def plain_fp64_2k(seed: int = 0) -> Workload:
    """1,000 singly charged 40-amu ions + 1,000 electrons at rest, uniform in a
    2 nm sphere; softening 0.1 nm; a0 = 0.05 linear, sin^2 over 20 cycles;
    dt = 0.02; 200 steps."""
    c = make_cluster(seed, 1000, 1000, nm_to_len(2.0), 1, MASS_40AMU)
    return Workload("ar1k_e1k_r2nm", c, a0=0.05, pol=0, env=ENV_SIN2, tau=40.0 * math.pi,
                    eps=nm_to_len(0.1), dt=0.02, nsteps=200)


def xe3_cluster(n_total: int, seed: int = 0, r0_nm: float | None = None) -> Workload:
    """Xe-like cluster, ions of fixed charge +3 and three electrons per ion,
    electrons Maxwellian at 10 eV, ions at rest, at the density of 100k ions in
    a 10 nm sphere unless r0_nm is given; a0 = 0.07 linear, sin^2 envelope of
    100 fs intensity FWHM; softening 0.1 nm; dt = 0.02."""
    n_ions = n_total // 4
    n_el = 3 * n_ions
    if r0_nm is None:
        r0_nm = 10.0 * (n_ions / 100000.0) ** (1.0 / 3.0)
    c = make_cluster(seed, n_ions, n_el, nm_to_len(r0_nm), 3, MASS_XE, kT_e_ev=10.0)
    return Workload(f"xe3_{n_ions // 1000}k_e{n_el // 1000}k_r{r0_nm:.2f}nm", c, a0=0.07,
                    pol=0, env=ENV_SIN2, tau=sin2_length_from_fwhm(fs_to_time(100.0)),
                    eps=nm_to_len(0.1), dt=0.02, nsteps=2000)


def headline_200k(seed: int = 0) -> Workload:
    """The N = 200,000 throughput workload: 50k Xe3+ + 150k electrons at the
    density of the 400k-particle Xe case (R0 = 10 nm * 0.5^(1/3))."""
    return xe3_cluster(200000, seed)


def precision_1m(seed: int = 0, a0: float = 0.0) -> Workload:
    """500k singly charged 40-amu ions + 500k electrons, R0 = 15 nm; laser off
    (a0 = 0) for the drift test, a0 = 0.1 for the driven run."""
    c = make_cluster(seed, 500000, 500000, nm_to_len(15.0), 1, MASS_40AMU)
    return Workload("ar500k_e500k_r15nm", c, a0=a0, pol=0, env=ENV_SIN2,
                    tau=sin2_length_from_fwhm(fs_to_time(100.0)), eps=nm_to_len(0.1),
                    dt=0.02, nsteps=200)


@dataclass
class ScanEntry:
    n_total: int
    z: int
    n_ions: int
    n_electrons: int
    r0: float
    a0: float
    tau: float
    seed: int


def batched_scan(n_clusters: int = 256, seed: int = 0, n_min: int = 1000,
                 n_max: int = 50000) -> list[ScanEntry]:
    """Parameter scan draw: N log-uniform in [n_min, n_max], Z uniform in 1..8,
    n_i = round(N/(1+Z)), n_e = Z n_i, R0 uniform 1-8 nm, a0 log-uniform
    0.01-0.3, intensity FWHM uniform 20-200 fs (sin^2 envelope)."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n_clusters):
        n = int(round(math.exp(rng.uniform(math.log(n_min), math.log(n_max)))))
        z = int(rng.integers(1, 9))
        ni = max(1, int(round(n / (1 + z))))
        r0 = nm_to_len(rng.uniform(1.0, 8.0))
        a0 = math.exp(rng.uniform(math.log(0.01), math.log(0.3)))
        tau = sin2_length_from_fwhm(fs_to_time(rng.uniform(20.0, 200.0)))
        out.append(ScanEntry(ni * (1 + z), z, ni, z * ni, r0, a0, tau, seed * 100003 + k + 1))
    return out


def scan_cluster(e: ScanEntry) -> Cluster:
    return make_cluster(e.seed, e.n_ions, e.n_electrons, e.r0, e.z, MASS_40AMU)


def neutral_ar_200k(seed: int = 0, n_atoms: int = 200000, zmax: int = 8,
                    r0_nm: float = 8.0) -> Cluster:
    """Neutral argon cluster with one inactive electron slot per possible
    ionization (zmax per atom)."""
    return make_cluster(seed, n_atoms, 0, nm_to_len(r0_nm), 0, MASS_AR,
                        n_electron_slots=n_atoms * zmax)


def ar_ionize(seed: int = 0, n_atoms: int = 200000) -> Workload:
    """Neutral argon cluster at the density of 200k atoms in an 8 nm sphere
    (R0 = 8 nm (n_atoms / 200000)^(1/3)), 8 inactive electron slots per atom,
    806 nm pulse of 8e15 W/cm^2 (a0 = 0.0617) with a 100 fs sin^2 envelope.
    The run starts 0.3 rad before the field crest nearest the envelope peak
    (a_x = a0 env(t) sin t), so its first steps ionize.  extra holds the
    ionization settings in paper units: zmax, the radius r_loc = 3 R_W of the
    local electron moments and the radius r_create = R_W of the ball a freed
    electron is placed in."""
    lam = 0.806
    c = make_cluster(seed, n_atoms, 0, nm_to_len(8.0 * (n_atoms / 200000) ** (1 / 3), lam), 0,
                     ARGON["mass"], n_electron_slots=8 * n_atoms)
    rw = nm_to_len(ARGON["r_w_nm"], lam)
    tau = sin2_length_from_fwhm(fs_to_time(100.0, lam))
    t0 = math.floor(tau / 2 / math.pi) * math.pi + 0.5 * math.pi - 0.3
    return Workload(f"ar{n_atoms // 1000}k_ionize", c, a0=0.0617, pol=0, env=ENV_SIN2, tau=tau,
                    eps=nm_to_len(0.1, lam), dt=0.02, nsteps=0, t0=t0, lambda_um=lam,
                    extra={"zmax": 8, "r_loc": 3 * rw, "r_create": rw})
