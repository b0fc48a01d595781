"""FP64 CPU oracle of the laser-cluster MD hot path (arXiv:1307.3711, Sec. II).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` load it; the product
library never does.  It shares no code with the CUDA path.

The arithmetic lives in plain C (``md_oracle.c``; ``ionize_oracle.c`` for
ionization, ``mlp_oracle.c`` for the MLP surrogate, ``generate_oracle.c`` for the
seeded placement of a cluster's records); this module only compiles it with gcc and
marshals numpy arrays through ctypes.  Every function states the passage of the
paper it follows; the readings of silent points are stated in the C sources.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libmd_oracle.so")
# a planted-mistake test compiles a mutant elsewhere and points here
_LIB_OVERRIDE = os.environ.get("MD_ORACLE_LIB")
_SOURCES = ["md_oracle.c", "ionize_oracle.c", "mlp_oracle.c", "generate_oracle.c"]
_lock = threading.Lock()
_lib = None

ENV_GAUSS, ENV_SIN2, ENV_LITERAL_EQ3, ENV_FLAT = 0, 1, 2, 3
BOUNDARY_OPEN, BOUNDARY_PERIODIC, BOUNDARY_MIXED = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile the oracle's C sources into ``_build/libmd_oracle.so`` (gcc, FP64,
    no FMA contraction so x86 and Arm give the same arithmetic)."""
    os.makedirs(_BUILD, exist_ok=True)
    srcs = [os.path.join(_HERE, s) for s in _SOURCES if os.path.exists(os.path.join(_HERE, s))]
    if not force and os.path.exists(_LIB_PATH):
        lib_m = os.path.getmtime(_LIB_PATH)
        if all(os.path.getmtime(s) <= lib_m for s in srcs):
            return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-std=c11", "-o", tmp] + srcs + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Params(C.Structure):
    """Mirror of ``or_params`` in md_oracle.c."""
    _fields_ = [("a0", C.c_double), ("tau", C.c_double), ("t0", C.c_double),
                ("dt", C.c_double), ("eps", C.c_double), ("kc", C.c_double),
                ("box", C.c_double), ("t_switch", C.c_double),
                ("pol", C.c_int), ("env", C.c_int), ("boundary", C.c_int),
                ("min_image", C.c_int)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            if _LIB_OVERRIDE:
                L = C.CDLL(_LIB_OVERRIDE)
            else:
                build()
                L = C.CDLL(_LIB_PATH)
            d, i, i64, p = C.c_double, C.c_int, C.c_int64, C.c_void_p
            L.or_coulomb_constant.restype = d
            L.or_coulomb_constant.argtypes = [d]
            L.or_a0_from_intensity.restype = d
            L.or_a0_from_intensity.argtypes = [d, d]
            L.or_n_atoms.restype = d
            L.or_n_atoms.argtypes = [d, d]
            L.or_envelope.restype = d
            L.or_envelope.argtypes = [d, i, d]
            L.or_laser_fields.restype = None
            L.or_laser_fields.argtypes = [d, d, i, i, d, p, p]
            L.or_coulomb_field.restype = None
            L.or_coulomb_field.argtypes = [i, p, p, i, p, p, d, d, p, p, i]
            L.or_coulomb_field_mi.restype = None
            L.or_coulomb_field_mi.argtypes = [i, p, p, i, p, p, d, d, d, p, p, i]
            L.or_boris_kick.restype = None
            L.or_boris_kick.argtypes = [p, p, p, d, d]
            L.or_drift.restype = None
            L.or_drift.argtypes = [p, p, d]
            L.or_md_steps.restype = None
            L.or_md_steps.argtypes = [i, p, p, p, p, p, C.POINTER(Params), i64, i, p, p, i]
            L.or_diagnostics.restype = None
            L.or_diagnostics.argtypes = [i, p, p, p, p, p, p, p, C.POINTER(Params), i64,
                                         p, p, p, p, i]
            L.or_detect.restype = None
            L.or_detect.argtypes = [i, p, p, p, p, p, p, p, d, d, d, i, p, p]
            L.or_iedf_inside.restype = None
            L.or_iedf_inside.argtypes = [i, p, p, p, p, p, d, i, p]
            L.io_philox4x32_10.restype = None
            L.io_philox4x32_10.argtypes = [p, p, p]
            L.io_uniform_open0.restype = d
            L.io_uniform_open0.argtypes = [C.c_uint32]
            L.io_e1.restype = d
            L.io_e1.argtypes = [d]
            L.io_adk_rate_au.restype = d
            L.io_adk_rate_au.argtypes = [d, d, d]
            L.io_lotz_rate_cgs.restype = d
            L.io_lotz_rate_cgs.argtypes = [d, d, d]
            L.io_rate_total.restype = d
            L.io_rate_total.argtypes = [d, i, d, d, p, p, d]
            L.io_local_moments.restype = None
            L.io_local_moments.argtypes = [i, p, i, p, p, p, p, p, d, d, p, p]
            L.io_local_moments_box.restype = None
            L.io_local_moments_box.argtypes = [i, p, i, p, p, p, p, p, d, d, d, p, p]
            L.mo_nparam.restype = i
            L.mo_nparam.argtypes = []
            L.mo_features.restype = None
            L.mo_features.argtypes = [d, i, d, d, d, d, p]
            L.mo_target.restype = d
            L.mo_target.argtypes = [d]
            L.mo_rate_from_output.restype = d
            L.mo_rate_from_output.argtypes = [d]
            L.mo_forward.restype = None
            L.mo_forward.argtypes = [p, i, p, p]
            L.mo_loss_grad.restype = d
            L.mo_loss_grad.argtypes = [p, i, p, p, p, p]
            L.or_generate_cluster.restype = None
            L.or_generate_cluster.argtypes = [d, p, d, d, d, d, i64, i64, i64, C.c_int32,
                                              C.c_uint64, p, p, p, p, p, p]
            L.io_decide.restype = None
            L.io_decide.argtypes = [i, p, p, p, p, p, p, p, i, d, d, C.c_uint64, i64, d, p, p,
                                    p]
            _lib = L
    return _lib


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p)


# ------------------------------------------------------------------ units ---

def coulomb_constant(lambda_um: float = 0.8) -> float:
    """K_C = r_e k = 2 pi r_e / lambda (Sec. II units; reading of the silent
    Coulomb constant)."""
    return lib().or_coulomb_constant(lambda_um)


def a0_from_intensity(intensity_wcm2: float, lambda_um: float) -> float:
    """Eq. 2."""
    return lib().or_a0_from_intensity(intensity_wcm2, lambda_um)


def n_atoms(r0: float, r_w: float) -> float:
    """Eq. 1."""
    return lib().or_n_atoms(r0, r_w)


def envelope(t: float, kind: int, tau: float) -> float:
    """Eq. 3 and its readings (see md_oracle.c)."""
    return lib().or_envelope(t, kind, tau)


def laser_fields(t: float, a0: float, pol: int, env: int, tau: float):
    """Eqs. 4-9: returns (a, b) as two length-3 arrays."""
    a = np.zeros(3)
    b = np.zeros(3)
    lib().or_laser_fields(t, a0, pol, env, tau, _ptr(a), _ptr(b))
    return a, b


# ------------------------------------------------------------ generation ---

def generate_cluster(r0, n_ions, n_electrons, n_slots=0, ion_charge=1, ion_mass=1.0,
                     weight=1.0, kt_e_ev=0.0, kt_i_ev=0.0, seed=0, center=(0.0, 0.0, 0.0)):
    """Seeded records of one cluster (Sec. II: atoms at random in the sphere
    of radius r0; Eq. 1: macro weight w): ions, electrons, then inactive
    electron slots; positions uniform in the ball by rejection from the cube,
    Maxwellian momenta (generate_oracle.c states the draws).  Returns a dict
    of x, u, z, mass, w, kind."""
    n = int(n_ions) + int(n_electrons) + int(n_slots)
    out = {"x": np.zeros((n, 3)), "u": np.zeros((n, 3)), "z": np.zeros(n, np.int32),
           "mass": np.zeros(n), "w": np.zeros(n), "kind": np.zeros(n, np.uint8)}
    c = _f64(center)
    lib().or_generate_cluster(float(r0), _ptr(c), float(ion_mass), float(weight),
                              float(kt_e_ev), float(kt_i_ev), int(n_ions), int(n_electrons),
                              int(n_slots), int(ion_charge), int(seed) & (2 ** 64 - 1),
                              _ptr(out["x"]), _ptr(out["u"]), _ptr(out["z"]), _ptr(out["mass"]),
                              _ptr(out["w"]), _ptr(out["kind"]))
    return out


# ------------------------------------------------------------ direct sum ---

def coulomb_field(x_targets, x_sources, q_sources, eps, kc, self_idx=None,
                  potential=False, nthreads=1, box=0.0):
    """Softened direct-sum field (and potential) at the targets (Sec. II: the
    Coulomb force of all other charged particles).  ``self_idx[i]`` is the
    source index of target i, excluded from its sum (-1: none).  box > 0:
    minimum-image displacements in the periodic cube of that side."""
    xt = _f64(x_targets, (-1, 3))
    xs = _f64(x_sources, (-1, 3))
    qs = _f64(q_sources).ravel()
    nt, ns = xt.shape[0], xs.shape[0]
    assert qs.shape[0] == ns
    e = np.zeros((nt, 3))
    phi = np.zeros(nt) if potential else None
    si = None
    if self_idx is not None:
        si = np.ascontiguousarray(self_idx, dtype=np.int64)
        assert si.shape[0] == nt
    if box > 0.0:
        lib().or_coulomb_field_mi(nt, _ptr(xt), _ptr(si) if si is not None else None, ns,
                                  _ptr(xs), _ptr(qs), float(eps), float(kc), float(box), _ptr(e),
                                  _ptr(phi) if phi is not None else None, int(nthreads))
    else:
        lib().or_coulomb_field(nt, _ptr(xt), _ptr(si) if si is not None else None, ns,
                               _ptr(xs), _ptr(qs), float(eps), float(kc), _ptr(e),
                               _ptr(phi) if phi is not None else None, int(nthreads))
    return (e, phi) if potential else e


def self_field(x, q, eps, kc, potential=False, nthreads=1, box=0.0):
    """Field of every particle from all the others (box > 0: minimum image)."""
    n = len(q)
    return coulomb_field(x, x, q, eps, kc, np.arange(n, dtype=np.int64),
                         potential=potential, nthreads=nthreads, box=box)


# ----------------------------------------------------------------- Boris ---

def boris_kick(u, e, b, qm, dt):
    """One relativistic Boris kick (Sec. II) of a single particle."""
    u = _f64(u).copy()
    lib().or_boris_kick(_ptr(u), _ptr(_f64(e)), _ptr(_f64(b)), float(qm), float(dt))
    return u


def drift(x, u, dt):
    x = _f64(x).copy()
    lib().or_drift(_ptr(x), _ptr(_f64(u)), float(dt))
    return x


# ------------------------------------------------------------------ steps ---

class State:
    """Particle state in the paper's units: x, u [n,3]; z [n] charge number;
    mass [n] in m_e; w [n] macro weight; active [n] uint8; step index."""

    def __init__(self, x, u, z, mass, w, active=None, step=0):
        self.x = _f64(x, (-1, 3)).copy()
        self.u = _f64(u, (-1, 3)).copy()
        self.z = np.ascontiguousarray(z, dtype=np.int32).copy()
        self.mass = _f64(mass).ravel().copy()
        self.w = _f64(w).ravel().copy()
        n = self.x.shape[0]
        self.active = (np.ones(n, np.uint8) if active is None
                       else np.ascontiguousarray(active, dtype=np.uint8).copy())
        self.step = int(step)

    @property
    def n(self):
        return self.x.shape[0]

    def q(self):
        """Macro charge w z; zero for inactive particles."""
        return np.where(self.active > 0, self.w * self.z, 0.0).astype(np.float64)

    def qm(self):
        return (self.z / self.mass).astype(np.float64)

    def copy(self):
        return State(self.x, self.u, self.z, self.mass, self.w, self.active, self.step)


def make_params(a0=0.0, tau=1.0, t0=0.0, dt=0.02, eps=0.0, kc=None, box=0.0,
                t_switch=0.0, pol=0, env=ENV_SIN2, boundary=BOUNDARY_OPEN,
                lambda_um=0.8, min_image=0):
    if kc is None:
        kc = coulomb_constant(lambda_um)
    return Params(a0, tau, t0, dt, eps, kc, box, t_switch, pol, env, boundary, int(min_image))


def md_steps(state: State, params: Params, nsteps: int, nthreads: int = 1) -> State:
    """Advance ``state`` by nsteps (Sec. II step; order stated in md_oracle.c).
    Modifies and returns ``state``."""
    n = state.n
    qm = state.qm()
    q = state.q()
    e = np.zeros((n, 3))
    si = np.zeros(n, np.int64)
    lib().or_md_steps(n, _ptr(state.x), _ptr(state.u), _ptr(qm), _ptr(q),
                      _ptr(state.active), C.byref(params), state.step, int(nsteps),
                      _ptr(e), _ptr(si), int(nthreads))
    state.step += int(nsteps)
    return state


def diagnostics(state: State, params: Params, nthreads: int = 1) -> dict:
    """Energies and momentum at integer time t_n (u^n from the half-step mean)."""
    n = state.n
    qm = state.qm()
    q = state.q()
    wm = (state.w * state.mass).astype(np.float64)
    e = np.zeros((n, 3))
    phi = np.zeros(n)
    si = np.zeros(n, np.int64)
    out = np.zeros(8)
    lib().or_diagnostics(n, _ptr(state.x), _ptr(state.u), _ptr(qm), _ptr(q), _ptr(wm),
                         _ptr(state.z), _ptr(state.active), C.byref(params), state.step,
                         _ptr(e), _ptr(phi), _ptr(si), _ptr(out), int(nthreads))
    return {"ke": out[0], "ke_ions": out[1], "ke_electrons": out[2], "pe": out[3],
            "p": out[4:7].copy(), "n_active": int(out[7]),
            "total": out[0] + out[3]}


# ------------------------------------------------------------- detectors ---
# Ion energy detectors at a fixed radius (Sec. III, Fig. 3); md_oracle.c.

DETECTORS = ("+x", "-x", "+y", "-y", "all")


class Detectors:
    """Detector sphere (radius, centre), cone half-angle (degrees), energy
    bins [0, e_max_ev) in nbins + overflow; hist[5][nbins + 1] of ion counts
    and the crossed flag of every record."""

    def __init__(self, n, radius, cone_deg=30.0, e_max_ev=1e4, nbins=100, center=(0, 0, 0)):
        self.radius, self.cone_deg, self.e_max_ev, self.nbins = radius, cone_deg, e_max_ev, nbins
        self.center = np.ascontiguousarray(center, dtype=np.float64)
        self.crossed = np.zeros(n, np.uint8)
        self.hist = np.zeros((5, nbins + 1), np.uint64)

    def record(self, x_prev, x_next, state: "State"):
        """Ions of `state` (u = u^{n+1/2}) that crossed between x_prev and x_next."""
        xp = _f64(x_prev, (-1, 3))
        xn = _f64(x_next, (-1, 3))
        lib().or_detect(state.n, _ptr(xp), _ptr(xn), _ptr(state.u), _ptr(state.mass),
                        _ptr(state.z), _ptr(state.active), _ptr(self.center),
                        float(self.radius), float(np.cos(np.radians(self.cone_deg))),
                        float(self.e_max_ev), int(self.nbins), _ptr(self.crossed),
                        _ptr(self.hist))

    def inside(self, state: "State"):
        h = np.zeros(self.nbins + 1, np.uint64)
        lib().or_iedf_inside(state.n, _ptr(state.u), _ptr(state.mass), _ptr(state.z),
                             _ptr(state.active), _ptr(self.crossed), float(self.e_max_ev),
                             int(self.nbins), _ptr(h))
        return h


def md_steps_detected(state: State, params: Params, nsteps: int, det: Detectors,
                      nthreads: int = 1) -> State:
    """md_steps one step at a time, recording detector crossings."""
    for _ in range(nsteps):
        x_prev = state.x.copy()
        md_steps(state, params, 1, nthreads)
        det.record(x_prev, state.x, state)
    return state


# ------------------------------------------------------------- ionization ---
# Sec. II ionization paragraph; arithmetic in ionize_oracle.c.

def philox4x32_10(ctr, key):
    """Philox4x32-10 block: four counter words, two key words -> four words."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, np.uint32)
    lib().io_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def uniform_open0(w):
    return lib().io_uniform_open0(int(w))


def e1(x):
    return lib().io_e1(float(x))


def adk_rate_au(field_au, ip_au, z_residual):
    return lib().io_adk_rate_au(float(field_au), float(ip_au), float(z_residual))


def lotz_rate_cgs(p_ev, t_ev, q):
    return lib().io_lotz_rate_cgs(float(p_ev), float(t_ev), float(q))


def _species(species):
    ip = np.ascontiguousarray(species["ip_ev"], dtype=np.float64)
    q = np.ascontiguousarray(species["q_outer"], dtype=np.float64)
    return ip, q


def rate_total(a_mag, z, ne, te, species, lambda_um=0.8):
    ip, q = _species(species)
    return lib().io_rate_total(float(a_mag), int(z), float(ne), float(te), _ptr(ip), _ptr(q),
                               float(lambda_um))


def local_moments(x_targets, state: "State", r_loc, lambda_um=0.8, box=0.0):
    """(ne [cm^-3], Te [eV]) of the active electrons within r_loc of each target
    (box > 0: nearest periodic images in the cube of that side)."""
    xt = _f64(x_targets, (-1, 3))
    ne = np.zeros(xt.shape[0])
    te = np.zeros(xt.shape[0])
    if box > 0.0:
        lib().io_local_moments_box(xt.shape[0], _ptr(xt), state.n, _ptr(state.x),
                                   _ptr(state.u), _ptr(state.w), _ptr(state.z),
                                   _ptr(state.active), float(r_loc), float(lambda_um), float(box),
                                   _ptr(ne), _ptr(te))
    else:
        lib().io_local_moments(xt.shape[0], _ptr(xt), state.n, _ptr(state.x), _ptr(state.u),
                               _ptr(state.w), _ptr(state.z), _ptr(state.active), float(r_loc),
                               float(lambda_um), _ptr(ne), _ptr(te))
    return ne, te


def decide(ids, z, a_mag, ne, te, species, zmax, seed, step, dt_ion, r_create,
           lambda_um=0.8):
    """Monte-Carlo decision (Sec. II): returns (new z, fired, offsets, P)."""
    ids = np.ascontiguousarray(ids, dtype=np.int64)
    z = np.ascontiguousarray(z, dtype=np.int32).copy()
    a = np.ascontiguousarray(a_mag, dtype=np.float64)
    ne = np.ascontiguousarray(ne, dtype=np.float64)
    te = np.ascontiguousarray(te, dtype=np.float64)
    ip, q = _species(species)
    n = ids.shape[0]
    fired = np.zeros(n, np.uint8)
    off = np.zeros((n, 3))
    prob = np.zeros(n)
    lib().io_decide(n, _ptr(ids), _ptr(z), _ptr(a), _ptr(ne), _ptr(te), _ptr(ip), _ptr(q),
                    int(zmax), float(lambda_um), float(dt_ion), int(seed) & (2 ** 64 - 1),
                    int(step), float(r_create), _ptr(fired), _ptr(off), _ptr(prob))
    return z, fired, off, prob


def next_free_slot(state: "State", slot_base, n_ion, zmax):
    """The record after the last active one in the electron-slot region
    [slot_base, slot_base + zmax n_ion), or slot_base if none is active."""
    region = state.active[slot_base:slot_base + zmax * n_ion]
    act = np.nonzero(region)[0]
    return slot_base + (int(act[-1]) + 1 if act.size else 0)


def ionize_pass(state: "State", params: Params, species, n_ion, slot_base, zmax, seed, dt_ion,
                r_loc, r_create, lambda_um=0.8, nthreads=1):
    """Without minimum-image forces; see ionize_pass_box."""
    return ionize_pass_box(state, params, species, n_ion, slot_base, zmax, seed, dt_ion, r_loc,
                           r_create, lambda_um, nthreads, box=0.0)


def ionize_pass_box(state: "State", params: Params, species, n_ion, slot_base, zmax, seed,
                    dt_ion, r_loc, r_create, lambda_um=0.8, nthreads=1, box=0.0):
    """One ionization pass at step state.step (Sec. II): for each ion record
    i < n_ion (id = i) of charge z < zmax, the field |E_coulomb + a(t_n)| at
    x_i, the local electron moments, the Philox decision; an ionizing ion gets
    z + 1 and frees an electron at x_i + offset with the ion's u and weight.
    The electrons freed in one pass take the next free slots (next_free_slot)
    in the order of their ions' indices.  box > 0: the field and the local
    moments use minimum-image distances in the periodic cube of that side.
    Returns (fired, field_mag, ne, te) of the ions; modifies state."""
    ions = np.arange(n_ion, dtype=np.int64)
    q = state.q()
    e = coulomb_field(state.x[:n_ion], state.x, q, params.eps, params.kc, self_idx=ions,
                      nthreads=nthreads, box=box)
    t = params.t0 + state.step * params.dt
    a, _ = laser_fields(t, params.a0, params.pol, params.env, params.tau)
    amag = np.linalg.norm(e + a[None, :], axis=1)
    ne, te = local_moments(state.x[:n_ion], state, r_loc, lambda_um, box=box)
    z_old = state.z[:n_ion].copy()
    z_new, fired, off, _ = decide(ions, z_old, amag, ne, te, species, zmax, seed, state.step,
                                  dt_ion, r_create, lambda_um)
    slot = next_free_slot(state, slot_base, n_ion, zmax)
    for i in np.nonzero(fired)[0]:
        assert slot < slot_base + zmax * n_ion and state.active[slot] == 0
        state.x[slot] = state.x[i] + off[i]
        state.u[slot] = state.u[i]
        state.z[slot] = -1
        state.mass[slot] = 1.0
        state.w[slot] = state.w[i]
        state.active[slot] = 1
        slot += 1
    state.z[:n_ion] = z_new
    return fired, amag, ne, te


# ------------------------------------------------------------ rate surrogate
# Learned stand-in for the rate evaluation; definition in mlp_oracle.c.

def mlp_nparam():
    return lib().mo_nparam()


def mlp_features(e_mag, z, ne, te, ip_ev, lambda_um=0.8):
    """Surrogate inputs of one ion; ip_ev = ionization energy of charge z."""
    f = np.zeros(4)
    lib().mo_features(float(e_mag), int(z), float(ne), float(te), float(ip_ev),
                      float(lambda_um), _ptr(f))
    return f


def mlp_target(nu):
    return lib().mo_target(float(nu))


def mlp_rate_from_output(y):
    return lib().mo_rate_from_output(float(y))


def mlp_forward(params, feats):
    p = _f64(params).ravel()
    f = _f64(feats, (-1, 4))
    y = np.zeros((f.shape[0], 8))
    lib().mo_forward(_ptr(p), f.shape[0], _ptr(f), _ptr(y))
    return y


def mlp_loss_grad(params, feats, z, target):
    p = _f64(params).ravel()
    f = _f64(feats, (-1, 4))
    zz = np.ascontiguousarray(z, dtype=np.int32)
    t = _f64(target).ravel()
    g = np.zeros(mlp_nparam())
    loss = lib().mo_loss_grad(_ptr(p), f.shape[0], _ptr(f), _ptr(zz), _ptr(t), _ptr(g))
    return loss, g
