"""FP64 CPU oracle of the laser-cluster MD hot path (arXiv:1307.3711, Sec. II).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` load it; the product
library never does.  It shares no code with the CUDA path.

The arithmetic lives in plain C (``md_oracle.c`` and, for ionization and the MLP
surrogate, ``ionize_oracle.c``); this module only compiles it with gcc and
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
_SOURCES = ["md_oracle.c"]
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
                ("pad", C.c_int)]


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
            L.or_boris_kick.restype = None
            L.or_boris_kick.argtypes = [p, p, p, d, d]
            L.or_drift.restype = None
            L.or_drift.argtypes = [p, p, d]
            L.or_md_steps.restype = None
            L.or_md_steps.argtypes = [i, p, p, p, p, p, C.POINTER(Params), i64, i, p, p, i]
            L.or_diagnostics.restype = None
            L.or_diagnostics.argtypes = [i, p, p, p, p, p, p, p, C.POINTER(Params), i64,
                                         p, p, p, p, i]
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


# ------------------------------------------------------------ direct sum ---

def coulomb_field(x_targets, x_sources, q_sources, eps, kc, self_idx=None,
                  potential=False, nthreads=1):
    """Softened direct-sum field (and potential) at the targets (Sec. II: the
    Coulomb force of all other charged particles).  ``self_idx[i]`` is the
    source index of target i, excluded from its sum (-1: none)."""
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
    lib().or_coulomb_field(nt, _ptr(xt), _ptr(si) if si is not None else None, ns,
                           _ptr(xs), _ptr(qs), float(eps), float(kc), _ptr(e),
                           _ptr(phi) if phi is not None else None, int(nthreads))
    return (e, phi) if potential else e


def self_field(x, q, eps, kc, potential=False, nthreads=1):
    """Field of every particle from all the others."""
    n = len(q)
    return coulomb_field(x, x, q, eps, kc, np.arange(n, dtype=np.int64),
                         potential=potential, nthreads=nthreads)


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
                lambda_um=0.8):
    if kc is None:
        kc = coulomb_constant(lambda_um)
    return Params(a0, tau, t0, dt, eps, kc, box, t_switch, pol, env, boundary, 0)


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
