"""Thin ctypes binding of the C ABI in ``include/md.h`` (libmd.so).

Argument marshalling only: every step of the hot path runs in the library's
CUDA kernels.  Importing this module loads ``_build/libmd.so`` and raises
``ImportError`` if it is missing (build it with ``paper_1307_3711_gb300.build``
or ``__graft_entry__.build()``); there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

# MD_CHECKED=1 selects the build with device-side bounds checks
_LIB_PATH = _build.LIB_CHECKED if os.environ.get("MD_CHECKED") == "1" else _build.LIB
if not os.path.exists(_LIB_PATH):
    raise ImportError(f"libmd.so not built ({_LIB_PATH}); run paper_1307_3711_gb300.build.build()")
_lib = C.CDLL(_LIB_PATH)

MD_OK, MD_ERR_ARG, MD_ERR_OOM, MD_ERR_CUDA, MD_ERR_TIMEOUT, MD_ERR_NONFINITE, MD_ERR_STATE, \
    MD_ERR_UNSUPPORTED = 0, -1, -2, -3, -4, -5, -6, -7
ENV_GAUSS, ENV_SIN2, ENV_LITERAL_EQ3, ENV_FLAT = 0, 1, 2, 3
BOUNDARY_OPEN, BOUNDARY_PERIODIC, BOUNDARY_MIXED = 0, 1, 2
KIND_ION, KIND_ELECTRON, KIND_INACTIVE = 0, 1, 2


class MDError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"md status {status}: {msg}")
        self.status = status


class Config(C.Structure):
    _fields_ = [("a0", C.c_double), ("tau", C.c_double), ("t0", C.c_double),
                ("dt", C.c_double), ("softening", C.c_double), ("box", C.c_double),
                ("t_switch", C.c_double), ("lambda_um", C.c_double),
                ("polarization", C.c_int32), ("envelope", C.c_int32),
                ("boundary", C.c_int32), ("rate_model", C.c_int32),
                ("ionize_every", C.c_int32), ("zmax", C.c_int32), ("n_ions", C.c_int32),
                ("min_image", C.c_int32), ("slot_base", C.c_int64), ("seed", C.c_uint64),
                ("r_loc", C.c_double), ("r_create", C.c_double),
                ("ip_ev", C.c_double * 16), ("q_outer", C.c_double * 16)]


class Particles(C.Structure):
    _fields_ = [("n", C.c_int64), ("x", C.c_void_p), ("u", C.c_void_p), ("z", C.c_void_p),
                ("mass", C.c_void_p), ("w", C.c_void_p), ("kind", C.c_void_p)]


class Diag(C.Structure):
    _fields_ = [("step", C.c_int64), ("t", C.c_double), ("ke", C.c_double),
                ("ke_ions", C.c_double), ("ke_electrons", C.c_double), ("pe", C.c_double),
                ("total", C.c_double), ("p", C.c_double * 3), ("n_active", C.c_int64),
                ("n_nonfinite", C.c_int64), ("charge_count", C.c_int64 * 16),
                ("charge_weight", C.c_double * 16)]


class Tuning(C.Structure):
    _fields_ = [("threads", C.c_int32), ("r", C.c_int32), ("tile", C.c_int32),
                ("ctas_per_sm", C.c_int32), ("jsplit", C.c_int32), ("packed", C.c_int32),
                ("min_blocks", C.c_int32)]

    def as_tuple(self):
        return (self.threads, self.r, self.tile, self.ctas_per_sm, self.jsplit, self.packed,
                self.min_blocks)


class MlpTrainConfig(C.Structure):
    _fields_ = [("ip_ev", C.c_double * 16), ("q_outer", C.c_double * 16), ("zmax", C.c_int32),
                ("epochs", C.c_int32), ("lambda_um", C.c_double), ("n_samples", C.c_int64),
                ("batch", C.c_int32), ("reserved", C.c_int32), ("lr", C.c_double),
                ("seed", C.c_uint64), ("e_min", C.c_double), ("e_max", C.c_double),
                ("ne_min", C.c_double), ("ne_max", C.c_double), ("te_min", C.c_double),
                ("te_max", C.c_double)]


class DetectorConfig(C.Structure):
    _fields_ = [("radius", C.c_double), ("cone_half_angle_deg", C.c_double),
                ("e_max_ev", C.c_double), ("n_bins", C.c_int32), ("reserved", C.c_int32),
                ("center", C.c_double * 3)]


DETECTORS = ("+x", "-x", "+y", "-y", "all")


class Generate(C.Structure):
    """Mirror of md_generate: seeded records of one cluster (see md.h)."""
    _fields_ = [("r0", C.c_double), ("center", C.c_double * 3), ("ion_mass", C.c_double),
                ("weight", C.c_double), ("kt_e_ev", C.c_double), ("kt_i_ev", C.c_double),
                ("n_ions", C.c_int64), ("n_electrons", C.c_int64), ("n_slots", C.c_int64),
                ("ion_charge", C.c_int32), ("reserved", C.c_int32), ("seed", C.c_uint64)]


def make_generate(r0, n_ions, n_electrons, n_slots=0, ion_charge=1, ion_mass=1.0, weight=1.0,
                  kt_e_ev=0.0, kt_i_ev=0.0, seed=0, center=(0.0, 0.0, 0.0)) -> Generate:
    g = Generate()
    g.r0, g.ion_mass, g.weight, g.kt_e_ev, g.kt_i_ev = r0, ion_mass, weight, kt_e_ev, kt_i_ev
    for k in range(3):
        g.center[k] = center[k]
    g.n_ions, g.n_electrons, g.n_slots = int(n_ions), int(n_electrons), int(n_slots)
    g.ion_charge, g.reserved, g.seed = int(ion_charge), 0, int(seed) & (2 ** 64 - 1)
    return g


class MlpReport(C.Structure):
    _fields_ = [("loss_first", C.c_double), ("loss_last", C.c_double),
                ("holdout_median_dlog10", C.c_double), ("holdout_p99_dlog10", C.c_double),
                ("holdout_max_dlog10", C.c_double), ("train_ms", C.c_double),
                ("n_holdout", C.c_int64), ("steps", C.c_int64)]


_ctx_p = C.c_void_p
_st = C.c_int
_p = C.c_void_p
_SIGS = {
    "md_init": (_st, [C.POINTER(_ctx_p), C.POINTER(Config), C.c_int32, C.POINTER(Particles), _p]),
    "md_init_generate": (_st, [C.POINTER(_ctx_p), C.POINTER(Config), C.POINTER(Generate),
                               C.c_int32, _p]),
    "md_destroy": (None, [_ctx_p]),
    "md_last_error": (C.c_char_p, []),
    "md_step": (_st, [_ctx_p, C.c_int32]),
    "md_sync": (_st, [_ctx_p]),
    "md_diagnostics": (_st, [_ctx_p, C.c_int32, C.POINTER(Diag)]),
    "md_count_active": (_st, [_ctx_p, C.c_int32, C.POINTER(C.c_int64)]),
    "md_step_diag": (_st, [_ctx_p, C.POINTER(Diag)]),
    "md_get_particles": (_st, [_ctx_p, C.c_int32, C.POINTER(Particles)]),
    "md_set_particles": (_st, [_ctx_p, C.c_int32, C.POINTER(Particles)]),
    "md_get_fields": (_st, [_ctx_p, C.c_int32, _p, _p]),
    "md_get_step": (_st, [_ctx_p, C.POINTER(C.c_int64)]),
    "md_set_step": (_st, [_ctx_p, C.c_int64]),
    "md_wait_selftest": (_st, [_ctx_p, C.c_double]),
    "md_set_slice": (_st, [_ctx_p, C.c_int32, C.c_int64, C.c_int64]),
    "md_get_jstream": (_st, [_ctx_p, C.c_int32, C.POINTER(C.c_void_p), C.POINTER(C.c_int64)]),
    "md_ionize": (_st, [_ctx_p]),
    "md_get_ionization": (_st, [_ctx_p, C.c_int32, _p, _p, _p, _p, _p]),
    "md_set_detectors": (_st, [_ctx_p, C.c_int32, C.POINTER(DetectorConfig)]),
    "md_coulomb_field_fp64_device": (_st, [_p, _p, C.c_int64, _p, _p, C.c_int64, C.c_double,
                                           C.c_double, _p, _p, _p]),
    "md_get_iedf": (_st, [_ctx_p, C.c_int32, _p, _p]),
    "md_tuning_list": (C.c_int32, [C.POINTER(Tuning), C.c_int32]),
    "md_plan_shares": (C.c_int, [C.POINTER(C.c_int32), C.c_int32, C.c_int32, C.c_int32,
                                 C.c_int64, C.POINTER(C.c_int32), C.c_int64,
                                 C.POINTER(C.c_int32), C.POINTER(C.c_int64),
                                 C.POINTER(C.c_int64)]),
    "md_set_tuning": (_st, [_ctx_p, C.POINTER(Tuning)]),
    "md_get_tuning": (_st, [_ctx_p, C.POINTER(Tuning)]),
    "md_autotune": (_st, [_ctx_p, C.c_int32, _p, C.c_int32]),
    "md_coulomb_field_device": (_st, [_p, C.c_int64, _p, C.c_int64, C.c_float, C.c_int64, _p,
                                      _p, _p]),
    "md_coulomb_field_device_noalloc": (_st, [_p, C.c_int64, _p, C.c_int64, C.c_float, C.c_int64,
                                              _p, _p, _p]),
    "md_field_device_status": (_st, [_p]),
    "md_field_wait_selftest": (_st, [C.c_double, _p]),
    "md_mlp_train": (_st, [C.POINTER(MlpTrainConfig), _p, C.POINTER(MlpReport), _p]),
    "md_set_rate_mlp": (_st, [_ctx_p, _p, C.POINTER(MlpTrainConfig)]),
    "md_mlp_forward_device": (_st, [_p, _p, C.c_int64, _p, _p]),
    "md_mlp_loss_grad_device": (_st, [_p, _p, _p, _p, C.c_int64, _p, _p, _p]),
    "md_mlp_samples_device": (_st, [C.POINTER(MlpTrainConfig), C.c_int64, C.c_uint64, _p, _p, _p,
                                    _p, _p]),
    "md_ion_rates_device": (_st, [C.POINTER(MlpTrainConfig), C.c_int32, _p, _p, _p, _p, _p,
                                  C.c_int64, _p, _p]),
    "md_coulomb_constant": (C.c_double, [C.c_double]),
    "md_a0_from_intensity": (C.c_double, [C.c_double, C.c_double]),
    "md_n_atoms": (C.c_double, [C.c_double, C.c_double]),
    "md_device_info": (_st, [C.POINTER(C.c_int32), C.c_char_p, C.c_int32]),
    "md_measure_fp32_peak": (_st, [C.POINTER(C.c_double), C.POINTER(C.c_double), _p]),
}
for _name, (_res, _args) in _SIGS.items():
    _fn = getattr(_lib, _name)
    _fn.restype = _res
    _fn.argtypes = _args

# every symbol include/md.h declares
EXPORTED = tuple(_SIGS)


def _check(st: int):
    if st != MD_OK:
        raise MDError(st, _lib.md_last_error().decode())


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def coulomb_constant(lambda_um: float = 0.8) -> float:
    return _lib.md_coulomb_constant(lambda_um)


def a0_from_intensity(intensity_wcm2: float, lambda_um: float) -> float:
    return _lib.md_a0_from_intensity(intensity_wcm2, lambda_um)


def n_atoms(r0: float, r_w: float) -> float:
    return _lib.md_n_atoms(r0, r_w)


def device_info():
    n = C.c_int32(0)
    buf = C.create_string_buffer(256)
    _check(_lib.md_device_info(C.byref(n), buf, 256))
    return int(n.value), buf.value.decode()


def measure_fp32_peak(stream=None):
    """(scalar FFMA, packed f32x2 FMA) lane operations per second of the GPU."""
    v = C.c_double(0)
    t = C.c_double(0)
    _check(_lib.md_measure_fp32_peak(C.byref(v), C.byref(t),
                                     C.c_void_p(stream) if stream else None))
    return float(v.value), float(t.value)


def tuning_list():
    n = _lib.md_tuning_list(None, 0)
    arr = (Tuning * n)()
    _lib.md_tuning_list(arr, n)
    return [t.as_tuple() for t in arr]


def plan_shares(n_pad, per, tile, shares):
    """md_plan_shares (host only): the step kernel's units under equal shares
    for clusters of n_pad records each.  Returns (units [n, 6] int32: cluster,
    i-block, piece, pieces of the i-block, first source, sources; first
    [S + 1] int32: each share's first unit)."""
    n_pad = np.ascontiguousarray(n_pad, dtype=np.int32).ravel()
    nu, ns = C.c_int64(0), C.c_int64(0)
    ip = C.POINTER(C.c_int32)
    _check(_lib.md_plan_shares(n_pad.ctypes.data_as(ip), len(n_pad), per, tile, shares, None, 0,
                               None, C.byref(nu), C.byref(ns)))
    units = np.zeros((nu.value, 6), np.int32)
    first = np.zeros(shares + 1, np.int32)
    _check(_lib.md_plan_shares(n_pad.ctypes.data_as(ip), len(n_pad), per, tile, shares,
                               units.ctypes.data_as(ip), nu.value, first.ctypes.data_as(ip),
                               C.byref(nu), C.byref(ns)))
    return units, first[: ns.value + 1]


class HostParticles:
    """Host arrays of one cluster in the layout md_particles expects; keeps the
    numpy arrays alive while a C struct points at them."""

    def __init__(self, x, u, z, mass, w, kind=None):
        self.x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 3)
        self.u = np.ascontiguousarray(u, dtype=np.float64).reshape(-1, 3)
        self.z = np.ascontiguousarray(z, dtype=np.int32).ravel()
        self.mass = np.ascontiguousarray(mass, dtype=np.float64).ravel()
        self.w = np.ascontiguousarray(w, dtype=np.float64).ravel()
        if kind is None:
            kind = np.where(self.z < 0, KIND_ELECTRON, KIND_ION)
        self.kind = np.ascontiguousarray(kind, dtype=np.uint8).ravel()

    @classmethod
    def empty(cls, n):
        return cls(np.zeros((n, 3)), np.zeros((n, 3)), np.zeros(n, np.int32), np.zeros(n),
                   np.zeros(n), np.zeros(n, np.uint8))

    @classmethod
    def from_cluster(cls, c):
        kind = np.where(c.active == 0, KIND_INACTIVE, np.where(c.z < 0, KIND_ELECTRON, KIND_ION))
        return cls(c.x, c.u, c.z, c.mass, c.w, kind)

    @property
    def n(self):
        return self.x.shape[0]

    def struct(self) -> Particles:
        return Particles(self.n, _ptr(self.x), _ptr(self.u), _ptr(self.z), _ptr(self.mass),
                         _ptr(self.w), _ptr(self.kind))


RATES_NONE, RATES_PLAIN, RATES_MLP = 0, 1, 2


def make_config(a0=0.0, tau=1.0, t0=0.0, dt=0.02, softening=1e-3, box=0.0, t_switch=0.0,
                lambda_um=0.8, polarization=0, envelope=ENV_SIN2,
                boundary=BOUNDARY_OPEN, rate_model=RATES_NONE, ionize_every=0, zmax=0,
                n_ions=0, slot_base=0, seed=0, r_loc=0.0, r_create=0.0, species=None,
                min_image=0) -> Config:
    c = Config()
    c.a0, c.tau, c.t0, c.dt, c.softening = a0, tau, t0, dt, softening
    c.box, c.t_switch, c.lambda_um = box, t_switch, lambda_um
    c.polarization, c.envelope, c.boundary = polarization, envelope, boundary
    c.rate_model, c.ionize_every, c.zmax, c.n_ions = rate_model, ionize_every, zmax, n_ions
    c.min_image, c.slot_base, c.seed = int(min_image), slot_base, seed & (2 ** 64 - 1)
    c.r_loc, c.r_create = r_loc, r_create
    if species is not None:
        for k, v in enumerate(species["ip_ev"]):
            c.ip_ev[k] = v
        for k, v in enumerate(species["q_outer"]):
            c.q_outer[k] = v
    return c


def config_from_workload(w) -> Config:
    """Config of a ``synth.Workload``."""
    return make_config(a0=w.a0, tau=w.tau, t0=w.t0, dt=w.dt, softening=w.eps, box=w.box,
                       t_switch=w.t_switch, lambda_um=w.lambda_um, polarization=w.pol,
                       envelope=w.env, boundary=w.boundary)


class Context:
    """An md_ctx: one or more clusters resident on the GPU."""

    def __init__(self, configs, particles, stream=None):
        configs = list(configs)
        particles = list(particles)
        assert len(configs) == len(particles) and configs
        self._cfgs = (Config * len(configs))(*configs)
        self._parts = (Particles * len(particles))(*[p.struct() for p in particles])
        self._keep = particles
        self.sizes = [p.n for p in particles]
        h = _ctx_p()
        _check(_lib.md_init(C.byref(h), self._cfgs, len(configs), self._parts,
                            C.c_void_p(stream) if stream else None))
        self._h = h

    @classmethod
    def generate(cls, configs, gens, stream=None) -> "Context":
        """A context whose clusters' records are generated on the device
        (md_init_generate) from `gens` (Generate structures)."""
        configs, gens = list(configs), list(gens)
        assert len(configs) == len(gens) and configs
        self = cls.__new__(cls)
        self._cfgs = (Config * len(configs))(*configs)
        self._gens = (Generate * len(gens))(*gens)
        self._keep = []
        self.sizes = [g.n_ions + g.n_electrons + g.n_slots for g in gens]
        h = _ctx_p()
        _check(_lib.md_init_generate(C.byref(h), self._cfgs, self._gens, len(configs),
                                     C.c_void_p(stream) if stream else None))
        self._h = h
        return self

    def close(self):
        if getattr(self, "_h", None):
            _lib.md_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def step(self, nsteps: int = 1):
        _check(_lib.md_step(self._h, int(nsteps)))

    def sync(self):
        _check(_lib.md_sync(self._h))

    def set_slice(self, cluster: int, i_begin: int, i_end: int):
        """Push only the records [i_begin, i_end) of the cluster (see md.h)."""
        _check(_lib.md_set_slice(self._h, int(cluster), int(i_begin), int(i_end)))

    def jstream(self, cluster: int = 0):
        """(device address, n_pad) of the cluster's current j-stream, float4
        records (x, y, z, K_C w z) read by the next step."""
        ptr, n = C.c_void_p(), C.c_int64()
        _check(_lib.md_get_jstream(self._h, int(cluster), C.byref(ptr), C.byref(n)))
        return int(ptr.value or 0), int(n.value)

    def step_index(self) -> int:
        v = C.c_int64(0)
        _check(_lib.md_get_step(self._h, C.byref(v)))
        return int(v.value)

    @staticmethod
    def _diag_dict(d: Diag) -> dict:
        return {"step": d.step, "t": d.t, "ke": d.ke, "ke_ions": d.ke_ions,
                "ke_electrons": d.ke_electrons, "pe": d.pe, "total": d.total,
                "p": np.array(d.p[:]), "n_active": d.n_active, "n_nonfinite": d.n_nonfinite,
                "charge_count": np.array(d.charge_count[:]),
                "charge_weight": np.array(d.charge_weight[:])}

    def diagnostics(self, cluster: int = 0) -> dict:
        d = Diag()
        _check(_lib.md_diagnostics(self._h, cluster, C.byref(d)))
        return self._diag_dict(d)

    def step_diag(self) -> list:
        """One step that also returns every cluster's diagnostics at its start."""
        arr = (Diag * len(self._cfgs))()
        _check(_lib.md_step_diag(self._h, arr))
        return [self._diag_dict(d) for d in arr]

    def get_particles(self, cluster: int = 0, out: HostParticles | None = None) -> HostParticles:
        out = out or HostParticles.empty(self.sizes[cluster])
        s = out.struct()
        _check(_lib.md_get_particles(self._h, cluster, C.byref(s)))
        return out

    def count_active(self, cluster: int = 0) -> int:
        """Records of the cluster that are not INACTIVE (an O(n) count)."""
        v = C.c_int64()
        _check(_lib.md_count_active(self._h, cluster, C.byref(v)))
        return v.value

    def set_particles(self, cluster: int, p: HostParticles):
        s = p.struct()
        _check(_lib.md_set_particles(self._h, cluster, C.byref(s)))

    def fields(self, cluster: int = 0, potential: bool = False):
        n = self.sizes[cluster]
        e = np.zeros((n, 3))
        phi = np.zeros(n) if potential else None
        _check(_lib.md_get_fields(self._h, cluster, _ptr(e), _ptr(phi)))
        return (e, phi) if potential else e

    def set_step(self, step: int):
        _check(_lib.md_set_step(self._h, int(step)))

    def wait_selftest(self, budget_ms: float) -> int:
        """Status of the bounded-wait self-test (MD_ERR_TIMEOUT expected)."""
        return int(_lib.md_wait_selftest(self._h, float(budget_ms)))

    def ionize(self):
        _check(_lib.md_ionize(self._h))

    def ionization(self, cluster: int = 0, n_ions: int | None = None) -> dict:
        n = int(n_ions if n_ions is not None else self._cfgs[cluster].n_ions)
        emag, ne, te, prob = (np.zeros(n) for _ in range(4))
        fired = np.zeros(n, np.uint8)
        _check(_lib.md_get_ionization(self._h, cluster, _ptr(emag), _ptr(ne), _ptr(te),
                                      _ptr(prob), _ptr(fired)))
        return {"emag": emag, "ne": ne, "te": te, "prob": prob, "fired": fired}

    def set_detectors(self, cluster, radius, cone_deg=30.0, e_max_ev=1e4, n_bins=100,
                      center=(0.0, 0.0, 0.0)):
        """Ion energy detectors on the sphere of `radius` (paper units); None
        as radius switches them off."""
        self._det_bins = getattr(self, "_det_bins", {})
        if radius is None:
            _check(_lib.md_set_detectors(self._h, cluster, None))
            self._det_bins.pop(cluster, None)
            return
        d = DetectorConfig(float(radius), float(cone_deg), float(e_max_ev), int(n_bins), 0,
                           (C.c_double * 3)(*center))
        _check(_lib.md_set_detectors(self._h, cluster, C.byref(d)))
        self._det_bins[cluster] = int(n_bins)

    def iedf(self, cluster=0):
        """(detected [5][n_bins + 1], inside [n_bins + 1]) ion counts per energy bin."""
        nb = getattr(self, "_det_bins", {}).get(cluster)
        if nb is None:  # no detectors: the library reports the state error
            _check(_lib.md_get_iedf(self._h, cluster, None, None))
        det = np.zeros((5, nb + 1), np.uint64)
        ins = np.zeros(nb + 1, np.uint64)
        _check(_lib.md_get_iedf(self._h, cluster, _ptr(det), _ptr(ins)))
        return det, ins

    def set_rate_mlp(self, params, domain: "MlpTrainConfig"):
        w = np.ascontiguousarray(params, dtype=np.float32)
        assert w.size == 5000
        _check(_lib.md_set_rate_mlp(self._h, _ptr(w), C.byref(domain)))

    def tuning(self):
        t = Tuning()
        _check(_lib.md_get_tuning(self._h, C.byref(t)))
        return t.as_tuple()

    def set_tuning(self, threads, r, tile, ctas_per_sm=0, jsplit=0, packed=0, min_blocks=-1):
        """md_set_tuning: one of tuning_list()'s configurations; jsplit > 0 that
        many source segments per i-block, 0 a count chosen for balance, -k equal
        shares, k per resident CTA (md_tuning in md.h)."""
        t = Tuning(threads, r, tile, ctas_per_sm, jsplit, packed, min_blocks)
        _check(_lib.md_set_tuning(self._h, C.byref(t)))

    def autotune(self, steps: int = 3):
        n = len(tuning_list())
        times = np.zeros(n)
        _check(_lib.md_autotune(self._h, int(steps), _ptr(times), n))
        return times


def coulomb_field_device(src_ptr: int, ns: int, tgt_ptr: int, nt: int, eps2: float,
                         self_offset: int, e_ptr: int, phi_ptr: int | None, stream: int | None):
    """Stateless field evaluation on caller-owned device buffers (raw device
    addresses, e.g. ``tensor.data_ptr()``)."""
    _check(_lib.md_coulomb_field_device(C.c_void_p(src_ptr), int(ns), C.c_void_p(tgt_ptr),
                                        int(nt), float(eps2), int(self_offset),
                                        C.c_void_p(e_ptr),
                                        C.c_void_p(phi_ptr) if phi_ptr else None,
                                        C.c_void_p(stream) if stream else None))


def coulomb_field_fp64_device(xs_ptr: int, qs_ptr: int, ns: int, xt_ptr: int, self_ptr: int,
                              nt: int, eps: float, kc: float, e_ptr: int, phi_ptr: int = 0,
                              stream=None):
    """FP64 reference direct sum on caller device buffers (see md.h)."""
    _check(_lib.md_coulomb_field_fp64_device(_vp(xs_ptr), _vp(qs_ptr), int(ns), _vp(xt_ptr),
                                             _vp(self_ptr), int(nt), float(eps), float(kc),
                                             _vp(e_ptr), _vp(phi_ptr), _vp(stream)))


def coulomb_field_device_noalloc(src_ptr: int, ns: int, tgt_ptr: int, nt: int, eps2: float,
                                 self_offset: int, e_ptr: int, phi_ptr: int | None,
                                 stream: int | None):
    """As ``coulomb_field_device`` without any device allocation: its scratch
    is a fixed array inside the library (nt <= 32768; overlapping calls race)."""
    _check(_lib.md_coulomb_field_device_noalloc(
        C.c_void_p(src_ptr), int(ns), C.c_void_p(tgt_ptr), int(nt), float(eps2),
        int(self_offset), C.c_void_p(e_ptr), C.c_void_p(phi_ptr) if phi_ptr else None,
        C.c_void_p(stream) if stream else None))


def field_device_status(stream=None) -> int:
    """Status of the stateless field calls on the current device since the
    last query (synchronises `stream`; the sticky error word is cleared).
    Returns MD_OK, MD_ERR_TIMEOUT or MD_ERR_STATE (no exception)."""
    return int(_lib.md_field_device_status(_vp(stream)))


def field_wait_selftest(budget_ms: float, stream=None):
    """Launches a wait that runs out after budget_ms and records it in the
    stateless field calls' error word (see md.h)."""
    _check(_lib.md_field_wait_selftest(float(budget_ms), _vp(stream)))


# ---------------------------------------------------------- rate surrogate --

def mlp_train_config(species, zmax=8, n_samples=1 << 20, epochs=8, batch=8192, lr=3e-3,
                     seed=1, lambda_um=0.8, e_range=(1e-3, 1.0), ne_range=(1e15, 1e24),
                     te_range=(0.1, 1e4)) -> MlpTrainConfig:
    c = MlpTrainConfig()
    for k, v in enumerate(species["ip_ev"]):
        c.ip_ev[k] = v
    for k, v in enumerate(species["q_outer"]):
        c.q_outer[k] = v
    c.zmax, c.epochs, c.lambda_um, c.n_samples = zmax, epochs, lambda_um, n_samples
    c.batch, c.reserved, c.lr, c.seed = batch, 0, lr, seed
    c.e_min, c.e_max = e_range
    c.ne_min, c.ne_max = ne_range
    c.te_min, c.te_max = te_range
    return c


def mlp_train(cfg: MlpTrainConfig, stream=None):
    """Train the surrogate on the GPU; returns (params float32[5000], report dict)."""
    out = np.zeros(5000, np.float32)
    rep = MlpReport()
    _check(_lib.md_mlp_train(C.byref(cfg), _ptr(out), C.byref(rep),
                             C.c_void_p(stream) if stream else None))
    return out, {k: getattr(rep, k) for k, _ in MlpReport._fields_}


def _vp(x):
    return C.c_void_p(x) if x else None


def mlp_forward_device(params_ptr, feats_ptr, n, y_ptr, stream=None):
    _check(_lib.md_mlp_forward_device(_vp(params_ptr), _vp(feats_ptr), int(n), _vp(y_ptr),
                                      _vp(stream)))


def mlp_loss_grad_device(params_ptr, feats_ptr, z_ptr, target_ptr, n, grad_ptr, loss_ptr,
                         stream=None):
    _check(_lib.md_mlp_loss_grad_device(_vp(params_ptr), _vp(feats_ptr), _vp(z_ptr),
                                        _vp(target_ptr), int(n), _vp(grad_ptr), _vp(loss_ptr),
                                        _vp(stream)))


def mlp_samples_device(cfg, n, seed, feats_ptr, z_ptr, target_ptr, raw_ptr=None, stream=None):
    _check(_lib.md_mlp_samples_device(C.byref(cfg), int(n), int(seed) & (2 ** 64 - 1),
                                      _vp(feats_ptr), _vp(z_ptr), _vp(target_ptr), _vp(raw_ptr),
                                      _vp(stream)))


def ion_rates_device(cfg, model, params_ptr, emag_ptr, z_ptr, ne_ptr, te_ptr, n, nu_ptr,
                     stream=None):
    _check(_lib.md_ion_rates_device(C.byref(cfg), int(model), _vp(params_ptr), _vp(emag_ptr),
                                    _vp(z_ptr), _vp(ne_ptr), _vp(te_ptr), int(n), _vp(nu_ptr),
                                    _vp(stream)))
