"""The C ABI library builds for sm_103a, loads, exports every symbol
include/md.h declares, and rejects bad arguments on the host (no GPU needed:
no compute call is made here)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import oracle
from paper_1307_3711_gb300 import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def md():
    build.build()
    from paper_1307_3711_gb300 import md as m
    return m


def header_symbols():
    txt = open(os.path.join(ROOT, "include", "md.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(md_[a-z0-9_]+)\s*\(", txt)))


def test_library_exports_every_declared_symbol(md):
    lib = C.CDLL(build.LIB)
    syms = header_symbols()
    assert len(syms) >= 15
    for s in syms:
        assert hasattr(lib, s), s
    assert set(syms) == set(md.EXPORTED)


def test_si_helpers_match_oracle(md):
    """Eqs. 1-2 and K_C on the library side agree with the oracle's own code."""
    for lam in (0.4, 0.8, 1.06):
        assert md.coulomb_constant(lam) == pytest.approx(oracle.coulomb_constant(lam), rel=1e-15)
    assert md.a0_from_intensity(1e16, 0.8) == pytest.approx(oracle.a0_from_intensity(1e16, 0.8),
                                                            rel=1e-15)
    assert md.n_atoms(82.0, 2.4) == pytest.approx(oracle.n_atoms(82.0, 2.4), rel=1e-15)


def test_tuning_list(md):
    lst = md.tuning_list()
    assert len(lst) >= 4
    for threads, r, tile, _, _, packed, minb in lst:
        assert threads % 32 == 0 and r >= 1 and tile % 16 == 0
        assert packed in (0, 1) and (not packed or r % 2 == 0)
        assert minb >= 0
    assert any(t[5] for t in lst) and any(not t[5] for t in lst)


def _one(md, **kw):
    p = md.HostParticles(np.zeros((2, 3)), np.zeros((2, 3)), [1, -1], [1000.0, 1.0], [1.0, 1.0])
    return md.make_config(**kw), p


@pytest.mark.parametrize("kw,what", [
    ({"dt": 0.0}, "dt"), ({"softening": 0.0}, "softening"), ({"lambda_um": -1.0}, "lambda"),
    ({"polarization": 2}, "polarization"), ({"envelope": 9}, "envelope"),
    ({"boundary": 1, "box": 0.0}, "box"), ({"tau": 0.0, "envelope": 1}, "tau"),
    ({"softening": 1e-30}, "softening"), ({"a0": float("nan")}, "finite"),
    ({"t0": float("inf")}, "finite"),
    ({"min_image": 2}, "min_image"), ({"min_image": 1}, "periodic or mixed boundary"),
])
def test_init_rejects_bad_config_on_host(md, kw, what):
    cfg, p = _one(md, **kw)
    with pytest.raises(md.MDError) as ei:
        md.Context([cfg], [p])
    assert ei.value.status == md.MD_ERR_ARG
    assert what in str(ei.value)


def test_init_rejects_inconsistent_particles(md):
    cfg = md.make_config()
    p = md.HostParticles(np.zeros((2, 3)), np.zeros((2, 3)), [1, 1], [1000.0, 1.0], [1.0, 1.0],
                         kind=[0, 1])
    with pytest.raises(md.MDError) as ei:
        md.Context([cfg], [p])
    assert ei.value.status == md.MD_ERR_ARG
    p = md.HostParticles(np.zeros((2, 3)), np.zeros((2, 3)), [1, -1], [0.0, 1.0], [1.0, 1.0])
    with pytest.raises(md.MDError):
        md.Context([cfg], [p])
    x = np.zeros((2, 3))
    x[1, 2] = np.nan
    p = md.HostParticles(x, np.zeros((2, 3)), [1, -1], [1000.0, 1.0], [1.0, 1.0])
    with pytest.raises(md.MDError) as ei:
        md.Context([cfg], [p])
    assert "non-finite" in str(ei.value)


def test_init_rejects_an_empty_cluster(md):
    """A cluster of no records is an argument error, found on the host."""
    cfg = md.make_config()
    p = md.HostParticles(np.zeros((0, 3)), np.zeros((0, 3)), np.zeros(0, np.int32),
                         np.zeros(0), np.zeros(0))
    with pytest.raises(md.MDError) as ei:
        md.Context([cfg], [p])
    assert ei.value.status == md.MD_ERR_ARG
    assert "n must be >= 1" in str(ei.value)


def test_init_without_gpu_fails_cleanly(md):
    """Valid arguments but no usable GPU: a CUDA error status, not a crash."""
    from tests.helpers import has_gpu
    if has_gpu():
        pytest.skip("a GPU is present")
    cfg, p = _one(md)
    with pytest.raises(md.MDError) as ei:
        md.Context([cfg], [p])
    assert ei.value.status in (md.MD_ERR_CUDA, md.MD_ERR_UNSUPPORTED)


def test_generate_rejects_bad_parameters(md):
    """md_init_generate checks its md_generate and the ionization settings
    against the generated record order on the host, before any GPU work."""
    from tests.test_gpu_generate import GENS, _configs
    cfg = _configs(md)[:1]
    bad = [dict(GENS[0], r0=0.0), dict(GENS[0], ion_mass=-1.0), dict(GENS[0], weight=0.0),
           dict(GENS[0], kt_e_ev=-1.0), dict(GENS[0], n_ions=0, n_electrons=0, n_slots=0),
           dict(GENS[0], ion_charge=-1)]
    for b in bad:
        with pytest.raises(md.MDError) as ei:
            md.Context.generate(cfg, [md.make_generate(**b)])
        assert ei.value.status == md.MD_ERR_ARG
    # ionization settings the generated records cannot hold: 1500 atoms need
    # 12000 slots for zmax = 8
    ion = _configs(md, True)[1]
    with pytest.raises(md.MDError) as ei:
        md.Context.generate([ion], [md.make_generate(**dict(GENS[1], n_slots=11999))])
    assert ei.value.status == md.MD_ERR_ARG
