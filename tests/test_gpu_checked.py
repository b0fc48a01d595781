"""The checked build (-DMD_CHECKED: device-side bounds checks that record an
error instead of accessing memory out of range) on scenarios that exercise
every checked access: split sources, ionization with slot assignment and the
local moments' cell list, detectors, a multi-cluster scan with segments and
with equal shares, and graph replay.  It must report no bounds
error and give the same bits as the normal build."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCENARIO = r"""
import hashlib, math, sys
import numpy as np
sys.path.insert(0, sys.argv[1])
from paper_1307_3711_gb300 import md, synth
AR = synth.ARGON
h = hashlib.sha256()
def feed(g):
    for k in ("x", "u", "z", "kind"):
        h.update(np.ascontiguousarray(getattr(g, k)).tobytes())
# ionizing argon cluster + exploding ion sphere with detectors, split sources
n = 1500
ca = synth.make_cluster(2, n, 0, synth.nm_to_len(2.5), 0, AR["mass"], n_electron_slots=8 * n)
rw = synth.nm_to_len(AR["r_w_nm"])
ka = md.make_config(a0=0.1, tau=1.0, dt=0.05, softening=synth.nm_to_len(0.1), envelope=3,
                    rate_model=1, ionize_every=1, zmax=8, n_ions=n, slot_base=n, seed=7,
                    r_loc=3 * rw, r_create=rw, species=AR)
r0 = synth.nm_to_len(2.0)
cb = synth.make_cluster(4, 700, 0, r0, 1, synth.MASS_40AMU)
tau = math.sqrt(synth.MASS_40AMU * r0 ** 3 / (md.coulomb_constant(0.8) * 700.0))
kb = md.make_config(a0=0.0, dt=tau / 40, softening=synth.nm_to_len(0.005),
                    envelope=synth.ENV_FLAT)
with md.Context([ka, kb], [md.HostParticles.from_cluster(ca),
                           md.HostParticles.from_cluster(cb)]) as ctx:
    ctx.set_tuning(128, 4, 512, 0, 3)
    ctx.set_detectors(1, 1.2 * r0, e_max_ev=500.0, n_bins=16)
    ctx.step(37)                      # two graph replays of 16 + 5 direct steps
    for k in range(2):
        feed(ctx.get_particles(k))
    det, ins = ctx.iedf(1)
    h.update(det.tobytes()); h.update(ins.tobytes())
    d = ctx.diagnostics(0)
    assert d["charge_count"][1:].sum() > 0 and det[4].sum() > 0
# a scan of 24 uneven clusters in one launch, packed path
ws = []
for e in synth.batched_scan(24, seed=3, n_max=8000):
    ws.append(synth.Workload("s", synth.scan_cluster(e), a0=e.a0, pol=0, env=synth.ENV_SIN2,
                             tau=e.tau, eps=synth.nm_to_len(0.1), dt=0.02, nsteps=0))
with md.Context([md.config_from_workload(w) for w in ws],
                [md.HostParticles.from_cluster(w.cluster) for w in ws]) as ctx:
    ctx.set_tuning(128, 4, 256, 0, 0, 1)
    ctx.step(3)
    for k in range(len(ws)):
        feed(ctx.get_particles(k))
    # the same scan with equal shares (pieces that cross i-blocks and clusters)
    ctx.set_tuning(128, 8, 256, 0, -4, 1)
    ctx.step(3)
    for k in range(len(ws)):
        feed(ctx.get_particles(k))
print("DIGEST", h.hexdigest())
"""


def _run(env_extra):
    env = dict(os.environ, **env_extra)
    r = subprocess.run([sys.executable, "-c", SCENARIO, ROOT], capture_output=True, text=True,
                       timeout=600, env=env, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-3000:]
    return [ln for ln in r.stdout.splitlines() if ln.startswith("DIGEST")][0]


def test_checked_build_reports_no_bounds_error_and_same_bits():
    from paper_1307_3711_gb300 import build
    build.build()
    build.build(checked=True)
    checked = _run({"MD_CHECKED": "1"})
    plain = _run({"MD_CHECKED": "0"})
    assert checked == plain
