"""GPU parity of the CUDA hot path (through the C ABI) against the FP64 oracle.

Field: floored relative error (per target, |E - E64| / max(|E64|, rms|E64|))
with p99 <= 2e-5 for the FP32/Kahan sum.  Trajectories: compared over a few
steps only (chaotic beyond); long runs by energy and momentum.
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_1307_3711_gb300 import synth
from tests.helpers import force_error, summary

pytestmark = pytest.mark.gpu

FORCE_P99 = 2e-5


@pytest.fixture(scope="module")
def md():
    from paper_1307_3711_gb300 import build
    build.build()
    from paper_1307_3711_gb300 import md as m
    return m


def ctx_for(md, w, **kw):
    return md.Context([md.config_from_workload(w)], [md.HostParticles.from_cluster(w.cluster)],
                      **kw)


def oracle_state(c):
    return oracle.State(c.x, c.u, c.z, c.mass, c.w, c.active)


def oracle_params(w, nthreads=1):
    return oracle.make_params(a0=w.a0, tau=w.tau, t0=w.t0, dt=w.dt, eps=w.eps,
                              box=w.box, t_switch=w.t_switch, pol=w.pol, env=w.env,
                              boundary=w.boundary, lambda_um=w.lambda_um)


# ------------------------------------------------------------------ field --

@pytest.mark.parametrize("n_ions,n_el", [(700, 2100), (1, 1), (5, 0), (1500, 1517),
                                         (5003, 15001)])
def test_field_parity_small(md, n_ions, n_el):
    """Several 512-source tiles plus a ragged tail, and degenerate sizes.  At
    20k records the sources are split into segments whose partials are added
    in order (with the potential's self term removed once)."""
    c = synth.make_cluster(3, n_ions, n_el, synth.nm_to_len(3.0), 3, synth.MASS_XE, kT_e_ev=10)
    w = synth.Workload("t", c, a0=0.07, pol=0, env=1, tau=300.0, eps=synth.nm_to_len(0.1),
                       dt=0.02, nsteps=1)
    with ctx_for(md, w) as ctx:
        e, phi = ctx.fields(0, potential=True)
    kc = oracle.coulomb_constant(0.8)
    e64, phi64 = oracle.self_field(c.x, c.w * c.z, w.eps, kc, potential=True,
                                   nthreads=os.cpu_count() or 1)
    if c.n == 1:
        assert np.all(e == 0) and np.all(np.abs(phi) < 1e-12)
        return
    err = force_error(e, e64)
    s = summary(err)
    assert s["p99"] <= FORCE_P99, s
    perr = np.abs(phi - phi64) / np.sqrt(np.mean(phi64 ** 2))
    assert np.percentile(perr, 99) < 2e-5


def test_field_parity_headline_sampled(md):
    """The 200k-particle workload in its benchmarked launch configuration:
    400 sampled targets against the oracle."""
    w = synth.headline_200k(0)
    c = w.cluster
    with ctx_for(md, w) as ctx:
        e = ctx.fields(0)
    rng = np.random.default_rng(5)
    idx = rng.choice(c.n, 400, replace=False)
    kc = oracle.coulomb_constant(0.8)
    e64 = oracle.coulomb_field(c.x[idx], c.x, c.w * c.z, w.eps, kc, self_idx=idx, nthreads=8)
    s = summary(force_error(e[idx], e64))
    assert s["p99"] <= FORCE_P99, s


def test_stateless_field_entry_point(md):
    """md_coulomb_field_device on caller (torch) device buffers; targets that
    are not sources, ragged sizes, and the self term removed from phi."""
    import torch
    rng = np.random.default_rng(9)
    kc = oracle.coulomb_constant(0.8)
    ns, nt = 1237, 777
    xs = rng.normal(size=(ns, 3)) * 0.02
    qs = rng.choice([-1.0, 1.0, 3.0], size=ns)
    xt = rng.normal(size=(nt, 3)) * 0.02
    eps = 1e-3
    src = torch.tensor(np.c_[xs, kc * qs], dtype=torch.float32, device="cuda")
    tgt = torch.tensor(np.c_[xt, np.zeros(nt)], dtype=torch.float32, device="cuda")
    e = torch.zeros((nt, 3), dtype=torch.float64, device="cuda")
    phi = torch.zeros(nt, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    md.coulomb_field_device(src.data_ptr(), ns, tgt.data_ptr(), nt, eps * eps, -1, e.data_ptr(),
                            phi.data_ptr(), stream)
    torch.cuda.synchronize()
    e64, phi64 = oracle.coulomb_field(xt, xs, qs, eps, kc, potential=True)
    assert summary(force_error(e.cpu().numpy(), e64))["p99"] <= FORCE_P99
    np.testing.assert_allclose(phi.cpu().numpy(), phi64, rtol=1e-5,
                               atol=1e-5 * np.abs(phi64).max())
    # targets = sources: self term excluded from phi, zero self force
    e2 = torch.zeros((ns, 3), dtype=torch.float64, device="cuda")
    phi2 = torch.zeros(ns, dtype=torch.float64, device="cuda")
    md.coulomb_field_device(src.data_ptr(), ns, src.data_ptr(), ns, eps * eps, 0, e2.data_ptr(),
                            phi2.data_ptr(), stream)
    torch.cuda.synchronize()
    e64, phi64 = oracle.self_field(xs, qs, eps, kc, potential=True)
    assert summary(force_error(e2.cpu().numpy(), e64))["p99"] <= FORCE_P99
    np.testing.assert_allclose(phi2.cpu().numpy(), phi64, rtol=1e-4,
                               atol=2e-5 * np.abs(phi64).max())
    with pytest.raises(md.MDError):
        md.coulomb_field_device(src.data_ptr() + 4, ns, tgt.data_ptr(), nt, eps * eps, -1,
                                e.data_ptr(), 0, stream)


def test_stateless_field_status_reports_a_timeout(md):
    """The stateless field calls return once launched; a device-side wait that
    runs out is recorded in a sticky per-device word.  A wait that nothing
    completes (50 ms budget) sets it: md_field_device_status reports
    MD_ERR_TIMEOUT once, clears it, and a field call afterwards is clean."""
    import torch
    stream = torch.cuda.current_stream().cuda_stream
    assert md.field_device_status(stream) == md.MD_OK
    md.field_wait_selftest(50.0, stream)
    assert md.field_device_status(stream) == md.MD_ERR_TIMEOUT
    assert md.field_device_status(stream) == md.MD_OK
    src = torch.zeros((64, 4), dtype=torch.float32, device="cuda")
    e = torch.zeros((64, 3), dtype=torch.float64, device="cuda")
    md.coulomb_field_device(src.data_ptr(), 64, src.data_ptr(), 64, 1e-6, 0, e.data_ptr(), 0,
                            stream)
    assert md.field_device_status(stream) == md.MD_OK


def test_stateless_field_few_targets_many_sources(md):
    """md_coulomb_field_device with 300 targets and 200k sources splits the
    sources into segments (stream-ordered partials) and adds them in order:
    the FP64 oracle's field and potential, the self term removed once when
    the targets are sources; the same call gives the same bits twice."""
    import torch
    rng = np.random.default_rng(29)
    kc = oracle.coulomb_constant(0.8)
    ns, nt = 200000, 300
    xs = rng.normal(size=(ns, 3)) * 0.05
    qs = rng.choice([-1.0, 1.0, 2.0], size=ns)
    eps = 1e-3
    src = torch.tensor(np.c_[xs, kc * qs], dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    out = []
    for _ in range(2):
        e = torch.zeros((nt, 3), dtype=torch.float64, device="cuda")
        phi = torch.zeros(nt, dtype=torch.float64, device="cuda")
        md.coulomb_field_device(src.data_ptr(), ns, src.data_ptr(), nt, eps * eps, 0,
                                e.data_ptr(), phi.data_ptr(), stream)
        torch.cuda.synchronize()
        out.append((e.cpu().numpy(), phi.cpu().numpy()))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
    idx = np.arange(nt)
    e64, phi64 = oracle.coulomb_field(xs[:nt], xs, qs, eps, kc, self_idx=idx, potential=True,
                                      nthreads=os.cpu_count() or 1)
    assert summary(force_error(out[0][0], e64))["p99"] <= FORCE_P99
    np.testing.assert_allclose(out[0][1], phi64, rtol=2e-5, atol=2e-5 * np.abs(phi64).max())


def test_stateless_field_calls_on_two_streams_overlap_safely(md):
    """Two split md_coulomb_field_device calls with different sources, issued
    back to back on two streams (their partials in each stream's own
    stream-ordered memory): each result equals the same call made alone."""
    import torch
    rng = np.random.default_rng(30)
    kc = oracle.coulomb_constant(0.8)
    ns, nt = 100000, 500
    srcs = [torch.tensor(np.c_[rng.normal(size=(ns, 3)) * 0.05,
                               kc * rng.choice([-1.0, 1.0], size=ns)],
                         dtype=torch.float32, device="cuda") for _ in range(2)]
    alone = []
    for src in srcs:
        e = torch.zeros((nt, 3), dtype=torch.float64, device="cuda")
        md.coulomb_field_device(src.data_ptr(), ns, src.data_ptr(), nt, 1e-6, 0, e.data_ptr(), 0,
                                torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        alone.append(e.cpu().numpy())
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    outs = [torch.zeros((nt, 3), dtype=torch.float64, device="cuda") for _ in range(2)]
    torch.cuda.synchronize()
    for _ in range(3):
        for src, st, e in zip(srcs, streams, outs):
            md.coulomb_field_device(src.data_ptr(), ns, src.data_ptr(), nt, 1e-6, 0,
                                    e.data_ptr(), 0, st.cuda_stream)
    torch.cuda.synchronize()
    for k in range(2):
        assert np.array_equal(outs[k].cpu().numpy(), alone[k])


def test_stateless_fields_on_empty_and_single_inputs(md):
    """Degenerate sizes of the stateless entry points (FP32/Kahan, allocation
    free, FP64 reference): no sources gives a zero field and potential at
    every target; no targets writes nothing; a lone source that is its own
    target feels nothing; a negative size is an argument error."""
    import torch
    kc = oracle.coulomb_constant(0.8)
    stream = torch.cuda.current_stream().cuda_stream
    src = torch.tensor([[0.01, -0.02, 0.03, kc]], dtype=torch.float32, device="cuda")
    tgt = torch.zeros((5, 4), dtype=torch.float32, device="cuda")
    for fn in (md.coulomb_field_device, md.coulomb_field_device_noalloc):
        e = torch.full((5, 3), float("nan"), dtype=torch.float64, device="cuda")
        phi = torch.full((5,), float("nan"), dtype=torch.float64, device="cuda")
        fn(src.data_ptr(), 0, tgt.data_ptr(), 5, 1e-6, -1, e.data_ptr(), phi.data_ptr(), stream)
        torch.cuda.synchronize()
        assert torch.all(e == 0) and torch.all(phi == 0)
        e.fill_(7.0)
        fn(src.data_ptr(), 1, tgt.data_ptr(), 0, 1e-6, -1, e.data_ptr(), phi.data_ptr(), stream)
        torch.cuda.synchronize()
        assert torch.all(e == 7.0)
        e1 = torch.full((1, 3), float("nan"), dtype=torch.float64, device="cuda")
        phi1 = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        fn(src.data_ptr(), 1, src.data_ptr(), 1, 1e-6, 0, e1.data_ptr(), phi1.data_ptr(), stream)
        torch.cuda.synchronize()
        assert torch.all(e1 == 0) and torch.all(phi1 == 0)
        with pytest.raises(md.MDError) as ei:
            fn(src.data_ptr(), -1, tgt.data_ptr(), 5, 1e-6, -1, e.data_ptr(), 0, stream)
        assert ei.value.status == md.MD_ERR_ARG
    xs = torch.zeros((1, 3), dtype=torch.float64, device="cuda")
    qs = torch.ones(1, dtype=torch.float64, device="cuda")
    xt = torch.ones((5, 3), dtype=torch.float64, device="cuda")
    e = torch.full((5, 3), float("nan"), dtype=torch.float64, device="cuda")
    phi = torch.full((5,), float("nan"), dtype=torch.float64, device="cuda")
    md.coulomb_field_fp64_device(xs.data_ptr(), qs.data_ptr(), 0, xt.data_ptr(), 0, 5, 1e-3, kc,
                                 e.data_ptr(), phi.data_ptr(), stream)
    torch.cuda.synchronize()
    assert torch.all(e == 0) and torch.all(phi == 0)


# ------------------------------------------------------------------ steps --

def test_step_parity_short_2k(md):
    """2k-particle 2 nm case: positions and momenta after 10 steps agree with
    the FP64 oracle (before chaos amplifies the FP32 field error)."""
    w = synth.plain_fp64_2k(0)
    with ctx_for(md, w) as ctx:
        ctx.step(10)
        g = ctx.get_particles(0)
    st = oracle_state(w.cluster)
    oracle.md_steps(st, oracle_params(w), 10, nthreads=4)
    r0 = synth.nm_to_len(2.0)
    assert np.abs(g.x - st.x).max() < 1e-6 * r0
    uscale = np.abs(st.u).max()
    assert np.percentile(np.abs(g.u - st.u).max(1), 99) < 2e-4 * uscale
    assert g.z.tolist() == w.cluster.z.tolist()


def test_diagnostics_parity_and_energy_conservation_2k(md):
    """FP64 diagnostics match the oracle's at step 0; over the 200 steps of the
    2k case with the laser off the GPU conserves energy like the oracle."""
    w = synth.plain_fp64_2k(0)
    w.a0 = 0.0
    with ctx_for(md, w) as ctx:
        d0 = ctx.diagnostics(0)
        st = oracle_state(w.cluster)
        p = oracle_params(w)
        o0 = oracle.diagnostics(st, p)
        scale = abs(o0["pe"])
        assert d0["pe"] == pytest.approx(o0["pe"], rel=1e-5)
        assert abs(d0["ke"] - o0["ke"]) < 1e-5 * scale
        ctx.step(w.nsteps)
        d1 = ctx.diagnostics(0)
        g = ctx.get_particles(0)
    oracle.md_steps(st, p, w.nsteps, nthreads=4)
    o1 = oracle.diagnostics(st, p)
    drift_gpu = abs(d1["total"] - d0["total"]) / d1["ke"]
    drift_cpu = abs(o1["total"] - o0["total"]) / o1["ke"]
    assert drift_gpu < 1.5e-3
    assert drift_gpu < 2 * drift_cpu + 1e-5
    # Newton's third law holds only to FP32 rounding in the per-target sums
    pscale = np.sum(g.w * g.mass * np.linalg.norm(g.u, axis=1))
    assert np.abs(d1["p"] - d0["p"]).max() < 1e-5 * pscale
    assert d1["n_active"] == w.cluster.n and d1["n_nonfinite"] == 0
    assert d1["charge_count"][1] == 1000


@pytest.mark.parametrize("split,packed", [(1, 0), (4, 0), (-4, 0), (1, 1), (-4, 1)])
def test_diagnostic_step_equals_diagnostics_then_step(md, split, packed):
    """md_step_diag sums the potential inside the step's Coulomb pass and takes
    the kinetic energy from the step's own kick: its diagnostics are those of
    md_diagnostics before the step (to FP32 summation order; the oracle's at
    step 0 for the 2k case), and the step it takes leaves the same state bit
    for bit, with one or with 4 source segments per i-block or with 4 equal
    shares per CTA, on the scalar and the packed path, for a context of two
    clusters."""
    ws = [synth.plain_fp64_2k(0), synth.xe3_cluster(30000, seed=9)]
    cfgs = [md.config_from_workload(w) for w in ws]
    out = []
    for fused in (False, True):
        with md.Context(cfgs, [md.HostParticles.from_cluster(w.cluster) for w in ws]) as ctx:
            ctx.set_tuning(128, 4, 512, 0, split, packed)
            ctx.step(3)
            if fused:
                d = ctx.step_diag()
            else:
                d = [ctx.diagnostics(k) for k in range(len(ws))]
                ctx.step(1)
            g = [ctx.get_particles(k) for k in range(len(ws))]
            out.append((d, g, ctx.step_index()))
    (da, ga, sa), (db, gb, sb) = out
    assert sa == sb == 4
    for k in range(len(ws)):
        for f in ("x", "u"):
            assert np.array_equal(getattr(ga[k], f), getattr(gb[k], f)), (k, f)
        assert db[k]["step"] == da[k]["step"] == 3 and db[k]["t"] == da[k]["t"]
        scale = abs(da[k]["pe"]) + da[k]["ke"]
        assert abs(db[k]["pe"] - da[k]["pe"]) < 1e-6 * scale, (k, db[k]["pe"], da[k]["pe"])
        assert abs(db[k]["ke"] - da[k]["ke"]) < 1e-6 * scale, (k, db[k]["ke"], da[k]["ke"])
        pscale = np.sum(ga[k].w * ga[k].mass * np.linalg.norm(ga[k].u, axis=1))
        assert np.abs(db[k]["p"] - da[k]["p"]).max() < 1e-8 * pscale
        assert db[k]["n_active"] == da[k]["n_active"]
        assert np.array_equal(db[k]["charge_count"], da[k]["charge_count"])
    # the 2k case at step 0 against the oracle, through the diagnostic step
    w = ws[0]
    with ctx_for(md, w) as ctx:
        d0 = ctx.step_diag()[0]
    o0 = oracle.diagnostics(oracle_state(w.cluster), oracle_params(w))
    assert d0["pe"] == pytest.approx(o0["pe"], rel=1e-5)
    assert abs(d0["ke"] - o0["ke"]) < 1e-5 * abs(o0["pe"])


def test_diagnostic_step_falls_back_with_detectors(md):
    """With detectors set, md_step_diag is md_diagnostics followed by
    md_step(1): the same numbers and the same state."""
    w = synth.xe3_cluster(4000, seed=10)
    out = []
    for fused in (False, True):
        with ctx_for(md, w) as ctx:
            ctx.set_detectors(0, 5 * synth.nm_to_len(2.0))
            if fused:
                d = ctx.step_diag()[0]
            else:
                d = ctx.diagnostics(0)
                ctx.step(1)
            out.append((d, ctx.get_particles(0)))
    (da, ga), (db, gb) = out
    assert da["pe"] == db["pe"] and da["ke"] == db["ke"]
    assert np.array_equal(ga.x, gb.x) and np.array_equal(ga.u, gb.u)


@pytest.mark.parametrize("pol", [0, 1])
def test_free_electron_light_cone_invariant_gpu(md, pol):
    """One electron in the laser of Eqs. 4-9 (b0 = a0): gamma - u_z = 1 and
    final drift ~ 0 after the sin^2 pulse, as in the oracle."""
    a0, T = 0.5, 40 * math.pi
    c = synth.Cluster(np.zeros((1, 3)), np.zeros((1, 3)), np.array([-1], np.int32), np.ones(1),
                      np.ones(1), np.ones(1, np.uint8))
    w = synth.Workload("e", c, a0=a0, pol=pol, env=1, tau=T, eps=1e-3, dt=0.02, nsteps=0)
    nsteps = int(T / 0.02) + 20
    with ctx_for(md, w) as ctx:
        for k in range(0, nsteps, 500):
            ctx.step(min(500, nsteps - k))
            u = ctx.get_particles(0).u[0]
            g = math.sqrt(1 + u @ u)
            assert abs(g - u[2] - 1) < 5e-4 * a0 ** 2
    st = oracle_state(c)
    oracle.md_steps(st, oracle_params(w), nsteps)
    np.testing.assert_allclose(u, st.u[0], atol=2e-5 * a0)


def test_two_ion_closed_form_gpu(md):
    """Two ions from rest (softening 1e-7 of the separation): t(r) closed form."""
    kc = oracle.coulomb_constant(0.8)
    q1, q2, m1, m2, d = 2, 3, 5000.0, 9000.0, 0.01
    mu = m1 * m2 / (m1 + m2)
    tc = math.sqrt(mu * d ** 3 / (2 * kc * q1 * q2))
    dt = tc / 2000
    f = kc * q1 * q2 / d ** 2
    x = np.array([[0.0, 0, 0], [d, 0, 0]])
    u = np.array([[+0.5 * dt * f / m1, 0, 0], [-0.5 * dt * f / m2, 0, 0]])
    c = synth.Cluster(x, u, np.array([q1, q2], np.int32), np.array([m1, m2]), np.ones(2),
                      np.ones(2, np.uint8))
    w = synth.Workload("2ion", c, a0=0.0, pol=0, env=3, tau=1.0, eps=1e-7 * d, dt=dt, nsteps=0)
    with ctx_for(md, w) as ctx:
        ctx.step(9000)
        g = ctx.get_particles(0)
    xr = (g.x[1, 0] - g.x[0, 0]) / d
    t_pred = tc * (math.sqrt(xr * (xr - 1)) + math.log(math.sqrt(xr) + math.sqrt(xr - 1)))
    assert t_pred == pytest.approx(9000 * dt, rel=1e-5)


# ------------------------------------------------- batching / determinism --

@pytest.mark.parametrize("jsplit", [1, 3])
def test_batched_clusters_equal_single_runs_bitwise(md, jsplit):
    """A parameter scan of uneven clusters in one persistent launch gives
    exactly the per-cluster results of separate contexts (same kernel
    configuration and source split)."""
    scan = synth.batched_scan(6, seed=3, n_min=200, n_max=3000)
    cfgs, parts = [], []
    for e in scan:
        cl = synth.scan_cluster(e)
        cfgs.append(md.make_config(a0=e.a0, tau=e.tau, dt=0.02, softening=synth.nm_to_len(0.1),
                                   envelope=md.ENV_SIN2))
        parts.append(md.HostParticles.from_cluster(cl))
    with md.Context(cfgs, parts) as ctx:
        ctx.set_tuning(128, 4, 256, 0, jsplit, 1)
        ctx.step(20)
        batched = [ctx.get_particles(k) for k in range(len(scan))]
    for k in range(len(scan)):
        with md.Context([cfgs[k]], [parts[k]]) as one:
            one.set_tuning(128, 4, 256, 0, jsplit, 1)
            one.step(20)
            g = one.get_particles(0)
        assert np.array_equal(g.x, batched[k].x)
        assert np.array_equal(g.u, batched[k].u)


def test_graph_replay_equals_direct_launches_and_tunings_agree(md):
    """md_step(n) through the captured graph equals n single-step calls; every
    kernel configuration with the same tile and source split gives identical
    bits, and every configuration agrees with the others to FP32 level."""
    w = synth.xe3_cluster(6000, seed=2)
    with ctx_for(md, w) as a:
        a.step(35)
        ga = a.get_particles(0)
        assert a.step_index() == 35
    with ctx_for(md, w) as b:
        for _ in range(35):
            b.step(1)
        gb = b.get_particles(0)
    assert np.array_equal(ga.x, gb.x) and np.array_equal(ga.u, gb.u)
    r0 = np.abs(w.cluster.x).max()
    first, by_tile = None, {}
    for threads, r, tile, _, _, packed, minb in md.tuning_list():
        for jsplit in (1, 0):
            with ctx_for(md, w) as c:
                c.set_tuning(threads, r, tile, 0, jsplit, packed, minb)
                assert c.tuning()[5] == packed
                c.step(17)
                g = c.get_particles(0)
            first = first or g
            if jsplit == 1:
                # same tile and split: the same sums in the same order, so every
                # configuration (scalar or packed f32x2) gives identical bits
                ref = by_tile.setdefault(tile, g)
                assert np.array_equal(g.x, ref.x) and np.array_equal(g.u, ref.u), \
                    (threads, r, tile, packed, minb)
            assert np.abs(g.x - first.x).max() < 1e-6 * r0


@pytest.mark.parametrize("jsplit", [5, 0, -4])
def test_split_sources_parity_and_determinism(md, jsplit):
    """Splitting the sources into pieces (partial fields in scratch, summed
    by the last piece's CTA) matches the oracle after a few steps and is
    bitwise reproducible: 5 equal segments per i-block, a segment count chosen
    for balance, or equal shares of all tiles (four per resident CTA), which
    at 20k records cut every i-block into several pieces, some of them
    sharing a CTA's share with a piece of the next i-block."""
    w = synth.xe3_cluster(20000, seed=7)
    outs = []
    for _ in range(2):
        with ctx_for(md, w) as c:
            c.set_tuning(256, 4, 256, 0, jsplit, 1)
            t = c.tuning()[4]
            assert t == jsplit if jsplit != 0 else t >= 1
            c.step(6)
            outs.append(c.get_particles(0))
    assert np.array_equal(outs[0].x, outs[1].x) and np.array_equal(outs[0].u, outs[1].u)
    st = oracle_state(w.cluster)
    oracle.md_steps(st, oracle_params(w), 6, nthreads=8)
    r0 = np.abs(w.cluster.x).max()
    assert np.abs(outs[0].x - st.x).max() < 1e-6 * r0
    du = np.abs(outs[0].u - st.u).max(1)
    assert np.percentile(du, 99) < 1e-4 * np.abs(st.u).max()


def test_autotune_restores_state(md):
    w = synth.xe3_cluster(8000, seed=4)
    with ctx_for(md, w) as ctx:
        ctx.step(3)
        before = ctx.get_particles(0)
        times = ctx.autotune(2)
        after = ctx.get_particles(0)
        assert ctx.step_index() == 3
        assert np.all((times > 0) | (times == -1.0)) and np.any(times > 0)
        assert np.array_equal(before.x, after.x) and np.array_equal(before.u, after.u)


def test_set_particles_round_trip(md):
    w = synth.xe3_cluster(3000, seed=6)
    with ctx_for(md, w) as ctx:
        ctx.step(4)
        g = ctx.get_particles(0)
        g.x[:] += 0.001
        ctx.set_particles(0, g)
        h = ctx.get_particles(0)
        assert np.array_equal(g.x, h.x) and np.array_equal(g.u, h.u)
        assert np.array_equal(g.kind, h.kind)


def test_set_particles_rejects_bad_records_on_the_device(md):
    """md_set_particles on a cluster without ionization checks the records on
    the staged device copy: the first bad record is reported with the host
    check's message, and a rejected block leaves the state unchanged."""
    w = synth.xe3_cluster(3000, seed=7)
    with ctx_for(md, w) as ctx:
        ctx.step(2)
        g0 = ctx.get_particles(0)

        def rejected(edit, what):
            g = ctx.get_particles(0)
            edit(g)
            with pytest.raises(md.MDError) as ei:
                ctx.set_particles(0, g)
            assert ei.value.status == md.MD_ERR_ARG and what in str(ei.value), str(ei.value)
            h = ctx.get_particles(0)
            for k in ("x", "u", "z", "mass", "w", "kind"):
                assert np.array_equal(getattr(h, k), getattr(g0, k)), k

        def nan_x(g):
            g.x[2900, 1] = np.nan
        rejected(nan_x, "record 2900: non-finite")

        def inf_w_and_bad_kind(g):
            g.w[1234] = np.inf
            g.kind[2500] = 7
        rejected(inf_w_and_bad_kind, "record 1234: non-finite")

        def electron_sign(g):
            e = int(np.flatnonzero(g.kind == md.KIND_ELECTRON)[5])
            g.z[e] = 1
            g.u[e + 3, 0] = np.nan
        e5 = int(np.flatnonzero(g0.kind == md.KIND_ELECTRON)[5])
        rejected(electron_sign, f"record {e5}: electron with z >= 0")

        def no_mass(g):
            g.mass[17] = 0.0
        rejected(no_mass, "record 17: mass must be > 0")

        def kind_range(g):
            g.kind[0] = 3
        rejected(kind_range, "record 0: bad kind")

        g = ctx.get_particles(0)
        g.x[:] += 0.002
        ctx.set_particles(0, g)
        assert np.array_equal(ctx.get_particles(0).x, g.x)


def test_periodic_boundary_wraps_into_box(md):
    """Sec. II periodic box: positions stay in [-L/2, L/2) and match the oracle
    over a few steps of a hot electron gas."""
    c = synth.make_cluster(8, 200, 600, 0.01, 3, synth.MASS_XE, kT_e_ev=5000.0)
    L = 0.02
    w = synth.Workload("box", c, a0=0.0, pol=0, env=3, tau=1.0, eps=1e-3, dt=0.05, nsteps=0,
                       boundary=1, box=L)
    with ctx_for(md, w) as ctx:
        ctx.step(40)
        g = ctx.get_particles(0)
    assert g.x.min() >= -L / 2 and g.x.max() <= L / 2
    st = oracle_state(c)
    oracle.md_steps(st, oracle_params(w), 40)
    d = np.abs(g.x - st.x)
    d = np.minimum(d, L - d)
    assert np.percentile(d.max(1), 90) < 1e-5 * L


def _box_gas(n_ions, n_el, L, seed):
    """Ions (Xe3+) and electrons uniform over the whole periodic cube, so that
    many pairs meet through the faces."""
    rng = np.random.default_rng(seed)
    n = n_ions + n_el
    x = rng.uniform(-0.5 * L, 0.5 * L, size=(n, 3))
    u = np.r_[np.zeros((n_ions, 3)), rng.normal(size=(n_el, 3)) * 4e-3]
    z = np.r_[np.full(n_ions, 3), np.full(n_el, -1)].astype(np.int32)
    mass = np.r_[np.full(n_ions, synth.MASS_XE), np.ones(n_el)]
    return x, u, z, mass, np.ones(n)


@pytest.mark.parametrize("split,tuning", [(1, (128, 4, 512, 0)), (4, (128, 4, 512, 0)),
                                          (-4, (128, 4, 512, 0)), (1, (128, 8, 256, 1)),
                                          (-4, (128, 8, 256, 1))])
def test_min_image_field_step_and_diagnostics_follow_oracle(md, split, tuning):
    """Periodic cube with minimum-image forces (the optional image forces of
    the periodic boundary, Sec. II): the field and potential, one step's kick
    and drift, and the diagnostics follow the FP64 oracle's minimum-image sums
    for a gas spread over the whole cube (many pairs meet through the faces),
    with one or 4 source segments or equal shares, on the scalar and the
    packed path; a periodic translation of the gas leaves the GPU's field
    unchanged, and the field without image forces differs."""
    L, eps, kc = 0.05, 1e-3, oracle.coulomb_constant(0.8)
    x, u, z, mass, w = _box_gas(1000, 3000, L, 31)
    q = w * z

    def ctx_of(xx, min_image=1, boundary=1, t_switch=0.0):
        cfg = md.make_config(a0=0.02, tau=1.0, dt=0.05, softening=eps, box=L,
                             t_switch=t_switch, envelope=synth.ENV_FLAT, boundary=boundary,
                             min_image=min_image)
        c = md.Context([cfg], [md.HostParticles(xx, u, z, mass, w)])
        c.set_tuning(tuning[0], tuning[1], tuning[2], 0, split, tuning[3])
        return c

    e64, p64 = oracle.self_field(x, q, eps, kc, potential=True, box=L,
                                 nthreads=os.cpu_count() or 1)
    with ctx_of(x) as ctx:
        e, phi = ctx.fields(0, potential=True)
        d = ctx.step_diag()[0]            # falls back to diagnostics + step
        g1 = ctx.get_particles(0)
    err = summary(force_error(e, e64))
    assert err["p99"] <= FORCE_P99, err
    perr = np.abs(phi - p64) / np.sqrt(np.mean(p64 ** 2))
    assert np.percentile(perr, 99) < 2e-5
    e_open = oracle.self_field(x, q, eps, kc)
    assert summary(force_error(e_open, e64))["median"] > 1e-2   # image forces matter here
    # one step against the oracle's minimum-image kick and drift
    a, b = oracle.laser_fields(0.0, 0.02, 0, synth.ENV_FLAT, 1.0)
    du_ref, dx_ref = [], []
    for i in range(len(q)):
        u1 = oracle.boris_kick(u[i], e64[i] + a, b, z[i] / mass[i], 0.05)
        du_ref.append(u1 - u[i])
        x1 = oracle.drift(x[i], u1, 0.05)
        dx_ref.append(x1 - x[i])
    du_ref, dx_ref = np.array(du_ref), np.array(dx_ref)
    dx_gpu = g1.x - x
    dx_gpu -= L * np.round(dx_gpu / L)                 # across the wrap
    assert summary(force_error(g1.u - u, du_ref))["p99"] <= FORCE_P99
    assert summary(force_error(dx_gpu, dx_ref))["p99"] <= FORCE_P99
    # diagnostics against the oracle's minimum-image diagnostics
    st = oracle.State(x, u, z, mass, w)
    o = oracle.diagnostics(st, oracle.make_params(a0=0.02, tau=1.0, dt=0.05, eps=eps, box=L,
                                                  boundary=oracle.BOUNDARY_PERIODIC,
                                                  env=synth.ENV_FLAT, min_image=1))
    assert d["pe"] == pytest.approx(o["pe"], rel=1e-5)
    assert abs(d["ke"] - o["ke"]) < 1e-5 * (abs(o["pe"]) + o["ke"])
    # periodic translation: the same field (up to FP32)
    xs = x + np.array([0.37, -0.21, 0.11]) * L
    xs -= L * np.floor((xs + 0.5 * L) / L)
    with ctx_of(xs) as ctx:
        e2 = ctx.fields(0)
    assert summary(force_error(e2, e64))["p99"] <= FORCE_P99
    # a mixed boundary already open at t = 0, and a cluster without the flag:
    # the open field
    for kw in ({"boundary": 2, "t_switch": -1.0}, {"min_image": 0}):
        with ctx_of(x, **kw) as ctx:
            e3 = ctx.fields(0)
        assert summary(force_error(e3, e_open))["p99"] <= FORCE_P99


@pytest.mark.parametrize("tuning", [(128, 4, 512, 0), (128, 8, 256, 1)])
def test_min_image_skips_tiles_within_half_a_box_bit_for_bit(md, tuning):
    """A compact cluster in a large periodic cube (20 R0, as in Sec. II): no
    pair is half a box apart, so with minimum-image forces every tile takes
    the plain sum and the run equals the run without image forces bit for
    bit (fields and 5 steps), on the scalar and the packed path."""
    w = synth.xe3_cluster(20000, seed=12)
    r0 = float(np.abs(w.cluster.x).max())
    out = []
    for mi in (0, 1):
        cfg = md.config_from_workload(w)
        cfg.boundary, cfg.box, cfg.min_image = 1, 20.0 * r0, mi
        with md.Context([cfg], [md.HostParticles.from_cluster(w.cluster)]) as ctx:
            ctx.set_tuning(tuning[0], tuning[1], tuning[2], 0, 2, tuning[3])
            e = ctx.fields(0)
            ctx.step(5)
            out.append((e, ctx.get_particles(0)))
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1].x, out[1][1].x) and np.array_equal(out[0][1].u, out[1][1].u)


def test_min_image_refuses_tunings_without_its_kernel(md):
    cfg = md.make_config(softening=1e-3, box=0.05, boundary=1, min_image=1)
    x, u, z, mass, w = _box_gas(10, 30, 0.05, 3)
    with md.Context([cfg], [md.HostParticles(x, u, z, mass, w)]) as ctx:
        with pytest.raises(md.MDError) as ei:
            ctx.set_tuning(128, 4, 256, 0, 0, 1)      # packed 128x4: no minimum-image kernel
        assert ei.value.status == md.MD_ERR_ARG
        ctx.set_tuning(128, 8, 256, 0, 0, 1)          # packed 128x8 has one
        ctx.set_tuning(256, 4, 512, 0, 0, 1)


def test_min_image_scalar_and_packed_give_the_same_bits(md):
    """The packed minimum-image reduction takes the scalar one's three rounded
    operations lane by lane: with one tile size (512) and source split, the
    scalar and the packed 256 x 4 configurations step a gas that fills the
    periodic cube identically."""
    L = 0.05
    x, u, z, mass, w = _box_gas(1000, 3000, L, 41)
    cfg = md.make_config(a0=0.02, tau=1.0, dt=0.05, softening=1e-3, box=L,
                         envelope=synth.ENV_FLAT, boundary=1, min_image=1)
    out = []
    for packed in (0, 1):
        with md.Context([cfg], [md.HostParticles(x, u, z, mass, w)]) as ctx:
            ctx.set_tuning(256, 4, 512, 0, 1, packed)
            ctx.step(4)
            out.append(ctx.get_particles(0))
    assert np.array_equal(out[0].x, out[1].x) and np.array_equal(out[0].u, out[1].u)


def test_checkpoint_resume_is_exact(md):
    """A checkpoint (particles + step) restored into a new context continues
    bit-identically, ionization included (Philox is keyed on the step)."""
    n = 600
    c = synth.make_cluster(3, n, 0, synth.nm_to_len(2.0), 0, synth.ARGON["mass"],
                           n_electron_slots=n * 8)
    rw = synth.nm_to_len(synth.ARGON["r_w_nm"])
    cfg = md.make_config(a0=0.1, tau=1.0, dt=0.05, softening=synth.nm_to_len(0.1), envelope=3,
                         rate_model=1, ionize_every=2, zmax=8, n_ions=n, slot_base=n, seed=5,
                         r_loc=3 * rw, r_create=rw, species=synth.ARGON)
    with md.Context([cfg], [md.HostParticles.from_cluster(c)]) as a:
        a.step(13)
        ck = a.get_particles(0)
        a.step(17)
        ref = a.get_particles(0)
    with md.Context([cfg], [md.HostParticles.from_cluster(c)]) as b:
        b.set_particles(0, ck)
        b.set_step(13)
        b.step(17)
        got = b.get_particles(0)
        assert b.step_index() == 30
    assert np.array_equal(got.x, ref.x) and np.array_equal(got.u, ref.u)
    assert np.array_equal(got.z, ref.z) and np.array_equal(got.kind, ref.kind)


def test_bounded_wait_times_out_and_context_survives(md):
    """A device wait that nothing completes returns MD_ERR_TIMEOUT after its
    budget; the context keeps working afterwards."""
    w = synth.xe3_cluster(2000, seed=1)
    with ctx_for(md, w) as ctx:
        assert ctx.wait_selftest(20.0) == md.MD_ERR_TIMEOUT
        ctx.step(3)
        ctx.sync()
        d = ctx.diagnostics(0)
        assert d["step"] == 3 and d["n_nonfinite"] == 0


def test_mixed_boundary_periodic_then_open(md):
    """Mixed boundary (Sec. II): wrapped while t < t_switch, free flight after."""
    c = synth.make_cluster(8, 100, 300, 0.01, 3, synth.MASS_XE, kT_e_ev=5000.0)
    L = 0.02
    w = synth.Workload("mixed", c, a0=0.0, pol=0, env=3, tau=1.0, eps=1e-3, dt=0.05, nsteps=0,
                       boundary=2, box=L, t_switch=1.0)
    with ctx_for(md, w) as ctx:
        ctx.step(19)                 # drifts up to t = 19 dt = 0.95 < t_switch: wrapped
        g1 = ctx.get_particles(0)
        ctx.step(41)                 # open from t = 1.0 on: fast electrons leave the box
        g2 = ctx.get_particles(0)
    assert g1.x.min() >= -L / 2 and g1.x.max() <= L / 2
    assert np.abs(g2.x).max() > L / 2
    st = oracle_state(c)
    oracle.md_steps(st, oracle_params(w), 60)
    assert np.percentile(np.abs(g2.x - st.x).max(1), 90) < 1e-4 * L


@pytest.mark.parametrize("boundary", [1, 2])
def test_free_flight_through_the_faces_closed_form(md, boundary):
    """Sec. II boundaries on free particles (neutral atoms: no force, laser
    off), against the straight line, not the oracle.  Periodic: after every
    step each particle sits at its wrapped line position in [-L/2, L/2).
    Mixed with t_switch = 9.5 dt: wrapped up to x^9; from x^10 on (the wrap of
    x^{n+1} is the one in force at t_{n+1}) the particles fly on unwrapped."""
    rng = np.random.default_rng(21)
    n, L, dt, steps = 64, 1.0, 0.2, 16
    x0 = rng.uniform(-0.5 * L, 0.5 * L, size=(n, 3))
    u0 = rng.normal(size=(n, 3)) * 2.0
    c = synth.Cluster(x0, u0, np.zeros(n, np.int32), np.full(n, 3.0), np.ones(n),
                      np.ones(n, np.uint8), n_ions=n)
    cfg = md.make_config(dt=dt, envelope=synth.ENV_FLAT, boundary=boundary, box=L,
                         t_switch=9.5 * dt)
    line = x0[None] + dt * np.arange(steps + 1)[:, None, None] * (
        u0 / np.sqrt(1.0 + (u0 * u0).sum(1, keepdims=True)))[None]
    wrap = lambda x: x - L * np.floor((x + 0.5 * L) / L)
    with md.Context([cfg], [md.HostParticles.from_cluster(c)]) as ctx:
        for k in range(1, steps + 1):
            ctx.step(1)
            g = ctx.get_particles(0)
            if boundary == 1 or k < 10:
                want = wrap(line[k])
                assert g.x.min() >= -0.5 * L and g.x.max() < 0.5 * L
            else:
                want = wrap(line[9]) + (line[k] - line[9])
            np.testing.assert_allclose(g.x, want, rtol=0, atol=1e-12)
        np.testing.assert_array_equal(g.u, u0)
    if boundary == 2:
        assert np.abs(g.x).max() > 0.5 * L  # some left the box after the switch
        # and some crossed a face during the step that ends after t_switch
        assert (np.floor((line[10] + 0.5 * L) / L) != np.floor((line[9] + 0.5 * L) / L)).any()


def test_fp64_reference_field_matches_oracle_bitwise(md):
    """The FP64 reference direct sum evaluates the oracle's formula in the
    oracle's order with every operation rounded to nearest: the same bits
    (ragged source tiles, self exclusion, uncharged sources skipped)."""
    import torch
    rng = np.random.default_rng(21)
    ns, nt = 3001, 517
    xs = rng.normal(size=(ns, 3)) * 0.01
    qs = rng.choice([-1.0, 0.0, 3.0], size=ns)
    sel = np.sort(rng.choice(ns, nt, replace=False))
    xt = xs[sel]
    self_idx = sel.astype(np.int64)
    self_idx[::7] = -1
    eps, kc = 7.854e-4, oracle.coulomb_constant(0.8)
    d = lambda a: torch.tensor(np.ascontiguousarray(a), device="cuda")
    dxs, dqs, dxt, dsi = d(xs), d(qs), d(xt), d(self_idx)
    e = torch.zeros((nt, 3), dtype=torch.float64, device="cuda")
    phi = torch.zeros(nt, dtype=torch.float64, device="cuda")
    md.coulomb_field_fp64_device(dxs.data_ptr(), dqs.data_ptr(), ns, dxt.data_ptr(),
                                 dsi.data_ptr(), nt, eps, kc, e.data_ptr(), phi.data_ptr())
    torch.cuda.synchronize()
    e_ref, phi_ref = oracle.coulomb_field(xt, xs, qs, eps, kc, self_idx=self_idx,
                                          potential=True)
    assert np.array_equal(e.cpu().numpy(), e_ref)
    assert np.array_equal(phi.cpu().numpy(), phi_ref)


def test_pinned_and_pageable_host_buffers_give_the_same_records(md):
    """md_set_particles / md_get_particles copy page-locked caller arrays
    directly and pageable ones through the staging buffer: same records."""
    import torch
    w = synth.plain_fp64_2k(seed=3)
    hp = md.HostParticles.from_cluster(w.cluster)

    def pinned(a):
        t = torch.empty(a.shape, dtype=getattr(torch, str(a.dtype)), pin_memory=True)
        t.numpy()[...] = a
        return t

    keep = [pinned(getattr(hp, k)) for k in ("x", "u", "z", "mass", "w", "kind")]
    hpp = md.HostParticles(*(t.numpy() for t in keep))
    with md.Context([md.config_from_workload(w)], [hp]) as a, \
            md.Context([md.config_from_workload(w)], [hp]) as b:
        a.set_particles(0, hp)
        b.set_particles(0, hpp)
        a.step(3)
        b.step(3)
        ga = a.get_particles(0)
        outp = md.HostParticles(*(pinned(np.zeros_like(getattr(hp, k))).numpy()
                                  for k in ("x", "u", "z", "mass", "w", "kind")))
        gb = b.get_particles(0, out=outp)
        for k in ("x", "u", "z", "mass", "w", "kind"):
            assert np.array_equal(getattr(ga, k), getattr(gb, k)), k


# ----------------------------------------------- full sizes, bench launch --

def _one_step_sampled(md, clusters, n_sample, seed, autotune=True):
    """One md_step of the given workloads in one context (the configuration the
    autotuner picks, as the bench times it), against the FP64 oracle's field +
    Boris kick + drift at sampled particles of each cluster: the momentum
    increment and the displacement, floored relative error per particle."""
    rng = np.random.default_rng(seed)
    cfgs = [md.config_from_workload(w) for w in clusters]
    parts = [md.HostParticles.from_cluster(w.cluster) for w in clusters]
    errs_u, errs_x = [], []
    with md.Context(cfgs, parts) as ctx:
        if autotune:
            ctx.autotune(2)
        g0 = [ctx.get_particles(k) for k in range(len(clusters))]
        ctx.step(1)
        g1 = [ctx.get_particles(k) for k in range(len(clusters))]
        tuning = ctx.tuning()
    for k, w in enumerate(clusters):
        c = w.cluster
        kc = oracle.coulomb_constant(w.lambda_um)
        q = np.where(g0[k].kind != md.KIND_INACTIVE, g0[k].w * g0[k].z, 0.0)
        idx = np.sort(rng.choice(c.n, min(n_sample, c.n), replace=False))
        e64 = oracle.coulomb_field(g0[k].x[idx], g0[k].x, q, w.eps, kc, self_idx=idx,
                                   nthreads=8)
        a, b = oracle.laser_fields(w.t0, w.a0, w.pol, w.env, w.tau)
        du_ref, dx_ref = [], []
        for m, i in enumerate(idx):
            qm = g0[k].z[i] / g0[k].mass[i]
            u1 = oracle.boris_kick(g0[k].u[i], e64[m] + a, b, qm, w.dt)
            du_ref.append(u1 - g0[k].u[i])
            dx_ref.append(oracle.drift(g0[k].x[i], u1, w.dt) - g0[k].x[i])
        du_ref, dx_ref = np.array(du_ref), np.array(dx_ref)
        errs_u.append(force_error(g1[k].u[idx] - g0[k].u[idx], du_ref))
        errs_x.append(force_error(g1[k].x[idx] - g0[k].x[idx], dx_ref))
    return np.concatenate(errs_u), np.concatenate(errs_x), tuning


def test_step_parity_headline_in_bench_configuration(md):
    """N = 200k (the bench's workload and autotuned launch): the kick of one
    step at 500 sampled particles is the FP64 oracle's within the force gate."""
    eu, ex, tuning = _one_step_sampled(md, [synth.headline_200k(0)], 500, 11)
    print("tuning", tuning, "kick", summary(eu), "drift", summary(ex))
    assert summary(eu)["p99"] <= FORCE_P99
    assert summary(ex)["p99"] <= FORCE_P99


def test_step_parity_precision_1m_sampled(md):
    """N = 1M (500k Ar+ + 500k e): one autotuned step, 200 sampled particles."""
    eu, ex, tuning = _one_step_sampled(md, [synth.precision_1m(0)], 200, 12)
    print("tuning", tuning, "kick", summary(eu), "drift", summary(ex))
    assert summary(eu)["p99"] <= FORCE_P99
    assert summary(ex)["p99"] <= FORCE_P99


def test_step_parity_batched_scan_sampled(md):
    """The 256-cluster scan in one persistent launch: one autotuned step, 8
    sampled particles in each of the 256 clusters."""
    scan = synth.batched_scan(256, seed=0)
    ws = []
    for e in scan:
        ws.append(synth.Workload(f"scan_{e.seed}", synth.scan_cluster(e), a0=e.a0, pol=0,
                                 env=synth.ENV_SIN2, tau=e.tau, eps=synth.nm_to_len(0.1),
                                 dt=0.02, nsteps=0))
    eu, ex, tuning = _one_step_sampled(md, ws, 8, 13)
    print("tuning", tuning, "kick", summary(eu), "drift", summary(ex))
    assert summary(eu)["p99"] <= FORCE_P99
    assert summary(ex)["p99"] <= FORCE_P99


def test_heterogeneous_context_equals_single_runs_bitwise(md):
    """One context with an ionizing argon cluster and a plain cluster with
    detectors (so the step kernel with the detector epilogue runs for both):
    with one source segment per i-block, every record, charge state and
    detector count equals the single-cluster runs of the same clusters.
    (Equal shares cut the sources by the whole context's work, so there a
    cluster's bits depend on the others.)"""
    AR = synth.ARGON
    n = 1200
    ca = synth.make_cluster(2, n, 0, synth.nm_to_len(2.5), 0, AR["mass"],
                            n_electron_slots=8 * n)
    rw = synth.nm_to_len(AR["r_w_nm"])
    ka = md.make_config(a0=0.1, tau=1.0, dt=0.05, softening=synth.nm_to_len(0.1), envelope=3,
                        rate_model=1, ionize_every=2, zmax=8, n_ions=n, slot_base=n,
                        seed=7, r_loc=3 * rw, r_create=rw, species=AR)
    # an exploding ion sphere: its ions reach the detectors within the run
    r0 = synth.nm_to_len(2.0)
    cb = synth.make_cluster(4, 600, 0, r0, 1, synth.MASS_40AMU)
    kcb = oracle.coulomb_constant(0.8)
    tau = math.sqrt(synth.MASS_40AMU * r0 ** 3 / (kcb * 600.0))
    kb = md.make_config(a0=0.0, dt=tau / 40, softening=synth.nm_to_len(0.005),
                        envelope=synth.ENV_FLAT)
    pa = md.HostParticles.from_cluster(ca)
    pb = md.HostParticles.from_cluster(cb)

    def run(cfgs, parts, det_on):
        with md.Context(cfgs, parts) as ctx:
            ctx.set_tuning(128, 4, 512, 0, 1)
            if det_on is not None:
                ctx.set_detectors(det_on, 1.1 * r0, e_max_ev=500.0, n_bins=32)
            ctx.step(40)
            out = [ctx.get_particles(k) for k in range(len(cfgs))]
            det = ctx.iedf(det_on)[0] if det_on is not None else None
        return out, det

    (ga, gb), det_both = run([ka, kb], [pa, pb], 1)
    (sa,), _ = run([ka], [pa], None)
    (sb,), det_b = run([kb], [pb], 0)
    for g, ref in ((ga, sa), (gb, sb)):
        for k in ("x", "u", "z", "kind"):
            assert np.array_equal(getattr(g, k), getattr(ref, k)), k
    assert np.array_equal(det_both, det_b)
    assert ga.z[:n].sum() > 0 and det_b[4].sum() > 0


def _weighted(w, seed):
    """The same workload with macro weights w = N_atoms/N_macro (Eq. 1) drawn in
    [0.5, 3]: charges K_C w z, kinetic energy w m (gamma - 1)."""
    rng = np.random.default_rng(seed)
    w.cluster.w = rng.uniform(0.5, 3.0, w.cluster.n)
    return w


def test_weighted_macroparticles_field_steps_and_diagnostics(md):
    """Non-unit macro weights: the field, 10 steps and the FP64 diagnostics
    agree with the oracle as for unit weights."""
    w = _weighted(synth.plain_fp64_2k(1), 3)
    c = w.cluster
    kc = oracle.coulomb_constant(0.8)
    with ctx_for(md, w) as ctx:
        e = ctx.fields(0)
        d0 = ctx.diagnostics(0)
        ctx.step(10)
        g = ctx.get_particles(0)
        d1 = ctx.diagnostics(0)
    e64 = oracle.self_field(c.x, c.w * c.z, w.eps, kc)
    assert summary(force_error(e, e64))["p99"] <= FORCE_P99
    st = oracle_state(c)
    p = oracle_params(w)
    o0 = oracle.diagnostics(st, p)
    assert d0["pe"] == pytest.approx(o0["pe"], rel=1e-5)
    oracle.md_steps(st, p, 10, nthreads=4)
    o1 = oracle.diagnostics(st, p)
    r0 = synth.nm_to_len(2.0)
    assert np.abs(g.x - st.x).max() < 1e-6 * r0
    assert np.percentile(np.abs(g.u - st.u).max(1), 99) < 2e-4 * np.abs(st.u).max()
    assert np.array_equal(g.w, c.w)
    assert d1["ke"] == pytest.approx(o1["ke"], rel=1e-4)
    assert d1["pe"] == pytest.approx(o1["pe"], rel=1e-4)


def test_weighted_ionization_inputs_and_freed_electron_weight(md):
    """Weighted argon atoms: the local density counts electron weights
    (n_e = sum w / V), and an ionizing atom frees an electron of its weight."""
    AR = synth.ARGON
    n = 800
    c = synth.make_cluster(2, n, 0, synth.nm_to_len(2.5), 0, AR["mass"],
                           n_electron_slots=n * 8)
    rng = np.random.default_rng(6)
    c.w[:n] = rng.uniform(0.5, 3.0, n)
    rw = synth.nm_to_len(AR["r_w_nm"])
    kw = dict(a0=0.1, tau=1.0, dt=0.05, softening=synth.nm_to_len(0.1), envelope=3,
              rate_model=1, ionize_every=0, zmax=8, n_ions=n, slot_base=n, seed=1234567,
              r_loc=3 * rw, r_create=rw, species=AR)
    with md.Context([md.make_config(**kw)], [md.HostParticles.from_cluster(c)]) as ctx:
        ctx.step(10)                     # a0 sin(t): the field is up by t = 0.5
        g0 = ctx.get_particles(0)
        ctx.ionize()
        fired = np.nonzero(ctx.ionization(0)["fired"])[0]
        g1 = ctx.get_particles(0)
        ctx.step(3)
        g2 = ctx.get_particles(0)
        ctx.ionize()
        info = ctx.ionization(0)
    assert len(fired) > 0.1 * n
    # the freed electrons fill the next slots in ion order, each with its atom's weight
    slots = n + np.arange(len(fired))
    assert np.array_equal(g1.kind[slots], np.full(len(fired), md.KIND_ELECTRON, np.uint8))
    assert np.array_equal(g1.w[slots], g0.w[fired])
    st = oracle.State(g2.x, g2.u, g2.z, g2.mass, g2.w,
                      (g2.kind != md.KIND_INACTIVE).astype(np.uint8))
    ne64, te64 = oracle.local_moments(g2.x[:n], st, kw["r_loc"])
    both = (ne64 > 0) & (info["ne"] > 0)
    assert both.sum() > 0.5 * (ne64 > 0).sum()
    same = np.isclose(info["ne"][both], ne64[both], rtol=1e-6)
    assert same.mean() > 0.95


@pytest.mark.parametrize("env,pol", [(synth.ENV_GAUSS, 0), (synth.ENV_GAUSS, 1),
                                     (synth.ENV_LITERAL_EQ3, 0), (synth.ENV_FLAT, 1)])
def test_envelopes_and_polarizations_follow_the_oracle(md, env, pol):
    """One electron through each envelope reading of Eq. 3 (intensity-FWHM
    Gaussian, the printed constant, flat) and both polarizations: the GPU's
    laser and push follow the oracle's trajectory (FP32 kick increments)."""
    a0, tau = 0.2, 30.0
    c = synth.Cluster(np.zeros((1, 3)), np.zeros((1, 3)), np.array([-1], np.int32),
                      np.ones(1), np.ones(1), np.ones(1, np.uint8))
    w = synth.Workload("e", c, a0=a0, pol=pol, env=env, tau=tau, eps=1e-3, dt=0.02, nsteps=0,
                       t0=5.0)
    nsteps = 4000   # t from 5 to 85: the Gaussian peaks at 2 tau = 60
    with ctx_for(md, w) as ctx:
        ctx.step(nsteps)
        g = ctx.get_particles(0)
    st = oracle_state(c)
    oracle.md_steps(st, oracle_params(w), nsteps)
    assert np.abs(st.u[0]).max() > 0.05 * a0          # the pulse did push it
    np.testing.assert_allclose(g.u[0], st.u[0], atol=2e-5 * a0)
    np.testing.assert_allclose(g.x[0], st.x[0], atol=1e-4 * max(1.0, np.abs(st.x[0]).max()))
