"""One cluster split by target records (md_set_slice) on one GPU: two contexts
push the two halves of a 20k-record cluster and hand each other their slices
of the j-stream (md_get_jstream) after every step, as ranks on two GPUs do
with an all-gather.  With the same kernel configuration and source split as an
unsplit context, every record's state matches it bit for bit; the slices'
diagnostics add up to the cluster's."""
import numpy as np
import pytest

from paper_1307_3711_gb300 import synth
from tests.helpers import force_error, summary

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def md():
    from paper_1307_3711_gb300 import build
    build.build()
    from paper_1307_3711_gb300 import md as m
    return m


def _ctx(md, w, jsplit):
    ctx = md.Context([md.config_from_workload(w)], [md.HostParticles.from_cluster(w.cluster)])
    ctx.set_tuning(128, 4, 512, 0, jsplit, 0)
    return ctx


@pytest.mark.parametrize("jsplit", [1, 3])
def test_two_slices_step_like_the_whole_cluster(md, jsplit):
    import torch
    from paper_1307_3711_gb300 import shard
    w = synth.xe3_cluster(20000, seed=3)
    n = w.cluster.n
    b1 = shard.slice_bounds(n, 2, 1)[0]
    whole, lo, hi = _ctx(md, w, jsplit), _ctx(md, w, jsplit), _ctx(md, w, jsplit)
    lo.set_slice(0, 0, b1)
    hi.set_slice(0, b1, n)
    for _ in range(5):
        for c in (whole, lo, hi):
            c.step(1)
        jl, jh = shard.jstream_tensor(lo), shard.jstream_tensor(hi)
        jl[b1:] = jh[b1:]
        jh[:b1] = jl[:b1]
        torch.cuda.synchronize()
    ref = whole.get_particles(0)
    pl, ph = lo.get_particles(0), hi.get_particles(0)
    np.testing.assert_array_equal(pl.x[:b1], ref.x[:b1])
    np.testing.assert_array_equal(pl.u[:b1], ref.u[:b1])
    np.testing.assert_array_equal(ph.x[b1:], ref.x[b1:])
    np.testing.assert_array_equal(ph.u[b1:], ref.u[b1:])
    # each slice's j-stream now holds the whole cluster's positions
    jw = shard.jstream_tensor(whole).cpu().numpy()
    np.testing.assert_array_equal(shard.jstream_tensor(lo).cpu().numpy(), jw)
    np.testing.assert_array_equal(shard.jstream_tensor(hi).cpu().numpy(), jw)
    # fields and diagnostics of the slices
    e_w = whole.fields(0)
    e_l, e_h = lo.fields(0), hi.fields(0)
    assert summary(force_error(np.r_[e_l[:b1], e_h[b1:]], e_w))["p99"] <= 2e-6
    dw, dl, dh = whole.diagnostics(0), lo.diagnostics(0), hi.diagnostics(0)
    assert dl["n_active"] + dh["n_active"] == dw["n_active"]
    for k in ("ke", "ke_ions", "ke_electrons"):
        assert dl[k] + dh[k] == pytest.approx(dw[k], rel=1e-12)
    assert dl["pe"] + dh["pe"] == pytest.approx(dw["pe"], rel=1e-6)
    np.testing.assert_allclose(np.add(dl["p"], dh["p"]), dw["p"], rtol=1e-6,
                               atol=1e-9 * np.abs(dw["p"]).max())
    for c in (whole, lo, hi):
        c.close()


def test_slices_with_equal_shares_step_like_the_whole_cluster(md):
    """With equal shares (jsplit -4, the autotuner's usual pick) each slice cuts
    its own i-blocks' sources into shares, so its pieces, and the order of its
    sums, differ from the unsplit context's: after 5 steps the slices' records
    agree with the whole cluster's to FP32 summation order."""
    import torch
    from paper_1307_3711_gb300 import shard
    w = synth.xe3_cluster(20000, seed=5)
    n = w.cluster.n
    b1 = shard.slice_bounds(n, 2, 1)[0]
    whole, lo, hi = _ctx(md, w, -4), _ctx(md, w, -4), _ctx(md, w, -4)
    assert whole.tuning()[4] == -4
    lo.set_slice(0, 0, b1)
    hi.set_slice(0, b1, n)
    for _ in range(5):
        for c in (whole, lo, hi):
            c.step(1)
        jl, jh = shard.jstream_tensor(lo), shard.jstream_tensor(hi)
        jl[b1:] = jh[b1:]
        jh[:b1] = jl[:b1]
        torch.cuda.synchronize()
    ref = whole.get_particles(0)
    pl, ph = lo.get_particles(0), hi.get_particles(0)
    x = np.r_[pl.x[:b1], ph.x[b1:]]
    u = np.r_[pl.u[:b1], ph.u[b1:]]
    r0 = np.abs(ref.x).max()
    assert np.abs(x - ref.x).max() < 1e-6 * r0
    du = np.abs(u - ref.u).max(1)
    assert np.percentile(du, 99) < 1e-4 * np.abs(ref.u).max()
    e_w = whole.fields(0)
    e_l, e_h = lo.fields(0), hi.fields(0)
    assert summary(force_error(np.r_[e_l[:b1], e_h[b1:]], e_w))["p99"] <= 2e-5
    for c in (whole, lo, hi):
        c.close()


def test_slice_arguments_and_states(md):
    w = synth.xe3_cluster(4000, seed=1)
    with _ctx(md, w, 0) as c:
        for b, e in ((0, 1000), (100, 4000), (-1024, 4000), (2048, 1024), (0, 5000)):
            with pytest.raises(md.MDError) as ei:
                c.set_slice(0, b, e)
            assert ei.value.status == md.MD_ERR_ARG
        c.set_slice(0, 4000, 4000)     # an empty slice: steps push nothing
        x0 = c.get_particles(0).x.copy()
        c.step(2)
        np.testing.assert_array_equal(c.get_particles(0).x, x0)
        c.set_slice(0, 0, 4000)        # the whole cluster again
        c.step(1)
        assert not np.array_equal(c.get_particles(0).x, x0)
        with pytest.raises(md.MDError) as ei:
            c.set_slice(0, 0, 2048)
            c.set_detectors(0, 1.0)
        assert ei.value.status == md.MD_ERR_STATE
    # ionizing contexts cannot be split
    cl = synth.make_cluster(2, 1024, 0, synth.nm_to_len(2.0), 0, synth.ARGON["mass"],
                            n_electron_slots=8 * 1024)
    cfg = md.make_config(a0=0.05, tau=300.0, softening=synth.nm_to_len(0.1),
                         rate_model=md.RATES_PLAIN, ionize_every=1, zmax=8, n_ions=1024,
                         slot_base=1024, r_loc=0.02, r_create=0.002, species=synth.ARGON)
    with md.Context([cfg], [md.HostParticles.from_cluster(cl)]) as c:
        with pytest.raises(md.MDError) as ei:
            c.set_slice(0, 0, 1024)
        assert ei.value.status == md.MD_ERR_STATE
