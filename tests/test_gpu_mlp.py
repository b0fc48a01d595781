"""The learned rate surrogate on the GPU: forward pass and gradients against
the FP64 oracle, training labels from the plain rate, training accuracy, the
ionization pass with the surrogate against the plain rates, and what it gains.

BF16 tolerance: weights and activations are rounded to 8-bit mantissas
(relative 2^-9) before each 64-term FP32 accumulation, so outputs carry a few
1e-3 relative error per layer; gradients are compared by relative norm."""
import time

import numpy as np
import pytest

import oracle
from paper_1307_3711_gb300 import synth

pytestmark = pytest.mark.gpu
AR = synth.ARGON


@pytest.fixture(scope="module")
def md():
    from paper_1307_3711_gb300 import build
    build.build()
    from paper_1307_3711_gb300 import md as m
    return m


def bf16_round(a):
    import torch
    return torch.tensor(np.asarray(a, np.float32)).to(torch.bfloat16).to(torch.float64).numpy()


def random_params(seed):
    rng = np.random.default_rng(seed)
    p = np.zeros(5000)
    p[0:256] = rng.uniform(-0.6, 0.6, 256)
    p[256:320] = rng.normal(0, 0.1, 64)
    p[320:4416] = rng.uniform(-0.3, 0.3, 4096)
    p[4416:4480] = rng.normal(0, 0.1, 64)
    p[4480:4992] = rng.uniform(-0.3, 0.3, 512)
    p[4992:5000] = rng.normal(0, 0.1, 8)
    return p.astype(np.float32)


def test_forward_matches_oracle(md):
    import torch
    p = random_params(1)
    rng = np.random.default_rng(2)
    n = 1000
    f = rng.uniform(-1.5, 1.5, size=(n, 4)).astype(np.float32)
    pd = torch.tensor(p, device="cuda")
    fd = torch.tensor(f, device="cuda")
    yd = torch.zeros((n, 8), dtype=torch.float32, device="cuda")
    md.mlp_forward_device(pd.data_ptr(), fd.data_ptr(), n, yd.data_ptr())
    torch.cuda.synchronize()
    y = yd.cpu().numpy()
    pb = bf16_round(p)
    y64 = oracle.mlp_forward(pb, bf16_round(f))
    err = np.abs(y - y64)
    # Error budget of the one rounding the oracle does not make: the GPU feeds
    # layer 2 with the layer-1 activations h1 rounded to BF16 (relative
    # 2^-9), so a2_j moves by at most 2^-9 sum_k |W2_jk| |h1_k|, h2 = silu(a2)
    # by at most max|silu'| (< 1.1) times that, and output i by
    # sum_j |W3_ij| times the h2 error; FP32 accumulation adds ~1e-6.
    w1, b1 = pb[0:256].reshape(64, 4), pb[256:320]
    w2, w3 = pb[320:4416].reshape(64, 64), pb[4480:4992].reshape(8, 64)
    a1 = bf16_round(f) @ w1.T + b1
    h1 = a1 / (1.0 + np.exp(-a1))
    bound = 1.1 * 2.0 ** -9 * (np.abs(h1) @ np.abs(w2).T) @ np.abs(w3).T + 1e-5
    print(f"forward: max |y - y64| {err.max():.3g} (max/bound {(err / bound).max():.3g}), "
          f"median {np.median(err):.3g}, scale {np.abs(y64).max():.3g}")
    assert np.all(err <= bound)
    assert np.median(err) < 0.003 * np.abs(y64).max()


def test_gradient_matches_oracle(md):
    import torch
    p = random_params(3)
    rng = np.random.default_rng(4)
    n = 3000
    f = rng.uniform(-1.5, 1.5, size=(n, 4)).astype(np.float32)
    z = rng.integers(0, 8, size=n).astype(np.int32)
    t = rng.normal(0, 0.5, size=n).astype(np.float32)
    dev = lambda a: torch.tensor(a, device="cuda")
    pd, fd, zd, td = dev(p), dev(f), dev(z), dev(t)
    gd = torch.zeros(5000, dtype=torch.float32, device="cuda")
    ld = torch.zeros(1, dtype=torch.float32, device="cuda")
    md.mlp_loss_grad_device(pd.data_ptr(), fd.data_ptr(), zd.data_ptr(), td.data_ptr(), n,
                            gd.data_ptr(), ld.data_ptr())
    g = gd.cpu().numpy().astype(np.float64)
    loss64, g64 = oracle.mlp_loss_grad(bf16_round(p), bf16_round(f), z, t)
    assert ld.item() / n == pytest.approx(loss64, rel=0.02)
    rel = np.linalg.norm(g - g64) / np.linalg.norm(g64)
    cos = g @ g64 / (np.linalg.norm(g) * np.linalg.norm(g64))
    assert rel < 0.05 and cos > 0.999, (rel, cos)
    for lo, hi in [(0, 256), (256, 320), (320, 4416), (4416, 4480), (4480, 4992), (4992, 5000)]:
        blk = np.linalg.norm(g[lo:hi] - g64[lo:hi]) / np.linalg.norm(g64[lo:hi])
        assert blk < 0.08, (lo, hi, blk)


def test_samples_are_labelled_by_the_plain_rate(md):
    import torch
    cfg = md.mlp_train_config(AR)
    n = 4000
    f = torch.zeros((n, 4), dtype=torch.float32, device="cuda")
    z = torch.zeros(n, dtype=torch.int32, device="cuda")
    t = torch.zeros(n, dtype=torch.float32, device="cuda")
    raw = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    md.mlp_samples_device(cfg, n, 77, f.data_ptr(), z.data_ptr(), t.data_ptr(), raw.data_ptr())
    torch.cuda.synchronize()
    raw, z, t, f = raw.cpu().numpy(), z.cpu().numpy(), t.cpu().numpy(), f.cpu().numpy()
    assert raw[:, 0].min() >= 1e-3 and raw[:, 0].max() <= 1.0
    assert set(np.unique(z)) == set(range(8))
    for k in range(0, n, 37):
        nu = oracle.rate_total(raw[k, 0], int(z[k]), raw[k, 1], raw[k, 2], AR)
        assert t[k] == pytest.approx(oracle.mlp_target(nu), abs=2e-7)
        np.testing.assert_allclose(f[k], oracle.mlp_features(raw[k, 0], int(z[k]), raw[k, 1],
                                                             raw[k, 2], AR["ip_ev"][int(z[k])]),
                                   atol=2e-6)


def test_plain_rate_entry_point_matches_oracle(md):
    import torch
    rng = np.random.default_rng(8)
    n = 500
    e = 10 ** rng.uniform(-3, 0, n)
    z = rng.integers(0, 8, n).astype(np.int32)
    ne = np.where(rng.random(n) < 0.2, 0.0, 10 ** rng.uniform(15, 24, n))
    te = np.where(ne > 0, 10 ** rng.uniform(-1, 4, n), 0.0)
    ed, zd, ned, ted = (torch.tensor(a, device="cuda") for a in (e, z, ne, te))
    nu = torch.zeros(n, dtype=torch.float64, device="cuda")
    cfg = md.mlp_train_config(AR)
    md.ion_rates_device(cfg, 1, 0, ed.data_ptr(), zd.data_ptr(), ned.data_ptr(), ted.data_ptr(),
                        n, nu.data_ptr())
    torch.cuda.synchronize()
    ref = np.array([oracle.rate_total(e[k], int(z[k]), ne[k], te[k], AR) for k in range(n)])
    np.testing.assert_allclose(nu.cpu().numpy(), ref, rtol=1e-11, atol=1e-300)


@pytest.fixture(scope="module")
def trained(md):
    cfg = md.mlp_train_config(AR, n_samples=8 << 20, epochs=80, batch=8192, lr=3e-3, seed=11)
    params, rep = md.mlp_train(cfg)
    return cfg, params, rep


def test_training_accuracy(md, trained):
    cfg, params, rep = trained
    print("surrogate training:", rep)
    assert rep["loss_last"] < 0.05 * rep["loss_first"]
    assert rep["holdout_median_dlog10"] < 0.05
    assert rep["holdout_p99_dlog10"] < 0.5


def test_surrogate_charge_states_match_plain_rates(md, trained):
    """The same Ar cluster and seed, ionized with the plain rates and with the
    surrogate: the charge-state fractions agree within 0.01 per state.  The
    runs decorrelate (chaotic dynamics), so each fraction carries binomial
    noise of about sqrt(p(1-p)/n): 50k atoms keep it near 0.0015, and a plain
    run with another seed shows the noise level."""
    cfg, params, _ = trained
    n = 50000
    c = synth.make_cluster(6, n, 0, synth.nm_to_len(5.7 * (n / 20000) ** (1 / 3)), 0,
                           AR["mass"], n_electron_slots=n * 8)
    rw = synth.nm_to_len(AR["r_w_nm"])
    fracs = []
    for model, seed in ((1, 99), (2, 99), (1, 98)):
        kw = dict(a0=0.07, tau=1.0, dt=0.05, softening=synth.nm_to_len(0.1), envelope=3,
                  rate_model=model, ionize_every=2, zmax=8, n_ions=n, slot_base=n, seed=seed,
                  r_loc=3 * rw, r_create=rw, species=AR)
        with md.Context([md.make_config(**kw)], [md.HostParticles.from_cluster(c)]) as ctx:
            if model == 2:
                ctx.set_rate_mlp(params, cfg)
            ctx.step(120)
            d = ctx.diagnostics(0)
        fracs.append(d["charge_count"][:9] / n)
    print("charge fractions plain", np.round(fracs[0], 4), "surrogate", np.round(fracs[1], 4),
          "plain, other seed", np.round(fracs[2], 4))
    assert fracs[0][1:].sum() > 0.3   # the run ionized
    assert np.abs(fracs[0] - fracs[2]).max() <= 0.01   # seed-to-seed noise below the bound
    assert np.abs(fracs[0] - fracs[1]).max() <= 0.01


def test_surrogate_charge_states_at_full_size(md):
    """The full-size ionizing workload: 200k neutral Ar atoms in an 8 nm
    sphere (1.8M records with the electron slots), 806 nm, 8e15 W/cm^2,
    100 fs sin^2 pulse, started at the field crest nearest the envelope peak,
    ionization before every step.  The surrogate is trained for argon at
    806 nm; after 10 ionizing steps the charge-state fractions of the
    surrogate run are within 0.01 of the plain-rate run on the same seed.
    At 200k atoms the binomial noise of a fraction is below 0.0012; a plain
    run with another seed shows it."""
    cfg = md.mlp_train_config(AR, n_samples=8 << 20, epochs=80, batch=8192, lr=3e-3, seed=11,
                              lambda_um=0.806)
    params, rep = md.mlp_train(cfg)
    assert rep["holdout_median_dlog10"] < 0.05
    n = 200000
    w = synth.ar_ionize(seed=0, n_atoms=n)
    fracs = []
    for model, seed in ((1, 1), (2, 1), (1, 2)):
        c = md.config_from_workload(w)
        ion = md.make_config(rate_model=model, ionize_every=1, zmax=w.extra["zmax"], n_ions=n,
                             slot_base=n, seed=seed, r_loc=w.extra["r_loc"],
                             r_create=w.extra["r_create"], species=AR)
        for f in ("rate_model", "ionize_every", "zmax", "n_ions", "slot_base", "seed", "r_loc",
                  "r_create", "ip_ev", "q_outer"):
            setattr(c, f, getattr(ion, f))
        with md.Context([c], [md.HostParticles.from_cluster(w.cluster)]) as ctx:
            if model == 2:
                ctx.set_rate_mlp(params, cfg)
            ctx.step(10)
            d = ctx.diagnostics(0)
        fracs.append(d["charge_count"][:9] / n)
    print("charge fractions plain", np.round(fracs[0], 4), "surrogate", np.round(fracs[1], 4),
          "plain, other seed", np.round(fracs[2], 4))
    assert fracs[0][1:].sum() > 0.5   # the run ionized
    assert np.abs(fracs[0] - fracs[2]).max() <= 0.005   # seed-to-seed noise
    assert np.abs(fracs[0] - fracs[1]).max() <= 0.01


def test_surrogate_gain_in_rate_evaluation(md, trained):
    """What the network buys: the rate evaluation of 200k ions with the
    surrogate (BF16 tensor cores) against the FP64 transcendental plain rate."""
    import torch
    cfg, params, _ = trained
    rng = np.random.default_rng(12)
    n = 200000
    dev = lambda a: torch.tensor(a, device="cuda")
    e = dev(10 ** rng.uniform(-2.5, -0.2, n))
    z = dev(rng.integers(0, 8, n).astype(np.int32))
    ne = dev(10 ** rng.uniform(19, 23, n))
    te = dev(10 ** rng.uniform(0, 3, n))
    pd = dev(params)
    nu1 = torch.zeros(n, dtype=torch.float64, device="cuda")
    nu2 = torch.zeros(n, dtype=torch.float64, device="cuda")
    times = {}
    for model, out in ((1, nu1), (2, nu2)):
        for _ in range(3):
            md.ion_rates_device(cfg, model, pd.data_ptr(), e.data_ptr(), z.data_ptr(),
                                ne.data_ptr(), te.data_ptr(), n, out.data_ptr())
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record()
        for _ in range(20):
            md.ion_rates_device(cfg, model, pd.data_ptr(), e.data_ptr(), z.data_ptr(),
                                ne.data_ptr(), te.data_ptr(), n, out.data_ptr())
        ev1.record()
        torch.cuda.synchronize()
        times[model] = ev0.elapsed_time(ev1) / 20
    d = np.abs(np.log10(nu2.cpu().numpy() + 1e-12) - np.log10(nu1.cpu().numpy() + 1e-12))
    print(f"rates of {n} ions: plain {times[1]:.4f} ms, surrogate {times[2]:.4f} ms, "
          f"speed-up {times[1] / times[2]:.2f}x, median |dlog10 nu| {np.median(d):.4f}")
    assert np.median(d) < 0.05
    assert times[2] < times[1]
