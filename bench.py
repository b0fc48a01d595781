#!/usr/bin/env python
"""Throughput of the fused Coulomb + laser + Boris MD step on GB300.

Metric: Coulomb pair interactions per second (N_i x N_j per step, self pair and
padding included in the work, only the N^2 real pairs counted) and steps per
second at N = 200,000 (50k Xe3+ + 150k electrons at 10 eV in a 7.94 nm sphere,
the density of the 400k-particle Xe case), one cluster per GPU; N GPUs run N
independent clusters (weak scaling).  The force error against the FP64 oracle
on sampled targets is reported beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]

Prints one JSON line (rank 0).  The `reference` arm times the FP64 CPU oracle on
the host cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1307_3711_gb300 import synth  # noqa: E402

METRIC = "Coulomb pair interactions/s & steps/s at N=200k on 1 GB300; force err vs FP64"
UNIT = "pair/s"
RECORD_BYTES = 3 * 8 + 3 * 8 + 4 + 8 + 8 + 1   # x, u, z, mass, w, kind per record
FP32_INSTR_PER_PAIR = 12
# DRAM bytes (read + write) per launch of the step kernel, from one 1-pass ncu
# capture (dram__bytes_read.sum + dram__bytes_write.sum) of the named workload
# at full size in the named kernel configuration (threads, r, tile, packed,
# jsplit); reported only when the timed run uses that configuration.
STEP_TRAFFIC_BYTES = {("xe3_200k", 200000, 128, 8, 512, True, 9): 15.77e6,
                      ("xe3_200k", 200000, 128, 8, 256, True, -4): 20.16e6}
L2_FLUSH_BYTES = 512 << 20
# step kernel configuration of the ionizing 200k-atom contexts (threads, r,
# tile, CTAs per SM, jsplit, packed, min_blocks): the fastest of four packed
# configurations timed on that workload (193.4 ms per step against 205.9 to
# 207.5 ms for 128 x 8 targets with 256- or 512-source tiles)
IONIZING_TUNING = (256, 4, 512, 0, 0, 1, 0)
WORKLOAD_TEXT = {
    "xe3_200k": "{name}: N={n} (Xe3+ ions + electrons, 10 eV), one cluster per GPU",
    "xe3_200k_shard": "{name}: N={n} (Xe3+ ions + electrons, 10 eV), one cluster split over "
                      "{ranks} GPU(s) by target records, j-stream all-gathered every step",
    "scan256": "parameter scan of {clusters} clusters (N log-uniform 1k-50k, Z 1-8, R0 1-8 nm, "
               "a0 0.01-0.3, 20-200 fs), {n} records in one persistent launch per step",
    "precision_1m": "{name}: N={n}, laser off (timed), then the same cluster driven at a0 = 0.1 "
                    "(precision.driven)",
    "ar_ionize": "{name}: {atoms} Ar atoms (neutral at the start) in an 8 nm sphere + 8 "
                 "electron slots each ({n} records), ADK + Lotz ionization before every step "
                 "({rates} rates), from the pulse peak",
}


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--n", type=int, default=None,
                    help="particles per cluster (ar_ionize: atoms; default 200000)")
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--cpu-seconds", type=float, default=12.0,
                    help="target CPU time of the oracle sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--shard", action="store_true",
                    help="xe3_200k under torchrun: one cluster split over the ranks by target "
                         "records, its j-stream all-gathered (NCCL) after every step (strong "
                         "scaling); without it every rank runs its own cluster (weak scaling)")
    ap.add_argument("--no-secondary", action="store_true",
                    help="skip the secondary measurements (scan256, ar_ionize plain/mlp, "
                         "precision_1m) that follow the headline at N = 1")
    ap.add_argument("--tuning", default=None,
                    help="force a kernel configuration: threads,r,tile,packed[,jsplit[,min_blocks]]")
    ap.add_argument("--workload", default="xe3_200k",
                    choices=["xe3_200k", "scan256", "precision_1m", "ar_ionize", "iedf",
                             "iedf_xe", "nscale"],
                    help="xe3_200k: the headline N=200k cluster; scan256: 256 clusters of a "
                         "parameter scan in one persistent launch; precision_1m: 500k Ar+ + 500k "
                         "e, laser off; ar_ionize: neutral Ar atoms ionizing; iedf: a small "
                         "ionizing Ar cluster through the whole pulse with ion energy detectors "
                         "at 9 R0 (the IEDF along and across the polarization); iedf_xe: the "
                         "same for the Xe_2600 cluster of Sec. III (16 charge states)")
    ap.add_argument("--rates", default="plain", choices=["plain", "mlp"],
                    help="ar_ionize: plain ADK + Lotz rates, or the BF16 surrogate trained on "
                         "the GPU before the run (plain rates outside its domain)")
    args = ap.parse_args()
    if args.n is None:
        args.n = 200000
    return args


# ----------------------------------------------------------- distributed --

def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


class Dist:
    def __init__(self, backend):
        self.world, self.rank, self.local = dist_env()
        self.pg = None
        if self.world > 1:
            import torch.distributed as td
            os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
            td.init_process_group(backend=backend)
            self.pg = td

    def barrier(self):
        if self.pg:
            self.pg.barrier()

    def max(self, v: float) -> float:
        if not self.pg:
            return v
        import torch
        dev = "cuda" if self.pg.get_backend() == "nccl" else "cpu"
        t = torch.tensor([v], dtype=torch.float64, device=dev)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.pg:
            self.pg.destroy_process_group()


def whole_job_value(world: int, pairs_per_step: float, steps: int, t_max: float) -> float:
    """Pairs per second of the whole job: every rank advances its own cluster
    (replicas, weak scaling) through the same number of steps, and the job
    takes as long as its slowest rank."""
    return world * pairs_per_step * steps / t_max


# --------------------------------------------------------------- clocks --

class ClockSampler:
    """nvidia-smi samples (every 200 ms) while the timed region runs."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.lines = []
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", gpu_id], stdout=subprocess.PIPE,
                stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except (OSError, ValueError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.th.join(timeout=2)
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
                power.append(float(f[3]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "power_w_max": max(power), "samples": len(sm), "reasons": sorted(reasons)}


def gpu_id_for(local_rank: int) -> str:
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        ids = [v.strip() for v in vis.split(",") if v.strip()]
        if local_rank < len(ids):
            return ids[local_rank]
    return str(local_rank)


# ------------------------------------------------------------ workloads --

def workload(n: int, seed: int):
    w = synth.xe3_cluster(n, seed=seed)
    return w


def cpu_oracle_rate(w, seconds: float, seed: int = 0, e_gpu=None):
    """The FP64 oracle's direct sum (OpenMP over targets, all host cores) on
    sampled targets of the workload, sized to about `seconds` of CPU time.
    With e_gpu (the GPU field of the same state) it also returns the floored
    relative field error |E - E64| / max(|E64|, rms |E64|) at those targets."""
    import oracle
    c = w.cluster
    kc = oracle.coulomb_constant(w.lambda_um)
    q = c.w * c.z * c.active
    threads = os.cpu_count() or 1
    rng = np.random.default_rng(seed)
    nt = 256
    while True:  # calibrate on a sample long enough to time
        idx = rng.choice(c.n, nt, replace=False)
        t0 = time.perf_counter()
        oracle.coulomb_field(c.x[idx], c.x, q, w.eps, kc, self_idx=idx, nthreads=threads)
        dt = time.perf_counter() - t0
        if dt > 0.25 or nt >= c.n:
            break
        nt = min(c.n, nt * 4)
    nt = int(min(c.n, max(64, nt * seconds / max(dt, 1e-6))))
    idx = np.sort(rng.choice(c.n, nt, replace=False))
    t0 = time.perf_counter()
    e64 = oracle.coulomb_field(c.x[idx], c.x, q, w.eps, kc, self_idx=idx, nthreads=threads)
    dt = time.perf_counter() - t0
    pairs = nt * c.n
    err = None
    if e_gpu is not None:
        live = c.active[idx] > 0
        nrm = np.linalg.norm(e64[live], axis=1)
        rel = np.linalg.norm(e_gpu[idx][live] - e64[live], axis=1) / np.maximum(
            nrm, np.sqrt(np.mean(nrm ** 2)))
        err = {"median": float(np.median(rel)), "p99": float(np.percentile(rel, 99)),
               "max": float(rel.max()), "n_targets": int(live.sum()),
               "metric": "|E - E_fp64| / max(|E_fp64|, rms|E_fp64|) at sampled targets, "
                         "GPU FP32/Kahan sum vs FP64 oracle, initial state"}
    return pairs / dt, threads, nt, dt, err


def ar_ionize_context(md, args, rank, stream):
    """Neutral argon cluster at the density of 200k atoms in an 8 nm sphere, 8
    inactive electron slots per atom, 806 nm pulse of 8e15 W/cm^2 (a0 = 0.0617)
    with a 100 fs sin^2 envelope, started just before a field crest at the
    envelope peak so that the timed steps ionize (synth.ar_ionize)."""
    return ionizing_context(md, args.n, args.rates, rank, stream)


def ionizing_context(md, n, rates, rank, stream, train=None):
    """The ar_ionize context with `rates` ("plain" or "mlp").  train: a
    previously trained (params, train_config) to install instead of training
    the surrogate again."""
    w = synth.ar_ionize(seed=rank, n_atoms=n)
    c = w.cluster
    cfg = md.config_from_workload(w)
    model = md.RATES_MLP if rates == "mlp" else md.RATES_PLAIN
    ion = md.make_config(rate_model=model, ionize_every=1, zmax=w.extra["zmax"], n_ions=n,
                         slot_base=n, seed=rank + 1, r_loc=w.extra["r_loc"],
                         r_create=w.extra["r_create"], species=synth.ARGON)
    for f in ("rate_model", "ionize_every", "zmax", "n_ions", "slot_base", "seed", "r_loc",
              "r_create", "ip_ev", "q_outer"):
        setattr(cfg, f, getattr(ion, f))
    ctx = md.Context([cfg], [md.HostParticles.from_cluster(c)], stream=stream)
    # ion field, inputs, (surrogate rates,) decision, apply, charge-change
    # correction, ion push, step
    info = {"rates": rates, "t0": w.t0,
            "kernels_per_step": 7 + (1 if model == md.RATES_MLP else 0)}
    if model == md.RATES_MLP:
        if train is None:
            tc = md.mlp_train_config(synth.ARGON, n_samples=10 << 20, epochs=80, batch=8192,
                                     lr=3e-3, seed=11, lambda_um=w.lambda_um)
            t_train = time.perf_counter()
            params, rep = md.mlp_train(tc, stream)
            info["surrogate_training"] = dict(rep, wall_s=time.perf_counter() - t_train,
                                              samples=tc.n_samples, epochs=tc.epochs,
                                              ms_per_epoch=rep["train_ms"] / tc.epochs)
            info["trained"] = (params, tc)
        else:
            params, tc = train
        ctx.set_rate_mlp(params, tc)
    return ctx, [w], None, info


def precision_study(md, ctx, w, n_targets=10000, n_oracle=2000, seed=0):
    """FP32/Kahan field of the state against the FP64 GPU reference on a
    seeded subset of targets, and the FP64 GPU reference against the FP64
    oracle (bitwise) on part of that subset."""
    import torch
    import oracle
    c = w.cluster
    kc = md.coulomb_constant(w.lambda_um)
    g = ctx.get_particles(0)
    rng = np.random.default_rng(seed)
    idx = np.sort(rng.choice(c.n, min(n_targets, c.n), replace=False)).astype(np.int64)
    q = np.where(g.kind != md.KIND_INACTIVE, g.w * g.z, 0.0)
    dev = lambda a: torch.tensor(np.ascontiguousarray(a), device="cuda")
    dxs, dqs, dxt, dsi = dev(g.x), dev(q), dev(g.x[idx]), dev(idx)
    e64 = torch.zeros((len(idx), 3), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    md.coulomb_field_fp64_device(dxs.data_ptr(), dqs.data_ptr(), c.n, dxt.data_ptr(),
                                 dsi.data_ptr(), len(idx), w.eps, kc, e64.data_ptr(), 0)
    torch.cuda.synchronize()
    t64 = time.perf_counter() - t0
    e64 = e64.cpu().numpy()
    e32 = ctx.fields(0)[idx]
    nrm = np.linalg.norm(e64, axis=1)
    rel = np.linalg.norm(e32 - e64, axis=1) / np.maximum(nrm, np.sqrt(np.mean(nrm ** 2)))
    m = min(n_oracle, len(idx))
    e_or = oracle.coulomb_field(g.x[idx[:m]], g.x, q, w.eps, kc, self_idx=idx[:m],
                                nthreads=os.cpu_count() or 1)
    return {"targets": int(len(idx)), "fp64_gpu_reference_s": t64,
            "fp32_kahan_vs_fp64_gpu": {"median": float(np.median(rel)),
                                       "p99": float(np.percentile(rel, 99)),
                                       "max": float(rel.max())},
            "fp64_gpu_vs_oracle_bitwise_equal": f"{int(np.sum(np.all(e_or == e64[:m], axis=1)))}"
                                                f"/{m} targets",
            "metric": "|E - E_fp64| / max(|E_fp64|, rms|E_fp64|), state after the timed steps"}


def driven_precision(md, args, rank, stream, tuning):
    """The precision case's driven run: the same 1M-particle cluster with the
    laser on (a0 = 0.1, 100 fs sin^2, from the envelope's peak), the same
    kernel configuration, as many
    steps as the timed run; then the FP32/Kahan field against the FP64 GPU
    reference (and the oracle) on the state the laser has pulled apart, and
    the energy the laser has put in."""
    import torch
    wd = synth.precision_1m(seed=rank, a0=0.1)
    wd.t0 = 0.5 * wd.tau          # from the peak of the sin^2 envelope
    with md.Context([md.config_from_workload(wd)], [md.HostParticles.from_cluster(wd.cluster)],
                    stream=stream.cuda_stream) as cd:
        cd.set_tuning(tuning[0], tuning[1], tuning[2], 0, tuning[4], tuning[5], tuning[6])
        d0 = cd.diagnostics(0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        cd.step(args.steps)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        d1 = cd.diagnostics(0)
        out = precision_study(md, cd, wd)
    out.update(a0=wd.a0, steps=args.steps, ms_per_step=ms,
               energy_gain_m_ec2=d1["total"] - d0["total"], ke_after=d1["ke"],
               t_end=d1["t"], laser="on, a0 = 0.1, 100 fs sin^2 from its peak")
    return out


def event_steps(ctx, stream, flush, steps, after=None):
    """Times `steps` single steps with CUDA events on `stream`, the L2 flushed
    before each outside the events; after(ctx) runs after each step (outside
    the events) and its results are returned beside the step times (ms)."""
    import torch
    ms, extra = [], []
    for _ in range(steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.step(1)
        e1.record(stream)
        if after is not None:
            extra.append(after(ctx))
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    return ms, extra


def alu_frac(pairs_per_s: float, sms: int, clocks: dict) -> dict:
    """Fraction of the FP32 roofline (128 lanes x SMs x clock / 12) at the
    median SM clock sampled during the run and at the maximum clock."""
    clk = clocks.get("sm_mhz") or 2070.0
    peak = 128.0 * sms * clk * 1e6 / FP32_INSTR_PER_PAIR
    return {"frac": pairs_per_s / peak, "peak_gpair_s": peak / 1e9, "sm_mhz": clk,
            "frac_at_max_clock": pairs_per_s / (128.0 * sms * 2070e6 / FP32_INSTR_PER_PAIR)}


def secondary_measurements(md, stream, flush, sms, gpu_id, tuning, steps=3, warmup=2):
    """Driver-visible numbers of the other configurations, each timed with
    CUDA events (L2 flushed between steps, outside the events) and its own
    nvidia-smi clock record:
      scan256      -- 256 uneven clusters in one persistent launch (autotuned);
      ar_ionize    -- 200k neutral Ar atoms ionizing before every step, plain
                      ADK + Lotz rates and the BF16 surrogate (trained here;
                      its training time per epoch), charge-state fractions of
                      both on the same seed;
      precision_1m -- 500k Ar+ + 500k e: the step time, and the FP32/Kahan
                      field against the FP64 GPU reference and the oracle.
    The 1M context runs the step kernel configuration and source split that
    the headline's autotuner chose (`tuning`); the ionizing contexts run
    IONIZING_TUNING with a segment count chosen for balance."""
    import torch
    out = {}
    cs = stream.cuda_stream

    # scan256
    t_wall = time.perf_counter()
    scan = synth.batched_scan(256, seed=0)
    cfgs, parts = [], []
    pairs = 0.0
    for e in scan:
        cl = synth.scan_cluster(e)
        w = synth.Workload(f"scan_{e.seed}", cl, a0=e.a0, pol=0, env=synth.ENV_SIN2, tau=e.tau,
                           eps=synth.nm_to_len(0.1), dt=0.02, nsteps=0)
        cfgs.append(md.config_from_workload(w))
        parts.append(md.HostParticles.from_cluster(cl))
        pairs += float(cl.n) ** 2
    with md.Context(cfgs, parts, stream=cs) as ctx:
        ctx.autotune(2)
        for _ in range(warmup):
            ctx.step(1)
        sampler = ClockSampler(gpu_id)
        time.sleep(0.3)
        ms, _ = event_steps(ctx, stream, flush, 2 * steps)
        clocks = sampler.stop()
        tun = ctx.tuning()
    rate = pairs / (statistics.mean(ms) / 1e3)
    out["scan256"] = dict({"clusters": 256, "records": int(sum(p.n for p in parts)),
                           "pairs_per_step": pairs, "steps": len(ms),
                           "ms_per_step": statistics.mean(ms), "pairs_per_s": rate,
                           "tuning": list(tun), "clocks": clocks, "gpu_launches": len(ms),
                           "wall_s": time.perf_counter() - t_wall}, **alu_frac(rate, sms, clocks))

    # ar_ionize, plain rates then the surrogate, same seed
    n_atoms = 200000
    trained = None
    for rates in ("plain", "mlp"):
        t_wall = time.perf_counter()
        ctx, ws, _, info = ionizing_context(md, n_atoms, rates, 0, cs)
        if rates == "mlp":
            trained = info.get("trained")
        ctx.set_tuning(*IONIZING_TUNING)
        with ctx:
            for _ in range(warmup):
                ctx.step(1)
            sampler = ClockSampler(gpu_id)
            time.sleep(0.3)
            ms, act = event_steps(ctx, stream, flush, steps, after=lambda c: c.count_active(0))
            clocks = sampler.stop()
            d = ctx.diagnostics(0)
        pairs = float(np.mean([float(a) ** 2 for a in act]))
        rate = pairs / (statistics.mean(ms) / 1e3)
        ent = dict({"atoms": n_atoms, "records": ws[0].cluster.n, "steps": steps,
                    "warmup": warmup, "ms_per_step": statistics.mean(ms),
                    "ms_per_timed_step": ms, "active_records_per_timed_step": act,
                    "pairs_per_s": rate,
                    "pairs_counted": "(active records after each step's ionization pass)^2",
                    "charge_fractions": (d["charge_count"][:9] / n_atoms).tolist(),
                    "clocks": clocks, "gpu_launches": steps * info["kernels_per_step"],
                    "wall_s": time.perf_counter() - t_wall},
                   **alu_frac(rate, sms, clocks))
        if "surrogate_training" in info:
            ent["surrogate_training"] = info["surrogate_training"]
        out[f"ar_ionize_{rates}"] = ent
    fp, fm = (np.array(out[f"ar_ionize_{r}"]["charge_fractions"]) for r in ("plain", "mlp"))
    out["ar_ionize_mlp"]["max_abs_fraction_diff_vs_plain"] = float(np.abs(fp - fm).max())
    out["ar_ionize_mlp"]["step_speedup_vs_plain"] = (out["ar_ionize_plain"]["ms_per_step"] /
                                                     out["ar_ionize_mlp"]["ms_per_step"])
    del trained

    # precision_1m: a short run of the 1M case, laser off
    t_wall = time.perf_counter()
    w = synth.precision_1m(seed=0, a0=0.0)
    with md.Context([md.config_from_workload(w)], [md.HostParticles.from_cluster(w.cluster)],
                    stream=cs) as ctx:
        ctx.set_tuning(tuning[0], tuning[1], tuning[2], 0, tuning[4], tuning[5], tuning[6])
        ctx.step(1)
        sampler = ClockSampler(gpu_id)
        time.sleep(0.3)
        ms, _ = event_steps(ctx, stream, flush, 2)
        clocks = sampler.stop()
        tun = ctx.tuning()
        prec = precision_study(md, ctx, w, n_targets=10000, n_oracle=1000)
    pairs = float(w.cluster.n) ** 2
    rate = pairs / (statistics.mean(ms) / 1e3)
    out["precision_1m"] = dict({"n_particles": w.cluster.n, "steps": len(ms),
                                "ms_per_step": statistics.mean(ms), "pairs_per_s": rate,
                                "tuning": list(tun), "clocks": clocks,
                                "gpu_launches": len(ms), "precision": prec,
                                "wall_s": time.perf_counter() - t_wall},
                               **alu_frac(rate, sms, clocks))
    torch.cuda.synchronize()
    return out


def single_thread_rate(w, seconds: float):
    """The same FP64 oracle sum on one host core (the paper's code without
    its OpenMP loop), on a sample sized to about `seconds`."""
    import oracle
    c = w.cluster
    kc = oracle.coulomb_constant(w.lambda_um)
    q = c.w * c.z * c.active
    rng = np.random.default_rng(1)
    nt = 16
    while True:
        idx = rng.choice(c.n, nt, replace=False)
        t0 = time.perf_counter()
        oracle.coulomb_field(c.x[idx], c.x, q, w.eps, kc, self_idx=idx, nthreads=1)
        dt = time.perf_counter() - t0
        if dt > 0.2 or nt >= c.n:
            break
        nt = min(c.n, nt * 4)
    nt = int(min(c.n, max(16, nt * seconds / max(dt, 1e-6))))
    idx = rng.choice(c.n, nt, replace=False)
    t0 = time.perf_counter()
    oracle.coulomb_field(c.x[idx], c.x, q, w.eps, kc, self_idx=idx, nthreads=1)
    dt = time.perf_counter() - t0
    return {"value": nt * c.n / dt, "unit": UNIT, "cores": 1,
            "sample": f"FP64 field at {nt} sampled targets from all {c.n} sources ({dt:.1f} s)"}


def oracle_step_scaling(ns=(20000, 50000, 100000), sweep_n=20000):
    """The paper's Fig. 7 on the host cores, with the FP64 oracle as it stands:
    one full step (field of every particle from all the others, laser, Boris
    push, drift; OpenMP over targets, the paper's own decomposition) of the
    same cluster family at several N on all cores (Fig. 7b: time ~ N^2), and
    at N = sweep_n on 1, 2, 4, ... cores (Fig. 7a)."""
    import oracle
    threads = os.cpu_count() or 1

    def one_step(n, nthreads):
        w = workload(n, seed=0)
        c = w.cluster
        st = oracle.State(c.x, c.u, c.z, c.mass, c.w, c.active)
        p = oracle.make_params(a0=w.a0, tau=w.tau, t0=w.t0, dt=w.dt, eps=w.eps, pol=w.pol,
                               env=w.env, boundary=w.boundary, box=w.box, t_switch=w.t_switch,
                               lambda_um=w.lambda_um)
        t0 = time.perf_counter()
        oracle.md_steps(st, p, 1, nthreads=nthreads)
        return time.perf_counter() - t0

    rows = []
    for n in ns:
        s = one_step(n, threads)
        rows.append({"n": n, "s_per_step": s, "pairs_per_s": float(n) ** 2 / s,
                     "ns_per_pair": 1e9 * s / float(n) ** 2})
    counts = sorted({k for k in (1, 2, 4, 8, 16, 32, 64, 128) if k < threads} | {threads})
    cores = []
    for k in counts:
        s = one_step(sweep_n, k)
        cores.append({"cores": k, "s_per_step": s})
    for r in cores:
        r["speedup"] = cores[0]["s_per_step"] / r["s_per_step"]
    return {"kind": "oracle", "cores": threads, "unit": UNIT,
            "what": "one full FP64 oracle step (all targets, OpenMP over targets) per row",
            "n_rows": rows, "n_for_core_rows": sweep_n, "core_rows": cores}


def run_nscale(args):
    """Step time against N for the headline cluster family (Xe3+ + 3 e per
    ion at the density of the 400k case), one autotuned context per N: the
    GPU counterpart of the paper's Fig. 7b (time ~ N^2)."""
    import torch
    from paper_1307_3711_gb300 import build
    build.build()
    from paper_1307_3711_gb300 import md
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    sms, gpu_name = md.device_info()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    rows = []
    for n in (20000, 50000, 100000, 200000, 400000):
        w = workload(n, seed=0)
        with md.Context([md.config_from_workload(w)], [md.HostParticles.from_cluster(w.cluster)],
                        stream=stream.cuda_stream) as ctx:
            ctx.autotune(3)
            for _ in range(3):
                ctx.step(1)
            ms = []
            for _ in range(max(args.steps // 6, 5)):
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                ctx.step(1)
                e1.record(stream)
                torch.cuda.synchronize()
                ms.append(e0.elapsed_time(e1))
            t = statistics.mean(ms)
            pairs = float(n) ** 2
            peak = 128.0 * sms * 2070e6 / FP32_INSTR_PER_PAIR
            rows.append({"n": n, "ms_per_step": t, "pairs_per_s": pairs / (t / 1e3),
                         "frac_at_max_clock": pairs / (t / 1e3) / peak,
                         "tuning": list(ctx.tuning())})
    cpu = None if args.no_cpu_baseline else oracle_step_scaling()
    print(json.dumps({"workload": "nscale: xe3 clusters at the density of the 400k case",
                      "device": gpu_name, "l2": "flushed between timed steps",
                      "rows": rows, "cpu_baseline": cpu}), flush=True)


def build_contexts(md, args, rank, stream):
    """The workload's clusters -> (context, list of workloads, pairs per step)."""
    if args.workload == "scan256":
        scan = synth.batched_scan(256, seed=rank)
        cfgs, parts, ws = [], [], []
        for e in scan:
            cl = synth.scan_cluster(e)
            w = synth.Workload(f"scan_{e.seed}", cl, a0=e.a0, pol=0, env=synth.ENV_SIN2, tau=e.tau,
                               eps=synth.nm_to_len(0.1), dt=0.02, nsteps=0)
            ws.append(w)
            cfgs.append(md.config_from_workload(w))
            parts.append(md.HostParticles.from_cluster(cl))
        pairs = float(sum(float(w.cluster.n) ** 2 for w in ws))
        return md.Context(cfgs, parts, stream=stream), ws, pairs, {}
    if args.workload == "precision_1m":
        w = synth.precision_1m(seed=rank, a0=0.0)
    elif args.workload == "ar_ionize":
        return ar_ionize_context(md, args, rank, stream)
    elif args.shard:
        # the same cluster on every rank, each pushing its slice of targets
        from paper_1307_3711_gb300 import shard
        world = dist_env()[0]
        w = workload(args.n, seed=0)
        ctx = md.Context([md.config_from_workload(w)], [md.HostParticles.from_cluster(w.cluster)],
                         stream=stream)
        b, e, per = shard.slice_bounds(w.cluster.n, world, rank)
        ctx.set_slice(0, b, e)
        return ctx, [w], float(w.cluster.n) ** 2, {"slice": (b, e, per)}
    else:
        w = workload(args.n, seed=rank)
    return (md.Context([md.config_from_workload(w)], [md.HostParticles.from_cluster(w.cluster)],
                       stream=stream), [w], float(w.cluster.n) ** 2, {})


# ------------------------------------------------------------------ iedf --

def iedf_case(args):
    """The two IEDF runs.  iedf: neutral Ar cluster (args.n atoms, default
    4000, at the density of 200k atoms in 8 nm), 806 nm, 8e15 W/cm^2 (a0 =
    0.0617), 100 fs sin^2 pulse, run to 1.5 pulse lengths, 8 charge states.
    iedf_xe: the Xe_2600 case of Sec. III (2600 atoms, R0 from Eq. 1 with the
    Wigner-Seitz radius of Sec. II), 790 nm, 4e15 W/cm^2 (a0 from Eq. 2),
    28 fs sin^2 pulse (intensity FWHM), run to the pulse length + 1 ps so
    most of the heavy ions reach the detectors, 16 charge states, Lotz
    collisional rates with the xenon table."""
    from paper_1307_3711_gb300 import md
    if args.workload == "iedf_xe":
        n = args.n if args.n != 200000 else 2600
        lam, sp, zmax = 0.79, synth.XENON, 16
        r0 = synth.nm_to_len(sp["r_w_nm"] * n ** (1 / 3), lam)
        a0 = md.a0_from_intensity(4e15, lam)
        tau = synth.sin2_length_from_fwhm(synth.fs_to_time(28.0, lam))
        t_end = tau + synth.fs_to_time(1000.0, lam)
        nb, e_max = 250, 5e5
        text = (f"iedf_xe{n}: {n} Xe atoms (neutral at t = 0) in {sp['r_w_nm'] * n ** (1 / 3):.2f}"
                f" nm + 16 slots each, 790 nm, 4e15 W/cm^2 (a0 {a0:.4f}), 28 fs sin^2, pulse "
                "+ 1 ps, detectors at 9 R0")
    else:
        n = args.n if args.n != 200000 else 4000
        lam, sp, zmax = 0.806, synth.ARGON, 8
        r0 = synth.nm_to_len(8.0 * (n / 200000) ** (1 / 3), lam)
        a0 = 0.0617
        tau = synth.sin2_length_from_fwhm(synth.fs_to_time(100.0, lam))
        t_end = 1.5 * tau
        nb, e_max = 200, 2e5
        text = (f"iedf_ar{n // 1000}k: {n} Ar atoms (neutral at t = 0) in "
                f"{r0 / synth.nm_to_len(1.0, lam):.2f} nm + 8 slots each, 806 nm, a0 0.0617, "
                "100 fs sin^2, 1.5 pulse lengths, detectors at 9 R0")
    return dict(n=n, lam=lam, species=sp, zmax=zmax, r0=r0, a0=a0, tau=tau, t_end=t_end,
                nb=nb, e_max=e_max, text=text)


def run_iedf(args):
    """A small ionizing cluster through the whole pulse with ionization before
    every step and detectors at 9 R0 (30-degree cones): ion counts and mean
    energies along (+-x) and across (+-y) the polarization (iedf_case)."""
    import torch
    from paper_1307_3711_gb300 import build
    build.build()
    from paper_1307_3711_gb300 import md
    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    k = iedf_case(args)
    n, lam, sp, zmax, r0 = k["n"], k["lam"], k["species"], k["zmax"], k["r0"]
    c = synth.make_cluster(rank + 1, n, 0, r0, 0, sp["mass"], n_electron_slots=zmax * n)
    rw = synth.nm_to_len(sp["r_w_nm"], lam)
    cfg = md.make_config(a0=k["a0"], tau=k["tau"], dt=0.02, softening=synth.nm_to_len(0.1, lam),
                         envelope=synth.ENV_SIN2, lambda_um=lam, rate_model=md.RATES_PLAIN,
                         ionize_every=1, zmax=zmax, n_ions=n, slot_base=n, seed=rank + 3,
                         r_loc=3 * rw, r_create=rw, species=sp)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    nb, e_max = k["nb"], k["e_max"]
    nsteps = int(k["t_end"] / 0.02)
    chunk = 2000
    with md.Context([cfg], [md.HostParticles.from_cluster(c)], stream=stream.cuda_stream) as ctx:
        ctx.set_detectors(0, 9 * r0, cone_deg=30.0, e_max_ev=e_max, n_bins=nb)
        ms, pairs, done = 0.0, 0.0, 0
        while done < nsteps:
            kk = min(chunk, nsteps - done)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ctx.step(kk)
            e1.record(stream)
            torch.cuda.synchronize()
            ms += e0.elapsed_time(e1)
            pairs += kk * float(ctx.count_active(0)) ** 2   # sampled per chunk
            done += kk
        zs = ctx.get_particles(0).z[:n]
        det, inside = ctx.iedf(0)
    if rank != 0:
        return
    centers = (np.arange(nb) + 0.5) * e_max / nb
    iedf = {}
    for j, name in enumerate(md.DETECTORS):
        h = det[j][:nb].astype(float)
        iedf[name] = {"ions": int(det[j].sum()),
                      "mean_kev": float((h * centers).sum() / max(h.sum(), 1.0) / 1e3),
                      "overflow": int(det[j][nb])}
    hin = inside[:nb].astype(float)
    line = {
        "metric": METRIC, "value": pairs / (ms / 1e3), "unit": UNIT, "n_gpus": 1,
        "steps": nsteps, "warmup": 0, "ms_per_step": ms / nsteps,
        "steps_per_s": nsteps / (ms / 1e3), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": k["text"],
                   "pairs_counted": "(active records)^2 sampled every 2000 steps",
                   "l2": "not flushed (a small cluster stays in L2)"},
        "ionization": {"charge_fractions": (np.bincount(zs, minlength=zmax + 1) / n).tolist(),
                       "mean_charge": float(zs.mean())},
        "iedf": iedf, "ions_inside": int(inside.sum()),
        "inside_mean_kev": float((hin * centers).sum() / max(hin.sum(), 1.0) / 1e3),
        # ion field, inputs, decision, apply, charge-change correction, ion push, step
        "gpu_launches": 7 * nsteps,
    }
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------- native --

def run_native(args):
    import torch

    from paper_1307_3711_gb300 import build
    build.build()
    from paper_1307_3711_gb300 import md

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = Dist("nccl")
    # one non-default stream shared by torch (events, L2 flush) and the library
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    ctx, ws, pairs_per_step, info = build_contexts(md, args, rank, stream.cuda_stream)
    ionizing = args.workload == "ar_ionize"
    w = ws[0]
    n = sum(x.cluster.n for x in ws)
    # FP32/Kahan field of the initial state, compared with the FP64 oracle in
    # the CPU-baseline leg below
    e_gpu0 = ctx.fields(0) if len(ws) == 1 and not ionizing else None
    sms, gpu_name = md.device_info()

    tune_ms = None
    if args.tuning:
        f = [int(v) for v in args.tuning.split(",")]
        ctx.set_tuning(f[0], f[1], f[2], 0, f[4] if len(f) > 4 else 0, f[3],
                       f[5] if len(f) > 5 else -1)
    elif not args.no_autotune:
        tune_ms = ctx.autotune(3).tolist()
    tuning = ctx.tuning()

    sliced = info.get("slice")

    def step_once():
        """One step of the workload: with --shard under several ranks, the
        rank's slice pushed, then the j-stream all-gathered."""
        ctx.step(1)
        if sliced and world > 1:
            from paper_1307_3711_gb300 import shard
            shard.exchange(shard.jstream_tensor(ctx), sliced[2], world, rank)

    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    for _ in range(max(args.warmup, 3)):
        flush.zero_()
        step_once()
    torch.cuda.synchronize()

    d_before = ctx.diagnostics(0) if args.workload == "precision_1m" else None
    sampler = ClockSampler(gpu_id_for(local))
    time.sleep(0.3)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    dist.barrier()
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    step_pairs = []
    for e0, e1 in evs:
        flush.zero_()                # L2 flushed between timed steps, outside the events
        e0.record(stream)
        step_once()
        e1.record(stream)
        if ionizing:
            # records active after the step's ionization pass (the pairs its
            # Coulomb sum covered); read outside the events
            step_pairs.append(float(ctx.count_active(0)) ** 2)
    torch.cuda.synchronize()
    dist.barrier()
    wall = time.perf_counter() - wall0
    clocks = sampler.stop()
    ctx.sync()
    step_ms = [a.elapsed_time(b) for a, b in evs]
    if ionizing:
        pairs_per_step = float(np.mean(step_pairs))
    t_local = sum(step_ms) / 1e3
    t_max = dist.max(t_local)
    ms_per_step = t_max * 1e3 / args.steps
    # a split cluster's ranks share its N^2 pairs; replicas each add theirs
    value = (pairs_per_step * args.steps / t_max if sliced
             else whole_job_value(world, pairs_per_step, args.steps, t_max))
    # pairs this GPU's kernel summed per step (its slice of targets x all sources)
    pairs_local = (float(sliced[1] - sliced[0]) * w.cluster.n if sliced else pairs_per_step)

    precision = None
    if args.workload == "precision_1m":
        d_after = ctx.diagnostics(0)
        precision = precision_study(md, ctx, w)
        precision["energy_drift"] = {
            "relative_to_pe0": (d_after["total"] - d_before["total"]) / abs(d_before["pe"]),
            "total_before": d_before["total"], "total_after": d_after["total"],
            "pe_before": d_before["pe"], "ke_after": d_after["ke"],
            "steps": args.steps, "dt": w.dt, "laser": "off",
            "what": "(E_total after - before) / |PE before| over the timed steps (the cluster "
                    "starts cold: KE = 0), FP64 sums, m_e c^2 units"}
        precision["driven"] = driven_precision(md, args, rank, stream, tuning)
    ion_state = None
    if ionizing:
        # the state the timed steps reached (the end-to-end leg below repeats
        # one step from it)
        d = ctx.diagnostics(0)
        ion_state = dict({k: v for k, v in info.items() if k != "trained"}, charge_fractions=(d["charge_count"][:9] / w.cluster.n_ions).tolist(),
                         active_records_after_timed_steps=int(d["n_active"]),
                         active_records_per_timed_step=[int(round(math.sqrt(p)))
                                                        for p in step_pairs],
                         ms_per_timed_step=step_ms,
                         pairs_counted="(active records after each step's ionization pass)^2, "
                                       "averaged over the timed steps",
                         step_includes="ionization field + moments, rate inputs, "
                                       + ("surrogate rates, " if args.rates == "mlp" else "")
                                       + "decision, fused Coulomb/laser/push step")

    # FP32 roofline of the step kernel (the only kernel of a step)
    ffma_per_s, ffma2_per_s = md.measure_fp32_peak(stream.cuda_stream)
    achieved = pairs_local / (statistics.mean(step_ms) / 1e3)
    peak_probe = max(ffma_per_s, ffma2_per_s) / FP32_INSTR_PER_PAIR
    clk = clocks.get("sm_mhz") or None
    peak_clock = 128.0 * sms * clk * 1e6 / FP32_INSTR_PER_PAIR if clk else None
    peak_max = 128.0 * sms * 2070e6 / FP32_INSTR_PER_PAIR

    # end to end through the C ABI with host buffers: upload, step, download.
    # An ionizing run repeats one step from the state its timed steps reached.
    reached = ctx.get_particles(0) if ionizing else None
    hps = []
    for x in ws:
        hx = reached if ionizing else md.HostParticles.from_cluster(x.cluster)
        pinned = {}
        for k in ("x", "u", "z", "mass", "w", "kind"):
            a = getattr(hx, k)
            t = torch.empty(a.shape, dtype=getattr(torch, str(a.dtype)), pin_memory=True)
            t.numpy()[...] = a
            pinned[k] = t
        hps.append(md.HostParticles(*(pinned[k].numpy()
                                      for k in ("x", "u", "z", "mass", "w", "kind"))))
    e2e_t, e2e_pairs = [], []
    for s_ in range(args.e2e_steps + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k, hp in enumerate(hps):
            ctx.set_particles(k, hp)
        step_once()
        for k, hp in enumerate(hps):
            ctx.get_particles(k, out=hp)
        t1 = time.perf_counter()
        if s_ > 0:
            e2e_t.append(t1 - t0)
            e2e_pairs.append(float(np.count_nonzero(hps[0].kind != md.KIND_INACTIVE)) ** 2
                             if ionizing else pairs_per_step)
        if ionizing:   # back to the reached state for the next end-to-end step
            for k in ("x", "u", "z", "mass", "w", "kind"):
                getattr(hps[0], k)[...] = getattr(reached, k)
    e2e_local = float(np.mean(e2e_t))
    e2e_max = dist.max(e2e_local)
    e2e_value = (1 if sliced else world) * float(np.mean(e2e_pairs)) / e2e_max

    cpu = None
    force_err = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, threads, nt, secs, force_err = cpu_oracle_rate(w, args.cpu_seconds, e_gpu=e_gpu0)
        cpu = {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": f"FP64 field at {nt} sampled targets from all {w.cluster.n} sources "
                         f"({nt * w.cluster.n:.3g} pairs, {secs:.1f} s, OpenMP over targets)",
               "steps_per_s": rate / (float(w.cluster.n) ** 2),
               "single_thread": single_thread_rate(w, 3.0)}

    launches_per_step = info.get("kernels_per_step", 1)
    ctx.close()
    secondary = None
    if (rank == 0 and world == 1 and args.workload == "xe3_200k" and not args.no_secondary):
        t_sec = time.perf_counter()
        secondary = secondary_measurements(md, stream, flush, sms, gpu_id_for(local), tuning)
        secondary["wall_s"] = time.perf_counter() - t_sec
    dist.close()
    if rank != 0:
        return
    line = {
        "metric": METRIC,
        "value": value,
        "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_per_step,
        "steps_per_s": 1e3 / ms_per_step,
        "higher_is_better": True,
        "scaling": "strong" if sliced else "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic",
        "config": {
            "workload": (WORKLOAD_TEXT["xe3_200k_shard"] if sliced else
                         WORKLOAD_TEXT[args.workload]).format(name=w.name, n=n,
                                                              clusters=len(ws), atoms=args.n,
                                                              rates=args.rates, ranks=world),
            "n_particles": n, "pairs_per_step": pairs_per_step, "ionization": ion_state,
            "softening_nm": 0.1, "dt": w.dt, "a0": w.a0, "envelope": "sin2, 100 fs FWHM",
            "l2": f"flushed between timed steps ({L2_FLUSH_BYTES >> 20} MB write outside the "
                  "timed events)",
            "tuning": {"threads": tuning[0], "r": tuning[1], "tile": tuning[2],
                       "source_split": (f"equal shares, {-tuning[4]} per resident CTA"
                                        if tuning[4] < 0 else
                                        f"{tuning[4]} segments per i-block"),
                       "jsplit": tuning[4], "packed_f32x2": bool(tuning[5]),
                       "min_blocks": tuning[6]},
            "autotune_configs": [list(t) for t in md.tuning_list()],
            "autotune_ms_per_step": tune_ms,
            "device": gpu_name, "sms": sms, "wall_s_timed_region": wall,
        },
        "roofline": {
            "bound": "alu",
            "achieved": achieved / 1e9,
            "peak": (peak_clock or peak_max) / 1e9,
            "unit": "Gpair/s",
            "frac": achieved / (peak_clock or peak_max),
            "peak_basis": ("128 FP32 lanes x SMs x median SM clock under load / 12 FP32 "
                           "instructions per pair" if peak_clock else
                           "128 FP32 lanes x SMs x 2070 MHz / 12"),
            "frac_at_max_clock": achieved / peak_max,
            "frac_of_measured_ffma": achieved / peak_probe,
            "measured_ffma_tflops": 2 * ffma_per_s / 1e12,
            "measured_packed_f32x2_fma_tflops": 2 * ffma2_per_s / 1e12,
            "traffic": STEP_TRAFFIC_BYTES.get((args.workload, n, tuning[0], tuning[1],
                                                tuning[2], bool(tuning[5]), tuning[4])),
            "traffic_unit": "B per launch (dram read + write, ncu)",
        },
        "clocks": clocks,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": RECORD_BYTES * n,
                "d2h_bytes_per_step": RECORD_BYTES * n, "wall_s_per_step": e2e_max,
                "what": "md_set_particles + md_step(1) + md_get_particles from pinned host "
                        "arrays, wall clock"},
        "gpu_launches": args.steps * launches_per_step,
        "cpu_baseline": cpu,
        "force_err_vs_fp64": force_err,
        "precision_study": precision,
        "secondary": secondary,
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------ reference --

def run_reference(args):
    """The FP64 oracle on the host cores: each step is a bounded sample (fields
    at sampled targets from all sources) of the same workload."""
    world, rank, _ = dist_env()
    if rank != 0:
        return
    w = workload(args.n, seed=0)
    n = w.cluster.n
    per_step = min(args.cpu_seconds, max(0.2, 150.0 / max(1, args.steps + args.warmup)))
    rates = []
    for s in range(args.warmup + args.steps):
        rate, threads, nt, secs, _ = cpu_oracle_rate(w, per_step, seed=s)
        if s >= args.warmup:
            rates.append((rate, nt, secs))
    value = float(np.mean([r[0] for r in rates]))
    pairs_per_step = float(n) * n
    ms = 1e3 * pairs_per_step / value
    line = {
        "metric": METRIC, "impl": "reference", "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "steps_per_s": value / pairs_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"{w.name}: N={n}", "n_particles": n,
                   "pairs_per_step": pairs_per_step},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": f"per step: FP64 field at ~{rates[0][1]} sampled targets "
                                   f"from all {n} sources"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload in ("iedf", "iedf_xe"):
        run_iedf(args)
    elif args.workload == "nscale":
        run_nscale(args)
    else:
        run_native(args)


if __name__ == "__main__":
    main()
