"""The multi-GPU split of one cluster by target records, on CPU: two or three
gloo ranks each push their slice of a 3000-record Xe3+ cluster with the
FP64 oracle's pieces (field of all sources at the slice's targets, laser,
Boris kick, drift) and exchange their slices of the j-stream with
shard.exchange after every step.  After three steps each rank's slice equals
the oracle's unsplit run, and each rank's j-stream holds every record's
position: the slice bounds, the padded all-gather and the copy-back cover the
cluster exactly once.  The partition itself is checked for several sizes."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
STEPS = 3
N = 3000


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_slice_bounds_partition_the_records():
    from paper_1307_3711_gb300 import shard
    for n in (1, 1023, 1024, 3000, 200000, 200003):
        for world in (1, 2, 3, 8):
            seen = np.zeros(n, np.int32)
            pers = set()
            for r in range(world):
                b, e, per = shard.slice_bounds(n, world, r)
                assert (b % shard.SLICE_ALIGN == 0 or b == e == n)
                assert per % shard.SLICE_ALIGN == 0
                assert e == n or e % shard.SLICE_ALIGN == 0
                assert 0 <= e - b <= per
                seen[b:e] += 1
                pers.add(per)
            assert (seen == 1).all() and len(pers) == 1


def _rank(rank, world, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    import oracle
    from paper_1307_3711_gb300 import shard, synth
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = synth.xe3_cluster(N, seed=4)
    c = w.cluster
    kc = oracle.coulomb_constant(w.lambda_um)
    st = oracle.State(c.x, c.u, c.z, c.mass, c.w)
    qs, qm = st.q(), st.qm()
    b, e, per = shard.slice_bounds(c.n, world, rank)
    x, u = st.x.copy(), st.u.copy()
    jst = torch.tensor(np.c_[x, kc * qs])      # the j-stream: (x, y, z, K_C w z)
    own = np.arange(b, e)
    for step in range(STEPS):
        t = w.t0 + step * w.dt
        xs = jst[:, :3].numpy().copy()
        ef = oracle.coulomb_field(xs[b:e], xs, qs, w.eps, kc, self_idx=own)
        a, bf = oracle.laser_fields(t, w.a0, w.pol, w.env, w.tau)
        for k, i in enumerate(own):
            u[i] = oracle.boris_kick(u[i], ef[k] + a, bf, qm[i], w.dt)
            x[i] = oracle.drift(x[i], u[i], w.dt)
        jst[b:e, :3] = torch.tensor(x[b:e])
        shard.exchange(jst, per, world, rank)
    q.put((rank, b, e, x[b:e].copy(), u[b:e].copy(), jst[:, :3].numpy().copy()))
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_gloo_ranks_split_one_cluster(world):
    import torch.multiprocessing as mp
    sys.path.insert(0, ROOT)
    import oracle
    from paper_1307_3711_gb300 import synth
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    ps = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in ps:
        p.start()
    out = sorted((q.get(timeout=300) for _ in ps), key=lambda o: o[0])
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    w = synth.xe3_cluster(N, seed=4)
    c = w.cluster
    ref = oracle.State(c.x, c.u, c.z, c.mass, c.w)
    p = oracle.make_params(a0=w.a0, tau=w.tau, t0=w.t0, dt=w.dt, eps=w.eps, pol=w.pol,
                           env=w.env, lambda_um=w.lambda_um)
    oracle.md_steps(ref, p, STEPS)
    assert out[0][1] == 0 and out[-1][2] == N
    assert all(out[k][2] == out[k + 1][1] for k in range(world - 1))
    scale = np.abs(ref.x).max()
    for _, b, e, x, u, jx in out:
        np.testing.assert_allclose(x, ref.x[b:e], rtol=0, atol=1e-12 * scale)
        np.testing.assert_allclose(u, ref.u[b:e], rtol=1e-10, atol=1e-14)
        # every rank's j-stream holds every record's new position
        np.testing.assert_allclose(jx, ref.x, rtol=0, atol=1e-12 * scale)
