"""Channel sharding for multi-GPU runs, on the CPU: the cost-balanced
contiguous partition covers every channel once and balances within one
channel's cost; two gloo ranks (127.0.0.1) split the batched workload the same
way, filter their own shards with the oracle, and the union equals the
unsharded result (no collective on the data path; the max over ranks of the
timing is the only exchange)."""
import multiprocessing as mp
import os
import socket

import numpy as np

from paper_2607_14054_gb300 import shard


def test_partition_covers_and_balances():
    rs = np.random.RandomState(3)
    for C, world in [(1, 1), (5, 8), (4096, 2), (4096, 8), (37, 3)]:
        lengths = rs.randint(1, 1 << 20, size=C)
        K = rs.randint(1, 9, size=C)
        costs = shard.channel_costs(lengths, K)
        parts = shard.partition_by_cost(costs, world)
        assert len(parts) == world and parts[0][0] == 0 and parts[-1][1] == C
        for (a, b), (c, d) in zip(parts, parts[1:]):
            assert b == c and a <= b
        loads = [sum(costs[a:b]) for a, b in parts]
        ideal = sum(costs) / world
        if C >= world:
            assert max(loads) - ideal <= max(costs) + 1e-6 * ideal


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank: int, port: int, q) -> None:
    os.environ.update(RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE="2",
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    import bench
    import oracle
    from synth import workloads
    r, w, _ = bench.dist_setup(2)
    wl = workloads.batched(n_channels=24, min_len=1000, max_len=20000, seed=5)
    lh = wl.lengths.tolist()
    parts = shard.partition_by_cost(shard.channel_costs(lh, wl.K.tolist()), w)
    c0, c1 = parts[r]
    xs, ss, ks, ls, zs = shard.shard(wl.x, wl.sos, wl.K, lh, wl.zi, c0, c1)
    y, _ = oracle.sosfilt(xs.double().numpy(), ss.numpy(), K=ks.numpy(), lengths=np.array(ls),
                          zi=zs.double().numpy())
    t = bench.reduce_max(float(len(y)), w)  # the one exchange: a max of a scalar
    q.put((r, c0, c1, y.tolist(), t))
    bench.barrier(w)
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_the_batch():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    try:
        got = sorted(q.get(timeout=180) for _ in range(2))
    finally:
        for p in ps:
            p.join(timeout=60)
            if p.is_alive():
                p.kill()
    assert all(p.exitcode == 0 for p in ps)
    import oracle
    from synth import workloads
    wl = workloads.batched(n_channels=24, min_len=1000, max_len=20000, seed=5)
    ref, _ = oracle.sosfilt(wl.x.double().numpy(), wl.sos.numpy(), K=wl.K.numpy(),
                            lengths=wl.lengths.numpy(), zi=wl.zi.double().numpy())
    (r0, a0, b0, y0, t0), (r1, a1, b1, y1, t1) = got
    assert (r0, r1) == (0, 1) and a0 == 0 and b0 == a1 and b1 == 24
    assert np.array_equal(np.concatenate([y0, y1]), ref)
    assert t0 == t1 == max(len(y0), len(y1))
