"""The bench's multi-rank host logic on the CPU: two gloo ranks (127.0.0.1),
process-group setup from the torchrun environment, the barrier, and the
max over ranks that the timing takes."""
import multiprocessing as mp
import os
import socket


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank: int, port: int, q) -> None:
    os.environ.update(RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE="2",
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    import bench
    r, w, _ = bench.dist_setup(2)
    bench.barrier(w)
    v = bench.reduce_max(1.5 * (r + 1), w)
    q.put((r, w, dist.get_backend(), v))
    bench.barrier(w)
    dist.destroy_process_group()


def test_two_gloo_ranks_max_over_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    try:
        got = sorted(q.get(timeout=120) for _ in range(2))
    finally:
        for p in ps:
            p.join(timeout=60)
            if p.is_alive():
                p.kill()
    assert got == [(0, 2, "gloo", 3.0), (1, 2, "gloo", 3.0)]
    assert all(p.exitcode == 0 for p in ps)
