"""The multi-GPU form of the benchmark on CPU: two gloo ranks (world size 2) run the
cross-rank steps bench.py uses -- the barrier around the timed region, the maximum of the
per-rank times, the whole-job throughput from it -- and draw disjoint per-rank
workloads (independent boxes: weak scaling, no data-path collective)."""
import multiprocessing as mp
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_2508_06012_gb300 import workloads as w
    bench.barrier(world)
    t_max = bench.max_over_ranks(1.5 * (rank + 1), world)      # per-rank seconds
    boxes = w.uneven_batch(base_seed=20250807 + rank, nbox=64)       # as bench.ours() draws them
    bench.barrier(world)
    q.put((rank, t_max, [b["seed"] for b in boxes], len(boxes) * world / t_max))
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_time_and_draw_disjoint_boxes():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = [q.get(timeout=120) for _ in ps]
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    assert out[0][1] == out[1][1] == pytest.approx(3.0)        # max over ranks
    assert out[0][3] == out[1][3] == pytest.approx(128 / 3.0)  # whole-job rate: all ranks' boxes
    assert not set(out[0][2]) & set(out[1][2])                 # independent boxes per rank
