"""The multi-GPU form of the benchmark is replicas (one image per rank, no
data exchange): its host logic -- rank environment, the whole-job time (the
slowest rank) and work (the sum over ranks), rank 0 alone reporting -- on
two gloo ranks on the CPU."""
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, ws, lr = bench.rank_env()
        # rank k took k + 1 seconds for 10 (k + 1) units
        t, w = bench.replica_totals(dist, "cpu", float(rank + 1), 10 * (rank + 1))
        q.put((rank, r, ws, lr, t, w))
    finally:
        dist.destroy_process_group()


def test_replica_totals_two_gloo_ranks():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(k, world, port, q)) for k in range(world)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, r, ws, lr, t, w in got:
        assert (r, ws, lr) == (rank, world, rank)
        assert t == 2.0          # the slowest rank's time
        assert w == 30.0         # the work of both ranks


def test_replica_totals_single_process():
    import bench
    assert bench.replica_totals(None, "cpu", 1.5, 7) == (1.5, 7.0)


def test_reference_arm_other_ranks_exit_quietly():
    # under torchrun only rank 0 runs and prints the reference line
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--gpus", "2", "--steps", "1", "--warmup", "0"],
                       env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_icd_critical_path_of_the_sweep_counts():
    """bench.py's critical path of an incomplete projection: per pass the tile
    with the most sweeps, over the pass's tile grid (offset (1 << i) mod B),
    summed; a count list of the wrong length gives None."""
    import numpy as np
    import bench
    H, W, K = 20, 27, 2                      # B = 4: offsets 1, 2, 0
    counts = [((H - (1 << i) % 4) // 4) * ((W - (1 << i) % 4) // 4) for i in range(3)]
    assert counts == [4 * 6, 4 * 6, 5 * 6]
    sw = np.ones(sum(counts), np.int32)
    sw[3] = 9                                # pass 0
    sw[counts[0] + 5] = 4                    # pass 1
    sw[-1] = 2                               # pass 2 (last tile)
    r = bench.icd_critical_path(sw, H, W, K, 30e-6)
    assert r["longest_tile_sweeps_per_pass"] == [9, 4, 2] and r["sweeps"] == 15
    assert abs(r["us_per_sweep_on_it"] - 2.0) < 1e-12
    assert bench.icd_critical_path(sw[:-1], H, W, K, 30e-6) is None
