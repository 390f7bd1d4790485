"""The N > 1 path of bench.py on CPU: two gloo ranks aggregate their step counts and times the
way the GPU ranks do (all ranks' DoF-steps over the slowest rank's time); every rank runs its
own independent cavity, so nothing else is exchanged."""
import json
import os
import socket

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    import torch.distributed as dist
    r, w, _ = bench.dist_env()
    bench.init_dist(w)
    units = 1000.0 * (r + 1)          # rank r did (r + 1) thousand DoF-steps ...
    seconds = 0.5 + 0.25 * r          # ... in 0.5 + 0.25 r seconds
    rate = bench.job_rate(units, seconds, w)
    mx = bench.reduce_max(seconds, w)
    dist.barrier()
    if r == 0:
        with open(out, "w") as f:
            json.dump({"rate": rate, "max": mx, "world": w}, f)
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_two_rank_aggregation(tmp_path, world):
    out = str(tmp_path / "agg.json")
    mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
    res = json.load(open(out))
    assert res["world"] == world
    assert res["max"] == pytest.approx(0.75)
    assert res["rate"] == pytest.approx((1000.0 + 2000.0) / 0.75)
