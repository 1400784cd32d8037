"""The bench's multi-GPU logic (replicas only, no collective on the data path) on
two CPU ranks over gloo: each rank gets its own images, the timing is the
slowest rank's, and the whole-job value counts all ranks' work."""
import json
import os
import socket

import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, outdir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local = 1.0 + 0.25 * rank                      # this rank's step time
    slowest = bench.max_over_ranks(local, world, device="cpu")
    seeds = list(bench.replica_seeds(rank, 8))
    dist.barrier()
    with open(os.path.join(outdir, f"r{rank}.json"), "w") as fh:
        json.dump({"slowest": slowest, "seeds": seeds}, fh)
    dist.destroy_process_group()


def test_two_replicas_over_gloo(tmp_path):
    world = 2
    mp.spawn(_rank, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    res = [json.load(open(tmp_path / f"r{r}.json")) for r in range(world)]
    assert res[0]["slowest"] == res[1]["slowest"] == 1.25
    assert not set(res[0]["seeds"]) & set(res[1]["seeds"])   # independent problems
    assert len(res[0]["seeds"]) == len(res[1]["seeds"]) == 8
    import bench
    # all ranks' pixels over the slowest rank's time
    assert abs(bench.whole_job_value(world, 481 * 321 * 256, 1.25e-3) - 2 * 481 * 321 * 256 / 1.25e-3 / 1e6) < 1e-9
    assert bench.max_over_ranks(3.5, 1) == 3.5
