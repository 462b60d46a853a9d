"""Host logic of bench.py's multi-rank (torchrun, N > 1) path, run as two gloo ranks on the
CPU: each rank's instance slice, the max-over-ranks timing reduction, the whole-job rate, and
the reference arm doing no work on ranks other than 0."""
import os
import socket

import numpy as np
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, outdir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    B, n, p, m = 3, 6, 5, 2
    batch, g = bench.rank_batch(rank, B, n, p, m)
    times = [1.0 + rank, 5.0 - rank, 2.0 * (rank + 1)]
    mx = bench.max_over_ranks(times, "cpu", dist)
    rate = bench.whole_job_rate(world, B, mx[0])
    ref_out = bench.run_reference(None) if rank != 0 else "skipped"
    np.savez(os.path.join(outdir, f"rank{rank}.npz"), Q=batch.Q, g=g, mx=np.array(mx),
             rate=rate, ref_none=ref_out is None)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_instances_and_reduce_timings(tmp_path):
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       join=True, start_method="spawn")
    import bench
    full, gfull = bench.rank_batch(0, 3 * world, 6, 5, 2)   # the single-process batch of N·B
    for rank in range(world):
        r = np.load(tmp_path / f"rank{rank}.npz")
        assert np.array_equal(r["Q"], full.Q[3 * rank:3 * rank + 3])       # disjoint slices
        assert np.array_equal(r["g"], gfull[3 * rank:3 * rank + 3])
        assert list(r["mx"]) == [2.0, 5.0, 4.0]                             # max over ranks
        assert abs(float(r["rate"]) - world * 3 / (2.0 / 1e3)) < 1e-9
    assert bool(np.load(tmp_path / "rank1.npz")["ref_none"])                # no work off rank 0
