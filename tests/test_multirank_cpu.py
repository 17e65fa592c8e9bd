"""The replica logic of bench.py under two gloo ranks on CPU: each rank draws
its own windows (no data-path collective), the job time is the slowest rank's
(all-reduce MAX) and the throughput counts every rank's work."""
import os
import socket

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench
from paper_2603_08386_gb300 import synth


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sc = synth.config3_window(0, 0, seed=bench.rank_seed(rank), W=64, H=48, mean_per_px=6.0)
    win = (sc.x, sc.y, sc.t, sc.p, sc.t0, sc.window_us, sc.n)
    terms = bench.terms_of(win, sc.W, sc.H, sc.grid[3])
    fake_ms = 100.0 + 50.0 * rank
    ms = bench.max_over_ranks(fake_ms, dist, "cpu")
    allt = torch.zeros(world, dtype=torch.float64)
    allt[rank] = terms
    dist.all_reduce(allt)
    digest = torch.tensor([float(np.int64(sc.t[:1000].sum() % 1_000_003))], dtype=torch.float64)
    ds = [torch.zeros(1, dtype=torch.float64) for _ in range(world)]
    dist.all_gather(ds, digest)
    dist.barrier()
    if rank == 0:
        out.put(dict(ms=ms, terms=allt.tolist(), digests=[float(d.item()) for d in ds],
                     value=bench.job_throughput(terms, world, 3, ms)))
    dist.destroy_process_group()


def test_two_gloo_ranks_replicas():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = q.get(timeout=240)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res["ms"] == 150.0                      # slowest rank
    assert res["digests"][0] != res["digests"][1]  # independent inputs per rank
    assert res["terms"][0] > 0 and res["terms"][1] > 0
    assert abs(res["value"] - res["terms"][0] * 2 * 3 / 0.150) < 1e-6 * res["value"]
