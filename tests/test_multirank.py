"""The N > 1 path of bench.py on CPU ranks (gloo, world size 2).

Under torchrun every rank runs an independent walker population (replicas:
walkers never interact within a step, so the path needs no data-path
collective).  What crosses ranks is only the measurement: the timed region's
maximum over ranks and the sums of electron moves and force evaluations.
These tests run those reductions, the rank-dependent seeding and the
"rank 0 prints one line" rule on two gloo processes.
"""
import json
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, out_dir):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(ws), MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port),
                      LOCAL_RANK=str(rank), QMC_BENCH_BACKEND="gloo")
    sys.path.insert(0, ROOT)
    import bench
    from paper_2504_07948_gb300 import synth
    r, w, dist = bench.dist_init()
    assert (r, w) == (rank, ws) and dist is not None
    # per-rank work and time as the GPU path would report them
    moves = 1000.0 * (rank + 1)
    sec = 0.5 + rank
    out = {
        "max_sec": bench.max_over_ranks(sec, dist),
        "sum_moves": bench.sum_over_ranks(moves, dist),
        # the replica's initial walkers: seeded by rank
        "R0_checksum": float(synth.initial_walkers(synth.water_system(1), 4,
                                                   seed=synth.SEED_WALKERS + rank).sum()),
    }
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump(out, f)
    dist.barrier()
    dist.destroy_process_group()


def test_replica_reductions_two_gloo_ranks(tmp_path):
    ws = 2
    mp.start_processes(_worker, args=(ws, _free_port(), str(tmp_path)), nprocs=ws, join=True, start_method="spawn")
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(ws)]
    for r in res:
        assert r["max_sec"] == pytest.approx(1.5)            # slowest rank sets the time
        assert r["sum_moves"] == pytest.approx(3000.0)       # whole-job moves
    # independent replicas: different initial populations
    assert res[0]["R0_checksum"] != res[1]["R0_checksum"]
    # value = all ranks' moves / max-over-ranks time
    assert res[0]["sum_moves"] / res[0]["max_sec"] == pytest.approx(2000.0)


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.0, None) == 3.0
    assert bench.sum_over_ranks(4.0, None) == 4.0
    env = {k: os.environ.pop(k) for k in ("WORLD_SIZE",) if k in os.environ}
    try:
        assert bench.dist_init() == (0, 1, None)
    finally:
        os.environ.update(env)
    assert np.isfinite(bench.FP32_PEAK_TFLOPS_NOMINAL)
