"""Walker sharding (one population over several ranks, one exchange per DMC
step) on CPU ranks: gloo, world size 2.

What crosses ranks is the step reduction the library calls back into
(shard.StepReducer) and the walkers that rebalancing moves; the trial
energy is the library's own (qmc_trial_energy, pure host code) applied to
the summed step sums.  The CUDA steps themselves are covered on the GPU by
tests/test_gpu_shard.py.
"""
import json
import math
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _qmc():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2504_07948_gb300 import qmc
    return qmc


def test_trial_energy_update():
    """Mean of the last (up to) 20 clipped-energy means, minus
    ln(W / W0) / (10 tau) for birth/death control; the window, the sign of
    the feedback and the fixed-population form."""
    Q = _qmc()
    h = np.arange(30, dtype=float)
    assert Q.qmc_trial_energy(h[:5], 100, 100, 0.01) == pytest.approx(2.0)
    assert Q.qmc_trial_energy(h, 100, 100, 0.01) == pytest.approx(np.mean(h[10:]))
    up = Q.qmc_trial_energy(h[:5], 110, 100, 0.01)
    assert up == pytest.approx(2.0 - math.log(1.1) / 0.1) and up < 2.0     # too many walkers: E_T drops
    assert Q.qmc_trial_energy(h[:5], 90, 100, 0.01) > 2.0
    assert Q.qmc_trial_energy(h[:5], 1e6, 100, 0.01, fixed_pop=True) == pytest.approx(2.0)
    with pytest.raises(Q.QmcError):
        Q.qmc_trial_energy(h[:5], 0, 100, 0.01)


@pytest.mark.parametrize("pops,mv", [
    ([37, 11], [(0, 1, 13)]),
    ([10, 10, 10], []),
    ([10, 11, 9], []),                       # within 10 % of the mean
    ([50, 0, 10, 20], [(0, 1, 20), (0, 2, 10)]),
])
def test_plan_rebalance(pops, mv):
    from paper_2504_07948_gb300 import shard
    plan = shard.plan_rebalance(pops, 0.1)
    assert plan == mv
    after = list(pops)
    for s, d, k in plan:
        assert k > 0
        after[s] -= k
        after[d] += k
    assert sum(after) == sum(pops)
    if plan:
        assert max(after) - min(after) <= 1


def _worker(rank, ws, port, out_dir):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(ws), MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    dist.init_process_group("gloo")
    Q = _qmc()
    from paper_2504_07948_gb300 import shard
    red = shard.StepReducer()
    out = {}
    # (1) the callback the library calls: each rank's step sums -> their sum
    rng = np.random.default_rng(rank)
    local = rng.uniform(1.0, 2.0, size=9)
    out["local"] = local.tolist()
    out["summed"] = red(local.copy()).tolist()
    # (2) the sharded trial energy: per-rank step sums (sum w, sum w clip(E),
    # population, reference population) of three steps; every rank sets E_T
    # from the sums over ranks with the library's own update
    hist = []
    et = None
    for step in range(3):
        w = rng.uniform(0.5, 1.5, size=20 + 5 * rank)
        e = rng.normal(-76.0, 1.0, size=w.shape[0])
        sums = red(np.array([w.sum(), (w * e).sum(), float(w.shape[0]), 20.0 + 5 * rank]))
        hist.append(sums[1] / sums[0])
        et = Q.qmc_trial_energy(np.array(hist), sums[2], sums[3], 0.01)
        out.setdefault("parts", []).append([w.sum(), (w * e).sum(), float(w.shape[0])])
    out["e_trial"] = et
    out["calls"] = red.calls
    # (3) rebalancing: 37 and 11 walkers -> 24 and 24, the walkers themselves
    # move (checked by their coordinates)
    R = np.arange((37 if rank == 0 else 11) * 2 * 3, dtype=float).reshape(-1, 2, 3) + 1000.0 * rank
    pops = shard.populations(R.shape[0])
    plan = shard.plan_rebalance(pops, 0.1)
    R2 = shard.exchange(R, plan, rank)
    out["pops"] = pops
    out["plan"] = plan
    out["R_after"] = R2.reshape(R2.shape[0], -1)[:, 0].tolist()
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump(out, f)
    dist.barrier()
    dist.destroy_process_group()


def test_sharded_reduction_trial_energy_and_rebalancing_two_gloo_ranks(tmp_path):
    ws = 2
    mp.start_processes(_worker, args=(ws, _free_port(), str(tmp_path)), nprocs=ws, join=True, start_method="spawn")
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(ws)]
    total = np.array(res[0]["local"]) + np.array(res[1]["local"])
    for r in res:
        assert np.allclose(r["summed"], total, rtol=1e-15)
        assert r["calls"] == 1 + 3
    # both ranks set the same trial energy, equal to the update over the
    # pooled samples of the whole population
    assert res[0]["e_trial"] == res[1]["e_trial"]
    Q = _qmc()
    hist = []
    for step in range(3):
        sw = res[0]["parts"][step][0] + res[1]["parts"][step][0]
        swe = res[0]["parts"][step][1] + res[1]["parts"][step][1]
        hist.append(swe / sw)
    pop = res[0]["parts"][2][2] + res[1]["parts"][2][2]
    assert res[0]["e_trial"] == pytest.approx(Q.qmc_trial_energy(np.array(hist), pop, 45.0, 0.01), rel=1e-14)
    # rebalancing moved the last 13 walkers of rank 0 to the end of rank 1
    assert res[0]["pops"] == [37, 11] and res[0]["plan"] == res[1]["plan"] == [[0, 1, 13]]
    first0 = [float(x) for x in np.arange(37 * 6).reshape(37, 6)[:, 0]]
    first1 = [float(x) + 1000.0 for x in np.arange(11 * 6).reshape(11, 6)[:, 0]]
    assert res[0]["R_after"] == first0[:24]
    assert res[1]["R_after"] == first1 + first0[24:]
