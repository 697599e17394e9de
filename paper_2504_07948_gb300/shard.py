"""Walker sharding across processes (one GPU per process).

One DMC population is split over the ranks of a torch.distributed process
group.  Within a step the walkers are independent (Sec. "Quantum Monte
Carlo"), so each rank sweeps, evaluates and branches its own walkers; the
only exchange per step is the sum of the step's sums (weights, weighted
energies, populations, reference populations and, when forces are sampled,
the force-estimator sums), which the library hands to a reduce callback
(``qmc_set_step_reduce``) and from which every rank sets the same trial
energy and records the same estimator samples.  Branching lets the shard
populations drift apart; ``rebalance`` moves whole walkers (positions; the
receiving rank rebuilds their state) from the fullest to the emptiest ranks.

This module only marshals: the arithmetic of the step (weights, trial
energy, estimators) stays in the library; here are the collective, the
bookkeeping of who sends how many walkers, and the point-to-point moves.
"""
from __future__ import annotations

import ctypes as C
from typing import List, Optional, Sequence, Tuple

import numpy as np

from . import qmc as Q


class StepReducer:
    """A REDUCE_FN that sums its buffer over the ranks of `group` with
    torch.distributed.all_reduce (on a CUDA tensor for the NCCL backend, a
    CPU tensor otherwise)."""

    def __init__(self, group=None, device: Optional[str] = None):
        import torch
        import torch.distributed as dist
        self.dist = dist
        self.group = group
        backend = dist.get_backend(group)
        self.device = device or ("cuda" if backend == "nccl" else "cpu")
        self.torch = torch
        self.calls = 0
        self.fn = Q.REDUCE_FN(self._reduce)

    def _reduce(self, buf, n, ctx) -> int:
        try:
            a = np.ctypeslib.as_array(buf, shape=(n,))
            t = self.torch.from_numpy(a.copy()).to(self.device)
            self.dist.all_reduce(t, group=self.group)
            a[:] = t.cpu().numpy()
            self.calls += 1
            return 0
        except Exception:   # a failed collective fails the DMC step (QMC_ERR_STATE)
            return 1

    def __call__(self, a: np.ndarray) -> np.ndarray:
        """Sums a float64 array over the ranks in place through the same path
        the library takes (for tests and for callers' own sums)."""
        a = np.ascontiguousarray(a, dtype=np.float64)
        st = self.fn(a.ctypes.data_as(C.POINTER(C.c_double)), int(a.shape[0]), None)
        if st != 0:
            raise RuntimeError("all-reduce failed")
        return a


def attach(qmc, reducer: StepReducer, pop_ref: Optional[float] = None):
    """Makes every later qmc_dmc step of `qmc` use the sums over all ranks.
    pop_ref: this rank's share of the reference population (default: its
    population now); keeping it fixed across rebalancing keeps the summed
    reference equal to the initial total population."""
    Q.qmc_set_step_reduce(qmc.h, reducer.fn)
    Q.qmc_set_population_reference(qmc.h, float(qmc.n_walkers if pop_ref is None else pop_ref))
    qmc._reducer = reducer   # keep the callback alive while the handle can call it


def detach(qmc):
    Q.qmc_set_step_reduce(qmc.h, None)
    Q.qmc_set_population_reference(qmc.h, 0.0)
    qmc._reducer = None


def plan_rebalance(pops: Sequence[int], threshold: float = 0.1) -> List[Tuple[int, int, int]]:
    """Moves (src, dst, count) that bring every rank's population to the mean
    (floor or ceiling; lower ranks take the remainder) when the largest
    deviation from the mean exceeds `threshold` of it; [] otherwise.  Greedy
    pairing of the largest surplus with the largest deficit, deterministic,
    so every rank computes the same plan from the same populations."""
    pops = [int(p) for p in pops]
    R = len(pops)
    tot = sum(pops)
    if R < 2 or tot == 0:
        return []
    mean = tot / R
    if max(abs(p - mean) for p in pops) <= threshold * mean:
        return []
    target = [tot // R + (1 if r < tot % R else 0) for r in range(R)]
    surplus = [p - t for p, t in zip(pops, target)]
    moves = []
    while True:
        s = max(range(R), key=lambda r: (surplus[r], -r))
        d = min(range(R), key=lambda r: (surplus[r], r))
        if surplus[s] <= 0 or surplus[d] >= 0:
            break
        k = min(surplus[s], -surplus[d])
        moves.append((s, d, k))
        surplus[s] -= k
        surplus[d] += k
    return moves


def exchange(R: np.ndarray, moves: Sequence[Tuple[int, int, int]], rank: int, group=None,
             device: str = "cpu") -> np.ndarray:
    """Applies a plan to this rank's walkers R [W, N, 3]: a sender gives away
    its last `count` walkers, a receiver appends what it gets.  Every rank
    walks the same list of moves, so sends and receives pair up."""
    import torch
    import torch.distributed as dist
    R = np.ascontiguousarray(R, dtype=np.float64)
    for (s, d, k) in moves:
        if rank == s:
            t = torch.from_numpy(np.ascontiguousarray(R[R.shape[0] - k:])).to(device)
            dist.send(t, dst=d, group=group)
            R = R[:R.shape[0] - k]
        elif rank == d:
            t = torch.empty((k,) + R.shape[1:], dtype=torch.float64, device=device)
            dist.recv(t, src=s, group=group)
            R = np.concatenate([R, t.cpu().numpy()], axis=0)
    return R


def populations(n_local: int, group=None, device: str = "cpu") -> List[int]:
    import torch
    import torch.distributed as dist
    t = torch.zeros(dist.get_world_size(group), dtype=torch.float64, device=device)
    t[dist.get_rank(group)] = float(n_local)
    dist.all_reduce(t, group=group)
    return [int(round(v)) for v in t.cpu().tolist()]


def rebalance(qmc, threshold: float = 0.1, group=None, device: str = "cpu") -> List[Tuple[int, int, int]]:
    """Evens out the shard populations of a sharded handle when they drift
    more than `threshold` from the mean: walker positions move between
    ranks, every rank that sent or received rebuilds its walkers' state
    (qmc_set_walkers), and the rank's reference population is left as it
    was.  Returns the plan (the same on every rank)."""
    import torch.distributed as dist
    rank = dist.get_rank(group)
    pops = populations(qmc.n_walkers, group, device)
    moves = plan_rebalance(pops, threshold)
    if any(rank in (s, d) for s, d, _ in moves):
        R, _ = qmc.get_walkers()
        # the reference population set by attach() is kept by the library
        # across qmc_set_walkers
        Q.qmc_set_walkers(qmc.h, exchange(R, moves, rank, group, device))
    return moves
