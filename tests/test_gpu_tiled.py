"""Walker-tiled mixed sweep (every walker moves the same electron; the
orbital contraction of Eq. 2 for all walkers is one tensor-core GEMM, the
delayed-update flush two batched tensor-core GEMMs) against the oracle and
against the fused one-CTA-per-walker delayed sweep, through the C ABI.

Mixed-form bounds of propagated state: the FP32 state against the oracle's
FP64 evaluation at the GPU's positions, ln|psi| 1e-5 and E_L 1e-3 relative
(the tensor-core contraction's error floor, about 4e-7 of sum |a b| per
element against 2e-8 for FP32 FMA chains, leaves the propagated local energy
at a few 1e-4 relative after two sweeps of these clusters); trajectories against the oracle's FP64 moves on the same random
stream agree walker by walker unless an acceptance test close to its
threshold flips (a flipped move shifts an electron by ~sqrt(tau)), so at
least 90 % of the walkers must match to 1e-3 bohr.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2504_07948_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def Q():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2504_07948_gb300 import qmc
    return qmc


def rel(a, b):
    a, b = np.asarray(a, dtype=float), np.asarray(b, dtype=float)
    return float((np.abs(a - b) / np.maximum(1.0, np.abs(b))).max())


def sweep_tiled(Q, monkeypatch, s, R, k, sweeps, tau, seed, tiled):
    monkeypatch.setenv("QMC_SWEEP_TILED", "1" if tiled else "0")
    monkeypatch.setenv("QMC_SWEEP_TILED_MIN_N", "4")
    g = Q.QMC(s, precision="mixed", seed=seed, delay_rank=k)
    g.set_walkers(R)
    Q.qmc_set_timing(g.h, True)
    g.vmc(sweeps, tau)
    ms, launches = Q.qmc_get_timing(g.h, "sweep_gemm")
    out = (g.get_walkers()[0], g.eval_cached(), g.evaluate(), launches)
    g.close()
    return out


@pytest.mark.parametrize("m,W,k", [(4, 37, 8), (4, 5, 4), (8, 70, 32)])
def test_tiled_sweep_follows_oracle(Q, monkeypatch, m, W, k):
    """4- and 8-water clusters (20 and 40 electrons per spin), ragged walker
    counts (several 4-walker CTAs, GEMM row tiles with a ragged tail), delay
    ranks 4, 8 and 32 (flushes inside and at the end of each spin block)."""
    s = synth.water_system(m)
    R = synth.initial_walkers(s, W, seed=40 + m)
    Rg, cached, fresh, launches = sweep_tiled(Q, monkeypatch, s, R, k, 2, 0.02, 818, True)
    N = s.n_elec
    assert launches == 2 * N   # one orbital GEMM per electron and sweep: the tiled sweep ran
    Ro, _, _ = O.Oracle(s).vmc(R, 2, 0.02, seed=818, step0=0, trace=False)
    same = np.abs(Rg - Ro).reshape(W, -1).max(axis=1) < 1e-3
    assert same.mean() >= 0.9, same.mean()
    ref = O.Oracle(s).evaluate(Rg)
    assert rel(cached["logpsi"], ref["logpsi"]) < 1e-5, rel(cached["logpsi"], ref["logpsi"])
    assert rel(cached["eloc"], ref["eloc"]) < 1e-3, rel(cached["eloc"], ref["eloc"])
    assert rel(fresh["logpsi"], ref["logpsi"]) < 1e-5


@pytest.mark.parametrize("groups,W,ng", [(2, 600, 2), (3, 1100, 3), (4, 1100, 3)])
def test_walker_groups_on_streams_match_one_group(Q, monkeypatch, groups, W, ng):
    """The tiled sweep's walker groups (whole 128-walker GEMM tiles, at least
    256 walkers each; here a ragged last group) run on separate streams and
    share no state: every GEMM row and every walker's move arithmetic is the
    one-group run's, so positions and the propagated state agree bit for
    bit."""
    s = synth.water_system(4)
    R = synth.initial_walkers(s, W, seed=77)
    monkeypatch.setenv("QMC_SWEEP_TILED_GROUPS", "1")
    a = sweep_tiled(Q, monkeypatch, s, R, 8, 2, 0.02, 919, True)
    monkeypatch.setenv("QMC_SWEEP_TILED_GROUPS", str(groups))
    b = sweep_tiled(Q, monkeypatch, s, R, 8, 2, 0.02, 919, True)
    N = s.n_elec
    assert a[3] == 2 * N and b[3] == 2 * N * ng   # one GEMM per electron, sweep and group
    assert np.array_equal(a[0], b[0])
    for key in ("logpsi", "eloc"):
        assert np.array_equal(a[1][key], b[1][key]), key
        assert np.array_equal(a[2][key], b[2][key]), key


def test_tiled_sweep_matches_fused_delayed_sweep_water32(Q, monkeypatch):
    """32-water cluster (160 electrons per spin, 768 GTOs), delay rank 32:
    the tiled and fused delayed sweeps make the same moves (FP32 rounding of
    the two contractions differs, a flipped decision would move an electron
    by ~0.14 bohr) and both propagated states match the oracle."""
    s = synth.water_system(32)
    R = synth.initial_walkers(s, 6, seed=23)
    a = sweep_tiled(Q, monkeypatch, s, R, 32, 2, 0.02, 717, True)
    b = sweep_tiled(Q, monkeypatch, s, R, 32, 2, 0.02, 717, False)
    assert a[3] == 2 * s.n_elec and b[3] == 0
    assert np.max(np.abs(a[0] - b[0])) < 2e-2
    ref = O.Oracle(s).evaluate(a[0])
    assert rel(a[1]["logpsi"], ref["logpsi"]) < 1e-5, rel(a[1]["logpsi"], ref["logpsi"])
    assert rel(a[1]["eloc"], ref["eloc"]) < 1e-3, rel(a[1]["eloc"], ref["eloc"])


def test_tiled_sweep_inside_dmc_with_forces(Q, monkeypatch):
    """The tiled sweep inside fixed-population DMC steps with forces (E_L,
    adjoint forces and branching read the state it leaves): finite energies
    and forces, the state consistent with a fresh evaluation."""
    monkeypatch.setenv("QMC_SWEEP_TILED_MIN_N", "4")
    s = synth.water_system(8)
    R = synth.initial_walkers(s, 24, seed=5)
    g = Q.QMC(s, precision="mixed", seed=99, delay_rank=16, fixed_population=True, cap_factor=4)
    g.set_walkers(R)
    out = g.dmc(3, 0.005, -600.0, forces_every=1)
    assert np.all(out["pop"] == 24) and np.all(np.isfinite(out["e_step"]))
    F, Fe = g.force_estimate(Q.QMC_EST_DMC)
    assert np.all(np.isfinite(F))
    cached, fresh = g.eval_cached(), g.evaluate()
    assert rel(cached["logpsi"], fresh["logpsi"]) < 1e-5
    g.close()
