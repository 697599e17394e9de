"""CUDA path against the FP64 oracle, through the C ABI.

FP64 tolerance (stated for the FP64 form): |gpu - oracle| <= 1e-10 max(1,
|oracle|) for ln|psi|, E_L, electron gradients and ionic derivatives.  Sizes span several
CTAs and ragged walker counts; the 6-water cluster is the forces workload.
"""
import math

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


def close(a, b, tol):
    a, b = np.asarray(a), np.asarray(b)
    err = np.abs(a - b) / np.maximum(1.0, np.abs(b))
    return float(err.max()) <= tol, float(err.max())


def systems():
    rng = np.random.default_rng(31)
    small = synth.random_small_system(rng, n_nuc=3, n_up=3, n_dn=2)
    return {
        "water1": synth.water_system(1),
        "water6": synth.water_system(6),
        "small_all_shells": small,
        "hydrogen_exact": synth.hydrogenic_exact(1.0),
    }


@pytest.mark.parametrize("name,W", [("water1", 37), ("water6", 19), ("small_all_shells", 33),
                                    ("hydrogen_exact", 5)])
def test_evaluate_fp64(Q, name, W):
    s = systems()[name]
    R = synth.initial_walkers(s, W, seed=11)
    g = Q.QMC(s, precision="fp64")
    g.set_walkers(R)
    ev = g.evaluate()
    ref = O.Oracle(s).evaluate(R)
    for k, tol in (("logpsi", 1e-10), ("eloc", 1e-10), ("grad", 1e-10)):
        ok, err = close(ev[k], ref[k], tol)
        assert ok, (k, err)
    assert np.array_equal(ev["sign"], ref["sign"])
    if name == "hydrogen_exact":
        assert np.all(np.abs(ev["eloc"] + 0.5) < 1e-13)
    g.close()


@pytest.mark.parametrize("name,W", [("water1", 13), ("water6", 5), ("small_all_shells", 9)])
def test_forces_fp64(Q, name, W):
    s = systems()[name]
    R = synth.initial_walkers(s, W, seed=12)
    g = Q.QMC(s, precision="fp64")
    g.set_walkers(R)
    rng = np.random.default_rng(3)
    gE, gL = rng.normal(size=W), rng.normal(size=W)
    dR, pw = g.forces(gE, gL)
    dEL, dlg = O.Oracle(s).forces(R)
    ok, err = close(pw[:, 0], dEL, 1e-10)
    assert ok, ("dEL", err)
    ok, err = close(pw[:, 1], dlg, 1e-10)
    assert ok, ("dlogpsi", err)
    ref = np.tensordot(gE, dEL, axes=(0, 0)) + np.tensordot(gL, dlg, axes=(0, 0))
    ok, err = close(dR, ref, 1e-10)
    assert ok, ("vjp", err)
    g.close()


def test_autograd_function_matches_estimator(Q):
    import torch
    from paper_2504_07948_gb300.forces import ForceFn, zvzb_force
    s = synth.water_system(1)
    R = synth.initial_walkers(s, 24, seed=5)
    g = Q.QMC(s, precision="fp64")
    g.set_walkers(R)
    Rn = torch.tensor(s.R, dtype=torch.float64, requires_grad=True)
    eloc, logpsi = ForceFn.apply(Rn, g)
    F = zvzb_force(torch.tensor(s.R, dtype=torch.float64), g).numpy()
    o = O.Oracle(s)
    ev = o.evaluate(R)
    dEL, dlg = o.forces(R)
    ok, err = close(eloc.detach().numpy(), ev["eloc"], 1e-10)
    assert ok, err
    Fref = O.force_estimator(ev["eloc"], dEL, dlg)
    ok, err = close(F, Fref, 1e-8)
    assert ok, err
    # moving a nucleus through the Function re-evaluates at the new geometry
    R2 = s.R.copy(); R2[1, 0] += 0.01
    e2, _ = ForceFn.apply(torch.tensor(R2), g)
    s2 = s.copy(); s2.R = R2
    ok, err = close(e2.numpy(), O.Oracle(s2).evaluate(R)["eloc"], 1e-10)
    assert ok, err
    g.close()


@pytest.mark.parametrize("name,W,tau,sweeps", [("water1", 16, 0.05, 4), ("water6", 6, 0.02, 2),
                                              ("small_all_shells", 10, 0.1, 3)])
def test_vmc_trajectory_parity(Q, name, W, tau, sweeps):
    """Same Philox stream on both sides: identical proposals and accept
    decisions, so positions agree to rounding after several sweeps."""
    s = systems()[name]
    R = synth.initial_walkers(s, W, seed=13)
    g = Q.QMC(s, precision="fp64", seed=424242)
    g.set_walkers(R)
    g.vmc(sweeps, tau)
    Rg, _ = g.get_walkers()
    Ro, acc, _ = O.Oracle(s).vmc(R, sweeps, tau, seed=424242, step0=0, trace=False)
    assert np.max(np.abs(Rg - Ro)) < 1e-8
    assert acc.sum() > 0
    # the incrementally updated state equals a fresh evaluation
    ev = g.evaluate()
    ref = O.Oracle(s).evaluate(Ro)
    ok, err = close(ev["logpsi"], ref["logpsi"], 1e-9)
    assert ok, err
    g.close()


def test_vmc_trajectory_parity_more_shells_than_threads(Q):
    """12-water cluster (144 shells, more than the sweep's 128 threads): the
    live-shell scan of every move runs in two rounds and the live shells are
    evaluated from the compacted list; trajectories follow the oracle's."""
    s = synth.water_system(12)
    R = synth.initial_walkers(s, 3, seed=14)
    g = Q.QMC(s, precision="fp64", seed=4343)
    g.set_walkers(R)
    g.vmc(1, 0.02)
    Rg, _ = g.get_walkers()
    Ro, acc, _ = O.Oracle(s).vmc(R, 1, 0.02, seed=4343, step0=0, trace=False)
    assert np.max(np.abs(Rg - Ro)) < 1e-8
    assert acc.sum() > 0
    g.close()


def test_incremental_state_matches_recompute(Q):
    """After many Sherman-Morrison updates, E_L from the cached inverse equals
    E_L after a from-scratch recompute."""
    s = synth.water_system(6)
    R = synth.initial_walkers(s, 64, seed=21)
    g = Q.QMC(s, precision="fp64")
    g.set_walkers(R)
    tr = g.vmc(5, 0.02, trace=True)
    ev = g.evaluate()
    ok, err = close(tr[-1], ev["eloc"], 1e-8)
    assert ok, err
    g.close()


def test_dmc_exact_hydrogen(Q):
    s = synth.hydrogenic_exact(1.0)
    R = synth.initial_walkers(s, 300, seed=1)
    g = Q.QMC(s)
    g.set_walkers(R)
    out = g.dmc(20, 0.01, -0.5)
    assert np.all(out["pop"] == 300)
    assert np.all(np.abs(out["e_step"] + 0.5) < 1e-13)
    g.close()


def test_dmc_branching_matches_oracle_first_steps(Q):
    """With identical random streams the first DMC steps agree exactly:
    same moves, same weights, same copies, hence the same population and
    step energies."""
    s = synth.water_system(1)
    R = synth.initial_walkers(s, 40, seed=3)
    g = Q.QMC(s, seed=99, cap_factor=4)
    g.set_walkers(R)
    out = g.dmc(3, 0.005, -70.0)
    ref = O.Oracle(s).dmc(R, 3, 0.005, -70.0, seed=99, step0=0)
    assert np.array_equal(out["pop"], ref["pop"])
    ok, err = close(out["e_step"], ref["e_step"], 1e-9)
    assert ok, err
    g.close()


def test_dmc_fixed_population_matches_oracle(Q):
    """Fixed-population DMC (systematic resampling with the branching
    weights): the same random streams give the same population (constant) and
    step energies and positions to rounding; the exact hydrogen ground state
    keeps every walker with E = -1/2."""
    s = synth.water_system(1)
    R = synth.initial_walkers(s, 40, seed=3)
    g = Q.QMC(s, seed=99, cap_factor=4, fixed_population=True)
    g.set_walkers(R)
    out = g.dmc(3, 0.005, -70.0)
    ref = O.Oracle(s).dmc(R, 3, 0.005, -70.0, seed=99, step0=0, fixed_pop=True)
    assert np.all(out["pop"] == 40) and np.array_equal(out["pop"], ref["pop"])
    ok, err = close(out["e_step"], ref["e_step"], 1e-9)
    assert ok, err
    Rg, _ = g.get_walkers()
    assert np.max(np.abs(Rg - ref["R"])) < 1e-8
    g.close()
    h = synth.hydrogenic_exact(1.0)
    g = Q.QMC(h, fixed_population=True)
    g.set_walkers(synth.initial_walkers(h, 200, seed=1))
    out = g.dmc(10, 0.01, -0.5)
    assert np.all(out["pop"] == 200) and np.all(np.abs(out["e_step"] + 0.5) < 1e-13)
    g.close()


def blocking_error(x):
    x = np.asarray(x, dtype=np.float64)
    best = x.std(ddof=1) / math.sqrt(len(x))
    while len(x) >= 16:
        x = 0.5 * (x[: len(x) // 2 * 2:2] + x[1: len(x) // 2 * 2:2])
        best = max(best, x.std(ddof=1) / math.sqrt(len(x)))
    return best


def test_dmc_helium_ground_state_gpu(Q):
    """The nodeless He trial function projects to -2.903724 Ha on the GPU
    (same physics pin as the oracle's), and agrees with the oracle's DMC
    run on an independent random stream."""
    s = synth.helium_nodeless()
    R0 = synth.initial_walkers(s, 512)
    g = Q.QMC(s, seed=2024, cap_factor=4)
    g.set_walkers(R0)
    tr = g.vmc(200, 0.1, trace=True)
    out = g.dmc(1200, 0.01, float(tr[50:].mean()))
    e = out["e_step"][300:]
    mean, err = e.mean(), blocking_error(e)
    assert abs(mean + 2.903724) < 4 * err + 0.01, (mean, err)
    o = O.Oracle(s)
    Rv, _, tro = o.vmc(R0, 200, 0.1, seed=777)
    outo = o.dmc(Rv, 1200, 0.01, tro[50:].mean(), seed=778, step0=1000)
    eo = outo["e_step"][300:]
    assert abs(mean - eo.mean()) < 4 * math.sqrt(err ** 2 + blocking_error(eo) ** 2)
    g.close()


def test_dmc_statistical_parity_water1(Q):
    """Water monomer on its full schedule (512 walkers, 200 VMC sweeps at
    tau = 0.05, 500 DMC steps at tau = 0.005, first 20 % of each phase
    discarded), GPU and oracle on independent random streams from the same
    initial walkers; the means agree within two combined standard errors.

    The standard errors come from independent samples, not from blocking
    one run: the synthetic trial function's local energy is heavy-tailed
    (single walkers from -3e4 to +4e4 Ha) and keeps drifting through the
    schedule, so two oracle runs with different seeds differ by ~6 blocked
    errors of either run.  VMC walkers are independent chains, so the error
    of a run's mean is the spread of the walkers' time averages over
    sqrt(512); DMC walkers interact through population control, so each side
    runs 16 independent fixed-population replicas of 32 walkers and the
    error is the spread of the replica means over sqrt(16)."""
    s = synth.water_system(1)
    R0 = synth.initial_walkers(s, 512)
    nv, nd, tau_v, tau_d, nrep = 200, 500, 0.05, 0.005, 16
    o = O.Oracle(s)
    # VMC: one run of 512 independent chains per side
    g = Q.QMC(s, seed=1005, cap_factor=4)
    g.set_walkers(R0)
    wg = g.vmc(nv, tau_v, trace=True)[nv // 5:].mean(axis=0)
    g.close()
    wo = o.vmc(R0, nv, tau_v, seed=777)[2][nv // 5:].mean(axis=0)
    se = math.sqrt(wg.var(ddof=1) / wg.size + wo.var(ddof=1) / wo.size)
    assert abs(wg.mean() - wo.mean()) < 2 * se, (wg.mean(), wo.mean(), se)
    # DMC: independent replicas, VMC equilibration then DMC on each
    W = R0.shape[0] // nrep
    mg, mo = [], []
    for r in range(nrep):
        Rr = R0[r * W:(r + 1) * W]
        g = Q.QMC(s, seed=2000 + r, cap_factor=4, fixed_population=True)
        g.set_walkers(Rr)
        ev = float(g.vmc(nv, tau_v, trace=True)[nv // 2:].mean())
        outg = g.dmc(nd, tau_d, ev)
        assert np.all(outg["pop"] == W)
        mg.append(outg["e_step"][nd // 5:].mean())
        g.close()
        Rv, _, tro = o.vmc(Rr, nv, tau_v, seed=3000 + r)
        outo = o.dmc(Rv, nd, tau_d, float(tro[nv // 2:].mean()), seed=4000 + r, step0=nv, cap_factor=4,
                     fixed_pop=True)
        assert outo["status"] == 0 and np.all(outo["pop"] == W)
        mo.append(outo["e_step"][nd // 5:].mean())
    mg, mo = np.array(mg), np.array(mo)
    se = math.sqrt(mg.var(ddof=1) / nrep + mo.var(ddof=1) / nrep)
    assert abs(mg.mean() - mo.mean()) < 2 * se, (mg.mean(), mo.mean(), se)


def test_errors_are_status_codes(Q):
    s = synth.water_system(1)
    g = Q.QMC(s)
    with pytest.raises(Q.QmcError) as e:
        g.evaluate()                      # no walkers yet
    assert e.value.code == -7
    s2 = s.copy()
    s2.C = s.C.copy()
    s2.C[0, :] = 0.0                      # occupied orbital 0 vanishes: singular A
    g2 = Q.QMC(s2)
    with pytest.raises(Q.QmcError) as e:
        g2.set_walkers(synth.initial_walkers(s, 4))
    assert e.value.code == -3
    with pytest.raises(Q.QmcError) as e:
        Q.qmc_set_precision(g.h, 0, 33, 0)  # delay rank beyond the supported 32
    assert e.value.code == -9
    bad = synth.initial_walkers(s, 2)
    bad[0, 0, 0] = np.nan
    with pytest.raises(Q.QmcError) as e:
        g.set_walkers(bad)
    assert e.value.code == -1
    g.close(); g2.close()


def test_checkpoint_roundtrip(Q, tmp_path):
    s = synth.water_system(1)
    g = Q.QMC(s)
    g.set_walkers(synth.initial_walkers(s, 20))
    g.vmc(2, 0.05)
    p = str(tmp_path / "ck.bin")
    Q.qmc_checkpoint(g.h, p)
    R1, _ = g.get_walkers()
    g.vmc(2, 0.05)
    Ra, _ = g.get_walkers()
    Q.qmc_restore(g.h, p)
    R2, _ = g.get_walkers()
    assert np.array_equal(R1, R2)
    g.vmc(2, 0.05)
    Rb, _ = g.get_walkers()
    assert np.max(np.abs(Ra - Rb)) < 1e-10   # resume is reproducible (counter-based RNG)
    g.close()


# ----------------------------------------------------------------------
# multi-determinant expansions (table method)
# ----------------------------------------------------------------------

def msd_systems():
    rng = np.random.default_rng(41)
    small = synth.random_small_system(rng, n_nuc=2, n_up=2, n_dn=2)
    return {
        "water1_30": synth.with_multidet(synth.water_system(1), 30, n_active=8, max_exc=4, seed=5),
        "water6_200": synth.with_multidet(synth.water_system(6), 200, n_active=20, max_exc=4, seed=6),
        "small_12": synth.with_multidet(small, 12, n_active=6, max_exc=2, seed=7),
        "water1_single": synth.with_multidet(synth.water_system(1), 1, n_active=4),
    }


@pytest.mark.parametrize("name,W", [("water1_30", 17), ("water6_200", 9), ("small_12", 11), ("water1_single", 5)])
def test_evaluate_multidet_fp64(Q, name, W):
    """Table-method ratios (small determinants of T = A0^-1 A_v) against the
    oracle's determinant-by-determinant LU sum."""
    s = msd_systems()[name]
    R = synth.initial_walkers(s, W, seed=14)
    g = Q.QMC(s, precision="fp64")
    g.set_walkers(R)
    ev = g.evaluate()
    ref = O.Oracle(s).evaluate(R)
    assert np.array_equal(ev["sign"], ref["sign"])
    for k, tol in (("logpsi", 1e-10), ("eloc", 1e-10), ("grad", 1e-10)):
        ok, err = close(ev[k], ref[k], tol)
        assert ok, (k, err)
    g.close()


def test_evaluate_multidet_10k_water6_sampled(Q):
    """The 10,000-determinant expansion of the 6-water cluster (up to
    quadruple excitations into 20 active virtuals): every walker evaluated
    on the GPU, two sampled walkers by the oracle."""
    s = synth.with_multidet(synth.water_system(6), 10_000, n_active=20, max_exc=4)
    R = synth.initial_walkers(s, 64, seed=15)
    g = Q.QMC(s, precision="fp64")
    g.set_walkers(R)
    ev = g.evaluate()
    idx = [3, 41]
    ref = O.Oracle(s).evaluate(R[idx])
    assert np.array_equal(ev["sign"][idx], ref["sign"])
    for k, tol in (("logpsi", 1e-10), ("eloc", 1e-9), ("grad", 1e-8)):
        ok, err = close(ev[k][idx], ref[k], tol)
        assert ok, (k, err)
    g.close()


@pytest.mark.parametrize("name,W,tau,sweeps", [("water1_30", 8, 0.05, 3), ("small_12", 10, 0.1, 3)])
def test_vmc_trajectory_parity_multidet(Q, name, W, tau, sweeps):
    """Table-method sweep (rank-1 table updates, string ratios, S'/S) against
    the oracle's VMC, which refactorises every determinant of the sum after
    each proposal: same stream, same positions."""
    s = msd_systems()[name]
    R = synth.initial_walkers(s, W, seed=16)
    g = Q.QMC(s, precision="fp64", seed=515)
    g.set_walkers(R)
    g.vmc(sweeps, tau)
    Rg, _ = g.get_walkers()
    Ro, acc, _ = O.Oracle(s).vmc(R, sweeps, tau, seed=515, step0=0, trace=False)
    assert np.max(np.abs(Rg - Ro)) < 1e-8
    assert acc.sum() > 0
    ev = g.eval_cached()
    ref = O.Oracle(s).evaluate(Ro)
    for k, tol in (("logpsi", 1e-9), ("eloc", 1e-8)):
        ok, err = close(ev[k], ref[k], tol)
        assert ok, (k, err)
    g.close()


def test_dmc_first_steps_multidet(Q):
    """Same stream: identical populations; step energies from the propagated
    (rank-1 updated) tables agree to 1e-8 relative, the bound used for all
    propagated multi-determinant state (E_L of an expansion is a ratio of
    sums with cancellation)."""
    s = msd_systems()["water1_30"]
    R = synth.initial_walkers(s, 40, seed=17)
    g = Q.QMC(s, seed=99, cap_factor=4)
    g.set_walkers(R)
    out = g.dmc(3, 0.005, -70.0)
    ref = O.Oracle(s).dmc(R, 3, 0.005, -70.0, seed=99, step0=0)
    assert np.array_equal(out["pop"], ref["pop"])
    ok, err = close(out["e_step"], ref["e_step"], 1e-8)
    assert ok, err
    g.close()


@pytest.mark.parametrize("name,W", [("water1_30", 7), ("small_12", 9), ("water6_200", 3), ("water1_single", 4)])
def test_forces_multidet_fp64(Q, name, W):
    """Adjoint of ln|psi| and E_L of a determinant expansion (cofactor
    weights of every string pulled back to basis space) against the
    oracle's forward-mode derivatives, term by term over determinants."""
    s = msd_systems()[name]
    R = synth.initial_walkers(s, W, seed=18)
    g = Q.QMC(s, precision="fp64")
    g.set_walkers(R)
    rng = np.random.default_rng(4)
    gE, gL = rng.normal(size=W), rng.normal(size=W)
    dR, pw = g.forces(gE, gL)
    dEL, dlg = O.Oracle(s).forces(R)
    ok, err = close(pw[:, 1], dlg, 1e-10)
    assert ok, ("dlogpsi", err)
    ok, err = close(pw[:, 0], dEL, 1e-10)
    assert ok, ("dEL", err)
    ref = np.tensordot(gE, dEL, axes=(0, 0)) + np.tensordot(gL, dlg, axes=(0, 0))
    ok, err = close(dR, ref, 1e-10)
    assert ok, ("vjp", err)
    g.close()


@pytest.mark.parametrize("name,W", [("water1_30", 7), ("water6_200", 3)])
def test_forces_multidet_mixed(Q, name, W):
    """Mixed form of the expansion's adjoint (FP32 string cofactors, weights,
    pull-back and third-order basis contraction; FP64 per-atom sums) against
    the oracle at fixed configurations: ln|psi| derivatives within 1e-3 and
    E_L derivatives within 1e-4 of the largest per-walker magnitude (FP32
    storage of the inverse, tables and orbital derivatives)."""
    s = msd_systems()[name]
    R = synth.initial_walkers(s, W, seed=18)
    g = Q.QMC(s, precision="mixed")
    g.set_walkers(R)
    _, pw = g.forces()
    dEL, dlg = O.Oracle(s).forces(R)
    sc = np.maximum(1.0, np.abs(dlg).max(axis=(1, 2), keepdims=True))
    assert float((np.abs(pw[:, 1] - dlg) / sc).max()) < 1e-3
    sc = np.maximum(1.0, np.abs(dEL).max(axis=(1, 2), keepdims=True))
    assert float((np.abs(pw[:, 0] - dEL) / sc).max()) < 1e-4
    g.close()


def test_forces_gemm_path_fp64(Q, monkeypatch):
    """The large-determinant force path (batched GEMMs for PT, Q, M, Y)
    forced on for the 6-water cluster, against the oracle."""
    monkeypatch.setenv("QMC_FORCE_GEMM_MIN_N", "1")
    s = synth.water_system(6)
    R = synth.initial_walkers(s, 6, seed=19)
    g = Q.QMC(s, precision="fp64")
    g.set_walkers(R)
    _, pw = g.forces()
    dEL, dlg = O.Oracle(s).forces(R)
    ok, err = close(pw[:, 0], dEL, 1e-10)
    assert ok, ("dEL", err)
    ok, err = close(pw[:, 1], dlg, 1e-10)
    assert ok, ("dlogpsi", err)
    g.close()


def test_forces_gemm_path_mixed_tensor_cores(Q, monkeypatch):
    """Mixed form, GEMM force path forced on for the 6-water cluster: the
    tensor-core (3xTF32) products against the same path on cuBLAS SGEMM
    (FP32 SIMT) -- both FP32 accurate, so they agree to FP32 rounding of the
    summed terms -- and against the oracle at the mixed-form bound."""
    monkeypatch.setenv("QMC_FORCE_GEMM_MIN_N", "1")
    s = synth.water_system(6)
    R = synth.initial_walkers(s, 6, seed=19)
    g = Q.QMC(s, precision="mixed")
    g.set_walkers(R)
    _, pw_tc = g.forces()
    g.close()
    monkeypatch.setenv("QMC_FORCE_GEMM_CUBLAS", "1")
    g = Q.QMC(s, precision="mixed")
    g.set_walkers(R)
    _, pw_blas = g.forces()
    g.close()
    scale = np.maximum(1.0, np.abs(pw_blas).max(axis=(2, 3), keepdims=True))
    assert float((np.abs(pw_tc - pw_blas) / scale).max()) < 1e-4
    dEL, dlg = O.Oracle(s).forces(R)
    ok, err = close(pw_tc[:, 1], dlg, 1e-3)
    assert ok, ("dlogpsi", err)
    sc = np.maximum(1.0, np.abs(dEL).max(axis=(1, 2), keepdims=True))
    assert float((np.abs(pw_tc[:, 0] - dEL) / sc).max()) < 1e-4


@pytest.fixture(scope="module")
def water32_reference():
    s = synth.water_system(32)
    R = synth.initial_walkers(s, 2, seed=20)
    o = O.Oracle(s)
    ref = o.evaluate(R)
    dEL, dlg = o.forces(R)
    return s, R, ref, dEL, dlg


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_water32_sampled(Q, prec, water32_reference):
    """32-water cluster (320 electrons, 160 per spin, 768 GTOs): FP64
    shared-memory inverse at n = 160 and the GEMM force path, two walkers
    checked against the oracle.  Mixed form (fresh FP64 evaluation stored
    in FP32): ln|psi| 1e-5 relative (the stated target), E_L 1e-5 relative,
    ionic derivatives 1e-2 relative per walker."""
    s, R, ref, dEL, dlg = water32_reference
    g = Q.QMC(s, precision=prec)
    g.set_walkers(R)
    ev = g.evaluate()
    _, pw = g.forces()
    tol = dict(fp64=(1e-10, 1e-10, 1e-10), mixed=(1e-5, 1e-5, 1e-2))[prec]
    for k, t in (("logpsi", tol[0]), ("eloc", tol[1])):
        ok, err = close(ev[k], ref[k], t)
        assert ok, (k, err)
    ok, err = close(pw[:, 0], dEL, tol[2])
    assert ok, ("dEL", err)
    ok, err = close(pw[:, 1], dlg, tol[2])
    assert ok, ("dlogpsi", err)
    g.close()


@pytest.mark.parametrize("k", [1, 3, 8, 32])
def test_delayed_updates_fp64(Q, k):
    """Woodbury-queued inverse updates (delay rank k) follow the oracle's
    trajectory (which refactorises after every proposal) and leave an
    inverse equal to a fresh FP64 evaluation; k = 1 is Sherman-Morrison
    through the queue-and-flush code path."""
    s = synth.water_system(6)
    R = synth.initial_walkers(s, 8, seed=22)
    g = Q.QMC(s, precision="fp64", seed=616, delay_rank=k)
    g.set_walkers(R)
    g.vmc(3, 0.02)
    Rg, _ = g.get_walkers()
    Ro, acc, _ = O.Oracle(s).vmc(R, 3, 0.02, seed=616, step0=0, trace=False)
    assert np.max(np.abs(Rg - Ro)) < 1e-8
    cached = g.eval_cached()
    fresh = g.evaluate()
    ok, err = close(cached["eloc"], fresh["eloc"], 1e-8)
    assert ok, err
    ok, err = close(cached["logpsi"], fresh["logpsi"], 1e-10)
    assert ok, err
    g.close()


def test_delayed_updates_mixed_water32(Q):
    """Delay rank 32 in the mixed form at n = 160: the same accept/reject
    decisions as the Sherman-Morrison mixed sweep (a flipped decision would
    move an electron by ~sqrt(tau) = 0.14 bohr; FP32 rounding of the drifts
    alone stays far below that), and a propagated state consistent with a
    fresh FP64 evaluation."""
    s = synth.water_system(32)
    R = synth.initial_walkers(s, 4, seed=23)
    out = {}
    for k in (1, 32):
        g = Q.QMC(s, precision="mixed", seed=717, delay_rank=k)
        g.set_walkers(R)
        g.vmc(2, 0.02)
        out[k] = (g.get_walkers()[0], g.eval_cached(), g.evaluate())
        g.close()
    assert np.max(np.abs(out[1][0] - out[32][0])) < 2e-2
    ok, err = close(out[32][1]["logpsi"], out[32][2]["logpsi"], 1e-5)
    assert ok, err
    # the propagated FP32 state of the delayed form (the walker-tiled sweep
    # at this size) against the oracle at the same positions: ln|psi| 1e-5
    # and E_L 1e-3 relative, the propagated-state bounds of the mixed form
    ref = O.Oracle(s).evaluate(out[32][0])
    ok, err = close(out[32][1]["logpsi"], ref["logpsi"], 1e-5)
    assert ok, ("logpsi", err)
    ok, err = close(out[32][1]["eloc"], ref["eloc"], 1e-3)
    assert ok, ("eloc", err)
