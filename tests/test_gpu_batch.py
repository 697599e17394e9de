"""Batches of uneven systems stepped together (persistent launches over all
systems, one CUDA graph per step) against the oracle and against the
per-handle DMC path, through the C ABI.

FP64 batches follow the oracle's DMC step for step (same random streams):
populations exactly, step energies and final positions to 1e-8 relative
(the bound of the single-handle DMC parity test).  Batch against per-handle
runs of the same kernels: 1e-12 (the trial-energy update runs on the device
in a batch and on the host per handle; the two agree to rounding).  In
the mixed form the batched and per-handle kernels are separate compilations
of the same FP32 code, which may contract multiply-adds differently: they
agree to FP32 rounding (1e-4 on step energies and positions, the size of
the mixed form's own E_L error against the oracle).
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2504_07948_gb300 import synth

pytestmark = pytest.mark.gpu

TAU = 0.005


@pytest.fixture(scope="module")
def Q():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2504_07948_gb300 import qmc
    return qmc


def uneven_systems():
    rng = np.random.default_rng(41)
    return [synth.water_system(2), synth.random_small_system(rng, n_nuc=3, n_up=3, n_dn=2),
            synth.water_system(1), synth.water_system(3, geom_seed=1011)]


WALKERS = [23, 17, 31, 9]
SEEDS = [501, 502, 503, 504]
E_TRIAL = [-150.0, -20.0, -76.0, -228.0]


def make_members(Q, precision="fp64", **kw):
    out = []
    for s, W, seed in zip(uneven_systems(), WALKERS, SEEDS):
        m = Q.QMC(s, precision=precision, seed=seed, cap_factor=4, **kw)
        m.set_walkers(synth.initial_walkers(s, W, seed=seed + 100))
        out.append(m)
    return out


def rel(a, b):
    a, b = np.asarray(a, dtype=float), np.asarray(b, dtype=float)
    return float((np.abs(a - b) / np.maximum(1.0, np.abs(b))).max())


def test_batch_fp64_follows_oracle(Q):
    members = make_members(Q)
    batch = Q.Batch(members)
    out = batch.dmc(3, TAU, E_TRIAL)
    for q, (s, W, seed) in enumerate(zip(uneven_systems(), WALKERS, SEEDS)):
        R0 = synth.initial_walkers(s, W, seed=seed + 100)
        ref = O.Oracle(s).dmc(R0, 3, TAU, E_TRIAL[q], seed=seed, step0=0)
        assert np.array_equal(out["pop"][:, q], ref["pop"]), q
        assert rel(out["e_step"][:, q], ref["e_step"]) < 1e-8, q
        R, _ = members[q].get_walkers()
        assert R.shape == ref["R"].shape
        assert rel(R, ref["R"]) < 1e-8, q
    batch.close()
    for m in members:
        m.close()


TOL = {"fp64": dict(e=1e-12, R=1e-12, f=1e-9), "mixed": dict(e=1e-4, R=1e-4, f=1e-3)}


def test_batch_fixed_population_follows_oracle(Q):
    """Fixed-population control inside the batch (comb resampling and trial
    energy on the device) against the oracle's fixed-population DMC."""
    members = []
    for s, W, seed in zip(uneven_systems(), WALKERS, SEEDS):
        m = Q.QMC(s, seed=seed, cap_factor=4, fixed_population=True)
        m.set_walkers(synth.initial_walkers(s, W, seed=seed + 100))
        members.append(m)
    batch = Q.Batch(members)
    out = batch.dmc(3, TAU, E_TRIAL)
    for q, (s, W, seed) in enumerate(zip(uneven_systems(), WALKERS, SEEDS)):
        R0 = synth.initial_walkers(s, W, seed=seed + 100)
        ref = O.Oracle(s).dmc(R0, 3, TAU, E_TRIAL[q], seed=seed, step0=0, fixed_pop=True)
        assert np.all(out["pop"][:, q] == W) and np.array_equal(out["pop"][:, q], ref["pop"]), q
        assert rel(out["e_step"][:, q], ref["e_step"]) < 1e-8, q
        R, _ = members[q].get_walkers()
        assert rel(R, ref["R"]) < 1e-8, q
    batch.close()
    for m in members:
        m.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batch_matches_per_handle_runs(Q, precision):
    """Forces every step and an FP64 recompute every second step."""
    kw = dict(recompute_period=2)
    tol = TOL[precision]
    a = make_members(Q, precision, **kw)
    b = make_members(Q, precision, **kw)
    batch = Q.Batch(a)
    out = batch.dmc(4, TAU, E_TRIAL, n_equil=0, forces_every=1)
    for q, m in enumerate(b):
        ref = m.dmc(4, TAU, E_TRIAL[q], forces_every=1)
        assert np.array_equal(out["pop"][:, q], ref["pop"]), q
        assert rel(out["e_step"][:, q], ref["e_step"]) < tol["e"], (q, rel(out["e_step"][:, q], ref["e_step"]))
        Ra, _ = a[q].get_walkers()
        Rb, _ = m.get_walkers()
        assert rel(Ra, Rb) < tol["R"], (q, rel(Ra, Rb))
        ea, eb = a[q].energy(), m.energy()
        # means of step energies of both signs: compare on the scale of the terms
        scale = max(1.0, float(np.abs(ref["e_step"]).max()))
        assert abs(ea["mean"] - eb["mean"]) < tol["e"] * scale
        assert ea["acceptance"] == eb["acceptance"]
        fa, fb = a[q].force_estimate(), m.force_estimate()
        fscale = max(1.0, float(np.abs(fb[0]).max()))
        assert float(np.abs(fa[0] - fb[0]).max()) < tol["f"] * fscale, q
    batch.close()
    for m in a + b:
        m.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batch_space_warp_matches_per_handle_runs(Q, precision):
    """Space-warped forces in a batch (two of the four members warped): the
    batched force launch writes the members' electron gradients and one
    persistent warp launch warps them; force estimates after DMC steps with
    forces equal the per-handle runs of the same members."""
    tol = TOL[precision]
    warped = [True, False, True, False]

    def members():
        out = make_members(Q, precision)
        for m, wq in zip(out, warped):
            if wq:
                Q.qmc_set_space_warp(m.h, True)
        return out
    a, b = members(), members()
    batch = Q.Batch(a)
    out = batch.dmc(3, TAU, E_TRIAL, n_equil=0, forces_every=1)
    for q, m in enumerate(b):
        ref = m.dmc(3, TAU, E_TRIAL[q], forces_every=1)
        assert np.array_equal(out["pop"][:, q], ref["pop"]), q
        fa, fb = a[q].force_estimate(), m.force_estimate()
        fscale = max(1.0, float(np.abs(fb[0]).max()))
        assert float(np.abs(fa[0] - fb[0]).max()) < tol["f"] * fscale, (q, fa[0], fb[0])
    # the warped members' per-walker derivatives against the oracle's warped ones
    if precision == "fp64":
        for q in (0, 2):
            R, _ = a[q].get_walkers()
            _, pw = a[q].forces()
            dELw, dlgw = O.Oracle(uneven_systems()[q]).warped_forces(R[:4])
            assert rel(pw[:4, 0], dELw) < 1e-9 and rel(pw[:4, 1], dlgw) < 1e-9
    batch.close()
    for m in a + b:
        m.close()


def test_batch_graph_and_plain_launches_agree(Q):
    a = make_members(Q)
    b = make_members(Q)
    ba, bb = Q.Batch(a), Q.Batch(b)
    bb.set_options(use_graph=False)
    oa = ba.dmc(5, TAU, E_TRIAL, forces_every=2)
    ob = bb.dmc(5, TAU, E_TRIAL, forces_every=2)
    assert np.array_equal(oa["pop"], ob["pop"])
    assert np.array_equal(oa["e_step"], ob["e_step"])
    for x, y in zip(a, b):
        assert np.array_equal(x.get_walkers()[0], y.get_walkers()[0])
    ba.close()
    bb.close()
    for m in a + b:
        m.close()


def test_batch_delayed_updates_match_per_handle(Q):
    """Delayed (rank 8) sweeps inside the batch against the per-handle
    delayed sweep of the same members."""
    a = make_members(Q, "mixed")
    b = make_members(Q, "mixed", delay_rank=8)
    batch = Q.Batch(a)
    batch.set_options(delay_rank=8, delay_min_electrons=0)
    out = batch.dmc(3, TAU, E_TRIAL)
    for q, m in enumerate(b):
        ref = m.dmc(3, TAU, E_TRIAL[q])
        assert np.array_equal(out["pop"][:, q], ref["pop"]), q
        assert rel(out["e_step"][:, q], ref["e_step"]) < TOL["mixed"]["e"], q
        # the batch's propagated (delayed-update) state against the oracle
        R, _ = a[q].get_walkers()
        ev = a[q].eval_cached()
        o = O.Oracle(uneven_systems()[q]).evaluate(R)
        assert rel(ev["logpsi"], o["logpsi"]) < 1e-5, q
        assert rel(ev["eloc"], o["eloc"]) < 1e-3, (q, rel(ev["eloc"], o["eloc"]))
    batch.close()
    for m in a + b:
        m.close()


def test_batch_autotune_and_timing(Q):
    members = make_members(Q, "mixed")
    batch = Q.Batch(members)
    cfg = batch.autotune(TAU)
    assert cfg["block"] in (128, 256) and cfg["grid"] > 0 and cfg["sweep_us"] > 0
    assert len(cfg["per_system"]) == len(members)
    for k, ainv in cfg["per_system"]:
        assert k in (1, 8, 16, 32) and ainv in (0, 1)
    Q.qmc_batch_set_timing(batch.b, True)
    out = batch.dmc(3, TAU, E_TRIAL, forces_every=1)
    ms, n = Q.qmc_batch_get_timing(batch.b, "sweep")
    assert ms > 0.0 and n == 3
    _, launches = Q.qmc_batch_get_timing(batch.b, "all")
    assert launches == 3 * 8
    assert np.all(np.isfinite(out["e_step"]))
    for m in members:
        assert np.isfinite(m.energy()["mean"])
    batch.close()
    for m in members:
        m.close()


def test_batch_errors_are_status_codes(Q):
    members = make_members(Q)
    msd = Q.QMC(synth.with_multidet(synth.water_system(1), 5, n_active=4, max_exc=2))
    msd.set_walkers(synth.initial_walkers(msd.sys, 4, seed=3))
    with pytest.raises(Q.QmcError) as e:
        Q.Batch(members + [msd])
    assert e.value.code == -9
    batch = Q.Batch(members)
    s = uneven_systems()[0]
    Q.qmc_set_jastrow(members[0].h, s.a_anti, s.a_par, 0.9, s.a_en, s.b_en)
    members[0].set_walkers(synth.initial_walkers(s, 8, seed=1))
    with pytest.raises(Q.QmcError) as e:
        batch.dmc(1, TAU, E_TRIAL)
    assert e.value.code == -7
    batch.close()
    msd.close()
    for m in members:
        m.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batch_large_members_follow_oracle(Q, precision):
    """Members of 13 and 16 waters (65 and 80 electrons per spin, the
    batched kernels' n > 64 code path) next to a 2-water member.  FP64:
    two fixed-population DMC steps with forces follow the oracle's step for
    step (populations, step energies and positions to 1e-8), and the
    propagated state of sampled walkers equals the oracle's evaluation at
    their positions (ln|psi|, E_L 1e-8).  Mixed: the propagated FP32 state
    of the same walkers against the oracle at their positions, ln|psi| 1e-5
    and E_L 1e-4 relative (the propagated-state bounds of the mixed form)."""
    systems = [synth.water_system(13, geom_seed=1113), synth.water_system(16, geom_seed=1116),
               synth.water_system(2)]
    Ws, seeds, ets = [6, 5, 9], [611, 612, 613], [-988.0, -1216.0, -152.0]
    members = []
    for s, W, seed in zip(systems, Ws, seeds):
        m = Q.QMC(s, precision=precision, seed=seed, cap_factor=4, fixed_population=True)
        m.set_walkers(synth.initial_walkers(s, W, seed=seed + 100))
        members.append(m)
    batch = Q.Batch(members)
    out = batch.dmc(2, TAU, ets, forces_every=1)
    for q, (s, W, seed) in enumerate(zip(systems, Ws, seeds)):
        o = O.Oracle(s)
        R, _ = members[q].get_walkers()
        cached = members[q].eval_cached()
        ref_at = o.evaluate(R)
        if precision == "fp64":
            R0 = synth.initial_walkers(s, W, seed=seed + 100)
            ref = o.dmc(R0, 2, TAU, ets[q], seed=seed, step0=0, fixed_pop=True)
            assert ref["status"] == 0
            assert np.array_equal(out["pop"][:, q], ref["pop"]), q
            assert rel(out["e_step"][:, q], ref["e_step"]) < 1e-8, (q, rel(out["e_step"][:, q], ref["e_step"]))
            assert rel(R, ref["R"]) < 1e-8, q
            tl, te = 1e-8, 1e-8
        else:
            tl, te = 1e-5, 1e-4
        assert rel(cached["logpsi"], ref_at["logpsi"]) < tl, (q, rel(cached["logpsi"], ref_at["logpsi"]))
        assert rel(cached["eloc"], ref_at["eloc"]) < te, (q, rel(cached["eloc"], ref_at["eloc"]))
    batch.close()
    for m in members:
        m.close()
