"""Space-warped ionic derivatives on the GPU against the FP64 oracle.

The oracle takes dE_L/dr_i forward mode over the electron coordinates and
combines it with the warp weights (pinned in test_oracle_pins.py against
finite differences of the warped coordinate map); the CUDA path gets
dE_L/dr_i from the same adjoint pass as the nuclear derivatives plus a pair
kernel for the Jastrow and potential terms.  Tolerances as for the plain
derivatives: FP64 1e-10 relative (1e-9 for determinant expansions), mixed
1e-3 (ln|psi|) and 1e-4 (E_L) of each walker's largest component.
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


def close(a, b, tol):
    a, b = np.asarray(a), np.asarray(b)
    err = np.abs(a - b) / np.maximum(1.0, np.abs(b))
    return float(err.max()) <= tol, float(err.max())


def rel_to_walker_max(a, b):
    sc = np.maximum(1.0, np.abs(b).max(axis=(1, 2), keepdims=True))
    return float((np.abs(a - b) / sc).max())


def sd_systems():
    rng = np.random.default_rng(31)
    return {"water1": synth.water_system(1), "water6": synth.water_system(6),
            "small_all_shells": synth.random_small_system(rng, n_nuc=3, n_up=3, n_dn=2)}


def msd_systems():
    rng = np.random.default_rng(41)
    small = synth.random_small_system(rng, n_nuc=2, n_up=2, n_dn=2)
    return {"water1_30": synth.with_multidet(synth.water_system(1), 30, n_active=8, max_exc=4, seed=5),
            "small_12": synth.with_multidet(small, 12, n_active=6, max_exc=2, seed=7)}


def warped(Q, s, R, precision="fp64"):
    g = Q.QMC(s, precision=precision, space_warp=True)
    g.set_walkers(R)
    rng = np.random.default_rng(8)
    gE, gL = rng.normal(size=R.shape[0]), rng.normal(size=R.shape[0])
    dR, pw = g.forces(gE, gL)
    g.close()
    return dR, pw, gE, gL


@pytest.mark.parametrize("name,W", [("water1", 13), ("water6", 5), ("small_all_shells", 9)])
def test_space_warp_fp64(Q, name, W):
    s = sd_systems()[name]
    R = synth.initial_walkers(s, W, seed=21)
    dR, pw, gE, gL = warped(Q, s, R)
    dELw, dlgw = O.Oracle(s).warped_forces(R)
    ok, err = close(pw[:, 0], dELw, 1e-10)
    assert ok, ("dEL", err)
    ok, err = close(pw[:, 1], dlgw, 1e-10)
    assert ok, ("dlogpsi", err)
    ref = np.tensordot(gE, dELw, axes=(0, 0)) + np.tensordot(gL, dlgw, axes=(0, 0))
    ok, err = close(dR, ref, 1e-10)
    assert ok, ("vjp", err)


def test_space_warp_gemm_path_fp64(Q, monkeypatch):
    """The large-determinant force path (batched GEMMs) forced on."""
    monkeypatch.setenv("QMC_FORCE_GEMM_MIN_N", "1")
    s = synth.water_system(6)
    R = synth.initial_walkers(s, 6, seed=22)
    _, pw, _, _ = warped(Q, s, R)
    dELw, dlgw = O.Oracle(s).warped_forces(R)
    ok, err = close(pw[:, 0], dELw, 1e-10)
    assert ok, ("dEL", err)
    ok, err = close(pw[:, 1], dlgw, 1e-10)
    assert ok, ("dlogpsi", err)


@pytest.mark.parametrize("name,W", [("water1_30", 7), ("small_12", 9)])
def test_space_warp_multidet_fp64(Q, name, W):
    s = msd_systems()[name]
    R = synth.initial_walkers(s, W, seed=23)
    _, pw, _, _ = warped(Q, s, R)
    dELw, dlgw = O.Oracle(s).warped_forces(R)
    ok, err = close(pw[:, 1], dlgw, 1e-10)
    assert ok, ("dlogpsi", err)
    ok, err = close(pw[:, 0], dELw, 1e-10)
    assert ok, ("dEL", err)


@pytest.mark.parametrize("case", ["fused", "gemm", "multidet"])
def test_space_warp_mixed(Q, monkeypatch, case):
    if case == "gemm":
        monkeypatch.setenv("QMC_FORCE_GEMM_MIN_N", "1")
    s = msd_systems()["water1_30"] if case == "multidet" else synth.water_system(6)
    R = synth.initial_walkers(s, 6, seed=24)
    _, pw, _, _ = warped(Q, s, R, precision="mixed")
    dELw, dlgw = O.Oracle(s).warped_forces(R)
    assert rel_to_walker_max(pw[:, 1], dlgw) < 1e-3
    assert rel_to_walker_max(pw[:, 0], dELw) < 1e-4


def test_space_warp_totals_vanish(Q):
    """sum_a of the warped derivatives is zero for every configuration (the
    weights are a partition of unity); one electron around one nucleus has
    zero warped derivatives although its plain ones are not."""
    s = synth.water_system(6)
    R = synth.initial_walkers(s, 8, seed=25)
    _, pw, _, _ = warped(Q, s, R)
    sc = np.maximum(1.0, np.abs(pw).max(axis=(2, 3)))
    assert np.all(np.abs(pw.sum(axis=2)).max(axis=2) <= 1e-9 * sc)
    a = synth.single_gaussian_atom(0.37, 1.0)
    Ra = np.random.default_rng(6).normal(0, 1.0, size=(16, 1, 3))
    _, pw, _, _ = warped(Q, a, Ra)
    assert np.abs(pw).max() < 1e-12


def test_space_warp_estimator_and_variance(Q):
    """VMC with forces: the warped estimator the handle accumulates equals the
    oracle's zero-variance zero-bias estimate from the warped derivatives at
    the same walkers, and the warp cuts the variance of the per-walker force
    samples on the oxygen by more than 100x (electrons near a nucleus no
    longer make dE_L/dR_a diverge)."""
    s = synth.water_system(1)
    R0 = synth.initial_walkers(s, 256, seed=26)
    g = Q.QMC(s, precision="fp64", space_warp=True)
    g.set_walkers(R0)
    g.vmc(30, 0.05)
    Q.qmc_reset_estimators(g.h)
    g.vmc(1, 0.05, forces_every=1)
    F, _ = g.force_estimate(Q.QMC_EST_VMC)
    R1, _ = g.get_walkers()
    g.close()
    o = O.Oracle(s)
    ev = o.evaluate(R1)
    dELw, dlgw = o.warped_forces(R1)
    ok, err = close(F, O.force_estimator(ev["eloc"], dELw, dlgw), 1e-8)
    assert ok, err
    dEL, dlg = o.forces(R1)
    E = ev["eloc"] - ev["eloc"].mean()
    var = lambda d, l: (-d - 2 * E[:, None, None] * l).var(axis=0)
    assert np.all(var(dEL, dlg)[0] > 100 * var(dELw, dlgw)[0])


def test_space_warp_flag_and_batch_setting(Q):
    """The flag takes 0 or 1; a batch reads each member's setting when it is
    created and refuses to step once a member's setting has changed."""
    s = synth.water_system(1)
    g = Q.QMC(s, precision="fp64")
    with pytest.raises(Q.QmcError):
        Q.qmc_set_space_warp(g.h, 2)
    Q.qmc_set_space_warp(g.h, True)
    g.set_walkers(synth.initial_walkers(s, 4))
    batch = Q.Batch([g])
    batch.dmc(1, 0.005, [-76.0], forces_every=1)
    Q.qmc_set_space_warp(g.h, False)
    with pytest.raises(Q.QmcError) as e:
        batch.dmc(1, 0.005, [-76.0], forces_every=1)
    assert e.value.code == -7
    batch.close()
    g.close()
