"""Three-body Jastrow and Jastrow parameter derivatives of the CUDA path
against the oracle (FP64 form), through the C ABI.

The three-body electron-electron-nucleus term (the third kind of Jastrow
term the paper's trial function carries, the paragraph after Eq. 2) enters
the fixed-configuration evaluation; the parameter derivatives d ln|psi|/dp
and dE_L/dp are what a linear-method optimisation step consumes per walker.
FP64 tolerance 1e-10 relative to max(1, |x|) as for every other evaluated
quantity; the Sherman-Morrison sweep carries it (trajectory parity), the
delayed sweeps, forces and batches refuse it.
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


def j3_systems():
    rng = np.random.default_rng(31)
    small = synth.random_small_system(rng, n_nuc=3, n_up=3, n_dn=2)
    return {"water1_j3": synth.with_three_body(synth.water_system(1), scale=0.2),
            "small_j3": synth.with_three_body(small, scale=0.3, b3=0.7),
            "water6_j3": synth.with_three_body(synth.water_system(6), scale=0.05)}


@pytest.mark.parametrize("name,W", [("water1_j3", 17), ("small_j3", 9), ("water6_j3", 5)])
def test_evaluate_with_three_body_jastrow(Q, name, W):
    s = j3_systems()[name]
    R = synth.initial_walkers(s, W, seed=14)
    g = Q.QMC(s, precision="fp64")
    g.set_walkers(R)
    ev = g.evaluate()
    ref = O.Oracle(s).evaluate(R)
    for k in ("logpsi", "eloc", "grad"):
        assert rel(ev[k], ref[k]) <= 1e-10, (k, rel(ev[k], ref[k]))
    g.close()
    m = Q.QMC(s, precision="mixed")
    m.set_walkers(R)
    ev = m.eval_cached()
    assert rel(ev["logpsi"], ref["logpsi"]) <= 1e-5
    assert rel(ev["eloc"], ref["eloc"]) <= 1e-5
    m.close()


@pytest.mark.parametrize("name,W", [("water1", 13), ("water1_j3", 13), ("small_j3", 7), ("water6_j3", 4)])
def test_jastrow_parameter_derivatives_match_oracle(Q, name, W):
    s = synth.water_system(1) if name == "water1" else j3_systems()[name]
    R = synth.initial_walkers(s, W, seed=15)
    g = Q.QMC(s, precision="fp64")
    g.set_walkers(R)
    dl, de = g.jastrow_derivs()
    rl, re_ = O.Oracle(s).jastrow_derivs(R)
    assert dl.shape == rl.shape
    assert rel(dl, rl) <= 1e-10, rel(dl, rl)
    assert rel(de, re_) <= 1e-10, rel(de, re_)
    g.close()


@pytest.mark.parametrize("name,W,sweeps", [("water1_j3", 16, 3), ("small_j3", 9, 3)])
def test_vmc_and_dmc_with_three_body_jastrow_follow_oracle(Q, name, W, sweeps):
    """The Sherman-Morrison sweep carries the three-body ratio and drift:
    with the same random stream the FP64 VMC trajectory equals the oracle's
    (which refactorises and recomputes the whole Jastrow after every
    proposal), and the first DMC steps give the same populations and step
    energies."""
    s = j3_systems()[name]
    R = synth.initial_walkers(s, W, seed=16)
    g = Q.QMC(s, precision="fp64", seed=919, cap_factor=4)
    g.set_walkers(R)
    g.vmc(sweeps, 0.05)
    Rg, _ = g.get_walkers()
    Ro, _, _ = O.Oracle(s).vmc(R, sweeps, 0.05, seed=919, step0=0, trace=False)
    assert np.max(np.abs(Rg - Ro)) < 1e-8
    cached, ref = g.eval_cached(), O.Oracle(s).evaluate(Rg)
    assert rel(cached["eloc"], ref["eloc"]) <= 1e-8 and rel(cached["logpsi"], ref["logpsi"]) <= 1e-10
    g.close()
    g = Q.QMC(s, precision="fp64", seed=99, cap_factor=4)
    g.set_walkers(R)
    et = float(np.median(O.Oracle(s).evaluate(R)["eloc"]))
    out = g.dmc(3, 0.005, et)
    ref = O.Oracle(s).dmc(R, 3, 0.005, et, seed=99, step0=0)
    assert np.array_equal(out["pop"], ref["pop"])
    assert rel(out["e_step"], ref["e_step"]) <= 1e-9
    g.close()


def test_three_body_jastrow_is_refused_where_not_carried(Q):
    s = j3_systems()["water1_j3"]
    g = Q.QMC(s, precision="fp64")
    g.set_walkers(synth.initial_walkers(s, 4, seed=1))
    with pytest.raises(Q.QmcError) as ex:
        g.forces()
    assert ex.value.code == -9
    with pytest.raises(Q.QmcError) as ex:
        Q.Batch([g])
    assert ex.value.code == -9
    g.close()
    d = Q.QMC(s, precision="fp64", delay_rank=4)
    d.set_walkers(synth.initial_walkers(s, 4, seed=1))
    with pytest.raises(Q.QmcError) as ex:
        d.vmc(1, 0.05)
    assert ex.value.code == -9
    # removing the term restores every path
    Q.qmc_set_jastrow3(d.h, np.zeros((0, 3), np.int32), np.zeros(0), 1.0)
    d.set_walkers(synth.initial_walkers(s, 4, seed=1))
    d.vmc(1, 0.05)
    d.forces()
    d.close()
