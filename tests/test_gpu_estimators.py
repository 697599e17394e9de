"""Force estimators of the CUDA path against the oracle's (FP64 form).

qmc_get_forces returns the zero-variance zero-bias estimate of Sec. "Single
Determinant QMC Forces" over the VMC samples (weight 1), over the DMC
samples (branching weights of Eq. 1) and the mixed estimator 2 F_DMC - F_VMC
of Sec. "Performance Measurement".  With the same random streams the FP64
form follows the oracle's moves, so the three estimates are compared with
the oracle's, built from its own per-walker forward-mode derivatives and its
own DMC force sums, at the FP64 tolerance 1e-10.  The estimator is a
difference of large averages (<E_L dln|psi|/dR> and <E_L><dln|psi|/dR> reach
~1e7 on these clusters while F is far smaller), so the 1e-10 is relative to
the magnitude of its terms, max(1, <|dE_L/dR|> + 2 <|E_L dln|psi|/dR|> +
2 |<E_L>| <|dln|psi|/dR|>) per component, the scale FP64 rounding of the
per-walker inputs acts on.
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


def scaled_err(a, b, scale):
    return float((np.abs(np.asarray(a) - np.asarray(b)) / np.maximum(1.0, scale)).max())


def term_scale(eloc, dEL, dlg):
    """Per-component magnitude of the estimator's terms over a sample."""
    E = eloc[:, None, None]
    return (np.abs(dEL).mean(axis=0) + 2.0 * np.abs(E * dlg).mean(axis=0)
            + 2.0 * abs(eloc.mean()) * np.abs(dlg).mean(axis=0))


@pytest.mark.parametrize("name,W", [("water1", 24), ("water6", 10)])
def test_vmc_dmc_mixed_force_estimates_match_oracle(Q, name, W):
    s = synth.water_system(1 if name == "water1" else 6)
    seed, tau_v, tau, n_vmc, n_dmc = 321, 0.05, 0.005, 2, 3
    R0 = synth.initial_walkers(s, W, seed=17)
    g = Q.QMC(s, precision="fp64", seed=seed, cap_factor=4)
    g.set_walkers(R0)
    g.vmc(n_vmc, tau_v, forces_every=1)
    # the oracle's VMC one sweep at a time on the same stream; the estimator
    # sums after every sweep (weight 1)
    o = O.Oracle(s)
    R = R0
    tot = 0.0
    for k in range(n_vmc):
        R, _, _ = o.vmc(R, 1, tau_v, seed=seed, step0=k, trace=False)
        ev = o.evaluate(R)
        dEL, dlg = o.forces(R)
        tot = tot + O.force_sums(ev["eloc"], dEL, dlg)
    F_vmc = O.force_from_sums(tot, s.n_nuc)
    scale = term_scale(ev["eloc"], dEL, dlg)
    Rg, _ = g.get_walkers()
    assert np.max(np.abs(Rg - R)) < 1e-8
    ET = float(np.median(ev["eloc"]))
    out = g.dmc(n_dmc, tau, ET, forces_every=1)
    ref = o.dmc(R, n_dmc, tau, ET, seed=seed, step0=n_vmc, forces_every=1, cap_factor=4)
    assert ref["status"] == 0
    assert np.array_equal(out["pop"], ref["pop"])
    F_dmc = O.force_from_sums(ref["facc"], s.n_nuc)
    F_mix = O.mixed_estimator(F_dmc, F_vmc)
    for est, Fo in ((Q.QMC_EST_VMC, F_vmc), (Q.QMC_EST_DMC, F_dmc), (Q.QMC_EST_MIXED, F_mix)):
        Fg, Fe = g.force_estimate(est)
        assert Fg.shape == Fo.shape and np.all(np.isfinite(Fe))
        err = scaled_err(Fg, Fo, (3.0 if est == Q.QMC_EST_MIXED else 1.0) * scale)
        assert err <= 1e-10, (est, err, float(np.abs(Fg - Fo).max()))
    g.close()


def test_force_estimate_over_current_walkers_matches_oracle(Q):
    """qmc_force_estimate (the estimator at fixed configurations, weighted
    and unweighted) against the oracle's estimator of its forward-mode
    derivatives at the same walkers."""
    import torch
    from paper_2504_07948_gb300.forces import zvzb_force
    s = synth.water_system(6)
    W = 16
    R = synth.initial_walkers(s, W, seed=23)
    g = Q.QMC(s, precision="fp64")
    g.set_walkers(R)
    o = O.Oracle(s)
    ev = o.evaluate(R)
    dEL, dlg = o.forces(R)
    scale = term_scale(ev["eloc"], dEL, dlg)
    w = np.random.default_rng(4).uniform(0.1, 3.0, W)
    for weights in (None, w):
        F = np.zeros((s.n_nuc, 3))
        Q.qmc_force_estimate(g.h, weights, F)
        Fo = O.force_estimator(ev["eloc"], dEL, dlg, weights=weights)
        assert scaled_err(F, Fo, scale) <= 1e-10, scaled_err(F, Fo, scale)
    Ft = zvzb_force(torch.tensor(s.R), g, weights=w).numpy()
    assert scaled_err(Ft, O.force_estimator(ev["eloc"], dEL, dlg, weights=w), scale) <= 1e-10
    g.close()


def test_init_walkers_follow_the_initial_distribution(Q):
    """qmc_init_walkers: round(Z_a) electrons per nucleus, spins alternating
    along that list, each Gaussian around its nucleus with sigma = 0.5 bohr.
    The electron -> nucleus map equals the input generator's (its centres at
    sigma = 0), per-electron means lie within 4.5 standard errors of those
    centres, the spread is 0.5 bohr within 5 %, and the draw is a function
    of the seed alone."""
    s = synth.water_system(6)
    W = 4096
    g = Q.QMC(s, precision="fp64")
    g.init_walkers(W, seed=77)
    R, wt = g.get_walkers()
    assert R.shape == (W, s.n_elec, 3) and np.all(wt == 1.0)
    centres = synth.initial_walkers(s, 1, sigma=0.0)[0]
    se = 0.5 / np.sqrt(W)
    assert np.all(np.abs(R.mean(axis=0) - centres) <= 4.5 * se)
    sd = R.std(axis=0, ddof=1)
    assert np.all(np.abs(sd - 0.5) <= 0.05 * 0.5), (sd.min(), sd.max())
    ev = g.evaluate()
    assert np.all(np.isfinite(ev["logpsi"])) and np.all(np.isfinite(ev["eloc"]))
    g.init_walkers(W, seed=77)
    R2, _ = g.get_walkers()
    assert np.array_equal(R, R2)
    g.init_walkers(W, seed=78)
    R3, _ = g.get_walkers()
    assert not np.allclose(R, R3)
    g.close()
