"""Semi-local pseudopotential of the CUDA path against the oracle, through
the C ABI.

The valence Hamiltonian with effective core potentials (Sec. "The
SPICE2(+)-ccECP dataset", Sec. "Quantum Monte Carlo") adds local radial
terms to E_L and a non-local term evaluated by a rotated quadrature rule in
the locality approximation.  The rotations come from the same counter-based
stream on both sides (Philox counter (sweep, nucleus, slot, 3), Shoemake's
quaternion), so fixed configurations compare element by element: FP64 at
1e-10 relative to max(1, |E_L|), the mixed form at the mixed E_L bound.  The
sampling drivers draw the rotations at the next sweep counter, which the
same-stream VMC trace and DMC steps check.
"""
import dataclasses

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


def pp_system(name):
    if name == "water1_pp":
        return synth.with_pseudopotential(synth.water_system(1))
    if name == "water6_pp":
        return synth.with_pseudopotential(synth.water_system(6))
    if name == "water1_pp_j3":
        return synth.with_three_body(synth.with_pseudopotential(synth.water_system(1)), scale=0.2)
    raise KeyError(name)


@pytest.mark.parametrize("name,W", [("water1_pp", 33), ("water6_pp", 6), ("water1_pp_j3", 9)])
@pytest.mark.parametrize("rotate", [True, False])
def test_evaluate_with_pseudopotential(Q, name, W, rotate):
    s = pp_system(name)
    R = synth.initial_walkers(s, W, seed=21)
    g = Q.QMC(s, precision="fp64", seed=4242, pp_rotate=rotate)
    Q.qmc_set_rng(g.h, 4242, 17)
    g.set_walkers(R)
    ev = g.evaluate()
    o = O.Oracle(s, pp_rotate=rotate)
    ref = o.evaluate(R, pp_seed=4242, pp_sweep=17)
    vnl = o.nonlocal_energy(R, pp_seed=4242, pp_sweep=17)
    assert np.abs(vnl).max() > 1e-3   # the non-local term is really there
    assert rel(ev["eloc"], ref["eloc"]) <= 1e-10, rel(ev["eloc"], ref["eloc"])
    assert rel(ev["logpsi"], ref["logpsi"]) <= 1e-10
    g.close()
    m = Q.QMC(s, precision="mixed", seed=4242, pp_rotate=rotate)
    Q.qmc_set_rng(m.h, 4242, 17)
    m.set_walkers(R)
    ev = m.eval_cached()
    assert rel(ev["eloc"], ref["eloc"]) <= 1e-5, rel(ev["eloc"], ref["eloc"])
    m.close()


def test_rotation_counter_changes_the_nonlocal_term(Q):
    s = pp_system("water1_pp")
    R = synth.initial_walkers(s, 8, seed=5)
    g = Q.QMC(s, precision="fp64", seed=7)
    g.set_walkers(R)
    e0 = g.evaluate()["eloc"]
    Q.qmc_set_rng(g.h, 7, 1)
    e1 = g.evaluate()["eloc"]
    assert np.abs(e1 - e0).max() > 1e-6
    ref = O.Oracle(s).evaluate(R, pp_seed=7, pp_sweep=1)["eloc"]
    assert rel(e1, ref) <= 1e-10
    g.close()


@pytest.mark.parametrize("name,W", [("water1_pp", 24), ("water1_pp_j3", 8)])
def test_vmc_and_dmc_with_pseudopotential_follow_oracle(Q, name, W):
    """Same stream: the FP64 VMC trajectory and its E_L trace (rotations at
    counter t + 1 after the sweep with counter t) equal the oracle's; the
    first DMC steps give the same populations and step energies."""
    s = pp_system(name)
    R = synth.initial_walkers(s, W, seed=16)
    g = Q.QMC(s, precision="fp64", seed=919, cap_factor=4)
    g.set_walkers(R)
    tr = g.vmc(3, 0.05, trace=True)
    Rg, _ = g.get_walkers()
    Ro, _, tro = O.Oracle(s).vmc(R, 3, 0.05, seed=919, step0=0)
    assert np.max(np.abs(Rg - Ro)) < 1e-8
    assert rel(tr, tro) <= 1e-9, rel(tr, tro)
    g.close()
    g = Q.QMC(s, precision="fp64", seed=99, cap_factor=4)
    g.set_walkers(R)
    et = float(np.median(O.Oracle(s).evaluate(R, pp_seed=99, pp_sweep=0)["eloc"]))
    out = g.dmc(3, 0.005, et)
    ref = O.Oracle(s).dmc(R, 3, 0.005, et, seed=99, step0=0)
    assert np.array_equal(out["pop"], ref["pop"])
    assert rel(out["e_step"], ref["e_step"]) <= 1e-9, rel(out["e_step"], ref["e_step"])
    g.close()


@pytest.mark.parametrize("delay_rank", [1, 8])
def test_mixed_sweep_local_energy_with_pseudopotential(Q, delay_rank):
    """Mixed form after sweeps (Sherman-Morrison or delayed updates): E_L of
    the propagated state at the GPU's positions against the oracle."""
    s = pp_system("water6_pp")
    R = synth.initial_walkers(s, 8, seed=3)
    m = Q.QMC(s, precision="mixed", seed=31, delay_rank=delay_rank, recompute_period=10)
    m.set_walkers(R)
    tr = m.vmc(4, 0.02, trace=True)
    Rg, _ = m.get_walkers()
    ref = O.Oracle(s).evaluate(Rg, pp_seed=31, pp_sweep=4)["eloc"]
    assert rel(tr[-1], ref) <= 1e-3, rel(tr[-1], ref)
    m.close()


def test_walker_tiled_sweep_with_pseudopotential_32_waters(Q):
    """32 waters with pseudopotentials on every O (128 electrons per spin):
    the mixed delayed sweep takes the walker-tiled tensor-core path; E_L
    after two sweeps on sampled walkers against the oracle at the GPU's
    positions."""
    s = synth.with_pseudopotential(synth.water_system(32))
    assert s.n_up == 128
    R = synth.initial_walkers(s, 64, seed=9)
    m = Q.QMC(s, precision="mixed", seed=5, delay_rank=32, recompute_period=100)
    m.set_walkers(R)
    Q.qmc_set_timing(m.h, 1)
    tr = m.vmc(2, 0.01, trace=True)
    _, launches = Q.qmc_get_timing(m.h, "sweep_gemm")
    assert launches == 2 * 2 * s.n_up   # the tiled sweep ran: one GEMM per electron per sweep
    Rg, _ = m.get_walkers()
    o = O.Oracle(s)
    for slot in (0, 37):
        ref = o.evaluate(Rg[slot:slot + 1], pp_seed=5, pp_sweep=2, pp_slot0=slot)["eloc"]
        assert rel(tr[-1][slot], ref[0]) <= 1e-3, (slot, tr[-1][slot], ref[0])
    m.close()


def vrel(a, b):
    a, b = np.asarray(a, dtype=float), np.asarray(b, dtype=float)
    sc = np.maximum(1.0, np.abs(b).reshape(b.shape[0], -1).max(axis=1))
    return float((np.abs(a - b).reshape(b.shape[0], -1).max(axis=1) / sc).max())


@pytest.mark.parametrize("path", ["kernel", "gemm"])
@pytest.mark.parametrize("name,W", [("water1_pp", 9), ("water6_pp", 4)])
def test_pseudopotential_forces_match_oracle(Q, name, W, path, monkeypatch):
    """Per-walker dE_L/dR_a and dln|psi|/dR_a with the pseudopotential: the
    local terms, the non-local rows of B (through X = A^-1 B A^-1) and the
    direct derivatives of the quadrature points, weights and Jastrow ratios,
    against the oracle's forward mode at the same rotations; through the
    per-walker force kernel and through the GEMM force path of large
    determinants (selected here for small ones)."""
    if path == "gemm":
        monkeypatch.setenv("QMC_FORCE_GEMM_MIN_N", "1")
    s = pp_system(name)
    R = synth.initial_walkers(s, W, seed=23)
    ref_E, ref_L = O.Oracle(s).forces(R, pp_seed=77, pp_sweep=6)
    for prec, tol in (("fp64", 1e-10), ("mixed", 1e-3)):
        g = Q.QMC(s, precision=prec, seed=77)
        Q.qmc_set_rng(g.h, 77, 6)
        g.set_walkers(R)
        _, pw = g.forces()
        assert vrel(pw[:, 0], ref_E) <= tol, (prec, vrel(pw[:, 0], ref_E))
        assert vrel(pw[:, 1], ref_L) <= tol, (prec, vrel(pw[:, 1], ref_L))
        g.close()


def test_dmc_force_sums_with_pseudopotential_follow_oracle(Q):
    """Same stream, FP64: three DMC steps with forces every step give the
    oracle's weighted force sums (the E_L and its derivatives of each step at
    that step's rotations)."""
    s = pp_system("water1_pp")
    R = synth.initial_walkers(s, 16, seed=12)
    et = float(np.median(O.Oracle(s).evaluate(R, pp_seed=55, pp_sweep=0)["eloc"]))
    ref = O.Oracle(s).dmc(R, 3, 0.005, et, seed=55, step0=0, forces_every=1, fixed_pop=True)
    g = Q.QMC(s, precision="fp64", seed=55, cap_factor=4, fixed_population=True)
    g.set_walkers(R)
    out = g.dmc(3, 0.005, et, forces_every=1)
    assert rel(out["e_step"], ref["e_step"]) <= 1e-9
    F, _ = g.force_estimate(Q.QMC_EST_DMC)
    Fo = O.force_from_sums(ref["facc"], s.n_nuc)
    scale = np.abs(ref["facc"][2:]).max() / ref["facc"][0]
    assert np.abs(F - Fo).max() <= 1e-9 * max(1.0, scale), (F, Fo)
    g.close()


def test_pseudopotential_is_refused_where_not_carried(Q):
    s = pp_system("water1_pp")
    g = Q.QMC(s, precision="fp64", space_warp=True)
    g.set_walkers(synth.initial_walkers(s, 4, seed=1))
    with pytest.raises(Q.QmcError) as ex:
        g.forces()
    assert ex.value.code == -9
    g.close()
    g = Q.QMC(s, precision="fp64")
    g.set_walkers(synth.initial_walkers(s, 4, seed=1))
    with pytest.raises(Q.QmcError) as ex:
        Q.Batch([g])
    assert ex.value.code == -9
    # removing the potential restores every path
    Q.qmc_set_pseudopotential(g.h, np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0, np.int32),
                              np.zeros(0), np.zeros(0), np.zeros(s.n_nuc), np.zeros((0, 3)), np.zeros(0))
    g.set_walkers(synth.initial_walkers(s, 4, seed=1))
    Q.Batch([g]).close()
    g.close()
    with pytest.raises(Q.QmcError) as ex:
        Q.QMC(synth.with_multidet(s, 4), precision="fp64").set_walkers(synth.initial_walkers(s, 2, seed=1))
    assert ex.value.code == -9


def test_pseudopotential_argument_checks(Q):
    s = pp_system("water1_pp")
    g = Q.QMC(s, precision="fp64")
    args = dict(nucleus=s.pp_nuc, l=s.pp_l, n=s.pp_n, alpha=s.pp_alpha, beta=s.pp_beta, rcut=s.pp_rcut,
                quad=s.pp_quad, weights=s.pp_qw)
    for key, bad in (("l", np.full_like(s.pp_l, 4)), ("nucleus", np.full_like(s.pp_nuc, 3)),
                     ("alpha", -s.pp_alpha), ("quad", 2.0 * s.pp_quad), ("rcut", -np.ones(s.n_nuc))):
        a = dict(args)
        a[key] = bad
        with pytest.raises(Q.QmcError) as ex:
            Q.qmc_set_pseudopotential(g.h, a["nucleus"], a["l"], a["n"], a["alpha"], a["beta"], a["rcut"],
                                      a["quad"], a["weights"])
        assert ex.value.code == -1, key
    g.close()


@pytest.mark.parametrize("name,W", [("water1_pp", 7), ("water1_pp_j3", 3), ("water6_pp", 3)])
def test_jastrow_parameter_derivatives_with_pseudopotential(Q, name, W):
    """dlog and deloc with the non-local term's Jastrow dependence, FP64 at
    1e-10 and mixed at 1e-5 relative to max(1, |ref|) per parameter column
    scale, rotations at a fixed sweep counter on both sides."""
    s = pp_system(name)
    R = synth.initial_walkers(s, W, seed=23)
    ref_l, ref_e = O.Oracle(s).jastrow_derivs(R, pp_seed=99, pp_sweep=5)
    # the non-local term's part is really there: with it cut off deloc differs
    off = dataclasses.replace(s, pp_rcut=np.zeros(s.n_nuc))
    assert np.abs(O.Oracle(off).jastrow_derivs(R)[1] - ref_e).max() > 1e-3
    for prec, tol in (("fp64", 1e-10), ("mixed", 1e-5)):
        g = Q.QMC(s, precision=prec, seed=99)
        Q.qmc_set_rng(g.h, 99, 5)
        g.set_walkers(R)
        dl, de = g.jastrow_derivs()
        scale = np.maximum(1.0, np.abs(ref_e).max(axis=0))
        assert np.abs(dl - ref_l).max() <= tol * max(1.0, np.abs(ref_l).max()), prec
        assert (np.abs(de - ref_e) / scale).max() <= tol, (prec, (np.abs(de - ref_e) / scale).max())
        g.close()


@pytest.mark.parametrize("name,W", [("water1_pp", 33), ("water6_pp", 40)])
def test_nonlocal_u_rows_from_tensor_cores(Q, monkeypatch, name, W):
    """Mixed form: u_k = C A^-1 e_k of every electron as batched tensor-core
    GEMMs (three-way split TF32) ahead of the non-local pass, or formed by the
    kernel itself in FP32 (QMC_NLPP_TC=0): E_L, forces and parameter
    derivatives agree with the oracle at the mixed bounds either way, and the
    GEMMs ran (one per spin and 256-column block of the basis).  The library
    takes the GEMM path from 64 electrons per spin; the test lowers that."""
    s = pp_system(name)
    R = synth.initial_walkers(s, W, seed=31)
    o = O.Oracle(s)
    ref = o.evaluate(R, pp_seed=77, pp_sweep=3)["eloc"]
    ref_E, _ = o.forces(R, pp_seed=77, pp_sweep=3)
    _, ref_de = o.jastrow_derivs(R, pp_seed=77, pp_sweep=3)
    blocks = 2 * ((s.n_basis + 255) // 256)
    monkeypatch.setenv("QMC_NLPP_TC_MIN_N", "1")   # small spin blocks take the GEMM path too
    for tc in ("1", "0"):
        monkeypatch.setenv("QMC_NLPP_TC", tc)
        m = Q.QMC(s, precision="mixed", seed=77)
        Q.qmc_set_rng(m.h, 77, 3)
        m.set_walkers(R)
        Q.qmc_set_timing(m.h, 1)
        ev = m.eval_cached()
        _, launches = Q.qmc_get_timing(m.h, "nlpp")
        assert launches == (1 + blocks if tc == "1" else 1), (tc, launches)
        assert rel(ev["eloc"], ref) <= 1e-5, (tc, rel(ev["eloc"], ref))
        _, pw = m.forces()
        assert vrel(pw[:, 0], ref_E) <= 1e-3, (tc, vrel(pw[:, 0], ref_E))
        _, de = m.jastrow_derivs()
        scale = np.maximum(1.0, np.abs(ref_de).max(axis=0))
        assert (np.abs(de - ref_de) / scale).max() <= 1e-5, (tc, (np.abs(de - ref_de) / scale).max())
        m.close()


def test_nonlocal_walker_slices_at_4096_walkers(Q):
    """Valence 32-water cluster at 4096 walkers (the full workload size): the
    tensor-core u_k rows take 2 GB at most, so the non-local pass runs in two
    walker slices (u_k GEMMs, then the kernel at a walker offset, per slice);
    E_L of walkers at both ends of both slices against the oracle at the same
    rotations."""
    s = synth.with_pseudopotential(synth.water_system(32))
    W = 4096
    R = synth.initial_walkers(s, W, seed=17)
    m = Q.QMC(s, precision="mixed", seed=61, delay_rank=32, recompute_period=100)
    Q.qmc_set_rng(m.h, 61, 8)
    m.set_walkers(R)
    Q.qmc_set_timing(m.h, 1)
    ev = m.eval_cached()
    _, launches = Q.qmc_get_timing(m.h, "nlpp")
    assert launches == 2 * (1 + 2 * 3), launches   # two slices: six GEMMs and one kernel each
    o = O.Oracle(s)
    for slot in (0, 2047, 2048, W - 1):
        ref = o.evaluate(R[slot:slot + 1], pp_seed=61, pp_sweep=8, pp_slot0=slot)["eloc"][0]
        assert rel(ev["eloc"][slot], ref) <= 1e-5, (slot, ev["eloc"][slot], ref)
    m.close()
