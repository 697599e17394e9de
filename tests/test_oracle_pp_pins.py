"""Pins of the oracle's semi-local pseudopotential (the valence Hamiltonian
with effective core potentials of Sec. "The SPICE2(+)-ccECP dataset" and
Sec. "Quantum Monte Carlo") against closed forms that do not go through the
oracle's quadrature path: the exact angular projection of an off-centre
Gaussian (modified spherical Bessel functions), the cofactor expansion of a
determinant of nucleus-centred s, p and d orbitals, the exactness degree of
the icosahedral rule, the local terms written out, and the statistics of a
uniform random rotation."""
from __future__ import annotations

import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2504_07948_gb300 import synth

scipy_special = pytest.importorskip("scipy.special")


def _product_rule(n_theta: int = 16, n_phi: int = 32):
    """Gauss-Legendre in cos(theta) times equally spaced phi: weights sum to
    1 and the rule is exact for harmonics of degree < min(2 n_theta, n_phi)."""
    t, g = np.polynomial.legendre.leggauss(n_theta)
    phi = 2.0 * np.pi * np.arange(n_phi) / n_phi
    st = np.sqrt(1.0 - t * t)
    P = np.stack([np.outer(st, np.cos(phi)), np.outer(st, np.sin(phi)), np.outer(t, np.ones(n_phi))],
                 axis=-1).reshape(-1, 3)
    w = np.outer(g / 2.0, np.full(n_phi, 1.0 / n_phi)).reshape(-1)
    return P, w


def _attach(sys, terms, rcut, rule):
    """Copy of sys with pseudopotential terms [(nucleus, l, n, alpha, beta)],
    cutoff radii [n_nuc] and quadrature rule (points, weights)."""
    s = sys.copy()
    s.pp_nuc = np.array([t[0] for t in terms], np.int32)
    s.pp_l = np.array([t[1] for t in terms], np.int32)
    s.pp_n = np.array([t[2] for t in terms], np.int32)
    s.pp_alpha = np.array([t[3] for t in terms], np.float64)
    s.pp_beta = np.array([t[4] for t in terms], np.float64)
    s.pp_rcut = np.asarray(rcut, np.float64)
    s.pp_quad = np.ascontiguousarray(rule[0], dtype=np.float64)
    s.pp_qw = np.ascontiguousarray(rule[1], dtype=np.float64)
    return s


def _radial(terms, a, l, r):
    return sum(b * r ** (n - 2) * math.exp(-al * r * r) for (nu, ll, n, al, b) in terms if nu == a and ll == l)


def _legendre(l, x):
    return [1.0, x, 0.5 * (3 * x * x - 1), 0.5 * (5 * x ** 3 - 3 * x)][l]


def test_icosahedron_rule_is_exact_to_degree_five():
    P, w = synth.icosahedron_rule()
    assert P.shape == (12, 3) and abs(w.sum() - 1.0) < 1e-15
    assert np.allclose(np.linalg.norm(P, axis=1), 1.0, atol=1e-15)

    def dfact(k):
        return math.prod(range(k, 0, -2)) if k > 0 else 1

    def sphere_mean(a, b, c):
        if a % 2 or b % 2 or c % 2:
            return 0.0
        return dfact(a - 1) * dfact(b - 1) * dfact(c - 1) / dfact(a + b + c + 1)

    worst6 = 0.0
    for deg in range(7):
        for a in range(deg + 1):
            for b in range(deg + 1 - a):
                c = deg - a - b
                q = float((w * P[:, 0] ** a * P[:, 1] ** b * P[:, 2] ** c).sum())
                if deg <= 5:
                    assert abs(q - sphere_mean(a, b, c)) < 1e-14, (a, b, c)
                else:
                    worst6 = max(worst6, abs(q - sphere_mean(a, b, c)))
    assert worst6 > 1e-3   # a 5-design, not a 6-design


def test_pp_rotation_is_a_uniform_rotation():
    Rs = np.array([O.pp_rotation(11, t, a, w) for t in range(25) for a in range(4) for w in range(40)])
    n = Rs.shape[0]
    assert np.abs(np.einsum("kji,kjl->kil", Rs, Rs) - np.eye(3)).max() < 1e-14
    assert np.abs(np.linalg.det(Rs) - 1.0).max() < 1e-13
    # Haar measure on SO(3): every entry has mean 0 and variance 1/3, the
    # trace 1 + 2 cos(theta) has mean 0, and R e_z is uniform on the sphere
    se = math.sqrt(1.0 / 3.0 / n)
    assert np.abs(Rs.mean(axis=0)).max() < 5 * se
    assert abs(np.trace(Rs, axis1=1, axis2=2).mean()) < 5 * math.sqrt(1.0 / n)
    z = Rs[:, :, 2]
    assert np.abs((z ** 2).mean(axis=0) - 1.0 / 3.0).max() < 5 * math.sqrt(4.0 / 45.0 / n)
    # a different counter gives a different rotation
    assert np.abs(O.pp_rotation(11, 0, 0, 0) - O.pp_rotation(11, 0, 0, 1)).max() > 1e-3


def _ghost_gaussian_system(Ra, c, alpha):
    """One electron, nucleus 0 at Ra (the pseudopotential site, Z = 1) and a
    charge-free centre at Ra + c carrying one s primitive exp(-alpha r^2);
    no Jastrow."""
    Ra = np.asarray(Ra, float)
    return synth.System(Z=np.array([1.0, 0.0]), R=np.array([Ra, Ra + np.asarray(c, float)]), n_up=1, n_dn=0,
                        shell_center=np.array([1], np.int32), shell_l=np.array([0], np.int32),
                        shell_pure=np.array([0], np.int32), shell_nprim=np.array([1], np.int32),
                        alpha=np.array([alpha]), coef=np.array([1.0]), C=np.array([[1.0]]),
                        occ_up=np.array([0], np.int32), occ_dn=np.zeros(0, np.int32),
                        a_anti=0.0, a_par=0.0, b_ee=0.0, a_en=np.zeros(2), b_en=0.0)


GHOST_TERMS = [(0, 0, 1, 1.1, 2.0), (0, 0, 2, 0.7, -1.5), (0, 1, 2, 0.9, 3.0), (0, 2, 3, 1.3, 0.8),
               (0, 3, 2, 1.0, 0.5)]


@pytest.mark.parametrize("rcut", [10.0, 1.0])
def test_nonlocal_projection_of_an_off_centre_gaussian(rcut):
    """psi(r) = exp(-alpha |r - Ra - c|^2).  With x = r - Ra on the sphere
    |x| = r, exp(2 alpha r c cos g) = sum_L (2L+1) i_L(2 alpha r c) P_L(cos g),
    and the addition theorem gives the exact projection
      (2l+1) <P_l(x_hat . d) psi(Ra + r d)>_d / psi(r)
        = (2l+1) i_l(2 alpha r c) P_l(x_hat . c_hat) exp(-alpha (r^2 + c^2)) / psi(r)."""
    Ra, c, alpha = np.array([0.3, -0.2, 0.5]), np.array([0.4, 0.25, -0.3]), 0.8
    s = _attach(_ghost_gaussian_system(Ra, c, alpha), GHOST_TERMS, [rcut, 0.0], _product_rule())
    rng = np.random.default_rng(3)
    W = 12
    dirs = rng.normal(size=(W, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    rad = rng.uniform(0.2, 2.0, size=W)
    R = (Ra + rad[:, None] * dirs)[:, None, :]
    got = O.Oracle(s).nonlocal_energy(R, pp_seed=5, pp_sweep=9)
    cn = np.linalg.norm(c)
    for w in range(W):
        x = R[w, 0] - Ra
        r = np.linalg.norm(x)
        cosg = float(x @ c) / (r * cn)
        psi = math.exp(-alpha * float((x - c) @ (x - c)))
        want = 0.0
        if r < rcut:
            for l in range(4):
                want += (_radial(GHOST_TERMS, 0, l, r) * (2 * l + 1) * scipy_special.spherical_in(l, 2 * alpha * r * cn)
                         * _legendre(l, cosg) * math.exp(-alpha * (r * r + cn * cn)) / psi)
        assert abs(got[w] - want) < 1e-12 * max(1.0, abs(want)), (w, got[w], want)


def test_nonlocal_of_nucleus_centred_orbitals_by_cofactor_expansion():
    """Orbitals built from s, p and pure-d functions on the pseudopotential
    nucleus: projecting electron i's angular dependence keeps, in each
    orbital, the functions of that l, so by the cofactor expansion of the
    determinant along row i the non-local term of electron i is
    sum_l v_l(r_i) sum_j (P_l phi_j)(r_i) (A^-1)_{ji}.  The electron-nucleus
    Jastrow is radial about the nucleus and drops out; the icosahedral rule
    is exact for these integrands (degree <= 4) under any rotation."""
    Ra = np.array([0.2, 0.1, -0.3])
    shells = [(0, 0, [3.0, 0.6], [0.5, 0.7]), (1, 0, [0.9], [1.0]), (2, 1, [0.7], [1.0])]
    lof = [0, 1, 1, 1, 2, 2, 2, 2, 2]
    sc, sl, sp, sn, al, co = [], [], [], [], [], []
    for (l, pure, a, cc) in shells:
        sc.append(0); sl.append(l); sp.append(pure); sn.append(len(a)); al.extend(a); co.extend(cc)
    nb = 9
    Q, _ = np.linalg.qr(np.random.default_rng(7).normal(size=(nb, nb)))
    base = synth.System(Z=np.array([3.0]), R=Ra[None, :].copy(), n_up=3, n_dn=2,
                        shell_center=np.array(sc, np.int32), shell_l=np.array(sl, np.int32),
                        shell_pure=np.array(sp, np.int32), shell_nprim=np.array(sn, np.int32),
                        alpha=np.array(al), coef=np.array(co), C=np.ascontiguousarray(Q.T),
                        occ_up=np.array([0, 1, 2], np.int32), occ_dn=np.array([0, 1], np.int32),
                        a_anti=0.0, a_par=0.0, b_ee=1.0, a_en=np.array([-0.7]), b_en=1.0)
    terms = [(0, -1, 2, 0.5, -1.0), (0, 0, 2, 0.8, 1.7), (0, 1, 1, 0.6, -0.9), (0, 2, 2, 1.1, 2.2)]
    rcut = 1.2
    s = _attach(base, terms, [rcut], synth.icosahedron_rule())
    o = O.Oracle(s)
    rng = np.random.default_rng(11)
    W = 6
    R = Ra + rng.normal(0.0, 0.8, size=(W, 5, 3))
    got = o.nonlocal_energy(R, pp_seed=21, pp_sweep=4)
    C = s.C
    for w in range(W):
        chi = np.array([o.basis(R[w, i])[:, 0] for i in range(5)])    # [electron, basis]
        want = 0.0
        for (i0, n, occ) in ((0, 3, s.occ_up), (3, 2, s.occ_dn)):
            A = chi[i0:i0 + n] @ C[occ].T                               # A_ij = phi_j(r_i)
            Ainv = np.linalg.inv(A)
            for k in range(n):
                x = R[w, i0 + k] - Ra
                r = np.linalg.norm(x)
                if r >= rcut:
                    continue
                for l in range(3):
                    mask = np.array([lb == l for lb in lof], float)
                    Pphi = C[occ] @ (mask * chi[i0 + k])               # (P_l phi_j)(r_i)
                    want += _radial(terms, 0, l, r) * float(Pphi @ Ainv[:, k])
        assert abs(got[w] - want) < 1e-11 * max(1.0, abs(want)), (w, got[w], want)


def test_local_terms_and_the_energy_split():
    """E_L with the pseudopotential minus E_L without it equals the local
    terms written out plus the non-local energy."""
    s = synth.with_pseudopotential(synth.water_system(1))
    bare = s.copy()
    bare.pp_nuc = None
    R = synth.initial_walkers(s, 6, seed=4)
    o = O.Oracle(s)
    e_pp = o.evaluate(R, pp_seed=1, pp_sweep=2)["eloc"]
    e_bare = O.Oracle(bare).evaluate(R)["eloc"]
    vnl = o.nonlocal_energy(R, pp_seed=1, pp_sweep=2)
    for w in range(R.shape[0]):
        loc = 0.0
        for t in range(s.n_pp):
            if s.pp_l[t] != -1:
                continue
            a = s.pp_nuc[t]
            for i in range(s.n_elec):
                r = np.linalg.norm(R[w, i] - s.R[a])
                loc += s.pp_beta[t] * r ** (s.pp_n[t] - 2) * math.exp(-s.pp_alpha[t] * r * r)
        assert abs(e_pp[w] - e_bare[w] - loc - vnl[w]) < 1e-10 * max(1.0, abs(e_pp[w]))
    assert np.all(np.abs(vnl) > 0)


def test_valence_system_counts():
    s = synth.with_pseudopotential(synth.water_system(2))
    assert s.n_up == s.n_dn == 8 and np.allclose(s.Z, [6, 1, 1, 6, 1, 1])
    assert s.n_elec == int(round(s.Z.sum()))
    assert np.all(s.a_en[s.Z == 6] == 0.0)


def test_sampling_drivers_draw_rotations_from_the_next_sweep_counter():
    """The VMC trace after the sweep with counter t is E_L with rotations
    from counter t + 1 (so a sweep's E_L and the next sweep's moves share a
    counter value but not a purpose)."""
    s = synth.with_pseudopotential(synth.water_system(1))
    o = O.Oracle(s)
    R0 = synth.initial_walkers(s, 4, seed=8)
    R, _, tr = o.vmc(R0, 2, 0.02, seed=77, step0=40)
    e = o.evaluate(R, pp_seed=77, pp_sweep=42)["eloc"]
    assert np.abs(tr[1] - e).max() < 1e-12 * np.abs(e).max()
    e_other = o.evaluate(R, pp_seed=77, pp_sweep=41)["eloc"]
    assert np.abs(tr[1] - e_other).max() > 1e-8


def _moved_pp(s, a, c, h):
    t = s.copy()
    t.R = t.R.copy()
    t.R[a, c] += h
    return O.Oracle(t, nthreads=1)


@pytest.mark.parametrize("case", ["water1", "water1_multidet", "small_l3"])
def test_pseudopotential_forces_by_central_differences(case):
    """dE_L/dR_a with the local and non-local pseudopotential terms (the
    quadrature points follow their nucleus; the rotations held fixed)
    against fourth-order central differences in every nuclear coordinate,
    h = 1e-4 bohr, relative 1e-6; ln|psi| is unchanged by the potential."""
    if case == "small_l3":
        base = synth.random_small_system(np.random.default_rng(5), n_nuc=2, n_up=2, n_dn=2)
        s = _attach(base, [(0, -1, 1, 2.0, 1.5), (0, 0, 2, 1.2, 3.0), (0, 1, 2, 0.9, -2.0), (0, 2, 3, 1.4, 0.7),
                           (0, 3, 2, 1.0, 0.4), (1, 1, 2, 1.1, 1.3)], [2.5, 2.0], synth.icosahedron_rule())
    else:
        s = synth.with_pseudopotential(synth.water_system(1))
        if case == "water1_multidet":
            s = synth.with_multidet(s, 5, n_active=4, max_exc=2, seed=3)
    o = O.Oracle(s, nthreads=1)
    R = synth.initial_walkers(s, 2, seed=4) if case != "small_l3" else \
        np.random.default_rng(8).normal(0, 0.9, size=(2, s.n_elec, 3))
    kw = dict(pp_seed=3, pp_sweep=5)
    dEL, dlg = o.forces(R, **kw)
    assert np.abs(o.nonlocal_energy(R, **kw)).max() > 1e-3
    h = 1e-4
    for a in range(s.n_nuc):
        for c in range(3):
            ev = {k: _moved_pp(s, a, c, k * h).evaluate(R, **kw) for k in (-2, -1, 1, 2)}
            d4 = lambda q: (ev[-2][q] - 8 * ev[-1][q] + 8 * ev[1][q] - ev[2][q]) / (12 * h)
            fdE, fdL = d4("eloc"), d4("logpsi")
            assert np.all(np.abs(fdE - dEL[:, a, c]) <= 1e-6 * np.maximum(1, np.abs(fdE))), (a, c, fdE, dEL[:, a, c])
            assert np.all(np.abs(fdL - dlg[:, a, c]) <= 1e-6 * np.maximum(1, np.abs(fdL)))


@pytest.mark.parametrize("three_body", [False, True])
def test_pseudopotential_jastrow_parameter_derivatives_by_central_differences(three_body):
    """dE_L/dp with the pseudopotential (the non-local ratios carry the
    Jastrow) against fourth-order central differences of E_L in every
    Jastrow parameter, rotations held fixed (relative 1e-6)."""
    s = synth.with_pseudopotential(synth.water_system(1))
    if three_body:
        s = synth.with_three_body(s, scale=0.2)
    o = O.Oracle(s, nthreads=1)
    R = synth.initial_walkers(s, 2, seed=6)
    kw = dict(pp_seed=9, pp_sweep=2)
    dlog, deloc = o.jastrow_derivs(R, **kw)
    P = dlog.shape[1]
    from test_oracle_pins import _with_param, _param_value
    for q in range(P):
        v = _param_value(s, q)
        h = 1e-4 * max(1.0, abs(v))
        ev = {k: O.Oracle(_with_param(s, q, v + k * h), nthreads=1).evaluate(R, **kw) for k in (-2, -1, 1, 2)}
        d4 = lambda key: (ev[-2][key] - 8 * ev[-1][key] + 8 * ev[1][key] - ev[2][key]) / (12 * h)
        fl, fe = d4("logpsi"), d4("eloc")
        assert np.all(np.abs(fl - dlog[:, q]) <= 1e-6 * np.maximum(1, np.abs(fl))), (q, fl, dlog[:, q])
        assert np.all(np.abs(fe - deloc[:, q]) <= 1e-6 * np.maximum(1, np.abs(fe))), (q, fe, deloc[:, q])
