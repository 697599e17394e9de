"""Pins of the CPU FP64 oracle against what physics and mathematics fix.

The paper prints no worked example for the DMC stage, so every pin here is a
closed form, an invariant, a brute-force evaluation on a tiny input, or a
finite difference; each one is chosen so that a plausible slip in the
oracle (a dropped term, a flipped sign, a transposed index) fails it.
"""
import itertools
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2504_07948_gb300 import synth


# ----------------------------------------------------------------------
# basis functions
# ----------------------------------------------------------------------

def _one_center_system(shells, center=(0.0, 0.0, 0.0)):
    """System with one nucleus and the given [(l, pure, alphas, coefs)]."""
    sc, sl, sp, sn, al, co = [], [], [], [], [], []
    for (l, pure, a, c) in shells:
        sc.append(0); sl.append(l); sp.append(pure); sn.append(len(a)); al.extend(a); co.extend(c)
    nb = sum(synth.shell_size(l, p) for l, p in zip(sl, sp))
    return synth.System(Z=np.array([1.0]), R=np.array([center], dtype=np.float64), n_up=1, n_dn=0,
                        shell_center=np.array(sc, np.int32), shell_l=np.array(sl, np.int32),
                        shell_pure=np.array(sp, np.int32), shell_nprim=np.array(sn, np.int32),
                        alpha=np.array(al), coef=np.array(co), C=np.eye(nb),
                        occ_up=np.array([0], np.int32), occ_dn=np.zeros(0, np.int32),
                        a_anti=0.0, a_par=0.0, b_ee=0.0, a_en=np.zeros(1), b_en=0.0)


def _overlap_by_quadrature(o, beta, n=48):
    """S_kl = int Phi_k Phi_l d^3r by a tensor Gauss-Hermite rule with
    weight exp(-beta r^2); the integrand divided by the weight is smooth."""
    x, w = np.polynomial.hermite.hermgauss(n)
    x = x / math.sqrt(beta)
    w = w / math.sqrt(beta)
    nb = o.sys.n_basis
    S = np.zeros((nb, nb))
    for i, j, k in itertools.product(range(n), repeat=3):
        r = (x[i], x[j], x[k])
        wt = w[i] * w[j] * w[k] * math.exp(beta * (x[i] ** 2 + x[j] ** 2 + x[k] ** 2))
        v = o.basis(r)[:, 0]
        S += wt * np.outer(v, v)
    return S


def test_basis_normalisation_and_orthogonality():
    """Every contracted s, p, pure-d and Cartesian-d function has unit norm;
    functions of one shell are orthogonal (real solid harmonics), and the
    pure d set is orthogonal to an s function on the same centre (traceless)."""
    shells = [(0, 0, [1.3, 0.6], [0.7, 0.4]),
              (1, 0, [1.1, 0.5, 0.8], [0.3, 0.9, 0.5]),
              (2, 1, [0.9, 0.55], [0.6, 0.8]),
              (2, 0, [1.0], [1.0])]
    o = O.Oracle(_one_center_system(shells), nthreads=1)
    S = _overlap_by_quadrature(o, beta=0.9, n=40)
    assert np.allclose(np.diag(S), 1.0, atol=1e-9), np.diag(S)
    # s=0, p=1..3, pure d=4..8, Cartesian d=9..14
    blocks = [range(1, 4), range(4, 9)]
    for b in blocks:
        for i in b:
            for j in b:
                if i != j:
                    assert abs(S[i, j]) < 1e-9
    for j in range(4, 9):   # pure d orthogonal to s
        assert abs(S[0, j]) < 1e-9
    # Cartesian xx and yy are not orthogonal: <xx|yy> = 1/3 for normalised functions
    assert abs(S[9, 12] - 1.0 / 3.0) < 1e-9


@pytest.mark.parametrize("order", [1, 2, 3])
def test_basis_derivatives_by_central_differences(order):
    """Each derivative slot of order k equals the central difference of a
    slot of order k-1 (h = 1e-4)."""
    rng = np.random.default_rng(7)
    s = synth.random_small_system(rng, n_nuc=2)
    o = O.Oracle(s, nthreads=1)
    slots = [(0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1), (2, 0, 0), (1, 1, 0), (1, 0, 1), (0, 2, 0),
             (0, 1, 1), (0, 0, 2), (3, 0, 0), (2, 1, 0), (2, 0, 1), (1, 2, 0), (1, 1, 1), (1, 0, 2),
             (0, 3, 0), (0, 2, 1), (0, 1, 2), (0, 0, 3)]
    idx = {m: k for k, m in enumerate(slots)}
    h = 1e-4
    for trial in range(4):
        r = rng.normal(0, 1.0, 3)
        B = o.basis(r)
        for k, m in enumerate(slots):
            if sum(m) != order:
                continue
            d = next(c for c in range(3) if m[c] > 0)
            lower = list(m); lower[d] -= 1
            e = np.zeros(3); e[d] = h
            fd = (o.basis(r + e)[:, idx[tuple(lower)]] - o.basis(r - e)[:, idx[tuple(lower)]]) / (2 * h)
            scale = np.maximum(1.0, np.abs(B[:, k]))
            assert np.all(np.abs(fd - B[:, k]) <= 2e-6 * scale), (m, np.max(np.abs(fd - B[:, k])))


def test_pure_d_is_harmonic_combination():
    """Pure d functions are solid harmonics: their angular parts are
    annihilated by the angular-free Laplacian test  lap(P e^{-ar^2}) =
    (4a^2 r^2 - 2a(2l+3)) P e^{-ar^2} for a single primitive."""
    a = 0.8
    o = O.Oracle(_one_center_system([(2, 1, [a], [1.0])]), nthreads=1)
    rng = np.random.default_rng(3)
    for _ in range(5):
        r = rng.normal(0, 1, 3)
        B = o.basis(r)
        lap = B[:, 4] + B[:, 7] + B[:, 9]
        r2 = float(r @ r)
        assert np.allclose(lap, (4 * a * a * r2 - 2 * a * 7) * B[:, 0], rtol=1e-12, atol=1e-14)


# ----------------------------------------------------------------------
# determinants (Eq. 3 notation: A_ij = phi_j(r_i))
# ----------------------------------------------------------------------

def _leibniz(A):
    n = A.shape[0]
    tot = 0.0
    for perm in itertools.permutations(range(n)):
        sgn = 1
        p = list(perm)
        for i in range(n):
            for j in range(i + 1, n):
                if p[i] > p[j]:
                    sgn = -sgn
        tot += sgn * np.prod([A[i, perm[i]] for i in range(n)])
    return tot


@pytest.mark.parametrize("n", [1, 2, 3, 4])
def test_lu_det_vs_leibniz(n):
    rng = np.random.default_rng(n)
    for _ in range(5):
        A = rng.normal(size=(n, n))
        la, sg, inv = O.lu_det(A)
        d = _leibniz(A)
        assert sg == np.sign(d)
        assert abs(la - math.log(abs(d))) < 1e-13
        assert np.allclose(A @ inv, np.eye(n), atol=1e-12)


def test_lu_det_vs_numpy_and_edge_cases():
    rng = np.random.default_rng(11)
    A = rng.normal(size=(30, 30))
    la, sg, inv = O.lu_det(A)
    s2, l2 = np.linalg.slogdet(A)
    assert sg == s2 and abs(la - l2) < 1e-11
    assert np.allclose(inv, np.linalg.inv(A), atol=1e-10)
    la, sg, _ = O.lu_det(np.zeros((0, 0)))
    assert la == 0.0 and sg == 1.0
    la, sg, _ = O.lu_det(np.ones((3, 3)), inverse=False)
    assert sg == 0.0 and la == -np.inf


def test_eq3_log_derivative_trace_identity():
    """d ln|det A|/dlambda = tr(A^-1 dA/dlambda) (Eq. 3), against a
    central difference of the oracle's LU log-determinant."""
    rng = np.random.default_rng(5)
    A0, A1, A2 = (rng.normal(size=(6, 6)) for _ in range(3))
    A = lambda t: A0 + t * A1 + t * t * A2
    lam, h = 0.3, 1e-5
    _, _, inv = O.lu_det(A(lam))
    analytic = np.trace(inv @ (A1 + 2 * lam * A2))
    fd = (O.lu_det(A(lam + h), False)[0] - O.lu_det(A(lam - h), False)[0]) / (2 * h)
    assert abs(analytic - fd) < 1e-7 * max(1, abs(fd))


def test_eq4_derivative_of_trace():
    """d tr(A^-1 B)/dlambda = tr(A^-1 dB - X dA), X = A^-1 B A^-1 (Eq. 4)."""
    rng = np.random.default_rng(6)
    A0, A1, B0, B1 = (rng.normal(size=(5, 5)) for _ in range(4))
    f = lambda t: np.trace(O.lu_det(A0 + t * A1)[2] @ (B0 + t * B1))
    _, _, inv = O.lu_det(A0)
    X = inv @ B0 @ inv
    analytic = np.trace(inv @ B1 - X @ A1)
    h = 1e-5
    assert abs(analytic - (f(h) - f(-h)) / (2 * h)) < 1e-6 * max(1, abs(analytic))


# ----------------------------------------------------------------------
# local energy closed forms
# ----------------------------------------------------------------------

@pytest.mark.parametrize("Zc", [1.0, 2.0, 3.0])
def test_exact_hydrogenic_local_energy(Zc):
    """psi = exp(-Z r) is exact: E_L = -Z^2/2 at every point, zero variance."""
    o = O.Oracle(synth.hydrogenic_exact(Zc), nthreads=1)
    R = np.random.default_rng(1).normal(0, 1.5, size=(64, 1, 3))
    ev = o.evaluate(R)
    assert np.all(np.abs(ev["eloc"] + 0.5 * Zc * Zc) < 1e-13)
    r = np.linalg.norm(R[:, 0, :], axis=1)
    assert np.allclose(ev["logpsi"], -Zc * r, atol=1e-14)


def test_single_gaussian_local_energy():
    """psi = exp(-a r^2) in the field of charge Z: E_L = 3a - 2a^2 r^2 - Z/r."""
    a, Zc = 0.37, 1.0
    o = O.Oracle(synth.single_gaussian_atom(a, Zc), nthreads=1)
    R = np.random.default_rng(2).normal(0, 1.0, size=(50, 1, 3))
    ev = o.evaluate(R)
    r = np.linalg.norm(R[:, 0, :], axis=1)
    assert np.allclose(ev["eloc"], 3 * a - 2 * a * a * r * r - Zc / r, rtol=1e-12, atol=1e-12)


def test_two_electron_and_two_centre_potentials():
    """Two electrons of opposite spin in one Gaussian each, no Jastrow, a
    bare second nucleus: E_L = sum_i (3a - 2a^2 r_i^2) - sum_{i,b} Z_b/r_ib
    + 1/r_12 + Z_0 Z_1 / R_01 (pins V_ee, V_en over centres, V_nn)."""
    a = 0.5
    s = synth.single_gaussian_atom(a, 2.0, n_up=1, n_dn=1)
    s.Z = np.array([2.0, 1.5]); s.R = np.array([[0.0, 0.0, 0.0], [0.3, -0.8, 1.1]])
    s.a_en = np.zeros(2)
    o = O.Oracle(s, nthreads=1)
    R = np.random.default_rng(4).normal(0, 1.0, size=(20, 2, 3))
    ev = o.evaluate(R)
    r0 = np.linalg.norm(R, axis=2)
    r1 = np.linalg.norm(R - s.R[1], axis=2)
    r12 = np.linalg.norm(R[:, 0] - R[:, 1], axis=1)
    exp = (np.sum(3 * a - 2 * a * a * r0 ** 2, axis=1) - np.sum(2.0 / r0 + 1.5 / r1, axis=1) + 1.0 / r12
           + 3.0 / np.linalg.norm(s.R[1]))
    assert np.allclose(ev["eloc"], exp, rtol=1e-12)


def _fd_check_system(seed=0):
    rng = np.random.default_rng(seed)
    return synth.random_small_system(rng, n_nuc=2, n_up=3, n_dn=2)


@pytest.mark.parametrize("multidet", [False, True])
def test_gradient_laplacian_and_local_energy_by_finite_differences(multidet):
    """grad ln|psi| and lap ln|psi| against central differences of the
    oracle's ln|psi|; then E_L = -1/2 sum(lap + |grad|^2) + V with V from a
    direct Coulomb sum and the kinetic part taken from the differences alone."""
    s = _fd_check_system(0)
    if multidet:
        s = synth.with_multidet(_fd_small_closed(), n_det=7, n_active=3, max_exc=3, seed=9)
    o = O.Oracle(s, nthreads=1)
    rng = np.random.default_rng(10)
    R = rng.normal(0, 1.0, size=(3, s.n_elec, 3))
    ev = o.evaluate(R)
    h1, h2 = 1e-5, 1e-3
    for w in range(R.shape[0]):
        kin, scale = 0.0, 1.0
        for i in range(s.n_elec):
            lap_fd = 0.0
            for c in range(3):
                Rp = R[w:w + 1].copy(); Rp[0, i, c] += h1
                Rm = R[w:w + 1].copy(); Rm[0, i, c] -= h1
                gp = (o.evaluate(Rp)["logpsi"][0] - o.evaluate(Rm)["logpsi"][0]) / (2 * h1)
                assert abs(gp - ev["grad"][w, i, c]) < 1e-6 * max(1, abs(gp))
                f = []
                for k in (-2, -1, 1, 2):
                    Rk = R[w:w + 1].copy(); Rk[0, i, c] += k * h2
                    f.append(o.evaluate(Rk)["logpsi"][0])
                # five-point second difference, error O(h^4)
                lap_fd += (-f[0] + 16 * f[1] - 30 * ev["logpsi"][w] + 16 * f[2] - f[3]) / (12 * h2 ** 2)
            assert abs(lap_fd - ev["lap"][w, i]) < 1e-6 * max(1, abs(lap_fd))
            g = ev["grad"][w, i]
            kin += -0.5 * (lap_fd + g @ g)
            scale += abs(lap_fd) + g @ g
        V = 0.0
        for i in range(s.n_elec):
            for j in range(i + 1, s.n_elec):
                V += 1 / np.linalg.norm(R[w, i] - R[w, j])
            for a in range(s.n_nuc):
                V -= s.Z[a] / np.linalg.norm(R[w, i] - s.R[a])
        for a in range(s.n_nuc):
            for b in range(a + 1, s.n_nuc):
                V += s.Z[a] * s.Z[b] / np.linalg.norm(s.R[a] - s.R[b])
        assert abs(kin + V - ev["eloc"][w]) < 1e-6 * scale


def test_antisymmetry_under_same_spin_exchange():
    s = synth.water_system(1)
    o = O.Oracle(s)
    R = synth.initial_walkers(s, 6)
    R2 = R.copy()
    R2[:, [1, 3]] = R2[:, [3, 1]]          # two up electrons
    R3 = R.copy()
    R3[:, [5, 8]] = R3[:, [8, 5]]          # two down electrons
    a, b, c = o.evaluate(R), o.evaluate(R2), o.evaluate(R3)
    for x in (b, c):
        assert np.all(x["sign"] == -a["sign"])
        assert np.allclose(x["logpsi"], a["logpsi"], atol=1e-11)
        assert np.allclose(x["eloc"], a["eloc"], rtol=1e-10, atol=1e-9)
    fa, ga = o.forces(R[:2])
    fb, gb = o.forces(R2[:2])
    assert np.allclose(fa, fb, rtol=1e-9, atol=1e-8) and np.allclose(ga, gb, rtol=1e-9, atol=1e-9)
    # unlike-spin exchange is not a symmetry of psi: it must change something
    R4 = R.copy()
    R4[:, [0, 5]] = R4[:, [5, 0]]
    assert not np.allclose(o.evaluate(R4)["logpsi"], a["logpsi"])


def test_cusp_cancellation():
    """With a_anti = 1/2 and a_en = -Z the 1/r singularities of the
    potential cancel exactly against the Jastrow kinetic terms."""
    s = synth.water_system(1)
    o = O.Oracle(s, nthreads=1)
    R = synth.initial_walkers(s, 1, seed=99)
    out = []
    for d in (1e-3, 1e-6, 1e-8):
        Rk = R.copy()
        Rk[0, 5] = Rk[0, 0] + np.array([d, 0.0, 0.0])      # up 0 and down 0 collide
        out.append(o.evaluate(Rk)["eloc"][0])
    assert abs(out[1] - out[2]) < 1e-3 * max(1.0, abs(out[2]))
    out = []
    for d in (1e-6, 1e-8):
        Rk = R.copy()
        Rk[0, 2] = s.R[1] + np.array([0.0, d, 0.0])           # electron on an H nucleus
        out.append(o.evaluate(Rk)["eloc"][0])
    assert abs(out[0] - out[1]) < 1e-3 * max(1.0, abs(out[1]))
    # without the e-n cusp the local energy diverges like -Z/r
    s2 = s.copy(); s2.a_en = np.zeros(3)
    o2 = O.Oracle(s2, nthreads=1)
    Rk = R.copy(); Rk[0, 2] = s.R[1] + np.array([0.0, 1e-8, 0.0])
    assert o2.evaluate(Rk)["eloc"][0] < -1e7


# ----------------------------------------------------------------------
# three-body (electron-electron-nucleus) Jastrow and the Jastrow parameter
# derivatives of a linear-method optimisation step (the Jastrow paragraph
# after Eq. 2)
# ----------------------------------------------------------------------

def _j3_system(seed=0):
    return synth.with_three_body(_fd_check_system(seed), seed=seed + 50, scale=0.3, b3=0.8)


def test_three_body_term_closed_form():
    """One nucleus, two electrons, one term: the three-body Jastrow adds
    exactly c (s1^m s2^n + s1^n s2^m) s12^o, s(r) = r / (1 + b r), to
    ln|psi| (the rest of the trial function unchanged)."""
    base = _one_center_system([(0, 0, [0.7], [1.0])])
    base.n_up, base.n_dn = 1, 1
    base.occ_dn = np.array([0], np.int32)
    s = base.copy()
    s.j3_exponents = np.array([[3, 2, 2]], np.int32)
    s.j3_coef = np.array([[0.37]])
    s.j3_b = 0.6
    R = np.array([[[0.3, -0.2, 0.5], [-0.4, 0.1, 0.2]]])
    sc = lambda r: r / (1.0 + 0.6 * r)
    r1, r2 = np.linalg.norm(R[0, 0]), np.linalg.norm(R[0, 1])
    r12 = np.linalg.norm(R[0, 0] - R[0, 1])
    expect = 0.37 * (sc(r1) ** 3 * sc(r2) ** 2 + sc(r1) ** 2 * sc(r2) ** 3) * sc(r12) ** 2
    d = O.Oracle(s, nthreads=1).evaluate(R)["logpsi"][0] - O.Oracle(base, nthreads=1).evaluate(R)["logpsi"][0]
    assert abs(d - expect) < 1e-14


def test_three_body_gradient_laplacian_and_local_energy_by_finite_differences():
    """grad and lap of ln|psi| with the three-body term on, against central
    differences of the oracle's ln|psi| (the same check as for the two-body
    trial function)."""
    s = _j3_system(0)
    o = O.Oracle(s, nthreads=1)
    R = np.random.default_rng(11).normal(0, 1.0, size=(2, s.n_elec, 3))
    ev = o.evaluate(R)
    h1, h2 = 1e-5, 1e-3
    for w in range(R.shape[0]):
        for i in range(s.n_elec):
            lap_fd = 0.0
            for c in range(3):
                Rp = R[w:w + 1].copy(); Rp[0, i, c] += h1
                Rm = R[w:w + 1].copy(); Rm[0, i, c] -= h1
                gp = (o.evaluate(Rp)["logpsi"][0] - o.evaluate(Rm)["logpsi"][0]) / (2 * h1)
                assert abs(gp - ev["grad"][w, i, c]) < 1e-6 * max(1, abs(gp))
                f = []
                for k in (-2, -1, 1, 2):
                    Rk = R[w:w + 1].copy(); Rk[0, i, c] += k * h2
                    f.append(o.evaluate(Rk)["logpsi"][0])
                lap_fd += (-f[0] + 16 * f[1] - 30 * ev["logpsi"][w] + 16 * f[2] - f[3]) / (12 * h2 ** 2)
            assert abs(lap_fd - ev["lap"][w, i]) < 1e-6 * max(1, abs(lap_fd))


def test_three_body_term_keeps_the_cusps():
    """Every power in the three-body terms is 0 or >= 2, so the electron-
    electron and electron-nucleus cusps of the two-body Jastrow still cancel
    the Coulomb singularities; a term with o = 1 breaks the e-e cusp and
    E_L diverges."""
    s = synth.with_three_body(synth.water_system(1), scale=0.5)
    o = O.Oracle(s, nthreads=1)
    R = synth.initial_walkers(s, 1, seed=99)
    out = []
    for d in (1e-6, 1e-8):
        Rk = R.copy(); Rk[0, 5] = Rk[0, 0] + np.array([d, 0.0, 0.0])
        out.append(o.evaluate(Rk)["eloc"][0])
    assert abs(out[0] - out[1]) < 1e-3 * max(1.0, abs(out[1]))
    out = []
    for d in (1e-6, 1e-8):
        Rk = R.copy(); Rk[0, 2] = s.R[1] + np.array([0.0, d, 0.0])
        out.append(o.evaluate(Rk)["eloc"][0])
    assert abs(out[0] - out[1]) < 1e-3 * max(1.0, abs(out[1]))
    bad = synth.with_three_body(synth.water_system(1), scale=0.5, terms=((0, 0, 1),))
    ob = O.Oracle(bad, nthreads=1)
    Rk = R.copy(); Rk[0, 5] = Rk[0, 0] + np.array([1e-8, 0.0, 0.0])
    Rl = R.copy(); Rl[0, 5] = Rl[0, 0] + np.array([1e-6, 0.0, 0.0])
    assert abs(ob.evaluate(Rk)["eloc"][0] - ob.evaluate(Rl)["eloc"][0]) > 1e3


def _with_param(s, q, v):
    """Copy of s with Jastrow parameter q (order a_anti, a_par, b_ee, b_en,
    a_en[n_nuc], c3[n_nuc][n3]) set to v."""
    t = s.copy()
    nn = s.n_nuc
    if q == 0:
        t.a_anti = v
    elif q == 1:
        t.a_par = v
    elif q == 2:
        t.b_ee = v
    elif q == 3:
        t.b_en = v
    elif q < 4 + nn:
        t.a_en = np.array(s.a_en, dtype=float).copy(); t.a_en[q - 4] = v
    else:
        t.j3_coef = np.array(s.j3_coef, dtype=float).copy(); t.j3_coef.reshape(-1)[q - 4 - nn] = v
    return t


def _param_value(s, q):
    nn = s.n_nuc
    if q < 4:
        return [s.a_anti, s.a_par, s.b_ee, s.b_en][q]
    if q < 4 + nn:
        return float(s.a_en[q - 4])
    return float(np.asarray(s.j3_coef).reshape(-1)[q - 4 - nn])


@pytest.mark.parametrize("three_body", [False, True])
def test_jastrow_parameter_derivatives_by_central_differences(three_body):
    """d ln|psi| / dp and dE_L / dp for every Jastrow parameter against
    fourth-order central differences of the oracle's ln|psi| and E_L in that
    parameter (h = 1e-4 of the parameter's scale, relative 1e-6)."""
    s = _j3_system(1) if three_body else _fd_check_system(1)
    o = O.Oracle(s, nthreads=1)
    R = np.random.default_rng(12).normal(0, 1.0, size=(3, s.n_elec, 3))
    dlog, deloc = o.jastrow_derivs(R)
    P = dlog.shape[1]
    assert P == 4 + s.n_nuc + (s.n_nuc * len(s.j3_exponents) if three_body else 0)
    for q in range(P):
        v = _param_value(s, q)
        h = 1e-4 * max(1.0, abs(v))
        ev = {k: O.Oracle(_with_param(s, q, v + k * h), nthreads=1).evaluate(R) for k in (-2, -1, 1, 2)}
        d4 = lambda key: (ev[-2][key] - 8 * ev[-1][key] + 8 * ev[1][key] - ev[2][key]) / (12 * h)
        fl, fe = d4("logpsi"), d4("eloc")
        assert np.all(np.abs(fl - dlog[:, q]) <= 1e-6 * np.maximum(1, np.abs(fl))), (q, fl, dlog[:, q])
        assert np.all(np.abs(fe - deloc[:, q]) <= 1e-6 * np.maximum(1, np.abs(fe))), (q, fe, deloc[:, q])


# ----------------------------------------------------------------------
# ionic derivatives
# ----------------------------------------------------------------------

def _moved(s, a, c, h):
    t = s.copy()
    t.R = t.R.copy()
    t.R[a, c] += h
    return O.Oracle(t, nthreads=1)


@pytest.mark.parametrize("multidet", [False, True])
def test_forces_by_central_differences(multidet):
    """dE_L/dR_a and dln|psi|/dR_a (forward mode) against fourth-order
    central differences in the nuclear coordinates, h = 1e-4 bohr (rel 1e-6)."""
    s = _fd_check_system(1)
    if multidet:
        s = synth.with_multidet(s.copy() if s.n_up == s.n_dn else _fd_small_closed(), n_det=6,
                                n_active=3, max_exc=2, seed=4)
    o = O.Oracle(s, nthreads=1)
    R = np.random.default_rng(12).normal(0, 1.0, size=(2, s.n_elec, 3))
    dEL, dlg = o.forces(R)
    h = 1e-4
    for a in range(s.n_nuc):
        for c in range(3):
            ev = {k: _moved(s, a, c, k * h).evaluate(R) for k in (-2, -1, 1, 2)}
            # fourth-order central difference
            d4 = lambda q: (ev[-2][q] - 8 * ev[-1][q] + 8 * ev[1][q] - ev[2][q]) / (12 * h)
            fdE, fdL = d4("eloc"), d4("logpsi")
            assert np.all(np.abs(fdE - dEL[:, a, c]) <= 1e-6 * np.maximum(1, np.abs(fdE))), (a, c, fdE, dEL[:, a, c])
            assert np.all(np.abs(fdL - dlg[:, a, c]) <= 1e-6 * np.maximum(1, np.abs(fdL)))


def _fd_small_closed():
    rng = np.random.default_rng(21)
    return synth.random_small_system(rng, n_nuc=2, n_up=2, n_dn=2)


def test_force_translation_identity():
    """Moving every nucleus and every electron together leaves psi and E_L
    unchanged, so sum_a dX/dR_a = -sum_i grad_i X for X = ln|psi|."""
    s = synth.water_system(1)
    o = O.Oracle(s)
    R = synth.initial_walkers(s, 4)
    ev = o.evaluate(R)
    dEL, dlg = o.forces(R)
    assert np.allclose(dlg.sum(axis=1), -ev["grad"].sum(axis=1), rtol=1e-9, atol=1e-9)
    # E_L: total derivative under a rigid shift vanishes; electron part by FD
    h = 1e-5
    for c in range(3):
        Rp = R.copy(); Rp[:, :, c] += h
        Rm = R.copy(); Rm[:, :, c] -= h
        dEe = (o.evaluate(Rp)["eloc"] - o.evaluate(Rm)["eloc"]) / (2 * h)
        assert np.allclose(dEL[:, :, c].sum(axis=1), -dEe, rtol=1e-5, atol=1e-5)


# ----------------------------------------------------------------------
# space warp (Filippi and Umrigar 2000, named in Sec. "Single Determinant
# QMC Forces" as the variance reduction of the force estimator)
# ----------------------------------------------------------------------

def _warp_case(multidet):
    s = _fd_check_system(1)
    if multidet:
        s = synth.with_multidet(_fd_small_closed(), n_det=6, n_active=3, max_exc=2, seed=4)
    R = np.random.default_rng(13).normal(0, 1.0, size=(2, s.n_elec, 3))
    return s, R


@pytest.mark.parametrize("multidet", [False, True])
def test_electron_gradient_of_local_energy_by_central_differences(multidet):
    """dE_L/dr_i (forward mode over electron coordinates) against
    fourth-order central differences of E_L (h = 1e-5: one electron of the
    second walker sits where E_L varies on a 1e-3 bohr scale, rel 1e-6);
    dln|psi|/dr_i against the evaluation's own gradient."""
    s, R = _warp_case(multidet)
    o = O.Oracle(s, nthreads=1)
    gEL, glg = o.electron_grad(R)
    assert np.allclose(glg, o.evaluate(R)["grad"], rtol=1e-10, atol=1e-10)
    h = 1e-5
    for i in range(s.n_elec):
        for c in range(3):
            ev = {}
            for k in (-2, -1, 1, 2):
                Rk = R.copy()
                Rk[:, i, c] += k * h
                ev[k] = o.evaluate(Rk)["eloc"]
            fd = (ev[-2] - 8 * ev[-1] + 8 * ev[1] - ev[2]) / (12 * h)
            assert np.all(np.abs(fd - gEL[:, i, c]) <= 1e-6 * np.maximum(1, np.abs(fd))), (i, c, fd, gEL[:, i, c])


def test_electron_gradient_translation_identity():
    """sum_i dE_L/dr_i = -sum_a dE_L/dR_a: the electron-coordinate forward mode
    against the independent nuclear one (water monomer, 10 electrons)."""
    s = synth.water_system(1)
    o = O.Oracle(s)
    R = synth.initial_walkers(s, 3)
    gEL, glg = o.electron_grad(R)
    dEL, dlg = o.forces(R)
    sc = np.maximum(1.0, np.abs(dEL).max())
    assert np.all(np.abs(gEL.sum(axis=1) + dEL.sum(axis=1)) <= 1e-9 * sc)
    assert np.allclose(glg.sum(axis=1), -dlg.sum(axis=1), rtol=1e-10, atol=1e-10)


def test_warp_weights_partition_of_unity_and_gradient():
    """omega_a sums to one, its gradients to zero, omega_a -> 1 at nucleus a,
    and the analytic gradient matches central differences."""
    s = synth.water_system(2)
    o = O.Oracle(s, nthreads=1)
    rng = np.random.default_rng(5)
    for _ in range(20):
        r = s.R[rng.integers(s.n_nuc)] + rng.normal(0, 1.2, 3)
        om, gom = o.warp_weights(r)
        assert abs(om.sum() - 1.0) < 1e-14 and np.all(om >= 0)
        assert np.all(np.abs(gom.sum(axis=0)) < 1e-12 * max(1.0, np.abs(gom).max()))
        h = 1e-5
        for c in range(3):
            e = np.zeros(3); e[c] = h
            fd = (o.warp_weights(r + e)[0] - o.warp_weights(r - e)[0]) / (2 * h)
            assert np.allclose(fd, gom[:, c], rtol=1e-6, atol=1e-8)
    a = 3
    om, _ = o.warp_weights(s.R[a] + np.array([1e-4, -2e-4, 1e-4]))
    assert abs(om[a] - 1.0) < 1e-10


@pytest.mark.parametrize("multidet", [False, True])
def test_warped_forces_by_central_differences_of_the_warped_map(multidet):
    """Warped derivatives against fourth-order central differences of the
    coordinate map itself (the route the paper takes for the space warp,
    Sec. "Performance Measurement"): nucleus a moves by delta e_c, every
    electron by omega_a(r_i) delta e_c; E_L and ln|psi| + 1/2 ln J are
    differenced, J taken as the determinant of the map's 3x3 Jacobian per
    electron by central differences of omega (h = 1e-5 bohr, rel 1e-6)."""
    s, R = _warp_case(multidet)
    o = O.Oracle(s, nthreads=1)
    dELw, dlgw = o.warped_forces(R)
    om = np.array([[o.warp_weights(R[w, i])[0] for i in range(s.n_elec)] for w in range(R.shape[0])])
    eta = 1e-6

    def logjac(w, a, c, delta):
        tot = 0.0
        for i in range(s.n_elec):
            Jm = np.eye(3)
            for q in range(3):
                e = np.zeros(3); e[q] = eta
                dom = (o.warp_weights(R[w, i] + e)[0][a] - o.warp_weights(R[w, i] - e)[0][a]) / (2 * eta)
                Jm[c, q] += delta * dom
            tot += np.log(np.linalg.det(Jm))
        return tot

    h = 1e-5
    for a in range(s.n_nuc):
        for c in range(3):
            ev, lj = {}, {}
            for k in (-2, -1, 1, 2):
                Rk = R + k * h * om[:, :, a, None] * np.eye(3)[c]
                ev[k] = _moved(s, a, c, k * h).evaluate(Rk)
                lj[k] = np.array([logjac(w, a, c, k * h) for w in range(R.shape[0])])
            d4 = lambda f: (f(-2) - 8 * f(-1) + 8 * f(1) - f(2)) / (12 * h)
            fdE = d4(lambda k: ev[k]["eloc"])
            fdL = d4(lambda k: ev[k]["logpsi"] + 0.5 * lj[k])
            assert np.all(np.abs(fdE - dELw[:, a, c]) <= 1e-6 * np.maximum(1, np.abs(fdE))), (a, c, fdE, dELw[:, a, c])
            assert np.all(np.abs(fdL - dlgw[:, a, c]) <= 1e-6 * np.maximum(1, np.abs(fdL))), (a, c, fdL, dlgw[:, a, c])


def test_warped_forces_sum_to_zero_per_configuration():
    """The warp weights are a partition of unity, so the warped derivatives
    are those of a rigid translation of the whole system summed over nuclei:
    sum_a dX^w/dR_a = 0 for every configuration (X = E_L, ln|psi|)."""
    s = synth.water_system(2)
    o = O.Oracle(s)
    R = synth.initial_walkers(s, 3)
    dELw, dlgw = o.warped_forces(R)
    dEL, dlg = o.forces(R)
    scE = np.maximum(1.0, np.abs(dEL).max(axis=(1, 2)))
    scL = np.maximum(1.0, np.abs(dlg).max(axis=(1, 2)))
    assert np.all(np.abs(dELw.sum(axis=1)) <= 1e-9 * scE[:, None])
    assert np.all(np.abs(dlgw.sum(axis=1)) <= 1e-9 * scL[:, None])
    assert np.all(np.abs(dEL.sum(axis=1)).max(axis=1) > 1e-3 * scE)   # the unwarped ones do not


def test_warped_forces_vanish_for_one_electron_around_one_nucleus():
    """One nucleus: omega = 1 everywhere, the warp is a rigid translation and
    the warped derivatives vanish identically, also for an inexact trial
    function whose unwarped derivatives do not."""
    o = O.Oracle(synth.single_gaussian_atom(0.37, 1.0), nthreads=1)
    R = np.random.default_rng(6).normal(0, 1.0, size=(16, 1, 3))
    dEL, _ = o.forces(R)
    dELw, dlgw = o.warped_forces(R)
    assert np.abs(dEL).max() > 0.1
    assert np.abs(dELw).max() < 1e-12 and np.abs(dlgw).max() < 1e-13


def test_space_warp_estimator_is_unbiased_and_cuts_variance():
    """Over |psi|^2 the warp is a change of integration variables, so the
    warped and plain zero-variance zero-bias force samples have the same
    mean: their paired difference over VMC walkers (independent chains, the
    final configuration of each) is zero within 4.5 standard errors in every
    component, while the oxygen's sample variance drops by more than 100x
    (electrons in its core no longer make dE_L/dR diverge)."""
    s = synth.water_system(1)
    o = O.Oracle(s)
    R = synth.initial_walkers(s, 256, seed=3)
    R, _, _ = o.vmc(R, 30, 0.05, seed=7, trace=False)
    E = o.evaluate(R)["eloc"]
    dEL, dlg = o.forces(R)
    dELw, dlgw = o.warped_forces(R)
    Ec = (E - E.mean())[:, None, None]
    f = -dEL - 2.0 * Ec * dlg
    fw = -dELw - 2.0 * Ec * dlgw
    diff = fw - f
    se = diff.std(axis=0, ddof=1) / np.sqrt(diff.shape[0])
    assert np.all(np.abs(diff.mean(axis=0)) <= 4.5 * se)
    assert np.all(f.var(axis=0)[0] > 100.0 * fw.var(axis=0)[0])


# ----------------------------------------------------------------------
# force estimators: the zero-variance zero-bias form (Sec. "Single
# Determinant QMC Forces") with VMC and DMC weights, and the mixed
# estimator 2 F_DMC - F_VMC (Sec. "Performance Measurement")
# ----------------------------------------------------------------------

def _reweighted_energy(s, a, c, h, R, logpsi0, w):
    """Energy of the wavefunction with nucleus a moved by h along c, estimated
    on the fixed configurations R by reweighting: sum w q E_L / sum w q,
    q = |psi_moved / psi|^2 at each configuration."""
    ev = _moved(s, a, c, h).evaluate(R)
    q = w * np.exp(2.0 * (ev["logpsi"] - logpsi0))
    return float((q * ev["eloc"]).sum() / q.sum())


@pytest.mark.parametrize("weighted", [False, True])
def test_force_estimator_is_minus_the_derivative_of_the_reweighted_energy(weighted):
    """On fixed configurations X_w with weights w_w (a VMC sample; random
    positive weights stand for the DMC ones), the reweighted energy
    E(R) = sum_w w_w q_w(R) E_L(R; X_w) / sum_w w_w q_w(R), q = |psi_R / psi_R0|^2,
    has at R0 the exact derivative <dE_L> + 2 (<E_L dln|psi|> - <E_L><dln|psi|>),
    so the zero-variance zero-bias force is F = -dE/dR.  Checked against
    fourth-order central differences of E(R) (h = 1e-4 bohr, every nuclear
    coordinate of the water monomer, 128 VMC configurations): a dropped
    covariance term, a flipped sign or a wrong weighting fails it."""
    s = synth.water_system(1)
    o = O.Oracle(s)
    R = synth.initial_walkers(s, 128, seed=41)
    R, _, _ = o.vmc(R, 10, 0.05, seed=42, trace=False)
    ev = o.evaluate(R)
    dEL, dlg = o.forces(R)
    w = np.random.default_rng(43).uniform(0.2, 2.0, R.shape[0]) if weighted else np.ones(R.shape[0])
    F = O.force_estimator(ev["eloc"], dEL, dlg, weights=w if weighted else None)
    h = 1e-4
    for a in range(s.n_nuc):
        for c in range(3):
            E = {k: _reweighted_energy(s, a, c, k * h, R, ev["logpsi"], w) for k in (-2, -1, 1, 2)}
            fd = (E[-2] - 8 * E[-1] + 8 * E[1] - E[2]) / (12 * h)
            assert abs(-fd - F[a, c]) <= 1e-6 * max(1.0, abs(F[a, c])), (a, c, -fd, F[a, c])


def test_dmc_force_sums_follow_the_branching_weights():
    """One DMC step of the oracle with forces: its accumulated sums equal the
    sums of the per-walker derivatives at the post-sweep configurations with
    the branching weights of Eq. 1 (energies clipped to E_T +- 0.2 sqrt(N/tau)),
    formed here independently; the estimator built from them equals the
    weighted zero-variance zero-bias estimate pinned above."""
    s = synth.water_system(1)
    o = O.Oracle(s)
    R0 = synth.initial_walkers(s, 24, seed=5)
    tau, ET = 0.005, -70.0
    out = o.dmc(R0, 1, tau, ET, seed=9, step0=0, forces_every=1)
    assert out["status"] == 0
    E_old = o.evaluate(R0)["eloc"]
    R1, _, _ = o.vmc(R0, 1, tau, seed=9, step0=0, trace=False)   # the same sweep stream
    ev1 = o.evaluate(R1)
    dEL, dlg = o.forces(R1)
    eps = 0.2 * math.sqrt(s.n_elec / tau)
    clip = lambda e: np.clip(e, ET - eps, ET + eps)
    w = np.exp(-tau * (0.5 * (clip(E_old) + clip(ev1["eloc"])) - ET))
    ref = O.force_sums(ev1["eloc"], dEL, dlg, w)
    assert np.allclose(out["facc"], ref, rtol=1e-12, atol=0.0)
    F = O.force_from_sums(out["facc"], s.n_nuc)
    Fw = O.force_estimator(ev1["eloc"], dEL, dlg, weights=w)
    assert np.allclose(F, Fw, rtol=1e-11, atol=1e-11 * np.abs(Fw).max())


def test_mixed_estimator_cancels_the_first_order_trial_error():
    """Trial psi = phi + eps chi around the exact ground state phi (chi
    orthogonal): the VMC average <psi|O|psi>/<psi|psi> and the DMC
    (mixed-distribution) average <phi|O|psi>/<phi|psi> both miss <phi|O|phi>
    at first order in eps, and 2 F_DMC - F_VMC cancels that order.  Discrete
    model (random symmetric H and O): halving eps halves the VMC and DMC
    errors but quarters the mixed estimator's; with the exact trial all
    three coincide.  A swapped coefficient (2 F_VMC - F_DMC) stays first
    order and fails."""
    rng = np.random.default_rng(5)
    n = 12
    H = rng.normal(size=(n, n))
    H = H + H.T
    Ob = rng.normal(size=(n, n))
    Ob = Ob + Ob.T
    phi = np.linalg.eigh(H)[1][:, 0]
    chi = rng.normal(size=n)
    chi -= (chi @ phi) * phi
    exact = phi @ Ob @ phi

    def errors(eps):
        psi = phi + eps * chi
        f_vmc = psi @ Ob @ psi / (psi @ psi)
        f_dmc = phi @ Ob @ psi / (phi @ psi)
        f_mix = float(O.mixed_estimator(np.array(f_dmc), np.array(f_vmc)))
        return np.array([f_vmc, f_dmc, f_mix]) - exact

    e1, e2 = errors(2e-3), errors(1e-3)
    assert 1.9 < e1[0] / e2[0] < 2.1 and 1.9 < e1[1] / e2[1] < 2.1
    assert 3.8 < e1[2] / e2[2] < 4.2
    assert abs(e2[2]) < 5e-2 * abs(e2[1])
    assert np.allclose(errors(0.0), 0.0, atol=1e-12)


# ----------------------------------------------------------------------
# multi-determinant sums (Eq. 2)
# ----------------------------------------------------------------------

def test_multidet_single_reference_reproduces_single_determinant():
    s = synth.water_system(1)
    m = synth.with_multidet(s, n_det=1, n_active=4)
    R = synth.initial_walkers(s, 5)
    a, b = O.Oracle(s).evaluate(R), O.Oracle(m).evaluate(R)
    for k in ("logpsi", "sign", "eloc", "grad", "lap"):
        assert np.allclose(a[k], b[k], rtol=1e-12, atol=1e-12), k


def test_multidet_two_determinants_by_brute_force():
    """psi = e^J (c1 D1up D1dn + c2 D2up D2dn) built from two
    single-determinant evaluations with the same Jastrow."""
    s = synth.water_system(1)
    m = synth.with_multidet(s, n_det=2, n_active=4, seed=8)
    R = synth.initial_walkers(s, 5)
    ev = O.Oracle(m).evaluate(R)
    parts = []
    for k in range(2):
        t = s.copy()
        ou = [b for b in range(64) if (int(m.det_up[k, 0]) >> b) & 1]
        od = [b for b in range(64) if (int(m.det_dn[k, 0]) >> b) & 1]
        t.occ_up = np.array(ou, np.int32); t.occ_dn = np.array(od, np.int32)
        parts.append(O.Oracle(t).evaluate(R))
    psi = sum(m.ci[k] * parts[k]["sign"] * np.exp(parts[k]["logpsi"] - parts[0]["logpsi"]) for k in range(2))
    assert np.allclose(ev["logpsi"], parts[0]["logpsi"] + np.log(np.abs(psi)), atol=1e-11)
    assert np.all(ev["sign"] == np.sign(psi))


def test_multidet_order_invariance():
    s = synth.water_system(1)
    m = synth.with_multidet(s, n_det=12, n_active=6, seed=2)
    p = m.copy()
    perm = np.random.default_rng(0).permutation(12)
    p.det_up, p.det_dn, p.ci = m.det_up[perm], m.det_dn[perm], m.ci[perm]
    R = synth.initial_walkers(s, 4)
    a, b = O.Oracle(m).evaluate(R), O.Oracle(p).evaluate(R)
    assert np.allclose(a["logpsi"], b["logpsi"], atol=1e-11)
    assert np.allclose(a["eloc"], b["eloc"], rtol=1e-10)


# ----------------------------------------------------------------------
# random numbers
# ----------------------------------------------------------------------

def test_philox_statistics():
    """Counter-based stream: uniform 32-bit words, independent across
    counter lanes and keys (chi^2 on 16 bins, lag correlation)."""
    n = 20000
    words = np.array([O.philox4x32([k, 7, 3, 0], [1005, 0]) for k in range(n)], dtype=np.float64)
    u = (words + 0.5) / 2 ** 32
    for lane in range(4):
        h, _ = np.histogram(u[:, lane], bins=16, range=(0, 1))
        chi2 = np.sum((h - n / 16) ** 2 / (n / 16))
        assert chi2 < 45.0       # 15 dof, p ~ 1e-4
        assert abs(u[:, lane].mean() - 0.5) < 0.01
    c = np.corrcoef(u.T)
    assert np.all(np.abs(c - np.eye(4)) < 0.03)
    assert abs(np.corrcoef(u[:-1, 0], u[1:, 0])[0, 1]) < 0.03
    a = O.philox4x32([1, 2, 3, 4], [5, 6])
    b = O.philox4x32([1, 2, 3, 4], [5, 7])
    assert not np.array_equal(a, b)


# ----------------------------------------------------------------------
# sampling
# ----------------------------------------------------------------------

def blocking_error(x):
    """Flyvbjerg-Petersen blocking: the plateau (max) of the naive
    standard error over successive pair-averagings."""
    x = np.asarray(x, dtype=np.float64)
    best = x.std(ddof=1) / math.sqrt(len(x))
    while len(x) >= 16:
        x = 0.5 * (x[: len(x) // 2 * 2:2] + x[1: len(x) // 2 * 2:2])
        best = max(best, x.std(ddof=1) / math.sqrt(len(x)))
    return best


def test_vmc_exact_hydrogen_zero_variance():
    o = O.Oracle(synth.hydrogenic_exact(1.0))
    R0 = np.random.default_rng(0).normal(0, 1, size=(32, 1, 3))
    R, acc, tr = o.vmc(R0, 20, 0.1, seed=1005)
    assert np.all(np.abs(tr + 0.5) < 1e-13)
    assert acc.sum() > 0.5 * 32 * 20


def test_vmc_single_gaussian_mean_energy():
    """<E_L> over |psi|^2 for psi = exp(-a r^2), Z = 1, is 3a/2 - 2 sqrt(2a/pi)."""
    a = 0.5
    o = O.Oracle(synth.single_gaussian_atom(a))
    R0 = np.random.default_rng(0).normal(0, 1, size=(256, 1, 3))
    R, acc, tr = o.vmc(R0, 300, 0.2, seed=77)
    x = tr[50:].mean(axis=1)
    mean, err = x.mean(), blocking_error(x)
    exact = 1.5 * a - 2.0 * math.sqrt(2 * a / math.pi)
    assert abs(mean - exact) < 4 * err + 1e-4, (mean, err, exact)


def test_dmc_exact_hydrogen_constant_population():
    """With the exact ground state every weight is 1: E = -1/2 each step and
    the population never changes."""
    o = O.Oracle(synth.hydrogenic_exact(1.0))
    R0 = np.random.default_rng(0).normal(0, 1, size=(64, 1, 3))
    out = o.dmc(R0, 30, 0.01, -0.5, seed=3)
    assert out["status"] == 0
    assert np.all(out["pop"] == 64)
    assert np.all(np.abs(out["e_step"] + 0.5) < 1e-13)


def test_dmc_projects_nodeless_trial_to_ground_state():
    """psi_T = exp(-r / (1 + 0.3 r)) for hydrogen: nodeless and cusp-correct
    but not exact (VMC energy ~ -0.26).  DMC (Eq. 1) must project it onto
    the exact ground state, -1/2 Ha, up to a small time-step bias."""
    s = synth.hydrogenic_exact(1.0)
    s.b_en = 0.3
    o = O.Oracle(s)
    R0 = np.random.default_rng(0).normal(0, 1, size=(512, 1, 3))
    R, _, tr = o.vmc(R0, 200, 0.3, seed=5)
    evmc = tr[20:].mean()
    out = o.dmc(R, 600, 0.05, evmc, seed=6, step0=1000)
    assert out["status"] == 0
    e = out["e_step"][100:]
    mean, err = e.mean(), blocking_error(e)
    assert abs(mean + 0.5) < 4 * err + 0.005, (mean, err)
    assert mean < evmc - 0.1


def test_dmc_fixed_population_projects_to_ground_state():
    """Fixed-population DMC (systematic resampling with the same branching
    weights) on the nodeless inexact hydrogen trial function: the population
    stays exactly at its initial size every step and the energy projects to
    the exact -1/2 Ha; on the exact ground state every weight is 1 and each
    walker keeps exactly one copy (E = -1/2 each step)."""
    s = synth.hydrogenic_exact(1.0)
    o = O.Oracle(s)
    R0 = np.random.default_rng(0).normal(0, 1, size=(64, 1, 3))
    out = o.dmc(R0, 10, 0.01, -0.5, seed=3, fixed_pop=True)
    assert out["status"] == 0 and np.all(out["pop"] == 64)
    assert np.array_equal(out["R"].shape, R0.shape)
    assert np.all(np.abs(out["e_step"] + 0.5) < 1e-13)
    s.b_en = 0.3
    o = O.Oracle(s)
    R0 = np.random.default_rng(1).normal(0, 1, size=(384, 1, 3))
    R, _, tr = o.vmc(R0, 150, 0.3, seed=5)
    evmc = tr[20:].mean()
    out = o.dmc(R, 600, 0.05, evmc, seed=7, step0=1000, fixed_pop=True)
    assert out["status"] == 0 and np.all(out["pop"] == 384)
    e = out["e_step"][100:]
    mean, err = e.mean(), blocking_error(e)
    assert abs(mean + 0.5) < 4 * err + 0.005, (mean, err)
    assert mean < evmc - 0.1


def test_dmc_helium_nodeless_reaches_ground_state():
    """Nodeless He trial function (both cusps, not exact: VMC ~ -1.85 Ha):
    fixed-node DMC is exact for a nodeless ground state, so it must reach
    the non-relativistic He energy -2.903724 Ha up to the time-step bias."""
    s = synth.helium_nodeless()
    o = O.Oracle(s)
    R0 = synth.initial_walkers(s, 512)
    Rv, _, tr = o.vmc(R0, 200, 0.1, seed=777)
    evmc = tr[50:].mean()
    out = o.dmc(Rv, 1200, 0.01, evmc, seed=778, step0=1000)
    assert out["status"] == 0
    e = out["e_step"][300:]
    mean, err = e.mean(), blocking_error(e)
    assert abs(mean + 2.903724) < 4 * err + 0.01, (mean, err)
    assert mean < evmc - 0.5
