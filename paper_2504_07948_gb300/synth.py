"""Seeded synthetic inputs for the walker-batched Slater-Jastrow DMC path.

This module only *draws* inputs: nuclear geometries, raw (unnormalised) basis
exponents and contraction weights, orbital coefficient matrices, Jastrow
parameters, determinant lists and initial walker positions.  It holds none of
the method's arithmetic (no basis normalisation, no orbital evaluation, no
determinants); both the CPU oracle and the CUDA library consume its arrays and
do their own arithmetic.

The paper's production inputs (DFT orbitals and basis sets for SPICE2/ANI-2X
molecules, Sec. "Dataset") are not available, so water monomers and rigid
water clusters stand in for the paper's water-cluster benchmarks (Sec.
"Performance Measurement", water monomer/dimer/trimer and 8-152 electron
clusters).  Recipes:

* water: O at the origin, two H at 0.9572 A with a 104.52 degree H-O-H angle,
  the molecule in the xz-plane before rotation;
* clusters: uniformly random rigid rotations (Shoemake's quaternion method),
  random sequential placement of O atoms in a cube of side 3.1 m^(1/3) A,
  rejecting O-O < 2.6 A and any intermolecular atom pair < 1.5 A; the cube
  grows by 5 % after 10^4 consecutive rejections;
* basis per species (shared by all atoms of a species): O = s,s,s,p,p,d(pure),
  H = s,s,p; three primitives per shell with exponents log-uniform in
  [0.1, 1e4] (sorted descending) and raw contraction weights uniform in
  [0.1, 1.0]; 24 functions per water;
* orbitals: QR of a seeded N(0,1) N_b x N_b matrix with columns flipped so that
  diag(R) > 0; orbital j has coefficients Q[:, j]; the lowest n are occupied
  for both spins;
* Jastrow: Pade e-e with a_anti = 1/2, a_par = 1/4, b_ee = 1, and e-n with
  a_a = -Z_a, b_en = 1;
* walkers: Z_a electrons around each nucleus drawn from N(R_a, 0.5^2 bohr^2),
  spins alternating along that list; up-spin electrons are stored first.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np

BOHR_PER_ANGSTROM = 1.0 / 0.529177210903  # CODATA 2018 bohr radius

# Fixed seeds of the synthetic workloads.
SEED_GEOMETRY = 1001
SEED_BASIS = 1002
SEED_MO = 1003
SEED_CI = 1004
SEED_WALKERS = 1005
SEED_CLUSTER_SIZES = 1006


@dataclasses.dataclass
class System:
    """A molecule plus a Slater-Jastrow wavefunction, as flat arrays.

    Basis functions are ordered shell by shell; within a shell: s -> (1),
    Cartesian p -> (x, y, z), pure d -> (m=-2, -1, 0, +1, +2) =
    (xy, yz, 3z^2-r^2, xz, x^2-y^2) type, Cartesian d -> (xx, xy, xz, yy, yz,
    zz).  Primitive arrays are concatenated in shell order.
    """

    Z: np.ndarray            # [n_nuc] float64 nuclear charges
    R: np.ndarray            # [n_nuc, 3] float64 positions (bohr)
    n_up: int
    n_dn: int
    shell_center: np.ndarray  # [n_shell] int32
    shell_l: np.ndarray       # [n_shell] int32
    shell_pure: np.ndarray    # [n_shell] int32 (1 = spherical d)
    shell_nprim: np.ndarray   # [n_shell] int32
    alpha: np.ndarray         # [n_prim] float64 exponents
    coef: np.ndarray          # [n_prim] float64 raw contraction weights
    C: np.ndarray             # [n_mo, n_basis] float64 orbital coefficients
    occ_up: np.ndarray        # [n_up] int32 orbital indices
    occ_dn: np.ndarray        # [n_dn] int32
    a_anti: float = 0.5
    a_par: float = 0.25
    b_ee: float = 1.0
    a_en: Optional[np.ndarray] = None  # [n_nuc]
    b_en: float = 1.0
    # optional multi-determinant expansion (bit strings over orbital index)
    det_up: Optional[np.ndarray] = None  # [n_det, n_words] uint64
    det_dn: Optional[np.ndarray] = None
    ci: Optional[np.ndarray] = None      # [n_det] float64
    # optional three-body (e-e-n) Jastrow: exponents [n3, 3] (m, n, o),
    # coefficients [n_nuc, n3], scale b3 of s(r) = r / (1 + b3 r)
    j3_exponents: Optional[np.ndarray] = None
    j3_coef: Optional[np.ndarray] = None
    j3_b: float = 1.0
    # optional semi-local pseudopotential: radial terms beta r^(n-2)
    # exp(-alpha r^2) of nucleus pp_nuc in channel pp_l (-1: local, added to
    # -Z/r; l >= 0: projector on angular momentum l about the nucleus), the
    # non-local cutoff radius per nucleus, and the quadrature rule (unit
    # vectors and weights summing to 1) of the non-local matrix elements
    pp_nuc: Optional[np.ndarray] = None    # [n_pp] int32
    pp_l: Optional[np.ndarray] = None      # [n_pp] int32
    pp_n: Optional[np.ndarray] = None      # [n_pp] int32
    pp_alpha: Optional[np.ndarray] = None  # [n_pp] float64
    pp_beta: Optional[np.ndarray] = None   # [n_pp] float64
    pp_rcut: Optional[np.ndarray] = None   # [n_nuc] float64
    pp_quad: Optional[np.ndarray] = None   # [n_q, 3] float64
    pp_qw: Optional[np.ndarray] = None     # [n_q] float64

    @property
    def n_nuc(self) -> int:
        return int(self.Z.shape[0])

    @property
    def n_elec(self) -> int:
        return self.n_up + self.n_dn

    @property
    def n_shell(self) -> int:
        return int(self.shell_l.shape[0])

    @property
    def n_basis(self) -> int:
        return int(sum(shell_size(int(l), int(p)) for l, p in zip(self.shell_l, self.shell_pure)))

    @property
    def n_mo(self) -> int:
        return int(self.C.shape[0])

    @property
    def n_det(self) -> int:
        return 0 if self.ci is None else int(self.ci.shape[0])

    @property
    def n_pp(self) -> int:
        return 0 if self.pp_nuc is None else int(self.pp_nuc.shape[0])

    def copy(self) -> "System":
        kw = {}
        for f in dataclasses.fields(self):
            v = getattr(self, f.name)
            kw[f.name] = v.copy() if isinstance(v, np.ndarray) else v
        return System(**kw)


def shell_size(l: int, pure: int) -> int:
    """Number of functions in a shell of angular momentum l."""
    if l == 0:
        return 1
    if l == 1:
        return 3
    if l == 2:
        return 5 if pure else 6
    raise ValueError("only s, p and d shells are supported")


# --------------------------------------------------------------------------
# geometry
# --------------------------------------------------------------------------

def water_monomer_angstrom() -> np.ndarray:
    """O, H, H positions in angstrom; molecule in the xz-plane."""
    d = 0.9572
    half = math.radians(104.52) / 2.0
    return np.array([[0.0, 0.0, 0.0],
                     [d * math.sin(half), 0.0, d * math.cos(half)],
                     [-d * math.sin(half), 0.0, d * math.cos(half)]])


def random_rotation(rng: np.random.Generator) -> np.ndarray:
    """Uniform random rotation matrix from a Shoemake (1992) quaternion."""
    u1, u2, u3 = rng.random(3)
    a = math.sqrt(1.0 - u1)
    b = math.sqrt(u1)
    q0 = a * math.sin(2 * math.pi * u2)
    q1 = a * math.cos(2 * math.pi * u2)
    q2 = b * math.sin(2 * math.pi * u3)
    q3 = b * math.cos(2 * math.pi * u3)
    w, x, y, z = q3, q0, q1, q2
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)],
    ])


def water_cluster_angstrom(m: int, seed: int = SEED_GEOMETRY) -> np.ndarray:
    """[3m, 3] positions (angstrom) of m rigid waters, O first in each triple."""
    mono = water_monomer_angstrom()
    if m == 1:
        return mono.copy()
    rng = np.random.default_rng(seed)
    side = 3.1 * m ** (1.0 / 3.0)
    placed: List[np.ndarray] = []
    fails = 0
    while len(placed) < m:
        rot = random_rotation(rng)
        origin = rng.random(3) * side
        mol = mono @ rot.T + origin
        ok = True
        for other in placed:
            if np.linalg.norm(other[0] - mol[0]) < 2.6:
                ok = False
                break
            dmin = np.min(np.linalg.norm(other[:, None, :] - mol[None, :, :], axis=-1))
            if dmin < 1.5:
                ok = False
                break
        if ok:
            placed.append(mol)
            fails = 0
        else:
            fails += 1
            if fails >= 10_000:
                side *= 1.05
                fails = 0
    return np.concatenate(placed, axis=0)


# --------------------------------------------------------------------------
# basis, orbitals, Jastrow
# --------------------------------------------------------------------------

SPECIES_SHELLS = {8: [(0, 0), (0, 0), (0, 0), (1, 0), (1, 0), (2, 1)],   # O 3s2p1d
                  1: [(0, 0), (0, 0), (1, 0)]}                           # H 2s1p


def species_basis(seed: int = SEED_BASIS, nprim: int = 3):
    """Per-species shells: {Z: [(l, pure, alphas[nprim], coefs[nprim]), ...]}."""
    rng = np.random.default_rng(seed)
    out = {}
    for zz in (8, 1):
        shells = []
        for (l, pure) in SPECIES_SHELLS[zz]:
            alphas = np.sort(10.0 ** rng.uniform(-1.0, 4.0, size=nprim))[::-1].copy()
            coefs = rng.uniform(0.1, 1.0, size=nprim)
            shells.append((l, pure, alphas, coefs))
        out[zz] = shells
    return out


def orbital_matrix(n_basis: int, seed: int = SEED_MO) -> np.ndarray:
    """[n_mo = n_basis, n_basis] coefficients: row j = Q[:, j] of a seeded QR."""
    rng = np.random.default_rng(seed)
    M = rng.standard_normal((n_basis, n_basis))
    Q, Rm = np.linalg.qr(M)
    s = np.sign(np.diag(Rm))
    s[s == 0] = 1.0
    Q = Q * s[None, :]
    return np.ascontiguousarray(Q.T)


def molecule(Z: Sequence[float], R_bohr: np.ndarray, basis_seed: int = SEED_BASIS,
             mo_seed: int = SEED_MO) -> System:
    """Water-like molecule with the per-species basis and QR orbitals."""
    Z = np.asarray(Z, dtype=np.float64)
    sb = species_basis(basis_seed)
    sc, sl, sp, sn, al, co = [], [], [], [], [], []
    for a, zz in enumerate(Z):
        for (l, pure, alphas, coefs) in sb[int(zz)]:
            sc.append(a); sl.append(l); sp.append(pure); sn.append(len(alphas))
            al.extend(alphas); co.extend(coefs)
    n_el = int(round(Z.sum()))
    n_up = (n_el + 1) // 2
    n_dn = n_el - n_up
    nb = int(sum(shell_size(l, p) for l, p in zip(sl, sp)))
    C = orbital_matrix(nb, mo_seed)
    return System(Z=Z, R=np.ascontiguousarray(R_bohr, dtype=np.float64), n_up=n_up, n_dn=n_dn,
                  shell_center=np.array(sc, np.int32), shell_l=np.array(sl, np.int32),
                  shell_pure=np.array(sp, np.int32), shell_nprim=np.array(sn, np.int32),
                  alpha=np.array(al, np.float64), coef=np.array(co, np.float64), C=C,
                  occ_up=np.arange(n_up, dtype=np.int32), occ_dn=np.arange(n_dn, dtype=np.int32),
                  a_anti=0.5, a_par=0.25, b_ee=1.0, a_en=-Z.copy(), b_en=1.0)


def water_system(m: int, geom_seed: int = SEED_GEOMETRY) -> System:
    """m-water cluster (m = 1 is the monomer at the origin)."""
    R = water_cluster_angstrom(m, geom_seed) * BOHR_PER_ANGSTROM
    Z = np.tile(np.array([8.0, 1.0, 1.0]), m)
    return molecule(Z, R)


def hydrogenic_exact(Zc: float = 1.0) -> System:
    """psi = exp(-Z r): a constant (alpha = 0) s orbital times an e-n Jastrow
    with a = -Z, b = 0.  Its local energy is -Z^2/2 everywhere."""
    return System(Z=np.array([Zc]), R=np.zeros((1, 3)), n_up=1, n_dn=0,
                  shell_center=np.array([0], np.int32), shell_l=np.array([0], np.int32),
                  shell_pure=np.array([0], np.int32), shell_nprim=np.array([1], np.int32),
                  alpha=np.array([0.0]), coef=np.array([1.0]), C=np.array([[1.0]]),
                  occ_up=np.array([0], np.int32), occ_dn=np.zeros(0, np.int32),
                  a_anti=0.0, a_par=0.0, b_ee=0.0, a_en=np.array([-Zc]), b_en=0.0)


def helium_nodeless(b_en: float = 0.4, b_ee: float = 0.5) -> System:
    """He: one constant orbital per spin times a Pade Jastrow with both cusps
    (a_en = -2, a_anti = 1/2).  Nodeless, not exact: DMC must reach the
    He ground state."""
    return System(Z=np.array([2.0]), R=np.zeros((1, 3)), n_up=1, n_dn=1,
                  shell_center=np.array([0], np.int32), shell_l=np.array([0], np.int32),
                  shell_pure=np.array([0], np.int32), shell_nprim=np.array([1], np.int32),
                  alpha=np.array([0.0]), coef=np.array([1.0]), C=np.array([[1.0]]),
                  occ_up=np.array([0], np.int32), occ_dn=np.array([0], np.int32),
                  a_anti=0.5, a_par=0.25, b_ee=b_ee, a_en=np.array([-2.0]), b_en=b_en)


def single_gaussian_atom(alpha: float, Zc: float = 1.0, n_up: int = 1, n_dn: int = 0) -> System:
    """One s primitive exp(-alpha r^2) per electron, no Jastrow."""
    return System(Z=np.array([Zc]), R=np.zeros((1, 3)), n_up=n_up, n_dn=n_dn,
                  shell_center=np.array([0], np.int32), shell_l=np.array([0], np.int32),
                  shell_pure=np.array([0], np.int32), shell_nprim=np.array([1], np.int32),
                  alpha=np.array([alpha]), coef=np.array([1.0]), C=np.array([[1.0]]),
                  occ_up=np.zeros(n_up, np.int32), occ_dn=np.zeros(n_dn, np.int32),
                  a_anti=0.0, a_par=0.0, b_ee=0.0, a_en=np.zeros(1), b_en=0.0)


def random_small_system(rng: np.random.Generator, n_nuc: int = 2, n_up: int = 2, n_dn: int = 2,
                        lmax: int = 2, with_cart_d: bool = True) -> System:
    """Small seeded system with every shell type, for unit tests."""
    Z = rng.integers(1, 4, size=n_nuc).astype(np.float64)
    R = rng.normal(0.0, 1.2, size=(n_nuc, 3))
    kinds = [(0, 0), (1, 0), (2, 1)] + ([(2, 0)] if with_cart_d else [])
    kinds = [k for k in kinds if k[0] <= lmax]
    sc, sl, sp, sn, al, co = [], [], [], [], [], []
    for a in range(n_nuc):
        for (l, pure) in kinds:
            npr = int(rng.integers(1, 4))
            sc.append(a); sl.append(l); sp.append(pure); sn.append(npr)
            al.extend(np.sort(10.0 ** rng.uniform(-0.7, 0.7, size=npr))[::-1])
            co.extend(rng.uniform(0.1, 1.0, size=npr))
    nb = int(sum(shell_size(l, p) for l, p in zip(sl, sp)))
    C = orbital_matrix(nb, int(rng.integers(1 << 30)))
    return System(Z=Z, R=R, n_up=n_up, n_dn=n_dn,
                  shell_center=np.array(sc, np.int32), shell_l=np.array(sl, np.int32),
                  shell_pure=np.array(sp, np.int32), shell_nprim=np.array(sn, np.int32),
                  alpha=np.array(al, np.float64), coef=np.array(co, np.float64), C=C,
                  occ_up=np.arange(n_up, dtype=np.int32), occ_dn=np.arange(n_dn, dtype=np.int32),
                  a_anti=0.5, a_par=0.25, b_ee=float(rng.uniform(0.5, 1.5)),
                  a_en=-Z.copy(), b_en=float(rng.uniform(0.5, 1.5)))


# --------------------------------------------------------------------------
# walkers
# --------------------------------------------------------------------------

def initial_walkers(sys: System, n_walkers: int, seed: int = SEED_WALKERS,
                    sigma: float = 0.5) -> np.ndarray:
    """[W, N, 3] float64 electron positions, up-spin electrons first."""
    rng = np.random.default_rng(seed)
    owners = []
    for a, zz in enumerate(sys.Z):
        owners.extend([a] * int(round(zz)))
    N = sys.n_elec
    if len(owners) < N:   # ions: extra electrons go to the first nucleus
        owners.extend([0] * (N - len(owners)))
    owners = owners[:N]
    up = [k for k in range(N) if k % 2 == 0][: sys.n_up]
    dn = [k for k in range(N) if k % 2 == 1][: sys.n_dn]
    if len(up) < sys.n_up or len(dn) < sys.n_dn:
        order = list(range(N))
        up, dn = order[: sys.n_up], order[sys.n_up:]
    centers = sys.R[np.array([owners[k] for k in up + dn], dtype=np.int64)]
    return centers[None, :, :] + rng.normal(0.0, sigma, size=(n_walkers, N, 3))


# --------------------------------------------------------------------------
# multi-determinant expansion
# --------------------------------------------------------------------------

def _bits(orbs: Sequence[int], n_words: int) -> np.ndarray:
    w = np.zeros(n_words, dtype=np.uint64)
    for o in orbs:
        w[o // 64] |= np.uint64(1) << np.uint64(o % 64)
    return w


def multidet_expansion(n_occ: int, n_active: int, n_det: int, max_exc: int = 4,
                       seed: int = SEED_CI):
    """Reference determinant plus n_det-1 distinct excited determinants.

    Holes are any of the n_occ occupied orbitals of a spin, particles any of
    the n_active lowest virtuals; the degrees (e_up, e_dn) satisfy
    e_up + e_dn <= max_exc.  The full space is far too large to enumerate,
    so determinants are drawn uniformly from it (degree pair with probability
    proportional to its count, then uniform hole/particle sets) without
    replacement.  CI weights are +-exp(-0.5 k) with random signs (k = rank),
    c_0 > 0, normalised to unit 2-norm.

    Returns (det_up, det_dn, ci) with bit strings over orbital indices.
    """
    rng = np.random.default_rng(seed)
    n_orb = n_occ + n_active
    n_words = (n_orb + 63) // 64
    pairs, weights = [], []
    for eu in range(max_exc + 1):
        for ed in range(max_exc + 1 - eu):
            cnt = (math.comb(n_occ, eu) * math.comb(n_active, eu)
                   * math.comb(n_occ, ed) * math.comb(n_active, ed))
            if eu + ed > 0 and cnt > 0:
                pairs.append((eu, ed)); weights.append(float(cnt))
    weights = np.array(weights) / np.sum(weights)
    total = int(sum(math.comb(n_occ, eu) * math.comb(n_active, eu) * math.comb(n_occ, ed)
                    * math.comb(n_active, ed) for eu, ed in pairs))
    if n_det - 1 > total:
        raise ValueError("requested more determinants than the excitation space holds")
    ref = tuple(range(n_occ))
    seen = {(ref, ref)}
    dets = [(ref, ref)]

    def excite(e):
        holes = set(rng.choice(n_occ, size=e, replace=False).tolist()) if e else set()
        parts = (rng.choice(n_active, size=e, replace=False) + n_occ).tolist() if e else []
        return tuple(sorted([o for o in range(n_occ) if o not in holes] + parts))

    while len(dets) < n_det:
        eu, ed = pairs[int(rng.choice(len(pairs), p=weights))]
        d = (excite(eu), excite(ed))
        if d not in seen:
            seen.add(d)
            dets.append(d)
    det_up = np.stack([_bits(u, n_words) for u, _ in dets])
    det_dn = np.stack([_bits(d, n_words) for _, d in dets])
    k = np.arange(n_det, dtype=np.float64)
    signs = rng.choice([-1.0, 1.0], size=n_det)
    signs[0] = 1.0
    ci = signs * np.exp(-0.5 * k)
    ci /= np.linalg.norm(ci)
    return det_up, det_dn, ci


def with_multidet(sys: System, n_det: int, n_active: int = 20, max_exc: int = 4,
                  seed: int = SEED_CI) -> System:
    assert sys.n_up == sys.n_dn, "expansion assumes a closed-shell reference"
    s = sys.copy()
    s.det_up, s.det_dn, s.ci = multidet_expansion(sys.n_up, n_active, n_det, max_exc, seed)
    return s


# --------------------------------------------------------------------------
# workloads
# --------------------------------------------------------------------------

# exponents (m, n, o) of the three-body terms: every power 0 or >= 2, so
# that neither the electron-electron nor the electron-nucleus cusp changes
THREE_BODY_TERMS = ((2, 2, 0), (2, 0, 2), (2, 2, 2), (3, 0, 2))


def with_three_body(sys: System, seed: int = SEED_MO + 7, scale: float = 0.05, b3: float = 1.0,
                    terms: Sequence[Sequence[int]] = THREE_BODY_TERMS) -> System:
    """A copy of `sys` with an electron-electron-nucleus Jastrow: the given
    exponent triples and coefficients drawn from N(0, scale^2) per nucleus
    and term (seeded)."""
    out = sys.copy()
    rng = np.random.default_rng(seed)
    out.j3_exponents = np.array(terms, dtype=np.int32).reshape(-1, 3)
    out.j3_coef = rng.normal(0.0, scale, size=(sys.n_nuc, out.j3_exponents.shape[0]))
    out.j3_b = float(b3)
    return out


# --------------------------------------------------------------------------
# semi-local pseudopotentials
# --------------------------------------------------------------------------
# The paper's production Hamiltonian replaces core electrons by ccECP
# pseudopotentials (Sec. "The SPICE2(+)-ccECP dataset"); their tables are not
# available here, so a synthetic potential of the same semi-local Gaussian
# form stands in: per species the core electrons it removes, and radial
# terms (channel l, power n, exponent alpha, coefficient beta) of
# beta r^(n-2) exp(-alpha r^2).  The local terms (l = -1) cancel the -Z_eff/r
# singularity at the nucleus (n = 1 with beta = Z_eff) and add a smooth
# well; the non-local channels are an s and a p projector.  The cutoff
# radius is where every non-local term is below 1e-10 Ha.
PP_SPECIES = {
    8: dict(core=2, rcut=1.6,
            terms=((-1, 1, 9.0, 6.0), (-1, 3, 8.0, 54.0), (-1, 2, 7.5, -30.0),
                   (0, 2, 12.0, 50.0), (1, 2, 10.0, -6.0))),
}


def icosahedron_rule():
    """The 12 vertices of a regular icosahedron (cyclic permutations of
    (0, +-1, +-golden ratio), normalised) with equal weights 1/12: a rule
    that integrates every spherical harmonic of degree <= 5 exactly."""
    g = (1.0 + math.sqrt(5.0)) / 2.0
    pts = []
    for a in (-1.0, 1.0):
        for b in (-g, g):
            pts += [(0.0, a, b), (a, b, 0.0), (b, 0.0, a)]
    P = np.array(pts, dtype=np.float64)
    P /= np.linalg.norm(P, axis=1, keepdims=True)
    return P, np.full(P.shape[0], 1.0 / P.shape[0])


def with_pseudopotential(sys: System, species=None, rule=None) -> System:
    """A valence-only copy of `sys`: every nucleus of a species in `species`
    (default PP_SPECIES) loses its core electrons from its charge and one
    electron per spin per core pair, carries that species' radial terms,
    and has no electron-nucleus Jastrow cusp (the potential is finite at the
    nucleus).  rule = (points [n_q, 3], weights [n_q]); default the
    icosahedral rule."""
    species = PP_SPECIES if species is None else species
    pts, wts = icosahedron_rule() if rule is None else rule
    out = sys.copy()
    Z = out.Z.copy()
    a_en = (out.a_en if out.a_en is not None else -out.Z).copy()
    rcut = np.zeros(out.n_nuc)
    nuc, ll, nn, al, be = [], [], [], [], []
    core = 0
    for a, z in enumerate(sys.Z):
        sp = species.get(int(round(z)))
        if sp is None:
            continue
        Z[a] = z - sp["core"]
        core += sp["core"]
        a_en[a] = 0.0
        rcut[a] = sp["rcut"]
        for (l, n, alpha, beta) in sp["terms"]:
            nuc.append(a); ll.append(l); nn.append(n); al.append(alpha); be.append(beta)
    assert core % 2 == 0 and core // 2 <= min(sys.n_up, sys.n_dn)
    out.Z = Z
    out.a_en = a_en
    out.n_up = sys.n_up - core // 2
    out.n_dn = sys.n_dn - core // 2
    out.occ_up = np.arange(out.n_up, dtype=np.int32)
    out.occ_dn = np.arange(out.n_dn, dtype=np.int32)
    out.pp_nuc = np.array(nuc, np.int32)
    out.pp_l = np.array(ll, np.int32)
    out.pp_n = np.array(nn, np.int32)
    out.pp_alpha = np.array(al, np.float64)
    out.pp_beta = np.array(be, np.float64)
    out.pp_rcut = rcut
    out.pp_quad = np.ascontiguousarray(pts, dtype=np.float64)
    out.pp_qw = np.ascontiguousarray(wts, dtype=np.float64)
    return out


@dataclasses.dataclass
class Workload:
    name: str
    n_water: int
    n_walkers: int
    precision: str          # "fp64" | "mixed"
    forces: bool
    vmc_sweeps: int
    dmc_steps: int
    tau: float
    n_det: int = 0
    delay_rank: int = 1
    recompute_period: int = 100
    pseudopotential: bool = False


WORKLOADS = {
    "water1_fp64": Workload("water1_fp64", 1, 512, "fp64", False, 200, 500, 0.005),
    "water6_fp64_forces": Workload("water6_fp64_forces", 6, 2048, "fp64", True, 20, 50, 0.005),
    "water32_mixed": Workload("water32_mixed", 32, 4096, "mixed", True, 20, 50, 0.005,
                              delay_rank=32, recompute_period=100),
    "water6_msd10k": Workload("water6_msd10k", 6, 2048, "mixed", True, 20, 50, 0.005, n_det=10_000),
    # the 32-water cluster in FP64 with forces (the large-determinant FP64
    # force path: batched DGEMMs between the preparation and contraction)
    "water32_fp64_forces": Workload("water32_fp64_forces", 32, 256, "fp64", True, 20, 50, 0.005),
    # valence-only 32-water cluster with the synthetic semi-local potential
    # on every O (8 electrons per water, 128 per spin)
    "water32_pp_mixed": Workload("water32_pp_mixed", 32, 4096, "mixed", False, 20, 50, 0.005,
                                 delay_rank=32, recompute_period=100, pseudopotential=True),
    # the same potential on the 6-water cluster (24 electrons per spin), forces every step
    "water6_pp_forces": Workload("water6_pp_forces", 6, 2048, "mixed", True, 20, 50, 0.005,
                                 pseudopotential=True),
}


def uneven_cluster_sizes(n_systems: int = 64, lo: int = 1, hi: int = 16,
                         seed: int = SEED_CLUSTER_SIZES) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.integers(lo, hi + 1, size=n_systems)
