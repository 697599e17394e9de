"""ctypes wrapper of the CPU FP64 oracle (``qmc_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by the tests, the smoke check and the
benchmark's CPU-baseline leg.  The product path (the CUDA library and its
binding) never imports this module.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from typing import Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "qmc_oracle.c")
LIB = os.path.join(HERE, "_build", "liboracle.so")

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with the host gcc (portable flags only)."""
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < max(
            os.path.getmtime(SRC), os.path.getmtime(os.path.join(HERE, "qmc_oracle.h"))):
        tmp = LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fno-fast-math",
                               "-ffp-contract=off", "-o", tmp, SRC, "-lm", "-lpthread"])
        os.replace(tmp, LIB)
    return LIB


class OSystem(C.Structure):
    _fields_ = [
        ("n_nuc", C.c_int), ("Z", C.c_void_p), ("R", C.c_void_p),
        ("n_up", C.c_int), ("n_dn", C.c_int),
        ("n_shell", C.c_int), ("sh_center", C.c_void_p), ("sh_l", C.c_void_p),
        ("sh_pure", C.c_void_p), ("sh_nprim", C.c_void_p),
        ("alpha", C.c_void_p), ("coef", C.c_void_p),
        ("n_mo", C.c_int), ("n_basis", C.c_int), ("C", C.c_void_p),
        ("occ_up", C.c_void_p), ("occ_dn", C.c_void_p),
        ("a_anti", C.c_double), ("a_par", C.c_double), ("b_ee", C.c_double),
        ("a_en", C.c_void_p), ("b_en", C.c_double),
        ("n_det", C.c_int), ("n_words", C.c_int),
        ("det_up", C.c_void_p), ("det_dn", C.c_void_p), ("ci", C.c_void_p),
        ("n3", C.c_int), ("e3", C.c_void_p), ("c3", C.c_void_p), ("b3", C.c_double),
        ("n_pp", C.c_int), ("pp_nuc", C.c_void_p), ("pp_l", C.c_void_p), ("pp_n", C.c_void_p),
        ("pp_alpha", C.c_void_p), ("pp_beta", C.c_void_p), ("pp_rcut", C.c_void_p),
        ("pp_nq", C.c_int), ("pp_quad", C.c_void_p), ("pp_qw", C.c_void_p),
        ("pp_rotate", C.c_int), ("pp_seed", C.c_uint64), ("pp_sweep", C.c_uint32), ("pp_slot0", C.c_uint32),
    ]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(LIB)
            vp, i, d = C.c_void_p, C.c_int, C.c_double
            L.oracle_n_basis.argtypes = [vp]
            L.oracle_basis.argtypes = [vp, vp, vp]
            L.oracle_lu_det.argtypes = [i, vp, vp, vp, vp]
            L.oracle_evaluate.argtypes = [vp, i, vp, vp, vp, vp, vp, vp, i]
            L.oracle_forces.argtypes = [vp, i, vp, vp, vp, i]
            L.oracle_electron_grad.argtypes = [vp, i, vp, vp, vp, i]
            L.oracle_warp_weights.argtypes = [vp, vp, vp, vp]
            L.oracle_warp_weights.restype = None
            L.oracle_space_warp.argtypes = [vp, i, vp, vp, vp, vp, vp, vp, vp]
            L.oracle_jastrow_derivs.argtypes = [vp, i, vp, vp, vp, i]
            L.oracle_nonlocal.argtypes = [vp, i, vp, vp, i]
            L.oracle_pp_rotation.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32, vp]
            L.oracle_pp_rotation.restype = None
            L.oracle_philox4x32.argtypes = [vp, vp, vp]
            L.oracle_philox4x32.restype = None
            L.oracle_vmc.argtypes = [vp, i, vp, i, d, C.c_uint64, C.c_uint32, vp, vp, i]
            L.oracle_dmc.argtypes = [vp, vp, i, vp, i, d, d, C.c_uint64, C.c_uint32, i, i,
                                     vp, vp, vp, vp, i, i]
            _lib = L
    return _lib


def _p(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data


class Oracle:
    """Holds a system's arrays (kept alive) and its C description."""

    def __init__(self, sys, nthreads: int = 0, pp_rotate: bool = True):
        self.sys = sys
        self.nthreads = nthreads or (os.cpu_count() or 1)
        f64 = lambda a: np.ascontiguousarray(a, dtype=np.float64)
        i32 = lambda a: np.ascontiguousarray(a, dtype=np.int32)
        self._keep = dict(
            Z=f64(sys.Z), R=f64(sys.R), sc=i32(sys.shell_center), sl=i32(sys.shell_l),
            sp=i32(sys.shell_pure), sn=i32(sys.shell_nprim), al=f64(sys.alpha), co=f64(sys.coef),
            C=f64(sys.C), ou=i32(sys.occ_up), od=i32(sys.occ_dn),
            aen=f64(sys.a_en if sys.a_en is not None else np.zeros(sys.n_nuc)))
        k = self._keep
        s = OSystem()
        s.n_nuc = sys.n_nuc; s.Z = _p(k["Z"]); s.R = _p(k["R"])
        s.n_up = sys.n_up; s.n_dn = sys.n_dn
        s.n_shell = sys.n_shell; s.sh_center = _p(k["sc"]); s.sh_l = _p(k["sl"])
        s.sh_pure = _p(k["sp"]); s.sh_nprim = _p(k["sn"]); s.alpha = _p(k["al"]); s.coef = _p(k["co"])
        s.n_mo = sys.C.shape[0]; s.n_basis = sys.C.shape[1]; s.C = _p(k["C"])
        s.occ_up = _p(k["ou"]); s.occ_dn = _p(k["od"])
        s.a_anti = sys.a_anti; s.a_par = sys.a_par; s.b_ee = sys.b_ee
        s.a_en = _p(k["aen"]); s.b_en = sys.b_en
        if sys.ci is not None:
            k["du"] = np.ascontiguousarray(sys.det_up, dtype=np.uint64)
            k["dd"] = np.ascontiguousarray(sys.det_dn, dtype=np.uint64)
            k["ci"] = f64(sys.ci)
            s.n_det = k["ci"].shape[0]; s.n_words = k["du"].shape[1]
            s.det_up = _p(k["du"]); s.det_dn = _p(k["dd"]); s.ci = _p(k["ci"])
        else:
            s.n_det = 0; s.n_words = 0
        e3 = getattr(sys, "j3_exponents", None)
        if e3 is not None and len(e3) > 0:
            k["e3"] = np.ascontiguousarray(e3, dtype=np.int32)
            k["c3"] = f64(sys.j3_coef)
            s.n3 = k["e3"].shape[0]; s.e3 = _p(k["e3"]); s.c3 = _p(k["c3"]); s.b3 = float(sys.j3_b)
        else:
            s.n3 = 0; s.b3 = 1.0
        if getattr(sys, "pp_nuc", None) is not None and len(sys.pp_nuc) > 0:
            k["ppn"] = i32(sys.pp_nuc); k["ppl"] = i32(sys.pp_l); k["ppp"] = i32(sys.pp_n)
            k["ppa"] = f64(sys.pp_alpha); k["ppb"] = f64(sys.pp_beta); k["ppr"] = f64(sys.pp_rcut)
            k["ppq"] = f64(sys.pp_quad); k["ppw"] = f64(sys.pp_qw)
            s.n_pp = k["ppn"].shape[0]
            s.pp_nuc = _p(k["ppn"]); s.pp_l = _p(k["ppl"]); s.pp_n = _p(k["ppp"])
            s.pp_alpha = _p(k["ppa"]); s.pp_beta = _p(k["ppb"]); s.pp_rcut = _p(k["ppr"])
            s.pp_nq = k["ppw"].shape[0]; s.pp_quad = _p(k["ppq"]); s.pp_qw = _p(k["ppw"])
            s.pp_rotate = int(bool(pp_rotate))
        else:
            s.n_pp = 0; s.pp_nq = 0; s.pp_rotate = 0
        self.cs = s
        self.ptr = C.addressof(s)
        assert lib().oracle_n_basis(self.ptr) == sys.C.shape[1], "C columns must match the basis size"

    # -- basis --------------------------------------------------------
    def basis(self, r) -> np.ndarray:
        """[n_basis, 20] derivatives of total order <= 3 at r."""
        r = np.ascontiguousarray(r, dtype=np.float64)
        out = np.zeros((self.sys.n_basis, 20))
        lib().oracle_basis(self.ptr, _p(r), _p(out))
        return out

    # -- fixed configurations -----------------------------------------
    def evaluate(self, R: np.ndarray, nthreads: int = 0, pp_seed: int = 0, pp_sweep: int = 0, pp_slot0: int = 0):
        """dict(logpsi, sign, eloc, grad [W,N,3], lap [W,N]) at R [W,N,3].
        With a pseudopotential, walker w's quadrature rotations come from
        Philox key pp_seed, counter (pp_sweep, nucleus, pp_slot0 + w, 3)."""
        self.cs.pp_seed = int(pp_seed); self.cs.pp_sweep = int(pp_sweep); self.cs.pp_slot0 = int(pp_slot0)
        R = np.ascontiguousarray(R, dtype=np.float64)
        W, N = R.shape[0], R.shape[1]
        out = dict(logpsi=np.zeros(W), sign=np.zeros(W), eloc=np.zeros(W),
                   grad=np.zeros((W, N, 3)), lap=np.zeros((W, N)))
        lib().oracle_evaluate(self.ptr, W, _p(R), _p(out["logpsi"]), _p(out["sign"]), _p(out["eloc"]),
                              _p(out["grad"]), _p(out["lap"]), nthreads or self.nthreads)
        return out

    def nonlocal_energy(self, R: np.ndarray, nthreads: int = 0, pp_seed: int = 0, pp_sweep: int = 0,
                        pp_slot0: int = 0):
        """[W] non-local pseudopotential energy (locality approximation) at
        R [W,N,3], rotations as in evaluate()."""
        self.cs.pp_seed = int(pp_seed); self.cs.pp_sweep = int(pp_sweep); self.cs.pp_slot0 = int(pp_slot0)
        R = np.ascontiguousarray(R, dtype=np.float64)
        out = np.zeros(R.shape[0])
        lib().oracle_nonlocal(self.ptr, R.shape[0], _p(R), _p(out), nthreads or self.nthreads)
        return out

    def forces(self, R: np.ndarray, nthreads: int = 0, pp_seed: int = 0, pp_sweep: int = 0, pp_slot0: int = 0):
        """(dEL [W,n_nuc,3], dlogpsi [W,n_nuc,3]) by forward mode (pseudopotential
        rotations as in evaluate())."""
        self.cs.pp_seed = int(pp_seed); self.cs.pp_sweep = int(pp_sweep); self.cs.pp_slot0 = int(pp_slot0)
        R = np.ascontiguousarray(R, dtype=np.float64)
        W = R.shape[0]
        dEL = np.zeros((W, self.sys.n_nuc, 3))
        dlg = np.zeros((W, self.sys.n_nuc, 3))
        if lib().oracle_forces(self.ptr, W, _p(R), _p(dEL), _p(dlg), nthreads or self.nthreads) != 0:
            raise ValueError("the oracle has no ionic derivatives of the three-body Jastrow")
        return dEL, dlg

    def jastrow_derivs(self, R: np.ndarray, nthreads: int = 0, pp_seed: int = 0, pp_sweep: int = 0, pp_slot0: int = 0):
        """(dlog [W,P], deloc [W,P]): d ln|psi| / dp and dE_L / dp for the
        Jastrow parameters (a_anti, a_par, b_ee, b_en, a_en[n_nuc],
        c3[n_nuc][n3])."""
        self.cs.pp_seed = int(pp_seed); self.cs.pp_sweep = int(pp_sweep); self.cs.pp_slot0 = int(pp_slot0)
        R = np.ascontiguousarray(R, dtype=np.float64)
        W = R.shape[0]
        P = 4 + self.sys.n_nuc + self.sys.n_nuc * int(self.cs.n3)
        dlog = np.zeros((W, P))
        deloc = np.zeros((W, P))
        lib().oracle_jastrow_derivs(self.ptr, W, _p(R), _p(dlog), _p(deloc), nthreads or self.nthreads)
        return dlog, deloc

    def electron_grad(self, R: np.ndarray, nthreads: int = 0):
        """(dE_L/dr_i [W,N,3], dln|psi|/dr_i [W,N,3]) by forward mode over the
        electron coordinates."""
        R = np.ascontiguousarray(R, dtype=np.float64)
        W, N = R.shape[0], R.shape[1]
        gEL = np.zeros((W, N, 3))
        glg = np.zeros((W, N, 3))
        lib().oracle_electron_grad(self.ptr, W, _p(R), _p(gEL), _p(glg), nthreads or self.nthreads)
        return gEL, glg

    def warp_weights(self, r):
        """(omega_a(r) [n_nuc], grad omega_a(r) [n_nuc,3]): space-warp weights
        of Filippi and Umrigar (2000) with F(d) = d^-4."""
        r = np.ascontiguousarray(r, dtype=np.float64)
        om = np.zeros(self.sys.n_nuc)
        gom = np.zeros((self.sys.n_nuc, 3))
        lib().oracle_warp_weights(self.ptr, _p(r), _p(om), _p(gom))
        return om, gom

    def warped_forces(self, R: np.ndarray, nthreads: int = 0):
        """Space-warped (dEL [W,n_nuc,3], dlogpsi [W,n_nuc,3]): the nuclear
        derivatives with every electron carried along by the warp weights,
        the log-derivative including half the Jacobian of that map."""
        R = np.ascontiguousarray(R, dtype=np.float64)
        W = R.shape[0]
        dEL, dlg = self.forces(R, nthreads)
        gEL, glg = self.electron_grad(R, nthreads)
        dELw = np.zeros_like(dEL)
        dlgw = np.zeros_like(dlg)
        lib().oracle_space_warp(self.ptr, W, _p(R), _p(dEL), _p(dlg), _p(gEL), _p(glg), _p(dELw), _p(dlgw))
        return dELw, dlgw

    # -- sampling ------------------------------------------------------
    def vmc(self, R: np.ndarray, n_sweeps: int, tau: float, seed: int, step0: int = 0,
            trace: bool = True, nthreads: int = 0):
        """Runs VMC in place on a copy; returns (R, n_accept[W], eloc_trace)."""
        R = np.array(R, dtype=np.float64, order="C", copy=True)
        W = R.shape[0]
        acc = np.zeros(W, dtype=np.int64)
        tr = np.zeros((n_sweeps, W)) if trace else None
        lib().oracle_vmc(self.ptr, W, _p(R), n_sweeps, tau, seed, step0, _p(acc), _p(tr),
                         nthreads or self.nthreads)
        return R, acc, tr

    def dmc(self, R: np.ndarray, n_steps: int, tau: float, e_trial: float, seed: int, step0: int = 0,
            cap_factor: int = 4, n_equil: int = 0, forces_every: int = 0, nthreads: int = 0,
            fixed_pop: bool = False):
        W0 = R.shape[0]
        N = R.shape[1]
        cap = cap_factor * W0
        Rb = np.zeros((cap, N, 3))
        Rb[:W0] = R
        Wio = np.array([W0], dtype=np.int32)
        e_step = np.zeros(n_steps)
        pop = np.zeros(n_steps, dtype=np.int32)
        e_tr = np.zeros(n_steps)
        nn = self.sys.n_nuc
        facc = np.zeros(2 + 9 * nn)
        st = lib().oracle_dmc(self.ptr, _p(Wio), cap, _p(Rb), n_steps, tau, e_trial, seed, step0,
                              n_equil, forces_every, _p(e_step), _p(pop), _p(e_tr), _p(facc),
                              nthreads or self.nthreads, int(bool(fixed_pop)))
        return dict(status=st, R=Rb[: int(Wio[0])].copy(), e_step=e_step, pop=pop, e_trial=e_tr,
                    facc=facc)


def lu_det(A: np.ndarray, inverse: bool = True):
    A = np.ascontiguousarray(A, dtype=np.float64)
    n = A.shape[0]
    la = np.zeros(1)
    sg = np.zeros(1)
    inv = np.zeros((n, n)) if inverse else None
    lib().oracle_lu_det(n, _p(A), _p(la), _p(sg), _p(inv))
    return float(la[0]), float(sg[0]), inv


def pp_rotation(seed: int, sweep: int, nucleus: int, slot: int) -> np.ndarray:
    """[3, 3] rotation of the quadrature rule for (slot, nucleus) at a sweep
    counter (Shoemake's quaternion from Philox counter (sweep, nucleus, slot, 3))."""
    out = np.zeros(9)
    lib().oracle_pp_rotation(int(seed), int(sweep), int(nucleus), int(slot), _p(out))
    return out.reshape(3, 3)


def philox4x32(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().oracle_philox4x32(_p(c), _p(k), _p(out))
    return out


def force_estimator(eloc: np.ndarray, dEL: np.ndarray, dlogpsi: np.ndarray,
                    weights: Optional[np.ndarray] = None) -> np.ndarray:
    """Zero-variance zero-bias force (Assaraf-Caffarel, via the formalism the
    paper follows, Sec. "Single Determinant QMC Forces"):
    F = -<dE_L/dR> - 2 (<E_L dln|psi|/dR> - <E_L><dln|psi|/dR>), with E_L
    including the nuclear repulsion so that its derivative carries the
    Hellmann-Feynman ion-ion term."""
    w = np.ones(eloc.shape[0]) if weights is None else weights
    sw = w.sum()
    m = lambda x: np.tensordot(w, x, axes=(0, 0)) / sw
    E = m(eloc)
    return -(m(dEL) + 2.0 * (m(eloc[:, None, None] * dlogpsi) - E * m(dlogpsi)))


def mixed_estimator(f_dmc: np.ndarray, f_vmc: np.ndarray) -> np.ndarray:
    """Mixed estimator F_mixed = 2 F_DMC - F_VMC (Sec. "Performance
    Measurement")."""
    return 2.0 * f_dmc - f_vmc


def force_sums(eloc: np.ndarray, dEL: np.ndarray, dlogpsi: np.ndarray,
               weights: Optional[np.ndarray] = None) -> np.ndarray:
    """Weighted sums a force estimate is built from, in the layout the
    oracle's DMC accumulates (``dmc(..., forces_every=...)["facc"]``):
    [sum w, sum w E_L, sum w dE_L/dR (3 n_nuc), sum w E_L dln|psi|/dR,
    sum w dln|psi|/dR]."""
    w = np.ones(eloc.shape[0]) if weights is None else np.asarray(weights, dtype=np.float64)
    K = dEL.shape[1] * dEL.shape[2]
    d = dEL.reshape(-1, K)
    g = dlogpsi.reshape(-1, K)
    return np.concatenate([[w.sum(), (w * eloc).sum()], w @ d, (w * eloc) @ g, w @ g])


def force_from_sums(tot: np.ndarray, n_nuc: int) -> np.ndarray:
    """The zero-variance zero-bias estimator of ``force_estimator`` from
    accumulated sums (``force_sums`` layout, possibly added over many steps):
    F = -(S_dE / S_w) - 2 (S_EdL / S_w - (S_E / S_w)(S_dL / S_w))."""
    K = 3 * n_nuc
    sw, E = tot[0], tot[1] / tot[0]
    dE, EdL, dL = tot[2:2 + K] / sw, tot[2 + K:2 + 2 * K] / sw, tot[2 + 2 * K:2 + 3 * K] / sw
    return (-(dE + 2.0 * (EdL - E * dL))).reshape(n_nuc, 3)
