"""Python binding of libqmc (``include/qmc.h``).

Argument marshalling only: every function below has the name of the C call it
wraps, converts numpy arrays / torch tensors to pointers and raises
``QmcError`` on a non-zero status.  All computation happens in the CUDA
library; there is no fallback.  ``QMC`` is a small convenience object over
the same calls.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional

import numpy as np

from .build import LIB

QMC_FP64, QMC_MIXED = 0, 1
QMC_EST_VMC, QMC_EST_DMC, QMC_EST_MIXED = 0, 1, 2
QMC_POP_BRANCH, QMC_POP_FIXED = 0, 1
STATUS = {0: "QMC_OK", -1: "QMC_ERR_ARG", -2: "QMC_ERR_CUDA", -3: "QMC_ERR_SINGULAR", -4: "QMC_ERR_NONFINITE",
          -5: "QMC_ERR_POPULATION", -6: "QMC_ERR_TIMEOUT", -7: "QMC_ERR_STATE", -8: "QMC_ERR_OOM",
          -9: "QMC_ERR_UNSUPPORTED"}

_lib = None


class QmcError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


def lib() -> C.CDLL:
    """Loads the in-tree libqmc.so; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB):
            raise RuntimeError(f"{LIB} is missing: build it with paper_2504_07948_gb300.build.build()")
        L = C.CDLL(LIB)
        vp, i, d, u64, u32 = C.c_void_p, C.c_int, C.c_double, C.c_uint64, C.c_uint32
        sig = {
            "qmc_create": [C.POINTER(vp), i, vp],
            "qmc_destroy": [vp],
            "qmc_last_error": [vp],
            "qmc_set_system": [vp, i, vp, vp, i, i],
            "qmc_set_nuclei": [vp, vp],
            "qmc_set_basis": [vp, i, vp, vp, vp, vp, vp, vp],
            "qmc_set_mos": [vp, i, i, vp, vp, vp],
            "qmc_set_jastrow": [vp, d, d, d, vp, d],
            "qmc_set_jastrow3": [vp, i, vp, vp, d],
            "qmc_jastrow_derivs": [vp, vp, vp, i],
            "qmc_set_pseudopotential": [vp, i, vp, vp, vp, vp, vp, vp, i, vp, vp, i],
            "qmc_set_multidet": [vp, i, i, vp, vp, vp],
            "qmc_set_precision": [vp, i, i, i],
            "qmc_set_rng": [vp, u64, u32],
            "qmc_set_population_control": [vp, i],
            "qmc_set_space_warp": [vp, i],
            "qmc_set_capacity_factor": [vp, i],
            "qmc_set_walkers": [vp, i, vp, i],
            "qmc_init_walkers": [vp, i, u64],
            "qmc_get_walkers": [vp, vp, vp, i],
            "qmc_n_walkers": [vp],
            "qmc_evaluate": [vp, vp, vp, vp, vp, i],
            "qmc_eval_cached": [vp, vp, vp, vp, vp, i],
            "qmc_force_vjp": [vp, vp, vp, vp, vp, i],
            "qmc_vmc": [vp, i, d, i, vp, i],
            "qmc_dmc": [vp, i, d, d, i, i, vp, vp, vp],
            "qmc_get_energy": [vp, i, vp, vp, vp, vp],
            "qmc_get_forces": [vp, i, vp, vp],
            "qmc_force_estimate": [vp, vp, vp, i],
            "qmc_reset_estimators": [vp],
            "qmc_trial_energy": [vp, i, d, d, d, i, vp],
            "qmc_set_step_reduce": [vp, vp, vp],
            "qmc_set_population_reference": [vp, d],
            "qmc_set_timing": [vp, i],
            "qmc_get_timing": [vp, C.c_char_p, vp, vp],
            "qmc_branch_noalloc": [i, vp, vp, d, d, d, u64, u32, i, vp, vp, vp],
            "qmc_checkpoint": [vp, C.c_char_p],
            "qmc_restore": [vp, C.c_char_p],
            "qmc_tc_gemm": [i, i, i, i, vp, C.c_longlong, i, vp, C.c_longlong, i, i, vp, C.c_longlong, i, vp],
            "qmc_tc_gemm_split": [i, i, i, vp, vp, i, vp, vp, i, vp, i, vp],
            "qmc_batch_create": [C.POINTER(vp), i, vp],
            "qmc_batch_destroy": [vp],
            "qmc_batch_last_error": [vp],
            "qmc_batch_set_options": [vp, i, i, i, i, i],
            "qmc_batch_autotune": [vp, d, vp],
            "qmc_batch_vmc": [vp, i, d],
            "qmc_batch_dmc": [vp, i, d, vp, i, i, vp, vp],
            "qmc_batch_set_timing": [vp, i],
            "qmc_batch_get_timing": [vp, C.c_char_p, vp, vp],
        }
        for name, args in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = C.c_char_p if name in ("qmc_last_error", "qmc_batch_last_error") else C.c_int
        _lib = L
    return _lib


def _check(h, st: int):
    if st != 0:
        msg = lib().qmc_last_error(h)
        raise QmcError(st, msg.decode() if msg else "")


def _host(a, dtype) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=dtype)


def _ptr(x):
    """(pointer, on_device) of a numpy array or a torch tensor (None -> NULL)."""
    if x is None:
        return None, None
    if isinstance(x, np.ndarray):
        if not x.flags.c_contiguous:
            raise ValueError("arrays passed to the library must be C-contiguous")
        return x.ctypes.data, False
    # torch tensor
    if not x.is_contiguous():
        raise ValueError("tensors passed to the library must be contiguous")
    return x.data_ptr(), bool(x.is_cuda)


def _ptrs(*xs, f64=False, min_sizes=None):
    """Pointers and the on-device flag of buffers passed to one C call.
    f64: every buffer must hold float64 (the C side reads or writes doubles);
    min_sizes: per buffer the smallest element count the call touches (None:
    not checked here), so that a short buffer is refused before the call."""
    ps, dev = [], None
    for k, x in enumerate(xs):
        if x is not None and f64 and str(x.dtype) not in ("float64", "torch.float64"):
            raise ValueError(f"buffer {k} must hold float64, not {x.dtype}")
        if x is not None and min_sizes is not None and min_sizes[k] is not None:
            n = x.size if isinstance(x, np.ndarray) else x.numel()
            if n < min_sizes[k]:
                raise ValueError(f"buffer {k} holds {n} elements, the call writes or reads {min_sizes[k]}")
        p, d = _ptr(x)
        ps.append(p)
        if d is not None:
            if dev is not None and d != dev:
                raise ValueError("mix of host and device buffers in one call")
            dev = d
    return ps, int(bool(dev))


# ---------------------------------------------------------------------------
# one wrapper per C call
# ---------------------------------------------------------------------------

def qmc_create(device: int = 0, stream: Optional[int] = None):
    h = C.c_void_p()
    st = lib().qmc_create(C.byref(h), device, stream)
    _check(None, st)
    return h


def qmc_destroy(h):
    _check(h, lib().qmc_destroy(h))


def qmc_last_error(h) -> str:
    m = lib().qmc_last_error(h)
    return m.decode() if m else ""


def qmc_set_system(h, Z, R, n_up: int, n_dn: int):
    Z, R = _host(Z, np.float64), _host(R, np.float64)
    _check(h, lib().qmc_set_system(h, Z.shape[0], Z.ctypes.data, R.ctypes.data, n_up, n_dn))


def qmc_set_nuclei(h, R):
    R = _host(R, np.float64)
    _check(h, lib().qmc_set_nuclei(h, R.ctypes.data))


def qmc_set_basis(h, center, l, pure, nprim, alpha, coef):
    a = [_host(x, np.int32) for x in (center, l, pure, nprim)] + [_host(alpha, np.float64), _host(coef, np.float64)]
    _check(h, lib().qmc_set_basis(h, a[0].shape[0], *[x.ctypes.data for x in a]))


def qmc_set_mos(h, Cmat, occ_up, occ_dn):
    Cm = _host(Cmat, np.float64)
    ou, od = _host(occ_up, np.int32), _host(occ_dn, np.int32)
    _check(h, lib().qmc_set_mos(h, Cm.shape[0], Cm.shape[1], Cm.ctypes.data, ou.ctypes.data if ou.size else None,
                                od.ctypes.data if od.size else None))


def qmc_set_jastrow(h, a_anti, a_par, b_ee, a_en, b_en):
    ae = _host(a_en, np.float64)
    _check(h, lib().qmc_set_jastrow(h, a_anti, a_par, b_ee, ae.ctypes.data, b_en))


def qmc_set_jastrow3(h, exponents, coef, b3: float):
    e = _host(exponents, np.int32).reshape(-1, 3)
    c = _host(coef, np.float64)
    _check(h, lib().qmc_set_jastrow3(h, int(e.shape[0]), e.ctypes.data, c.ctypes.data, float(b3)))


def qmc_set_pseudopotential(h, nucleus, l, n, alpha, beta, rcut, quad, weights, rotate: bool = True):
    nu = _host(nucleus, np.int32)
    ll = _host(l, np.int32)
    nn = _host(n, np.int32)
    al = _host(alpha, np.float64)
    be = _host(beta, np.float64)
    rc = _host(rcut, np.float64)
    q = _host(quad, np.float64).reshape(-1, 3)
    w = _host(weights, np.float64)
    _check(h, lib().qmc_set_pseudopotential(h, int(nu.shape[0]), nu.ctypes.data, ll.ctypes.data, nn.ctypes.data,
                                            al.ctypes.data, be.ctypes.data, rc.ctypes.data, int(w.shape[0]),
                                            q.ctypes.data, w.ctypes.data, int(bool(rotate))))


def qmc_jastrow_derivs(h, dlog, deloc):
    """dlog, deloc [W, P] (host or device)."""
    (pl, pe), dev = _ptrs(dlog, deloc, f64=True)
    _check(h, lib().qmc_jastrow_derivs(h, pl, pe, dev))


def qmc_set_multidet(h, det_up, det_dn, ci):
    if ci is None or len(ci) == 0:
        _check(h, lib().qmc_set_multidet(h, 0, 0, None, None, None))
        return
    du = np.ascontiguousarray(det_up, dtype=np.uint64)
    dd = np.ascontiguousarray(det_dn, dtype=np.uint64)
    c = _host(ci, np.float64)
    _check(h, lib().qmc_set_multidet(h, c.shape[0], du.shape[1], du.ctypes.data, dd.ctypes.data, c.ctypes.data))


def qmc_set_precision(h, mode: int, delay_rank: int = 1, recompute_period: int = 0):
    _check(h, lib().qmc_set_precision(h, mode, delay_rank, recompute_period))


def qmc_set_population_control(h, mode: int):
    _check(h, lib().qmc_set_population_control(h, mode))


def qmc_set_space_warp(h, enable: bool):
    _check(h, lib().qmc_set_space_warp(h, int(enable)))


def qmc_set_rng(h, seed: int, sweep: int = 0):
    _check(h, lib().qmc_set_rng(h, seed, sweep))


def qmc_set_capacity_factor(h, f: int):
    _check(h, lib().qmc_set_capacity_factor(h, f))


def qmc_set_walkers(h, R):
    if isinstance(R, np.ndarray):
        R = _host(R, np.float64)
    (p,), dev = _ptrs(R, f64=True)
    _check(h, lib().qmc_set_walkers(h, R.shape[0], p, dev))


def qmc_init_walkers(h, n_walkers: int, seed: int):
    _check(h, lib().qmc_init_walkers(h, n_walkers, seed))


def qmc_get_walkers(h, R=None, weight=None):
    W = qmc_n_walkers(h) if weight is not None else 0
    (pr, pw), dev = _ptrs(R, weight, f64=True, min_sizes=[None, W])
    _check(h, lib().qmc_get_walkers(h, pr, pw, dev))


def qmc_n_walkers(h) -> int:
    n = lib().qmc_n_walkers(h)
    if n < 0:
        _check(h, n)
    return n


def _per_walker(h, *xs):
    """Walker count of the handle when any of the buffers is given."""
    return qmc_n_walkers(h) if any(x is not None for x in xs) else 0


def qmc_evaluate(h, logpsi=None, sign=None, eloc=None, grad=None):
    W = _per_walker(h, logpsi, sign, eloc)
    ps, dev = _ptrs(logpsi, sign, eloc, grad, f64=True, min_sizes=[W, W, W, None])
    _check(h, lib().qmc_evaluate(h, *ps, dev))


def qmc_eval_cached(h, logpsi=None, sign=None, eloc=None, grad=None):
    W = _per_walker(h, logpsi, sign, eloc)
    ps, dev = _ptrs(logpsi, sign, eloc, grad, f64=True, min_sizes=[W, W, W, None])
    _check(h, lib().qmc_eval_cached(h, *ps, dev))


def qmc_force_vjp(h, g_eloc=None, g_logpsi=None, dR=None, per_walker=None):
    W = _per_walker(h, g_eloc, g_logpsi)
    ps, dev = _ptrs(g_eloc, g_logpsi, dR, per_walker, f64=True, min_sizes=[W, W, None, None])
    _check(h, lib().qmc_force_vjp(h, *ps, dev))


def qmc_vmc(h, n_sweeps: int, tau: float, forces_every: int = 0, eloc_trace=None):
    W = _per_walker(h, eloc_trace)
    (p,), dev = _ptrs(eloc_trace, f64=True, min_sizes=[int(n_sweeps) * W])
    _check(h, lib().qmc_vmc(h, n_sweeps, tau, forces_every, p, dev))


def qmc_dmc(h, n_steps: int, tau: float, e_trial: float, n_equil: int = 0, forces_every: int = 0,
            e_step=None, pop=None, e_trial_out=None):
    for a in (e_step, pop, e_trial_out):
        assert a is None or isinstance(a, np.ndarray)
    _check(h, lib().qmc_dmc(h, n_steps, tau, e_trial, n_equil, forces_every,
                            None if e_step is None else e_step.ctypes.data,
                            None if pop is None else pop.ctypes.data,
                            None if e_trial_out is None else e_trial_out.ctypes.data))


def qmc_get_energy(h, estimator: int):
    out = np.zeros(4)
    _check(h, lib().qmc_get_energy(h, estimator, *[out[k:k + 1].ctypes.data for k in range(4)]))
    return dict(mean=out[0], stderr=out[1], variance=out[2], acceptance=out[3])


def qmc_get_forces(h, estimator: int, n_nuc: int):
    F, E = np.zeros((n_nuc, 3)), np.zeros((n_nuc, 3))
    _check(h, lib().qmc_get_forces(h, estimator, F.ctypes.data, E.ctypes.data))
    return F, E


def qmc_force_estimate(h, weights, F):
    """Zero-variance zero-bias force over the current walkers into F
    [n_nuc, 3] (host or device, like weights [W] or None)."""
    W = _per_walker(h, weights)
    (pw, pF), dev = _ptrs(weights, F, f64=True, min_sizes=[W, None])
    _check(h, lib().qmc_force_estimate(h, pw, pF, dev))


REDUCE_FN = C.CFUNCTYPE(C.c_int, C.POINTER(C.c_double), C.c_int, C.c_void_p)


def qmc_trial_energy(hist, pop: float, pop0: float, tau: float, fixed_pop: bool = False) -> float:
    hh = _host(hist, np.float64)
    out = np.zeros(1)
    st = lib().qmc_trial_energy(hh.ctypes.data, int(hh.shape[0]), float(pop), float(pop0), float(tau),
                                int(bool(fixed_pop)), out.ctypes.data)
    if st != 0:
        raise QmcError(st, "qmc_trial_energy rejected its arguments")
    return float(out[0])


def qmc_set_step_reduce(h, fn):
    """fn: a REDUCE_FN (keep a reference to it while the handle uses it) or
    None."""
    _check(h, lib().qmc_set_step_reduce(h, C.cast(fn, C.c_void_p) if fn is not None else None, None))


def qmc_set_population_reference(h, pop0: float):
    _check(h, lib().qmc_set_population_reference(h, float(pop0)))


def qmc_reset_estimators(h):
    _check(h, lib().qmc_reset_estimators(h))


def qmc_set_timing(h, enable: bool):
    _check(h, lib().qmc_set_timing(h, int(bool(enable))))


def qmc_get_timing(h, family: str = "all"):
    """(total device milliseconds, kernel launches) of a kernel family."""
    ms = np.zeros(1)
    n = np.zeros(1, dtype=np.int64)
    _check(h, lib().qmc_get_timing(h, family.encode(), ms.ctypes.data, n.ctypes.data))
    return float(ms[0]), int(n[0])


def qmc_branch_noalloc(eloc_old, eloc_new, tau: float, e_trial: float, e_cut: float, seed: int, sweep: int,
                       parent, stats, stream: Optional[int] = None):
    """Allocation-free branching on caller-owned device tensors (see
    include/qmc.h); enqueued on `stream`, returns without waiting."""
    import torch
    ts = (eloc_old, eloc_new, parent, stats)
    if not all(isinstance(t, torch.Tensor) and t.is_cuda for t in ts):
        raise ValueError("qmc_branch_noalloc takes CUDA tensors")
    cur = torch.cuda.current_device()
    if any(t.device.index != cur for t in ts):
        raise ValueError("qmc_branch_noalloc: every tensor must be on the current CUDA device")
    if not all(t.is_contiguous() for t in ts):
        raise ValueError("qmc_branch_noalloc: tensors must be contiguous")
    if eloc_old.dtype != torch.float64 or eloc_new.dtype != torch.float64 or stats.dtype != torch.float64:
        raise ValueError("qmc_branch_noalloc: energies and stats must be float64")
    if parent.dtype != torch.int32:
        raise ValueError("qmc_branch_noalloc: parent must be int32")
    if eloc_new.numel() != eloc_old.numel():
        raise ValueError("qmc_branch_noalloc: eloc_old and eloc_new differ in length")
    if stats.numel() < 5:
        raise ValueError("qmc_branch_noalloc: stats needs at least 5 entries")
    (po, pn, pp, ps), dev = _ptrs(eloc_old, eloc_new, parent, stats)
    st = lib().qmc_branch_noalloc(int(eloc_old.numel()), po, pn, tau, e_trial, e_cut, seed, sweep,
                                  int(parent.numel()), pp, ps, stream)
    if st != 0:
        raise QmcError(st, "qmc_branch_noalloc rejected its arguments" if st in (-1, -9) else "launch failed")


def qmc_checkpoint(h, path: str):
    _check(h, lib().qmc_checkpoint(h, path.encode()))


def qmc_restore(h, path: str):
    _check(h, lib().qmc_restore(h, path.encode()))


def _need_f32_cuda(*ts):
    """Contiguous float32 CUDA tensors on one device, else ValueError."""
    import torch
    dev = None
    for t in ts:
        if not isinstance(t, torch.Tensor) or not t.is_cuda:
            raise ValueError("the tensor-core GEMMs take CUDA tensors")
        if t.dtype != torch.float32 or not t.is_contiguous():
            raise ValueError("the tensor-core GEMMs take contiguous float32 tensors")
        if dev is not None and t.device != dev:
            raise ValueError("all tensors must be on one device")
        dev = t.device


def qmc_tc_gemm(A, B, D, b_trans: bool = False, stream: Optional[int] = None):
    """D[b] = A[b] @ B[b]^T (or A[b] @ B[b] when b_trans) on the tensor cores
    for float32 CUDA tensors A [batch|1, M, K], B [batch|1, N, K] ([K, N] when
    b_trans), D [batch, M, N]; a leading dimension of 1 shares the operand."""
    _need_f32_cuda(A, B, D)
    if A.dim() != 3 or B.dim() != 3 or D.dim() != 3:
        raise ValueError("qmc_tc_gemm takes 3-D tensors A, B, D")
    batch, M, N = D.shape
    K = A.shape[-1]
    if A.shape[0] not in (1, batch) or A.shape[1] != M:
        raise ValueError("A must be [batch or 1, M, K] for D [batch, M, N]")
    if B.shape[0] not in (1, batch) or tuple(B.shape[1:]) != ((K, N) if b_trans else (N, K)):
        raise ValueError("B must be [batch or 1, K, N] (b_trans) or [batch or 1, N, K]")
    sA = 0 if A.shape[0] == 1 else M * K
    sB = 0 if B.shape[0] == 1 else B.shape[1] * B.shape[2]
    ldb = N if b_trans else K
    st = lib().qmc_tc_gemm(batch, M, N, K, A.data_ptr(), sA, K, B.data_ptr(), sB, ldb, int(bool(b_trans)),
                           D.data_ptr(), M * N, N, stream)
    if st != 0:
        raise QmcError(st, "qmc_tc_gemm failed")


def qmc_tc_gemm_split(A_hi, A_lo, B_hi, B_lo, D, stream: Optional[int] = None):
    """D = (A_hi + A_lo) @ (B_hi + B_lo)^T (lo*lo dropped) for float32 CUDA
    tensors [M, K], [N, K] holding TF32-exact halves; D [M, N]."""
    _need_f32_cuda(A_hi, A_lo, B_hi, B_lo, D)
    if any(t.dim() != 2 for t in (A_hi, A_lo, B_hi, B_lo, D)):
        raise ValueError("qmc_tc_gemm_split takes 2-D tensors")
    M, K = A_hi.shape
    N = B_hi.shape[0]
    if tuple(A_lo.shape) != (M, K) or tuple(B_hi.shape) != (N, K) or tuple(B_lo.shape) != (N, K) \
            or tuple(D.shape) != (M, N):
        raise ValueError("shapes must be A_hi, A_lo [M, K], B_hi, B_lo [N, K], D [M, N]")
    st = lib().qmc_tc_gemm_split(M, N, K, A_hi.data_ptr(), A_lo.data_ptr(), K, B_hi.data_ptr(), B_lo.data_ptr(), K,
                                 D.data_ptr(), N, stream)
    if st != 0:
        raise QmcError(st, "qmc_tc_gemm_split failed")


def _check_b(b, st: int):
    if st != 0:
        msg = lib().qmc_batch_last_error(b)
        raise QmcError(st, msg.decode() if msg else "")


def qmc_batch_create(handles):
    """A batch over the given handles (a sequence of qmc_t)."""
    arr = (C.c_void_p * len(handles))(*[h.value if isinstance(h, C.c_void_p) else h for h in handles])
    b = C.c_void_p()
    st = lib().qmc_batch_create(C.byref(b), len(handles), arr)
    if st != 0:
        msg = lib().qmc_batch_last_error(None)
        raise QmcError(st, msg.decode() if msg else "")
    return b


def qmc_batch_destroy(b):
    _check_b(b, lib().qmc_batch_destroy(b))


def qmc_batch_last_error(b) -> str:
    msg = lib().qmc_batch_last_error(b)
    return msg.decode() if msg else ""


def qmc_batch_set_options(b, use_graph: bool = True, sweep_block: int = 128, delay_rank: int = 1,
                          delay_min_electrons: int = 0, smem_budget: int = 100 * 1024):
    _check_b(b, lib().qmc_batch_set_options(b, int(bool(use_graph)), sweep_block, delay_rank, delay_min_electrons,
                                            smem_budget))


def qmc_batch_autotune(b, tau: float, n_systems: int):
    """Chosen configuration: dict(block, smem, grid, sweep_us, per_system=[(delay_rank, ainv_smem)])."""
    out = np.zeros(4 + n_systems, dtype=np.int32)
    _check_b(b, lib().qmc_batch_autotune(b, tau, out.ctypes.data))
    return dict(block=int(out[0]), smem=int(out[1]), grid=int(out[2]), sweep_us=int(out[3]),
                per_system=[(int(v) // 2, int(v) % 2) for v in out[4:]])


def qmc_batch_vmc(b, n_sweeps: int, tau: float):
    _check_b(b, lib().qmc_batch_vmc(b, n_sweeps, tau))


def qmc_batch_dmc(b, n_steps: int, tau: float, e_trial, n_equil: int = 0, forces_every: int = 0, e_step=None,
                  pop=None):
    et = _host(e_trial, np.float64)
    (pe, pp), _ = _ptrs(e_step, pop)
    _check_b(b, lib().qmc_batch_dmc(b, n_steps, tau, et.ctypes.data, n_equil, forces_every, pe, pp))


def qmc_batch_set_timing(b, enable: bool):
    _check_b(b, lib().qmc_batch_set_timing(b, int(bool(enable))))


def qmc_batch_get_timing(b, family: str = "all"):
    ms = np.zeros(1)
    n = np.zeros(1, dtype=np.int64)
    _check_b(b, lib().qmc_batch_get_timing(b, family.encode(), ms.ctypes.data, n.ctypes.data))
    return float(ms[0]), int(n[0])


# ---------------------------------------------------------------------------
# convenience objects
# ---------------------------------------------------------------------------

class QMC:
    """One handle holding a system (anything with the fields of
    ``synth.System``) and its walkers."""

    def __init__(self, system, device: int = 0, precision: str = "fp64", recompute_period: int = 0,
                 seed: int = 1005, stream: Optional[int] = None, cap_factor: int = 2, delay_rank: int = 1,
                 fixed_population: bool = False, space_warp: bool = False, pp_rotate: bool = True):
        self.sys = system
        self.h = qmc_create(device, stream)
        s = system
        qmc_set_system(self.h, s.Z, s.R, s.n_up, s.n_dn)
        qmc_set_basis(self.h, s.shell_center, s.shell_l, s.shell_pure, s.shell_nprim, s.alpha, s.coef)
        qmc_set_mos(self.h, s.C, s.occ_up, s.occ_dn)
        qmc_set_jastrow(self.h, s.a_anti, s.a_par, s.b_ee, s.a_en, s.b_en)
        if getattr(s, "ci", None) is not None:
            qmc_set_multidet(self.h, s.det_up, s.det_dn, s.ci)
        if getattr(s, "j3_exponents", None) is not None and len(s.j3_exponents) > 0:
            qmc_set_jastrow3(self.h, s.j3_exponents, s.j3_coef, s.j3_b)
        if getattr(s, "pp_nuc", None) is not None and len(s.pp_nuc) > 0:
            qmc_set_pseudopotential(self.h, s.pp_nuc, s.pp_l, s.pp_n, s.pp_alpha, s.pp_beta, s.pp_rcut,
                                    s.pp_quad, s.pp_qw, pp_rotate)
        qmc_set_precision(self.h, QMC_MIXED if precision == "mixed" else QMC_FP64, delay_rank, recompute_period)
        qmc_set_rng(self.h, seed, 0)
        qmc_set_capacity_factor(self.h, cap_factor)
        if fixed_population:
            qmc_set_population_control(self.h, QMC_POP_FIXED)
        if space_warp:
            qmc_set_space_warp(self.h, True)

    def close(self):
        if self.h is not None:
            qmc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def n_walkers(self) -> int:
        return qmc_n_walkers(self.h)

    def set_walkers(self, R):
        qmc_set_walkers(self.h, R)

    def init_walkers(self, n_walkers: int, seed: int = 1005):
        qmc_init_walkers(self.h, n_walkers, seed)

    def get_walkers(self):
        W = self.n_walkers
        R = np.zeros((W, self.sys.n_elec, 3))
        w = np.zeros(W)
        qmc_get_walkers(self.h, R, w)
        return R, w

    def evaluate(self):
        W, N = self.n_walkers, self.sys.n_elec
        out = dict(logpsi=np.zeros(W), sign=np.zeros(W), eloc=np.zeros(W), grad=np.zeros((W, N, 3)))
        qmc_evaluate(self.h, out["logpsi"], out["sign"], out["eloc"], out["grad"])
        return out

    def eval_cached(self):
        W, N = self.n_walkers, self.sys.n_elec
        out = dict(logpsi=np.zeros(W), sign=np.zeros(W), eloc=np.zeros(W), grad=np.zeros((W, N, 3)))
        qmc_eval_cached(self.h, out["logpsi"], out["sign"], out["eloc"], out["grad"])
        return out

    def forces(self, g_eloc=None, g_logpsi=None):
        """(dR [n_nuc,3], per_walker [W,2,n_nuc,3])."""
        W, nn = self.n_walkers, self.sys.n_nuc
        dR = np.zeros((nn, 3))
        pw = np.zeros((W, 2, nn, 3))
        gE = None if g_eloc is None else _host(g_eloc, np.float64)
        gL = None if g_logpsi is None else _host(g_logpsi, np.float64)
        qmc_force_vjp(self.h, gE, gL, dR, pw)
        return dR, pw

    def vmc(self, n_sweeps: int, tau: float, forces_every: int = 0, trace: bool = False):
        tr = np.zeros((n_sweeps, self.n_walkers)) if trace else None
        qmc_vmc(self.h, n_sweeps, tau, forces_every, tr)
        return tr

    def dmc(self, n_steps: int, tau: float, e_trial: float, n_equil: int = 0, forces_every: int = 0):
        e = np.zeros(n_steps)
        pop = np.zeros(n_steps, dtype=np.int32)
        et = np.zeros(n_steps)
        qmc_dmc(self.h, n_steps, tau, e_trial, n_equil, forces_every, e, pop, et)
        return dict(e_step=e, pop=pop, e_trial=et)

    def jastrow_derivs(self):
        """(dlog [W, P], deloc [W, P]) at the current walkers."""
        P = 4 + self.sys.n_nuc + (self.sys.n_nuc * len(self.sys.j3_exponents)
                                  if getattr(self.sys, "j3_exponents", None) is not None else 0)
        dlog = np.zeros((self.n_walkers, P))
        deloc = np.zeros((self.n_walkers, P))
        qmc_jastrow_derivs(self.h, dlog, deloc)
        return dlog, deloc

    def energy(self, estimator: int = QMC_EST_DMC):
        return qmc_get_energy(self.h, estimator)

    def force_estimate(self, estimator: int = QMC_EST_DMC):
        return qmc_get_forces(self.h, estimator, self.sys.n_nuc)


class Batch:
    """A batch over several ``QMC`` objects (which must outlive it)."""

    def __init__(self, members):
        self.members = list(members)
        self.b = qmc_batch_create([m.h for m in self.members])

    def close(self):
        if self.b is not None:
            qmc_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_options(self, **kw):
        qmc_batch_set_options(self.b, **kw)

    def autotune(self, tau: float):
        return qmc_batch_autotune(self.b, tau, len(self.members))

    def vmc(self, n_sweeps: int, tau: float):
        qmc_batch_vmc(self.b, n_sweeps, tau)

    def dmc(self, n_steps: int, tau: float, e_trial, n_equil: int = 0, forces_every: int = 0):
        n = len(self.members)
        e = np.zeros((n_steps, n))
        pop = np.zeros((n_steps, n), dtype=np.int32)
        qmc_batch_dmc(self.b, n_steps, tau, e_trial, n_equil, forces_every, e, pop)
        return dict(e_step=e, pop=pop)
