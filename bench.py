#!/usr/bin/env python
"""Throughput of the walker-batched Slater-Jastrow DMC step on GB300.

Workload (default): 6-water cluster (18 nuclei, 60 electrons, 144 GTOs), 2048
walkers, FP64 throughout, forces on every step.  One step = one
particle-by-particle sweep of all walkers (60 electron moves each), the local
energy, the ionic derivatives of E_L and ln|psi| for every walker (adjoint
kernel), the force-estimator reductions and branching.  Metric:
electron-moves/s (proposals, accepted or not); force evaluations/s is
reported beside it.  The same workload in mixed precision is reported under
"mixed" with its error against the FP64 oracle.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun each rank runs an independent replica (its own population);
value = all ranks' moves / max-over-ranks time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
# nvidia-smi clock samples of the timed regions (CSV per run)
CLOCK_DIR = os.environ.get("QMC_CLOCK_DIR", os.path.join(tempfile.gettempdir(), "qmc_clocks"))

METRIC = "electron-moves/s of a full DMC step (sweep + E_L + forces + branching); force evals/s beside"
FP64_PEAK_TFLOPS_NOMINAL = 1.25     # GB300 FP64 (recipe table)
TF32_OVER_BF16_NOMINAL = 1.1 / 2.25  # nominal dense TF32 / BF16 tensor rates (recipe table)
FP32_PEAK_TFLOPS_NOMINAL = 152 * 128 * 2 * 2.07e9 / 1e12   # 152 SMs x 128 FP32 lanes x FMA x 2.07 GHz


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f)
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "fallback": True}


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one launch of
# the dominant sweep kernel, per walker in the launch, from one ncu capture of
# each workload (walkers in the capture; the full-size launches are scaled by
# walker count).  They describe the sweep kernel as it was when captured:
# `traffic` is reported only while the sources that kernel is compiled from
# still hash to the value recorded with the capture, else it is null.
_SRC_SM = ("k_sweep.cu", "qmc_internal.cuh", "sweep_sm.cuh")
_SRC_BATCH = ("batch.cuh", "k_sweep_delayed.cu", "qmc_internal.cuh", "sweep_sm.cuh")
_SRC_MSD = ("k_msd.cu", "msd_small.cuh", "qmc_internal.cuh")
_SRC_GEMM = ("k_tc_gemm.cu", "qmc_internal.cuh")
_SRC_NLPP = ("k_nlpp.cu", "qmc_internal.cuh")
PROFILED_TRAFFIC = {
    # (workload, kernel form): (bytes per walker, summary, walkers in the capture, sources, their hash[,
    # bytes that do not grow with the walkers])
    ("water6_fp64_forces", "fp64"): (214_323_968 / 2048, "profiles/k_sweep_water6.md", 2048, _SRC_SM,
                                     "fde49d1880530800"),
    ("water6_fp64_forces", "mixed"): (94_340_096 / 2048, "profiles/k_sweep_water6.md", 2048, _SRC_SM,
                                      "fde49d1880530800"),
    # the orbital GEMM of the walker-tiled sweep (one launch per walker
    # group): the basis rows grow with the walkers, the coefficients
    # (2 x 160 x 768 x 4 bytes) do not
    ("water32_mixed", "gemm"): ((8_868_352 - 983_040) / 256, "profiles/k_tiled_sweep_water32.md", 256, _SRC_GEMM,
                                "57f23b21afebd826", 983_040.0),
    ("water6_msd10k", "mixed"): (210_295_808 / 512, "profiles/k_sweep_msd_water6_10k.md", 512, _SRC_MSD,
                                 "1b3e15a60b78925a"),
    ("batch64_uneven", "mixed"): (296_749_568 / 2048, "profiles/k_batch_kernels_batch64_uneven.md", 2048, _SRC_BATCH,
                                  "d348a963ce01d23d"),
    ("water32_pp_mixed", "nlpp"): (314_676_480 / 512, "profiles/k_nlpp_water32_pp.md", 512, _SRC_NLPP,
                                   "e9555c1f7d29d3e3"),
    ("water6_pp_forces", "nlpp"): (3_070_208 / 512, "profiles/k_nlpp_water32_pp.md", 512, _SRC_NLPP,
                                   "e9555c1f7d29d3e3"),
}


def sources_sha(files) -> str:
    import hashlib
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2504_07948_gb300", "csrc")
    for f in sorted(files):
        h.update(f.encode())
        with open(os.path.join(d, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(workload: str, precision: str, walkers_per_launch: float):
    """(bytes per launch, note) from the stored capture, or (None, why)."""
    rec = PROFILED_TRAFFIC.get((workload, precision))
    if rec is None:
        return None, "no ncu capture of this workload and form"
    per_walker, where, w_cap, files, digest = rec[:5]
    fixed = rec[5] if len(rec) > 5 else 0.0   # bytes that do not grow with the walkers
    if sources_sha(files) != digest:
        return None, "kernel sources changed since the ncu capture"
    note = f"ncu dram bytes of one launch at {w_cap} walkers ({where})"
    if abs(walkers_per_launch - w_cap) > 0.5:
        note += f", scaled by walker count to {walkers_per_launch:.0f}"
        if fixed:
            note += f" ({fixed / 1e6:.2f} MB of it fixed)"
    return per_walker * walkers_per_launch + fixed, note


def time_recompute(Q, g, s, R, period, steps, step_s, live=None):
    """The periodic FP64 rebuild (inverse, log-determinant and gradient cache
    from FP64 orbitals, every `period` steps; at the bench's step counts it
    falls outside the timed steps): one rebuild of the population R timed on
    its own (qmc_set_walkers rebuilds from scratch), its FP64 flops (per
    electron 10 n_s N_b for the orbitals with gradients and Laplacians, per
    spin 2 n_s^3 for the inverse; the contraction skips the exactly-zero rows
    of screened shells, so beside the dense count the executed one over the
    live fraction of the rows) and the step time with the rebuild's share
    amortised over the period."""
    if period <= 0:
        return None
    Q.qmc_set_timing(g.h, True)
    g.set_walkers(R)
    ms, n = Q.qmc_get_timing(g.h, "recompute")
    Q.qmc_set_timing(g.h, False)
    W = R.shape[0]
    fl = W * sum(ns * 10.0 * ns * s.n_basis + 2.0 * ns ** 3 for ns in (s.n_up, s.n_dn))
    fl_x = None if live is None else W * sum(ns * 10.0 * ns * s.n_basis * live + 2.0 * ns ** 3
                                             for ns in (s.n_up, s.n_dn))
    ex = {} if fl_x is None or ms <= 0 else {
        "live_basis_fraction": live, "achieved_fp64_tflops_executed": fl_x / (ms / 1e3) / 1e12,
        "frac_fp64_executed": fl_x / (ms / 1e3) / 1e12 / FP64_PEAK_TFLOPS_NOMINAL}
    return {"ms": ms, "kernels": n, "walkers": W, "period_steps": period, **ex,
            "ms_per_step_amortised": ms / period,
            "step_ms_with_recompute_amortised": step_s * 1e3 + ms / period,
            "achieved_fp64_tflops": fl / (ms / 1e3) / 1e12 if ms > 0 else None,
            "frac_fp64": fl / (ms / 1e3) / 1e12 / FP64_PEAK_TFLOPS_NOMINAL if ms > 0 else None,
            "flops_counted": "per electron 10 n_s N_b (FP64 orbitals, gradients, Laplacians), per spin 2 n_s^3"}


SCREEN_EXPONENT = 60.0   # a shell is screened where (smallest exponent) r^2 exceeds this


# FP operations of an e x e determinant (cofactor forms of sizes 1-4)
DET_FLOPS = {0: 0, 1: 0, 2: 3, 3: 14, 4: 47}


def msd_string_flops(s):
    """(up, down) FP operations per move over the unique spin strings of an
    expansion, by excitation level e: at the current position the e
    column-replaced determinants of the minor and the drift terms (e D(e) +
    6e), after the proposal the rank-1 bordered minor, its determinant, the e
    column-replaced determinants and the gradient terms (2e^2 + D(e) +
    e D(e) + 6e)."""
    out = []
    for bits, occ in ((s.det_up, s.occ_up), (s.det_dn, s.occ_dn)):
        uniq = np.unique(np.asarray(bits, dtype=np.uint64), axis=0)
        ref = np.zeros(uniq.shape[1], dtype=np.uint64)
        for o in occ:
            ref[o // 64] |= np.uint64(1) << np.uint64(o % 64)
        tot = 0.0
        for row in uniq:
            e = sum(bin(int(w) & ~int(r)).count("1") for w, r in zip(row, ref))
            d = DET_FLOPS[min(e, 4)]
            tot += (e * d + 6 * e) + (2 * e * e + d + e * d + 6 * e)
        out.append(tot)
    return out


def live_basis_fraction(s, R, max_walkers: int = 64) -> float:
    """Mean fraction of basis functions on unscreened shells at the electron
    positions R [W, N, 3] (a sample of walkers): the sweeps contract only
    those rows, so they are the algorithmic work of a move."""
    R = np.asarray(R)[:max_walkers]
    off = np.concatenate([[0], np.cumsum(s.shell_nprim)])
    amin = np.array([s.alpha[off[i]:off[i + 1]].min() if off[i + 1] > off[i] else np.inf
                     for i in range(s.n_shell)])
    nfn = np.array([(1 if l == 0 else 3 if l == 1 else (5 if p else 6)) for l, p in zip(s.shell_l, s.shell_pure)])
    ctr = np.asarray(s.R)[np.asarray(s.shell_center)]
    live = np.zeros(R.shape[:2])
    for q in range(s.n_shell):
        d2 = ((R - ctr[q]) ** 2).sum(axis=-1)
        live += np.where(amin[q] * d2 <= SCREEN_EXPONENT, nfn[q], 0)
    return float(live.mean() / nfn.sum())


def sweep_flops_per_move(s, live_frac: float = 1.0) -> float:
    """Algorithmic FP work of one proposed move: orbital contraction 2 n N_b
    for each of value, gradient (3) and Laplacian (dense; live_frac < 1
    counts only the unscreened rows the kernels visit), determinant ratio and
    new drift 8 n, and the drift at the current position 6 n.  The
    Sherman-Morrison update (4 n^2 per accepted move) is added by the caller
    with the measured acceptance."""
    n = max(s.n_up, s.n_dn)
    return 10.0 * n * s.n_basis * live_frac + 14.0 * n


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    def __init__(self, out_path):
        self.out_path = out_path
        self.proc = None
        os.makedirs(os.path.dirname(out_path), exist_ok=True)

    def __enter__(self):
        try:
            self.f = open(self.out_path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self, device_index=0):
        try:
            rows = [l.split(",") for l in open(self.out_path).read().strip().splitlines()]
        except Exception:
            return None
        rows = [[c.strip() for c in r] for r in rows if len(r) >= 9 and r[0].strip() == str(device_index)]
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def dist_init():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws <= 1:
        return 0, 1, None
    import torch.distributed as dist
    rank = int(os.environ["RANK"])
    backend = "nccl" if os.environ.get("QMC_BENCH_BACKEND", "nccl") == "nccl" else "gloo"
    dist.init_process_group(backend)
    return rank, ws, dist


def max_over_ranks(x, dist):
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if dist.get_backend() == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x, dist):
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if dist.get_backend() == "nccl" else "cpu")
    dist.all_reduce(t)
    return float(t.item())


def cpu_baseline(system, R, tau, e_trial, seconds_target=15.0, forces=True, max_walkers=0):
    """The oracle as it stands on the host cores: DMC steps (with forces
    unless forces=False) on a bounded sample of walkers; electron-moves/s and
    force-evals/s."""
    from oracle import oracle as O
    o = O.Oracle(system)
    cores = o.nthreads
    W = max(cores, 4) if max_walkers <= 0 else min(max(cores, 4), max_walkers)
    sample = R[:W]
    fe = 1 if forces else 0
    t0 = time.perf_counter()
    out = o.dmc(sample, 1, tau, e_trial, seed=4242, step0=10_000, cap_factor=4, n_equil=0, forces_every=fe)
    dt = time.perf_counter() - t0
    # scale the sample so the measurement is roughly seconds_target long
    steps = 1
    while dt * (steps + 1) / steps < seconds_target and steps < 4 and dt < seconds_target / 2:
        t1 = time.perf_counter()
        o.dmc(sample, 1, tau, e_trial, seed=4242 + steps, step0=10_000 + steps, cap_factor=4, forces_every=fe)
        dt += time.perf_counter() - t1
        steps += 1
    moves = steps * W * system.n_elec
    return {"value": moves / dt, "unit": "electron-moves/s", "force_evals_per_s": steps * W / dt if forces else 0.0,
            "cores": cores, "kind": "oracle",
            "sample": f"{steps} DMC step(s) {'with' if forces else 'without'} forces of {W} walkers of the same "
                      f"workload ({moves} electron moves, {dt:.1f} s, LU per move"
                      f"{', forward-mode forces' if forces else ''})"}


def workload_system(synth, wl):
    s = synth.water_system(wl.n_water)
    if wl.n_det > 0:
        s = synth.with_multidet(s, wl.n_det, n_active=20, max_exc=4)
    if getattr(wl, "pseudopotential", False):
        s = synth.with_pseudopotential(s)
    return s


def run_gpu(args, rank, ws, dist):
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2504_07948_gb300 import qmc as Q, synth
    from oracle import oracle as O

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    wl = synth.WORKLOADS[args.workload]
    s = workload_system(synth, wl)
    W = args.walkers or wl.n_walkers
    R0 = synth.initial_walkers(s, W, seed=synth.SEED_WALKERS + rank)
    stream = torch.cuda.current_stream()
    tau = wl.tau
    peaks = load_peaks()

    def make(precision, space_warp=False):
        g = Q.QMC(s, precision=precision, recompute_period=wl.recompute_period, seed=synth.SEED_WALKERS + rank,
                  stream=stream.cuda_stream, cap_factor=4,
                  delay_rank=wl.delay_rank if (precision == "mixed" and wl.n_det == 0) else 1,
                  fixed_population=not args.birth_death, space_warp=space_warp)
        g.set_walkers(R0)
        return g

    def equilibrate(g):
        tr = g.vmc(args.vmc_sweeps, 0.05, trace=True)
        return float(tr[-max(1, args.vmc_sweeps // 2):].mean())

    def timed(g, precision, e_trial):
        out = g.dmc(args.warmup, tau, e_trial, forces_every=1 if wl.forces else 0)
        et = float(out["e_trial"][-1]) if args.warmup else e_trial
        W_before = g.n_walkers
        Q.qmc_reset_estimators(g.h)
        Q.qmc_set_timing(g.h, True)
        clocks = ClockSampler(os.path.join(CLOCK_DIR, f"clocks_{precision}_r{rank}.csv"))
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        with clocks:
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            out = g.dmc(args.steps, tau, et, forces_every=1 if wl.forces else 0)
            ev1.record(stream)
            torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        ms = ev0.elapsed_time(ev1)
        fam = {f: Q.qmc_get_timing(g.h, f) for f in ("sweep", "sweep_gemm", "eloc", "force", "branch", "recompute",
                                                     "reduce", "all")}
        Q.qmc_set_timing(g.h, False)
        return ms, out, fam, clocks.summary(int(os.environ.get("LOCAL_RANK", "0"))), W_before

    result = {}
    for precision in (["fp64", "mixed"] if wl.precision == "fp64" and not args.only_primary else [wl.precision]):
        g = make(precision)
        e_v = equilibrate(g)
        ms, out, fam, clk, W_before = timed(g, precision, e_v)
        # walkers swept in step k = population entering step k
        entering = np.concatenate([[W_before], out["pop"][:-1]])
        moves = float(sum(entering)) * s.n_elec
        force_evals = float(sum(entering)) if wl.forces else 0.0
        sec = max_over_ranks(ms / 1e3, dist)
        moves_all = sum_over_ranks(moves, dist)
        fe_all = sum_over_ranks(force_evals, dist)
        sweep_ms, sweep_n = fam["sweep"]
        acc = Q.qmc_get_energy(g.h, Q.QMC_EST_DMC)["acceptance"]
        n = max(s.n_up, s.n_dn)
        live = live_basis_fraction(s, g.get_walkers()[0])
        # algorithmic work per move: the dense contraction over every basis
        # row; the kernels visit only the live rows, counted beside it
        flops_sweep = moves * (sweep_flops_per_move(s) + 4.0 * n * n * acc) / max(1, args.steps)
        flops_exec = moves * (sweep_flops_per_move(s, live) + 4.0 * n * n * acc) / max(1, args.steps)
        if s.n_det > 0:
            # per move also the virtual-orbital contraction (10 n_vir N_b) and
            # the string work of the moving spin (msd_string_flops)
            n_vir = 20
            str_fl = msd_string_flops(s)
            per_move = 10.0 * n_vir * s.n_basis + (s.n_up * str_fl[0] + s.n_dn * str_fl[1]) / s.n_elec
            flops_sweep += moves * per_move / max(1, args.steps)
            flops_exec += moves * per_move / max(1, args.steps)
        sweep_avg_s = sweep_ms / 1e3 / max(1, sweep_n)
        ach_tflops = flops_sweep / sweep_avg_s / 1e12 if sweep_avg_s > 0 else 0.0
        ach_exec = flops_exec / sweep_avg_s / 1e12 if sweep_avg_s > 0 else 0.0
        peak = FP64_PEAK_TFLOPS_NOMINAL if precision == "fp64" else FP32_PEAK_TFLOPS_NOMINAL
        traffic, traffic_note = profiled_traffic(args.workload, precision, float(np.mean(entering)))
        sweep_kernel = ("k_sweep_msd" if s.n_det > 0 else
                        "k_sweep_delayed" if precision == "mixed" and wl.delay_rank > 1 else "k_sweep")
        gemm_ms, gemm_n = fam["sweep_gemm"]
        result[precision] = {
            "value": moves_all / sec, "force_evals_per_s": fe_all / sec, "ms_per_step": ms / args.steps,
            "kernel_ms": {k: v[0] / args.steps for k, v in fam.items()},
            "gpu_launches": fam["all"][1], "acceptance": acc,
            "roofline": {"kernel": sweep_kernel, "bound": "alu", "achieved": ach_tflops, "peak": peak,
                         "unit": "TFLOP/s", "frac": ach_tflops / peak,
                         "flops_counted": "per move 10 n N_b (dense contraction) + 14 n, + 4 n^2 per accepted move",
                         "live_basis_fraction": live, "achieved_executed": ach_exec, "frac_executed": ach_exec / peak,
                         "executed_counted": "the contraction over the live basis rows only (fraction estimated at "
                                             "the final walker positions)",
                         "traffic": traffic,
                         "traffic_unit": "bytes per launch", "traffic_source": traffic_note,
                         "peak_source": "nominal FP64 1.25 TFLOP/s (recipe table)" if precision == "fp64"
                         else "nominal FP32 FMA rate, 152 SMs x 128 lanes x 2.07 GHz"},
            "clocks": clk, "population_last": int(out["pop"][-1]), "e_step_mean": float(out["e_step"].mean()),
        }
        if wl.forces and fam["force"][0] > 0:
            # the force pass beside the sweep: per walker sum over spins of
            # 4 n_s^2 N_b (M = C A^-1 and Y = C Q^T) + 2 n_s^3 (P) and
            # 30 N N_b for the third-order basis contraction
            f_flops = sum(4.0 * ns * ns * s.n_basis + 2.0 * ns ** 3 for ns in (s.n_up, s.n_dn)) \
                + 30.0 * s.n_elec * s.n_basis
            fl = f_flops * force_evals / max(1, args.steps)
            fsec = fam["force"][0] / 1e3 / max(1, args.steps)
            fpeak = FP64_PEAK_TFLOPS_NOMINAL if precision == "fp64" else FP32_PEAK_TFLOPS_NOMINAL
            result[precision]["roofline_force"] = {
                "kernel": "k_force" if max(s.n_up, s.n_dn) < 65 else "k_force_prep + GEMMs + k_force_contract",
                "bound": "alu", "achieved": fl / fsec / 1e12, "peak": fpeak, "unit": "TFLOP/s",
                "frac": fl / fsec / 1e12 / fpeak, "flops_per_walker": f_flops,
                "flops_counted": "per walker sum_s (4 n_s^2 N_b + 2 n_s^3) + 30 N N_b (dense)",
                "peak_source": "nominal FP64 1.25 TFLOP/s (recipe table)" if precision == "fp64"
                else "nominal FP32 FMA rate, 152 SMs x 128 lanes x 2.07 GHz"}
        if gemm_n > 0:
            # walker-tiled sweep: its dominant dense work is the orbital GEMM
            # on the tensor cores (10 n N_b flops per move, counted once;
            # 3xTF32 issues three TF32 products per flop pair)
            # the "sweep" span of the tiled sweep covers its GEMMs, which run
            # on the walker groups' streams beside the accept/propose launches
            sweep_total_ms = sweep_ms / max(1, args.steps)
            gemm_step_ms = gemm_ms / max(1, args.steps)
            groups = max(1, int(round(gemm_n / max(1, args.steps) / s.n_elec)))
            flops_gemm = moves * 10.0 * n * s.n_basis / max(1, args.steps)
            ach_g = flops_gemm / (gemm_step_ms / 1e3) / 1e12 if gemm_step_ms > 0 else 0.0
            peak_tf32 = peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops", 1700.0)) * TF32_OVER_BF16_NOMINAL
            peak_g = peak_tf32 / 3.0
            result[precision]["roofline"] = {
                "kernel": "k_tc_gemm_split", "bound": "tensor", "achieved": ach_g, "peak": peak_g,
                "unit": "TFLOP/s", "frac": ach_g / peak_g,
                "flops_counted": "per move 10 n N_b (the dense basis->orbital contraction, FP32-equivalent)",
                "traffic": None, "traffic_source": None,
                "peak_source": "measured sustained bf16 cuBLAS rate (MEASURED_PEAKS.json) x nominal TF32/BF16 "
                               "ratio 1.1/2.25, divided by 3 for the 3xTF32 split (of measured)",
                "gemm_ms_per_step": gemm_step_ms, "gemm_launches_per_step": gemm_n / max(1, args.steps),
                "walker_groups": groups,
                "note": "the walker groups' launches run on separate streams: a GEMM launch's event-timed duration "
                        "includes the time its CTAs wait for SMs held by the other group's accept/propose launches",
                "sweep_ms_per_step": sweep_total_ms,
                "sweep_achieved_fp32_tflops": flops_sweep / (sweep_total_ms / 1e3) / 1e12,
                "sweep_frac_of_fp32_peak": flops_sweep / (sweep_total_ms / 1e3) / 1e12 / FP32_PEAK_TFLOPS_NOMINAL,
                "kernel_of_sweep": "k_sweep_tiled (propose, tcgen05 orbital GEMM, accept, tensor-core flush)"}
            result[precision]["kernel_ms"]["sweep"] = sweep_total_ms
            tg, tg_note = profiled_traffic(args.workload, "gemm", float(np.mean(entering)) / groups)
            result[precision]["roofline"]["traffic"] = tg
            result[precision]["roofline"]["traffic_source"] = tg_note
            result[precision]["roofline"]["traffic_unit"] = "bytes per launch"
            if tg:
                # the GEMM streams its operands once: its HBM rate against the copy peak
                result[precision]["roofline"]["hbm_achieved_gbs"] = tg / (gemm_step_ms / 1e3 / max(1.0, gemm_n / max(1, args.steps))) / 1e9
                result[precision]["roofline"]["hbm_peak_gbs"] = peaks.get("hbm_gbs")
        # accuracy of this form as it ran: the incrementally maintained state
        # (cached inverse and gradients after the timed steps) against the FP64
        # oracle at the same walker positions, on a sample of the population
        Rg, _ = g.get_walkers()
        ev = g.eval_cached()
        _, pw = g.forces()
        n_sample = args.error_sample if s.n_elec <= 60 and s.n_det <= 1000 else 4
        idx = np.linspace(0, Rg.shape[0] - 1, n_sample).astype(int)
        o = O.Oracle(s)
        ref = o.evaluate(Rg[idx])
        # forward-mode oracle forces of a 10^4-determinant expansion take
        # minutes per walker: the force comparison is left to the tests there
        with_f = s.n_det <= 1000
        dEL, dlg = o.forces(Rg[idx]) if with_f else (pw[idx, 0], pw[idx, 1])
        el = np.abs(ev["eloc"][idx] - ref["eloc"])
        Fg = O.force_estimator(ev["eloc"][idx], pw[idx, 0], pw[idx, 1])
        Fo = O.force_estimator(ref["eloc"], dEL, dlg)
        rel = lambda a, b: np.abs(a - b) / np.maximum(1.0, np.abs(b))

        def vrel(a, b):
            sc = np.maximum(1.0, np.abs(b).reshape(b.shape[0], -1).max(axis=1))
            return float((np.abs(a - b).reshape(b.shape[0], -1).max(axis=1) / sc).max())
        result[precision]["error_vs_oracle"] = {
            "logpsi_rel_max": float(rel(ev["logpsi"][idx], ref["logpsi"]).max()),
            "eloc_abs_max_Ha": float(el.max()), "eloc_abs_median_Ha": float(np.median(el)),
            "eloc_abs_p99_Ha": float(np.percentile(el, 99)),
            "eloc_rel_max": float(rel(ev["eloc"][idx], ref["eloc"]).max()),
            "eloc_magnitude_max_Ha": float(np.abs(ref["eloc"]).max()),
            # per-walker vectors: error relative to the walker's largest
            # component (components span several orders of magnitude)
            "grad_rel_max": vrel(ev["grad"][idx], ref["grad"]),
            "dEL_rel_max": vrel(pw[idx, 0], dEL) if with_f else None,
            "dlogpsi_rel_max": vrel(pw[idx, 1], dlg) if with_f else None,
            "force_estimator_abs_max_Ha_per_bohr": float(np.abs(Fg - Fo).max()) if with_f else None,
            "force_estimator_rel_max": float((np.abs(Fg - Fo) / np.maximum(1.0, np.abs(Fo))).max()) if with_f else None,
            "forces_compared": bool(with_f),
            "sample": f"{len(idx)} walkers of the final population, state as propagated (no recompute)"}
        if precision == "mixed" and with_f:
            # the same walkers after an FP64 rebuild of their state (inverse
            # and gradient cache recomputed, stored in FP32): separates the
            # drift of the propagated FP32 state from the rounding of the
            # force kernels themselves
            g.set_walkers(Rg[idx])
            _, pw2 = g.forces()
            ev2 = g.eval_cached()
            Fg2 = O.force_estimator(ev2["eloc"], pw2[:, 0], pw2[:, 1])
            mag = np.abs(pw2[:, 0]).max()
            result[precision]["error_vs_oracle"]["after_fp64_rebuild"] = {
                "dEL_rel_max": vrel(pw2[:, 0], dEL), "dlogpsi_rel_max": vrel(pw2[:, 1], dlg),
                "force_estimator_abs_max_Ha_per_bohr": float(np.abs(Fg2 - Fo).max()),
                "eloc_rel_max": float(rel(ev2["eloc"], ref["eloc"]).max()),
                "dEL_magnitude_max": float(mag),
                "fp32_rounding_of_largest_dEL_Ha_per_bohr": float(mag) * 2.0 ** -24}
        rc = time_recompute(Q, g, s, Rg, wl.recompute_period, args.steps, sec / max(1, args.steps), live)
        if rc is not None:
            rc["value_with_recompute_amortised"] = moves_all / (sec + rc["ms"] / 1e3 * args.steps / rc["period_steps"])
        result[precision]["recompute"] = rc
        g.close()

    primary = result[wl.precision]
    # space-warped forces (same step, warped ionic derivatives): throughput,
    # error against the oracle's warped derivatives and the variance cut of
    # the per-walker force samples, both forms of the derivatives taken by
    # the GPU at the same walkers
    warp = None
    if wl.forces and not args.no_space_warp:
        g = make(wl.precision, space_warp=True)
        e_v = equilibrate(g)
        ms, out, fam, clk, W_before = timed(g, wl.precision + "_warp", e_v)
        entering = np.concatenate([[W_before], out["pop"][:-1]])
        sec = max_over_ranks(ms / 1e3, dist)
        Rg, _ = g.get_walkers()
        ev = g.eval_cached()
        _, pw = g.forces()
        g0 = make(wl.precision)
        g0.set_walkers(Rg)
        _, pw0 = g0.forces()
        g0.close()
        E = ev["eloc"] - ev["eloc"].mean()
        var = lambda p: (-p[:, 0] - 2.0 * E[:, None, None] * p[:, 1]).var(axis=0)
        ratio = var(pw0) / np.maximum(var(pw), 1e-300)
        # the oracle's forward-mode electron derivatives of a 10^4-determinant
        # expansion take minutes per walker: compared by the tests there
        idx = np.linspace(0, Rg.shape[0] - 1, 8 if s.n_elec <= 60 else 2).astype(int)
        vrel = lambda a, b: float((np.abs(a - b).reshape(b.shape[0], -1).max(axis=1)
                                   / np.maximum(1.0, np.abs(b).reshape(b.shape[0], -1).max(axis=1))).max())
        if s.n_det <= 1000:
            dELw, dlgw = O.Oracle(s).warped_forces(Rg[idx])
            werr = {"dEL_rel_max": vrel(pw[idx, 0], dELw), "dlogpsi_rel_max": vrel(pw[idx, 1], dlgw),
                    "sample": f"{len(idx)} walkers of the final population"}
        else:
            werr = None
        warp = {"value": sum_over_ranks(float(entering.sum()) * s.n_elec, dist) / sec,
                "force_evals_per_s": sum_over_ranks(float(entering.sum()), dist) / sec,
                "ms_per_step": ms / args.steps, "kernel_ms_per_step": {k: v[0] / args.steps for k, v in fam.items()},
                "force_sample_variance_reduction": {"median": float(np.median(ratio)), "min": float(ratio.min()),
                                                    "max": float(ratio.max())},
                "error_vs_oracle": werr,
                "clocks": clk}
        g.close()
    # end-to-end: host walkers in, K DMC steps with forces, walkers/energies/forces out
    e2e = None
    if not args.no_e2e:
        import torch
        g = make(wl.precision)
        e_v = equilibrate(g)
        Rh = torch.from_numpy(np.ascontiguousarray(g.get_walkers()[0])).pin_memory()
        Wh = Rh.shape[0]
        g.dmc(args.warmup, tau, e_v, forces_every=1 if wl.forces else 0)
        Rout = torch.empty((3 * Wh, s.n_elec, 3), dtype=torch.float64).pin_memory()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        Q.qmc_set_walkers(g.h, Rh.numpy())
        out = g.dmc(args.steps, tau, e_v, forces_every=1 if wl.forces else 0)
        Wn = g.n_walkers
        Q.qmc_get_walkers(g.h, Rout[:Wn].numpy(), None)
        F, Fe = g.force_estimate(Q.QMC_EST_DMC) if wl.forces else (None, None)
        dt = time.perf_counter() - t0
        entering = np.concatenate([[Wh], out["pop"][:-1]])
        moves = float(entering.sum()) * s.n_elec
        sec = max_over_ranks(dt, dist)
        h2d = Wh * s.n_elec * 3 * 8 / args.steps
        d2h = (Wn * s.n_elec * 3 * 8 + 2 * 3 * s.n_nuc * 8 + 3 * 8 * args.steps) / args.steps
        e2e = {"value": sum_over_ranks(moves, dist) / sec, "unit": "electron-moves/s",
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
               "what": f"qmc_set_walkers from pinned host memory, {args.steps} DMC steps with forces, "
                       "walkers + force estimate back to host; wall clock"}
        g.close()

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline(s, R0, tau, primary["e_step_mean"])
    return s, wl, W, primary, result, e2e, cpu, peaks, warp


BATCH_WORKLOAD = "batch64_uneven"


def batch_systems(synth, n_systems):
    """64 water clusters of seeded sizes U{1..16} (10-160 electrons), each
    with its own seeded geometry."""
    sizes = synth.uneven_cluster_sizes(n_systems)
    return sizes, [synth.water_system(int(m), geom_seed=synth.SEED_GEOMETRY + 100 + i) for i, m in enumerate(sizes)]


def run_batch(args, rank, dist):
    """Batched uneven systems: every kernel family one persistent launch over
    all systems, one CUDA graph per step, autotuned sweep configuration.
    Mixed precision is the primary form; the FP64 form runs beside it."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2504_07948_gb300 import qmc as Q, synth
    from oracle import oracle as O

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    n_sys = 64
    W = args.walkers or 256
    sizes, systems = batch_systems(synth, n_sys)
    tau = 0.005
    stream = torch.cuda.current_stream()
    result = {}
    for precision in (["mixed", "fp64"] if not args.only_primary else ["mixed"]):
        members = []
        for i, s in enumerate(systems):
            g = Q.QMC(s, precision=precision, recompute_period=100, seed=synth.SEED_WALKERS + 1000 * rank + i,
                      stream=stream.cuda_stream, cap_factor=4, fixed_population=not args.birth_death)
            g.set_walkers(synth.initial_walkers(s, W, seed=synth.SEED_WALKERS + 1000 * rank + i))
            members.append(g)
        batch = Q.Batch(members)
        batch.vmc(args.vmc_sweeps, 0.05)
        tuned = batch.autotune(tau)
        e0 = np.array([float(np.mean(g.eval_cached()["eloc"])) for g in members])
        out = batch.dmc(args.warmup, tau, e0, forces_every=1)
        et = out["e_step"][-1]
        pops0 = np.array([g.n_walkers for g in members])
        for g in members:
            Q.qmc_reset_estimators(g.h)
        clocks = ClockSampler(os.path.join(CLOCK_DIR, f"clocks_batch_{precision}_r{rank}.csv"))
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        with clocks:
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            out = batch.dmc(args.steps, tau, et, forces_every=1)
            ev1.record(stream)
            torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        ms = ev0.elapsed_time(ev1)
        _, launches = Q.qmc_batch_get_timing(batch.b, "all")
        entering = np.vstack([pops0[None, :], out["pop"][:-1]])          # [steps, n_sys]
        n_elec = np.array([s.n_elec for s in systems], dtype=float)
        moves = float((entering * n_elec[None, :]).sum())
        fevals = float(entering.sum())
        sec = max_over_ranks(ms / 1e3, dist)
        # per-family device time from plain launches of the same steps
        Q.qmc_batch_set_timing(batch.b, True)
        out_t = batch.dmc(2, tau, out["e_step"][-1], forces_every=1)
        fam = {f: Q.qmc_batch_get_timing(batch.b, f) for f in ("sweep", "eloc", "force", "branch", "recompute")}
        Q.qmc_batch_set_timing(batch.b, False)
        ent_t = np.vstack([out["pop"][-1][None, :], out_t["pop"][:-1]])
        flops = 0.0
        flops_exec = 0.0
        live_w = 0.0
        for q, sq in enumerate(systems):
            n = max(sq.n_up, sq.n_dn)
            lf = live_basis_fraction(sq, members[q].get_walkers()[0], max_walkers=16)
            live_w += lf * float(ent_t[:, q].sum()) * sq.n_elec * sq.n_basis
            flops += float(ent_t[:, q].sum()) * sq.n_elec * (sweep_flops_per_move(sq) + 4.0 * n * n * 0.5)
            flops_exec += float(ent_t[:, q].sum()) * sq.n_elec * (sweep_flops_per_move(sq, lf) + 4.0 * n * n * 0.5)
        live_w /= max(1.0, sum(float(ent_t[:, q].sum()) * sq.n_elec * sq.n_basis for q, sq in enumerate(systems)))
        sweep_s = fam["sweep"][0] / 1e3
        ach = flops / sweep_s / 1e12 if sweep_s > 0 else 0.0
        ach_exec = flops_exec / sweep_s / 1e12 if sweep_s > 0 else 0.0
        peak = FP64_PEAK_TFLOPS_NOMINAL if precision == "fp64" else FP32_PEAK_TFLOPS_NOMINAL
        traffic, traffic_note = profiled_traffic(BATCH_WORKLOAD, precision, float(ent_t.sum(axis=1).mean()))
        # accuracy: propagated state of the two smallest and the two largest
        # members (the batched kernels' n <= 64 and n > 64 paths) against the oracle
        errs = []
        order = np.argsort(sizes)
        for q in list(order[:2]) + list(order[-2:]):
            g = members[q]
            Rg, _ = g.get_walkers()
            ev = g.eval_cached()
            idx = np.linspace(0, Rg.shape[0] - 1, 4).astype(int)
            ref = O.Oracle(systems[q]).evaluate(Rg[idx])
            errs.append((float(np.max(np.abs(ev["logpsi"][idx] - ref["logpsi"]) / np.maximum(1, np.abs(ref["logpsi"])))),
                         float(np.max(np.abs(ev["eloc"][idx] - ref["eloc"]))),
                         float(np.max(np.abs(ev["eloc"][idx] - ref["eloc"]) / np.maximum(1, np.abs(ref["eloc"]))))))
        result[precision] = {
            "value": sum_over_ranks(moves, dist) / sec, "force_evals_per_s": sum_over_ranks(fevals, dist) / sec,
            "ms_per_step": ms / args.steps, "gpu_launches": launches,
            "kernel_ms_per_step": {k: v[0] / 2 for k, v in fam.items()},
            "roofline": {"kernel": "k_sweep_batch", "bound": "alu", "achieved": ach, "peak": peak,
                         "unit": "TFLOP/s", "frac": ach / peak,
                         "flops_counted": "per move 10 n N_b (dense contraction) + 14 n, + 4 n^2 per accepted move "
                                          "at acceptance 1/2",
                         "live_basis_fraction": live_w, "achieved_executed": ach_exec, "frac_executed": ach_exec / peak,
                         "executed_counted": "the contraction over the live basis rows only (per member, estimated at "
                                             "its final walker positions)",
                         "traffic": traffic,
                         "traffic_unit": "bytes per launch", "traffic_source": traffic_note,
                         "peak_source": "nominal FP64 1.25 TFLOP/s (recipe table)" if precision == "fp64"
                         else "nominal FP32 FMA rate, 152 SMs x 128 lanes x 2.07 GHz"},
            "autotune": {k: v for k, v in tuned.items() if k != "per_system"},
            "delayed_systems": int(sum(1 for k, _ in tuned["per_system"] if k > 1)),
            "clocks": clocks.summary(int(os.environ.get("LOCAL_RANK", "0"))),
            "error_vs_oracle": {"logpsi_rel_max": max(e[0] for e in errs), "eloc_abs_max_Ha": max(e[1] for e in errs),
                                "eloc_rel_max": max(e[2] for e in errs),
                                "sample": "4 walkers of each of the 2 smallest and the 2 largest members, state as "
                                          "propagated"},
            "population_last": int(out["pop"][-1].sum()),
        }
        if precision == "mixed" and not args.no_e2e:
            # end to end through the C ABI with host buffers: every member's
            # walkers in from pinned host memory, K batched DMC steps with
            # forces, walkers and force estimates back to the host
            Rh = [torch.from_numpy(np.ascontiguousarray(g.get_walkers()[0])).pin_memory() for g in members]
            Ro = [torch.empty((4 * r.shape[0], r.shape[1], 3), dtype=torch.float64).pin_memory() for r in Rh]
            et2 = np.array([float(v) for v in out["e_step"][-1]])
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for g, r in zip(members, Rh):
                Q.qmc_set_walkers(g.h, r.numpy())
            out2 = batch.dmc(args.steps, tau, et2, forces_every=1)
            for g, r in zip(members, Ro):
                Wn = g.n_walkers
                Q.qmc_get_walkers(g.h, r[:Wn].numpy(), None)
                g.force_estimate(Q.QMC_EST_DMC)
            dt = time.perf_counter() - t0
            ent2 = np.vstack([np.array([r.shape[0] for r in Rh])[None, :], out2["pop"][:-1]])
            moves2 = float((ent2 * n_elec[None, :]).sum())
            h2d = sum(r.numel() * 8 for r in Rh) / args.steps
            d2h = (sum(int(g.n_walkers) * s.n_elec * 3 * 8 + 2 * 3 * s.n_nuc * 8 for g, s in zip(members, systems))
                   + 2 * 8 * n_sys * args.steps) / args.steps
            result[precision]["e2e"] = {
                "value": sum_over_ranks(moves2, dist) / max_over_ranks(dt, dist), "unit": "electron-moves/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "what": f"qmc_set_walkers of all {n_sys} members from pinned host memory, {args.steps} batched DMC "
                        "steps with forces, walkers and DMC force estimates back to host; wall clock"}
        batch.close()
        for g in members:
            g.close()
    prim = result["mixed"]
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        mid = int(np.argsort(sizes)[n_sys // 2])
        sm = systems[mid]
        cpu = cpu_baseline(sm, synth.initial_walkers(sm, 64), tau, -76.0 * int(sizes[mid]))
        cpu["sample"] = f"member {mid} ({int(sizes[mid])} waters): " + cpu["sample"]
    line = {
        "metric": METRIC,
        "value": prim["value"], "unit": "electron-moves/s", "n_gpus": (dist.get_world_size() if dist else 1),
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": prim["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": BATCH_WORKLOAD, "n_systems": n_sys, "waters_per_system": [int(m) for m in sizes],
                   "walkers_per_system": W, "walkers_per_gpu": W * n_sys, "tau": tau, "forces": True,
                   "precision": "mixed", "recompute_period": 100, "graph": True,
                   "l2": "inputs larger than L2 (walker state of 64 systems)"},
        "force_evals_per_s": prim["force_evals_per_s"], "roofline": prim["roofline"],
        "gpu_launches": prim["gpu_launches"], "kernel_ms_per_step": prim["kernel_ms_per_step"],
        "clocks": prim["clocks"], "error_vs_oracle": prim["error_vs_oracle"], "autotune": prim["autotune"],
        "e2e": None, "cpu_baseline": cpu,
    }
    if "fp64" in result:
        f = result["fp64"]
        line["fp64"] = {k: f[k] for k in ("value", "force_evals_per_s", "ms_per_step", "roofline", "kernel_ms_per_step",
                                           "error_vs_oracle", "autotune", "clocks")}
        line["mixed_speedup_vs_fp64"] = prim["value"] / f["value"]
    line["e2e"] = prim.get("e2e")
    return line


PP_WORKLOAD = "water32_pp_mixed"
PP_FORCE_WORKLOAD = "water6_pp_forces"


def nlpp_counts(s, R):
    """(electrons within a cutoff, electron-nucleus pairs) per walker, means
    over the walkers R [W, N, 3]."""
    cut = np.asarray(s.pp_rcut)
    nl = sorted({int(a) for a, l in zip(s.pp_nuc, s.pp_l) if l >= 0 and cut[a] > 0})
    d = np.linalg.norm(R[:, :, None, :] - np.asarray(s.R)[nl][None, None], axis=-1) < cut[nl][None, None]
    return float(d.any(axis=2).sum(axis=1).mean()), float(d.sum(axis=(1, 2)).mean())


def run_pp_workload(args, rank, dist, name=PP_WORKLOAD):
    """A valence-only cluster with the semi-local pseudopotential: the
    32-water cluster (mixed form, delayed walker-tiled sweep, no forces) or
    the 6-water cluster with forces every step: electron-moves/s (and
    force-evals/s) with the non-local energy evaluated after every sweep,
    that kernel's share and counted rate, E_L (and the per-walker ionic
    derivatives) against the oracle on sampled walkers at the same quadrature
    rotations, end-to-end through the C ABI and the oracle's CPU rate on a
    bounded sample."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2504_07948_gb300 import qmc as Q, synth
    from oracle import oracle as O
    wl = synth.WORKLOADS[name]
    s = workload_system(synth, wl)
    W = args.walkers or wl.n_walkers
    fe = 1 if wl.forces else 0
    seed = synth.SEED_WALKERS + rank
    R0 = synth.initial_walkers(s, W, seed=seed)
    stream = torch.cuda.current_stream()

    def make():
        g = Q.QMC(s, precision="mixed", recompute_period=wl.recompute_period, seed=seed, stream=stream.cuda_stream,
                  cap_factor=4, delay_rank=wl.delay_rank, fixed_population=not args.birth_death)
        g.set_walkers(R0)
        return g

    g = make()
    e_v = float(g.vmc(args.vmc_sweeps, 0.05, trace=True)[-max(1, args.vmc_sweeps // 2):].mean())
    out = g.dmc(args.warmup, wl.tau, e_v, forces_every=fe)
    et = float(out["e_trial"][-1])
    W_before = g.n_walkers
    Q.qmc_set_timing(g.h, True)
    clocks = ClockSampler(os.path.join(CLOCK_DIR, f"clocks_pp_r{rank}.csv"))
    torch.cuda.synchronize()
    with clocks:
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        out = g.dmc(args.steps, wl.tau, et, forces_every=fe)
        ev1.record(stream)
        torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    fam = {f: Q.qmc_get_timing(g.h, f) for f in ("sweep", "sweep_gemm", "eloc", "nlpp", "force", "branch",
                                                 "recompute", "reduce", "all")}
    Q.qmc_set_timing(g.h, False)
    entering = np.concatenate([[W_before], out["pop"][:-1]])
    moves = float(entering.sum()) * s.n_elec
    Rg, _ = g.get_walkers()
    n_in, n_pairs = nlpp_counts(s, Rg[:256])
    n = max(s.n_up, s.n_dn)
    nq = len(s.pp_qw)
    # counted work of the non-local pass: u_k = C A^-1 e_k per electron in
    # range (2 n N_b) and the dot chi(r') . u_k per quadrature point (2 N_b)
    flops_walker = n_in * 2.0 * n * s.n_basis + n_pairs * nq * 2.0 * s.n_basis
    # one non-local evaluation per DMC step: from 64 electrons per spin u_k
    # comes from tensor-core GEMMs launched inside the same timed span, and
    # the walkers run in slices of at most 2 GB of u_k rows (one k_nlpp
    # launch per slice), so the time and traffic are per evaluation
    nl_ms, nl_n = fam["nlpp"]
    tr_nl, tr_note = profiled_traffic(name, "nlpp", float(entering.mean()))
    nl_s = nl_ms / 1e3 / max(1, args.steps)
    ach = flops_walker * float(entering.mean()) / nl_s / 1e12 if nl_s > 0 else 0.0
    tc_rows = n >= 64 and s.n_up % 4 == 0 and s.n_dn % 4 == 0
    # accuracy: E_L of the propagated state (rotations at a pinned counter)
    # against the oracle on two sampled walker slots
    t_pin = 1_000_000
    Q.qmc_set_rng(g.h, seed, t_pin)
    ev = g.eval_cached()
    o = O.Oracle(s)
    errs, ferrs = [], []
    if wl.forces:
        _, pw = g.forces()
    for slot in (0, Rg.shape[0] // 2):
        ref = o.evaluate(Rg[slot:slot + 1], pp_seed=seed, pp_sweep=t_pin, pp_slot0=slot)["eloc"][0]
        errs.append((abs(ev["eloc"][slot] - ref), abs(ref)))
        if wl.forces:
            dE, _ = o.forces(Rg[slot:slot + 1], pp_seed=seed, pp_sweep=t_pin, pp_slot0=slot)
            ferrs.append(float(np.abs(pw[slot, 0] - dE[0]).max() / max(1.0, np.abs(dE[0]).max())))
    rc = time_recompute(Q, g, s, Rg, wl.recompute_period, args.steps, ms / 1e3 / max(1, args.steps))
    if rc is not None:
        rc["value_with_recompute_amortised"] = moves / (ms / 1e3 + rc["ms"] / 1e3 * args.steps / rc["period_steps"])
    g.close()
    # end to end: walkers from pinned host memory, K DMC steps, walkers and
    # step energies back to the host
    e2e = None
    if not args.no_e2e:
        g = make()
        g.vmc(2, 0.05)
        Rh = torch.from_numpy(np.ascontiguousarray(g.get_walkers()[0])).pin_memory()
        Wh = Rh.shape[0]
        Rout = torch.empty((3 * Wh, s.n_elec, 3), dtype=torch.float64).pin_memory()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        Q.qmc_set_walkers(g.h, Rh.numpy())
        o2 = g.dmc(args.steps, wl.tau, et, forces_every=fe)
        Wn = g.n_walkers
        Q.qmc_get_walkers(g.h, Rout[:Wn].numpy(), None)
        if fe:
            g.force_estimate(Q.QMC_EST_DMC)
        dt = time.perf_counter() - t0
        ent = np.concatenate([[Wh], o2["pop"][:-1]])
        e2e = {"value": float(ent.sum()) * s.n_elec / dt, "unit": "electron-moves/s",
               "h2d_bytes_per_step": Wh * s.n_elec * 3 * 8 / args.steps,
               "d2h_bytes_per_step": (Wn * s.n_elec * 3 * 8 + 3 * 8 * args.steps +
                                      (2 * 3 * s.n_nuc * 8 if fe else 0)) / args.steps,
               "what": f"qmc_set_walkers from pinned host memory, {args.steps} DMC steps (E_L with the "
                       f"non-local term every step{', forces every step' if fe else ''}), walkers, step energies"
                       f"{' and the force estimate' if fe else ''} back to host; wall clock"}
        g.close()
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline(s, R0, wl.tau, float(out["e_step"].mean()), forces=bool(fe), max_walkers=8)
    return {
        "config": {"n_water": wl.n_water, "valence_electrons": s.n_elec, "walkers_per_gpu": W,
                   "precision": "mixed", "delay_rank": wl.delay_rank, "recompute_period": wl.recompute_period,
                   "tau": wl.tau, "forces": bool(wl.forces), "quadrature_points": nq,
                   "pseudopotential": "synthetic semi-local Gaussian-expansion potential on every O (2 core "
                                      "electrons removed), s and p projectors, cutoff 1.6 bohr"},
        "value": moves / (ms / 1e3), "unit": "electron-moves/s", "ms_per_step": ms / args.steps,
        "force_evals_per_s": float(entering.sum()) / (ms / 1e3) if fe else None,
        "kernel_ms_per_step": {k: v[0] / args.steps for k, v in fam.items()},
        "gpu_launches": fam["all"][1],
        "recompute": rc,
        "roofline_nlpp": {"kernel": "k_nlpp" + (" with u_k from k_tc_gemm_pipe (3xTF32)" if tc_rows else ""),
                          "bound": "alu", "achieved": ach, "peak": FP32_PEAK_TFLOPS_NOMINAL,
                          "unit": "TFLOP/s", "frac": ach / FP32_PEAK_TFLOPS_NOMINAL,
                          "ms_per_evaluation": nl_s * 1e3, "launches_per_evaluation": nl_n / max(1, args.steps),
                          "electrons_in_range_per_walker": n_in, "pairs_per_walker": n_pairs,
                          "traffic": tr_nl, "traffic_source": tr_note,
                          "traffic_unit": "bytes per evaluation (the k_nlpp launches" +
                                          ("; the u_k GEMMs' operands and rows not included)" if tc_rows else ")"),
                          "flops_counted": "per electron in range 2 n N_b (u_k = C A^-1 e_k), per quadrature "
                                           "point 2 N_b (chi(r') . u_k); basis exponentials and Jastrow terms "
                                           "not counted",
                          "peak_source": "nominal FP32 FMA rate, 152 SMs x 128 lanes x 2.07 GHz"},
        "error_vs_oracle": {"eloc_abs_max_Ha": max(e for e, _ in errs),
                            "eloc_rel_max": max(e / max(1.0, m) for e, m in errs),
                            "dEL_rel_max": max(ferrs) if ferrs else None,
                            "sample": "2 walker slots of the final population, state as propagated, rotations "
                                      "at a pinned counter on both sides"},
        "clocks": clocks.summary(int(os.environ.get("LOCAL_RANK", "0"))),
        "e2e": e2e, "cpu_baseline": cpu}


def run_workloads(args, rank, ws, dist):
    """The larger configurations beside the default line: the 32-water
    cluster in the mixed form with delayed updates (4096 walkers), the batch
    of 64 uneven clusters (mixed and FP64 forms) and the valence-only
    32-water cluster with pseudopotentials, each with its own roofline,
    oracle CPU baseline and end-to-end figure."""
    out = {}
    a2 = argparse.Namespace(**vars(args))
    a2.workload, a2.only_primary, a2.no_space_warp, a2.walkers = "water32_mixed", True, True, 0
    _, wl2, W2, prim2, _, e2e2, cpu2, _, _ = run_gpu(a2, rank, ws, dist)
    out["water32_mixed"] = {
        "config": {"n_water": wl2.n_water, "walkers_per_gpu": W2, "precision": wl2.precision,
                   "delay_rank": wl2.delay_rank, "recompute_period": wl2.recompute_period, "tau": wl2.tau,
                   "forces": wl2.forces},
        "value": prim2["value"], "unit": "electron-moves/s", "force_evals_per_s": prim2["force_evals_per_s"],
        "ms_per_step": prim2["ms_per_step"], "kernel_ms_per_step": prim2["kernel_ms"],
        "gpu_launches": prim2["gpu_launches"], "roofline": prim2["roofline"],
        "roofline_force": prim2.get("roofline_force"),
        "error_vs_oracle": prim2.get("error_vs_oracle"), "recompute": prim2.get("recompute"),
        "clocks": prim2["clocks"], "e2e": e2e2, "cpu_baseline": cpu2}
    a4 = argparse.Namespace(**vars(args))
    a4.workload, a4.walkers = BATCH_WORKLOAD, 0
    line4 = run_batch(a4, rank, dist)
    out[BATCH_WORKLOAD] = {k: v for k, v in line4.items() if k not in ("metric", "n_gpus", "steps", "warmup",
                                                                       "higher_is_better", "scaling", "vs_baseline",
                                                                       "data")}
    out[PP_WORKLOAD] = run_pp_workload(args, rank, dist)
    out[PP_FORCE_WORKLOAD] = run_pp_workload(args, rank, dist, PP_FORCE_WORKLOAD)
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="water6_fp64_forces")
    ap.add_argument("--walkers", type=int, default=0)
    ap.add_argument("--vmc-sweeps", type=int, default=20)
    ap.add_argument("--birth-death", action="store_true",
                    help="birth/death population control instead of the fixed population")
    ap.add_argument("--only-primary", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--error-sample", type=int, default=64)
    ap.add_argument("--no-space-warp", action="store_true",
                    help="skip the space-warped force measurement")
    ap.add_argument("--no-workloads", action="store_true",
                    help="skip the 32-water and batched-cluster entries of the default line")
    args = ap.parse_args()
    assert args.warmup >= 3 or args.impl == "reference", "at least 3 warm-up steps"
    rank, ws, dist = dist_init()

    if args.impl == "reference":
        if rank != 0:
            return
        from paper_2504_07948_gb300 import synth
        wl = synth.WORKLOADS[args.workload]
        s = workload_system(synth, wl)
        R0 = synth.initial_walkers(s, args.walkers or wl.n_walkers)
        from oracle import oracle as O
        O.build()
        t_all, moves_all, fe_all = 0.0, 0.0, 0.0
        o = O.Oracle(s)
        Wsamp = max(o.nthreads, 4)
        e_guess = float(np.mean(o.evaluate(R0[:Wsamp])["eloc"]))
        for k in range(args.warmup + args.steps):
            t0 = time.perf_counter()
            out = o.dmc(R0[:Wsamp], 1, wl.tau, e_guess, seed=99 + k, step0=k, cap_factor=4,
                        forces_every=1 if wl.forces else 0)
            dt = time.perf_counter() - t0
            if k >= args.warmup:
                t_all += dt
                moves_all += Wsamp * s.n_elec
                fe_all += Wsamp
        line = {"impl": "reference", "metric": METRIC, "value": moves_all / t_all,
                "unit": "electron-moves/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": 1e3 * t_all / args.steps, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": args.workload, "walkers_per_step_sample": Wsamp,
                           "n_electrons": s.n_elec, "n_basis": s.n_basis, "n_nuclei": s.n_nuc},
                "force_evals_per_s": fe_all / t_all,
                "cpu_baseline": {"value": moves_all / t_all, "unit": "electron-moves/s", "cores": o.nthreads,
                                 "kind": "oracle",
                                 "sample": f"each step: one DMC step with forces of {Wsamp} walkers of the workload"},
                "e2e": {"value": moves_all / t_all, "unit": "electron-moves/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    if args.workload == BATCH_WORKLOAD:
        line = run_batch(args, rank, dist)
        if rank == 0:
            print(json.dumps(line))
        return
    if args.workload in (PP_WORKLOAD, PP_FORCE_WORKLOAD):
        r = run_pp_workload(args, rank, dist, args.workload)
        if rank == 0:
            line = {"metric": METRIC, "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                    "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
                    "data": "synthetic", **r}
            line["config"] = {"workload": args.workload, **r["config"]}
            print(json.dumps(line))
        return
    s, wl, W, primary, result, e2e, cpu, peaks, warp = run_gpu(args, rank, ws, dist)
    workloads = None
    if not args.no_workloads and ws == 1:
        workloads = run_workloads(args, rank, ws, dist)
    if rank != 0:
        return
    line = {
        "metric": METRIC,
        "value": primary["value"], "unit": "electron-moves/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": primary["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if wl.precision == "fp64" else "f32+f64",
        "data": "synthetic",
        "config": {"workload": args.workload, "n_water": wl.n_water, "n_electrons": s.n_elec,
                   "n_nuclei": s.n_nuc, "n_basis": s.n_basis, "walkers_per_gpu": W, "tau": wl.tau,
                   "forces": wl.forces, "precision": wl.precision, "delay_rank": wl.delay_rank,
                   "recompute_period": wl.recompute_period, "n_det": wl.n_det,
                   "population_control": "birth-death" if args.birth_death else "fixed (systematic resampling)",
                   "l2": "inputs larger than L2 (walker state ~150 MB per buffer at 2048 walkers FP64)"},
        "force_evals_per_s": primary["force_evals_per_s"],
        "roofline": primary["roofline"],
        "roofline_force": primary.get("roofline_force"),
        "gpu_launches": primary["gpu_launches"],
        "kernel_ms_per_step": primary["kernel_ms"],
        "clocks": primary["clocks"],
        "acceptance": primary["acceptance"],
        "population_last": primary["population_last"],
        "error_vs_oracle": primary.get("error_vs_oracle"),
        "recompute": primary.get("recompute"),
        "e2e": e2e,
        "cpu_baseline": cpu,
        "space_warp": warp,
        "workloads": workloads,
    }
    if "mixed" in result and wl.precision == "fp64":
        m = result["mixed"]
        line["mixed"] = {"value": m["value"], "force_evals_per_s": m["force_evals_per_s"],
                         "ms_per_step": m["ms_per_step"], "speedup_vs_fp64": m["value"] / primary["value"],
                         "roofline": m["roofline"], "roofline_force": m.get("roofline_force"),
                         "kernel_ms_per_step": m["kernel_ms"],
                         "error_vs_oracle": m.get("error_vs_oracle"), "recompute": m.get("recompute"),
                         "clocks": m["clocks"]}
    print(json.dumps(line))


if __name__ == "__main__":
    main()
