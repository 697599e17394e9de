// Batches of independent systems (different molecules, electron counts and
// populations) stepped together: every kernel family of a DMC step runs as
// one persistent launch over the work items of all systems, and the step's
// launches are captured in one CUDA graph.
//
// Work items are counted in three units: walkers, (walker, electron) pairs
// and (walker, spin) pairs.  A plan kernel at the start of every step turns
// the current populations into prefix offsets per unit; persistent CTAs then
// take items from a counter (dynamic scheduling) and find their system by
// binary search over the offsets.  Systems are ordered by decreasing cost per
// walker, so the largest items are taken first and the smallest fill the
// tail.
#pragma once

#include "qmc_internal.cuh"

namespace qmc {

constexpr int kMaxBatchSystems = 1024;
constexpr int kBatchCounters = 16;
constexpr int kBatchHist = 20;   // energies kept for the trial-energy estimate

enum BatchUnit : int { kUnitWalker = 0, kUnitElectron = 1, kUnitSpin = 2, kUnitCount = 3 };

// One system of a batch as the batched kernels see it (device memory).
struct BatchSys {
    DevSys s;
    DevWalkers wk[2];
    uint2 key;             // RNG key of the system
    int cap;               // walker capacity of each buffer
    int delay_rank;        // 1: Sherman-Morrison sweep, > 1: delayed updates
    int ainv_smem;         // the Sherman-Morrison sweep keeps A^-1 in shared memory
    int elem;              // bytes per stored wavefunction element (4 or 8)
    double* eloc_new;      // [cap]
    double* wts;           // [cap]
    int* copies;           // [cap]
    int* offsets;          // [cap]
    double* dEL;           // [cap][3 n_nuc]
    double* dlog;          // [cap][3 n_nuc]
    double* Bscr;          // [cap][nmax^2] force scratch
    double* Pscr;
    const double* dvnn;    // [3 n_nuc] nuclear-repulsion derivative
    unsigned* err;         // the system's device error flags
    int space_warp;        // the system's ionic derivatives are space-warped
    int pad_;
    double* gEdet;         // [cap][N][3] determinant part of dE_L/dr_i (space warp)
    double* gtot;          // [cap][N][3] grad_i ln|psi| (space warp)
};

// DMC control of one system (device memory, updated by the scan kernel).
struct BatchCtl {
    double e_trial;        // current trial energy
    double e_cut;          // local-energy clipping half-width 0.2 sqrt(N / tau)
    double feedback;       // population feedback 1 / (10 tau)
    double W0;             // target population
    double hist[kBatchHist];
    int n_hist, head;      // ring of the last clipped step energies
    int pop;               // current population
    int status;            // 0 ok, 1 capacity exceeded, 2 population died out
    uint32_t sweep;        // RNG sweep counter of the system
    int fixed_pop;         // > 0: fixed-population resampling to this many walkers
};

struct BatchPlan {
    int n_sys;
    int step;                              // history row of the current step
    int total[kUnitCount];
    unsigned counter[kBatchCounters];      // dynamic-scheduling counters, zeroed per step
    int off[kUnitCount][kMaxBatchSystems + 1];
};

// History row per system and step:
//   [0] sum w, [1] sum w E, [2] new population, [3] capacity exceeded,
//   [4] sum w clip(E), [5] sum w E^2, [6] trial energy after the step,
//   [7] population before the step, then (forces) sum w, sum w E,
//   sum w dE_L/dR [K], sum w E dln|psi|/dR [K], sum w dln|psi|/dR [K].
constexpr int kHistHead = 8;

__device__ __forceinline__ int batch_find(const BatchPlan* plan, int unit, int t) {
    int lo = 0, hi = plan->n_sys - 1;
    while (lo < hi) {   // last system whose offset is <= t
        const int mid = (lo + hi + 1) >> 1;
        if (plan->off[unit][mid] <= t)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// Thread 0 takes the next item of a unit from counter ctr: sys = -1 when
// none is left.
__device__ __forceinline__ void batch_next(BatchPlan* plan, int unit, int ctr, int* sys, int* idx) {
    const int t = (int)atomicAdd(&plan->counter[ctr], 1u);
    if (t >= plan->total[unit]) {
        *sys = -1;
        return;
    }
    const int q = batch_find(plan, unit, t);
    *sys = q;
    *idx = t - plan->off[unit][q];
}

// Cooperative copy of a system descriptor into shared memory.
__device__ __forceinline__ void batch_load(BatchSys* dst, const BatchSys* src) {
    static_assert(sizeof(BatchSys) % 8 == 0, "descriptor size");
    const unsigned long long* s = (const unsigned long long*)src;
    unsigned long long* d = (unsigned long long*)dst;
    for (int q = threadIdx.x; q < (int)(sizeof(BatchSys) / 8); q += blockDim.x) d[q] = s[q];
}

// Launchers (defined next to the bodies they run).  The *_prepare calls set
// a kernel's dynamic shared memory limit and return its resident CTAs per
// SM; they run before any launch (and before graph capture).
template <typename T>
size_t sweep_batch_smem(const DevSys& s, int delay_rank, int ainv_smem);
template <typename T>
int sweep_batch_prepare(int block, size_t smem, int delayed);
template <typename T>
cudaError_t launch_sweep_batch(const BatchSys* sys, BatchPlan* plan, const BatchCtl* ctl, int parity, double tau,
                               int ctr, int grid, int block, size_t smem, int delayed, cudaStream_t st);
int wf_batch_prepare(int family, int block, size_t smem);
template <typename T>
cudaError_t launch_orbitals_batch(const BatchSys* sys, BatchPlan* plan, int parity, int ctr, int grid, size_t smem,
                                  cudaStream_t st);
cudaError_t launch_invert_batch(const BatchSys* sys, BatchPlan* plan, int parity, int store_fp32, int ctr, int grid,
                                size_t smem, cudaStream_t st);
template <typename T>
cudaError_t launch_eloc_batch(const BatchSys* sys, BatchPlan* plan, int parity, int into_walker, int ctr, int grid,
                              size_t smem, cudaStream_t st);
size_t force_batch_smem_bytes(const DevSys& s, int elem, int space_warp);
template <typename T>
int force_batch_prepare(size_t smem, int any_warp);
template <typename T>
cudaError_t launch_force_batch(const BatchSys* sys, BatchPlan* plan, int parity, int ctr, int grid, size_t smem,
                               int any_warp, cudaStream_t st);
// Space warp of the ionic derivatives of the systems that have it on (the
// others' walker items are skipped).
size_t space_warp_batch_smem_bytes(const DevSys& s, int elem);
template <typename T>
int space_warp_batch_prepare(size_t smem);
template <typename T>
cudaError_t launch_space_warp_batch(const BatchSys* sys, BatchPlan* plan, int parity, int ctr, int grid, size_t smem,
                                    cudaStream_t st);
cudaError_t launch_batch_plan(BatchPlan* plan, const BatchCtl* ctl, const BatchSys* sys, int n_sys, cudaStream_t st);
cudaError_t launch_batch_advance(BatchCtl* ctl, int n_sys, cudaStream_t st);
cudaError_t launch_branch_batch(const BatchSys* sys, BatchPlan* plan, BatchCtl* ctl, int n_sys, int parity,
                                double tau, double* hist, int hist_stride, int forces, int copy_grid,
                                cudaStream_t st);

}  // namespace qmc
