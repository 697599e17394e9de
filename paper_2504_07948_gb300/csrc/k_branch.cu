// Branching step of diffusion Monte Carlo (the projection of Eq. 1 with
// population control, following Reynolds et al. 1982).
//
//   w = exp(-tau [ (E_old + E_new)/2 - E_T ]),  E clipped to E_T +- e_cut,
//   copies = min(floor(w + u), 3), each copy restarts with weight 1.
// Walkers are compacted into a second buffer in source order: the copies of
// walker w occupy slots offsets[w] .. offsets[w] + copies[w] - 1.
#include "batch.cuh"
#include "qmc_internal.cuh"

namespace qmc {

__device__ __forceinline__ void branch_weight(const double* eloc_old, const double* eloc_new, int w, double tau,
                                              double e_trial, double e_cut, uint2 key, uint32_t sweep, int* copies,
                                              double* wts) {
    const double lo = e_trial - e_cut, hi = e_trial + e_cut;
    const double eo = fmin(fmax(eloc_old[w], lo), hi);
    const double en = fmin(fmax(eloc_new[w], lo), hi);
    double wt = exp(-tau * (0.5 * (eo + en) - e_trial));
    if (!isfinite(eloc_new[w])) wt = 0.0;  // a broken walker is dropped
    const double u = draw_uniform(key, sweep, 0xFFFFFFFFu, (uint32_t)w, 2u);
    int m = (int)floor(wt + u);
    copies[w] = m > 3 ? 3 : m;
    wts[w] = wt;
}

__global__ void k_branch_weights(DevWalkers src, int W, const double* eloc_new, BranchParams p, int* copies,
                                 double* wts) {
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= W) return;
    branch_weight(src.eloc, eloc_new, w, p.tau, p.e_trial, p.e_cut, p.key, p.sweep, copies, wts);
}

// Single CTA: exclusive scan of copies, ordered sums of w, w E_new and
// w clip(E_new) (the clipped energy drives the trial-energy feedback).
// fixed_pop > 0: the copies are drawn here instead, by systematic
// resampling of fixed_pop walkers: a comb of fixed_pop teeth with spacing
// sum(w) / fixed_pop and offset uc over the cumulative weights C_w; walker w
// keeps ceil(C_{w+1} / d - uc) - ceil(C_w / d - uc) copies (the counts add up
// to fixed_pop exactly).
// Block-wide exclusive prefix of one value per thread (threads in order),
// with the block total in *total.  blockDim.x is a multiple of 32; sh holds
// 33 entries and is free again on return.  Shuffle scans inside each warp,
// then one warp scans the warp totals: log-depth chains instead of a serial
// walk by one thread (an FP64 add costs the SM's FP64 pipe 64 FP32 adds).
template <typename V>
__device__ __forceinline__ V block_scan_excl(V v, V* sh, V* total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    V x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const V y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[wid] = x;
    __syncthreads();
    if (wid == 0) {
        const V a = lane < nw ? sh[lane] : V(0);
        V t = a;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const V y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        sh[lane] = t - a;
        if (lane == 31) sh[32] = t;
    }
    __syncthreads();
    const V r = sh[wid] + (x - v);
    *total = sh[32];
    __syncthreads();
    return r;
}

__device__ __forceinline__ void branch_scan_block(int W, int* copies, const double* wts, const double* eloc_new,
                                                  double lo, double hi, int cap, int* offsets, double* stats,
                                                  int fixed_pop = 0, double uc = 0.5) {
    __shared__ double s_d[33];
    __shared__ int s_i[33];
    const int t = threadIdx.x, nt = blockDim.x;
    const int chunk = (W + nt - 1) / nt;
    const int b = min(W, t * chunk), e = min(W, b + chunk);
    int c = 0;
    double sw = 0.0, swe = 0.0, swc = 0.0;
    for (int w = b; w < e; ++w) {
        if (!fixed_pop) c += copies[w];
        sw += wts[w];
        if (wts[w] != 0.0) {
            swe += wts[w] * eloc_new[w];
            swc += wts[w] * fmin(fmax(eloc_new[w], lo), hi);
        }
    }
    double tot_w;
    const double pre_w = block_scan_excl<double>(sw, s_d, &tot_w);
    if (fixed_pop) {
        const double d = tot_w / (double)fixed_pop;
        const bool live = tot_w > 0.0 && isfinite(tot_w);   // else every walker was dropped
        double cum = pre_w;
        for (int w = b; w < e; ++w) {
            const double lo_t = ceil(cum / d - uc);
            cum += wts[w];
            const int m = live ? (int)(ceil(cum / d - uc) - lo_t) : 0;
            copies[w] = m;
            c += m;
        }
    }
    int tot_c;
    const int pre_c = block_scan_excl<int>(c, s_i, &tot_c);
    double tot_we, tot_wc;
    block_scan_excl<double>(swe, s_d, &tot_we);
    block_scan_excl<double>(swc, s_d, &tot_wc);
    if (t == 0) {
        stats[0] = tot_w;
        stats[1] = tot_we;
        stats[2] = (double)tot_c;
        stats[3] = tot_c > cap ? 1.0 : 0.0;
        stats[4] = tot_wc;
    }
    int run = pre_c;
    for (int w = b; w < e; ++w) {
        offsets[w] = run;
        run += copies[w];
    }
}

__global__ void k_branch_scan(int W, int* copies, const double* wts, const double* eloc_new, double lo, double hi,
                              int cap, int* offsets, double* stats, int fixed_pop, uint2 key, uint32_t sweep) {
    const double uc = fixed_pop ? draw_uniform(key, sweep, 0xFFFFFFFFu, 0xFFFFFFFFu, 2u) : 0.5;
    branch_scan_block(W, copies, wts, eloc_new, lo, hi, cap, offsets, stats, fixed_pop, uc);
}

// CTA copy of one contiguous array; four loads in flight per thread before
// their stores (the pointers never overlap: two different walker buffers).
template <typename V>
__device__ __forceinline__ void cta_copy_v(V* __restrict__ d, const V* __restrict__ s, size_t n) {
    const size_t step = blockDim.x;
    size_t q = threadIdx.x;
    for (; q + 3 * step < n; q += 4 * step) {
        const V a = s[q], b = s[q + step], c = s[q + 2 * step], e = s[q + 3 * step];
        d[q] = a;
        d[q + step] = b;
        d[q + 2 * step] = c;
        d[q + 3 * step] = e;
    }
    for (; q < n; q += step) d[q] = s[q];
}

__device__ __forceinline__ void cta_copy(void* dst, const void* src, size_t bytes) {
    if ((((uintptr_t)dst | (uintptr_t)src | bytes) & 15) == 0)
        cta_copy_v<uint4>((uint4*)dst, (const uint4*)src, bytes / 16);
    else
        cta_copy_v<uint32_t>((uint32_t*)dst, (const uint32_t*)src, bytes / 4);
}

// Arrays of one walker's state, copied by separate CTAs: 0 positions and the
// scalars, 1-2 A^-1 of each spin, 3-4 the gradient caches, then for a
// determinant expansion five tables per spin.
constexpr int kCopySegs = 15;
__device__ __forceinline__ int copy_segments(const DevSys& s) { return s.msd ? kCopySegs : 5; }

__device__ __forceinline__ void copy_walker_seg(const DevSys& s, const DevWalkers& src, const DevWalkers& dst, int w,
                                                int seg, const int* copies, const int* offsets,
                                                const double* eloc_new, int elem) {
    const int m = copies[w], off = offsets[w];
    const int N = s.N, nu = s.n_up, nd = s.n_dn;
    const size_t a0 = (size_t)nu * nu * elem, a1 = (size_t)nd * nd * elem;
    for (int t = 0; t < m; ++t) {
        const int d = off + t;
        switch (seg) {
            case 0:
                cta_copy(dst.R + (size_t)d * 3 * N, src.R + (size_t)w * 3 * N, sizeof(double) * 3 * N);
                if (threadIdx.x == 0) {
                    dst.logdet[2 * d] = src.logdet[2 * w];
                    dst.logdet[2 * d + 1] = src.logdet[2 * w + 1];
                    dst.sgn[2 * d] = src.sgn[2 * w];
                    dst.sgn[2 * d + 1] = src.sgn[2 * w + 1];
                    dst.eloc[d] = eloc_new[w];
                    dst.weight[d] = 1.0;
                    if (s.msd) dst.Ssum[d] = src.Ssum[w];
                }
                break;
            case 1: cta_copy((char*)dst.Ainv[0] + d * a0, (const char*)src.Ainv[0] + w * a0, a0); break;
            case 2: cta_copy((char*)dst.Ainv[1] + d * a1, (const char*)src.Ainv[1] + w * a1, a1); break;
            case 3: cta_copy((char*)dst.G[0] + d * 4 * a0, (const char*)src.G[0] + w * 4 * a0, 4 * a0); break;
            case 4: cta_copy((char*)dst.G[1] + d * 4 * a1, (const char*)src.G[1] + w * 4 * a1, 4 * a1); break;
            default: {
                if (!s.msd) break;
                const int spin = (seg - 5) / 5, k = (seg - 5) % 5;
                const size_t n = spin ? nd : nu, nv = s.n_vir[spin], ns = s.n_str[spin];
                const size_t ta = n * nv * elem, tr = ns * elem;
                if (k == 0) cta_copy((char*)dst.Av[spin] + d * ta, (const char*)src.Av[spin] + w * ta, ta);
                if (k == 1) cta_copy((char*)dst.Gv[spin] + d * 4 * ta, (const char*)src.Gv[spin] + w * 4 * ta, 4 * ta);
                if (k == 2) cta_copy((char*)dst.Tt[spin] + d * ta, (const char*)src.Tt[spin] + w * ta, ta);
                if (k == 3) cta_copy((char*)dst.Rs[spin] + d * tr, (const char*)src.Rs[spin] + w * tr, tr);
                if (k == 4) cta_copy((char*)dst.Cd[spin] + d * tr, (const char*)src.Cd[spin] + w * tr, tr);
            }
        }
    }
}

// grid (W, segments): one CTA per (source walker, array).
__global__ void k_branch_copy(DevSys s, DevWalkers src, DevWalkers dst, int W, const int* copies,
                              const int* offsets, const double* eloc_new, const double* stats, int elem) {
    const int w = blockIdx.x;
    if (w >= W || stats[3] != 0.0) return;
    copy_walker_seg(s, src, dst, w, blockIdx.y, copies, offsets, eloc_new, elem);
}

cudaError_t launch_branch(const DevSys& s, const DevWalkers& src, const DevWalkers& dst, int W,
                          const double* eloc_new, const BranchParams& p, int* copies, int* offsets, double* wts,
                          double* stats, int elem_bytes, cudaStream_t st) {
    if (W == 0) return cudaSuccess;
    k_branch_weights<<<(W + 255) / 256, 256, 0, st>>>(src, W, eloc_new, p, copies, wts);
    k_branch_scan<<<1, 1024, 0, st>>>(W, copies, wts, eloc_new, p.e_trial - p.e_cut, p.e_trial + p.e_cut, p.cap,
                                      offsets, stats, p.fixed_pop, p.key, p.sweep);
    k_branch_copy<<<dim3(W, s.msd ? kCopySegs : 5), 256, 0, st>>>(s, src, dst, W, copies, offsets, eloc_new, stats,
                                                                  elem_bytes);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------
// Batched systems: plan, branching and per-step estimator sums.
// ---------------------------------------------------------------------

// Prefix offsets of the work items of the step from the current
// populations (systems that stopped contribute none), a new history row and
// zeroed scheduling counters.
__global__ void k_batch_plan(BatchPlan* plan, const BatchCtl* ctl, const BatchSys* sys, int n_sys) {
    if (threadIdx.x < kBatchCounters) plan->counter[threadIdx.x] = 0u;
    if (threadIdx.x != 0) return;
    plan->n_sys = n_sys;
    plan->step += 1;
    int o0 = 0, o1 = 0, o2 = 0;
    for (int q = 0; q < n_sys; ++q) {
        plan->off[kUnitWalker][q] = o0;
        plan->off[kUnitElectron][q] = o1;
        plan->off[kUnitSpin][q] = o2;
        const int pop = ctl[q].status ? 0 : ctl[q].pop;
        o0 += pop;
        o1 += pop * sys[q].s.N;
        o2 += 2 * pop;
    }
    plan->off[kUnitWalker][n_sys] = o0;
    plan->off[kUnitElectron][n_sys] = o1;
    plan->off[kUnitSpin][n_sys] = o2;
    plan->total[kUnitWalker] = o0;
    plan->total[kUnitElectron] = o1;
    plan->total[kUnitSpin] = o2;
}

__global__ void k_branch_weights_batch(const BatchSys* __restrict__ sys, const BatchPlan* plan,
                                       const BatchCtl* __restrict__ ctl, int parity, double tau) {
    const int total = plan->total[kUnitWalker];
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
        const int q = batch_find(plan, kUnitWalker, t);
        const int w = t - plan->off[kUnitWalker][q];
        const BatchSys& b = sys[q];
        branch_weight(b.wk[parity].eloc, b.eloc_new, w, tau, ctl[q].e_trial, ctl[q].e_cut, b.key, ctl[q].sweep,
                      b.copies, b.wts);
    }
}

// One CTA per system: the scan of the single-system path, then the history
// row and the trial-energy update (the mean clipped energy of the last
// kBatchHist steps minus the population feedback), all on the device.
__global__ void k_branch_scan_batch(const BatchSys* __restrict__ sys, const BatchPlan* plan, BatchCtl* ctl,
                                    double* hist, int stride) {
    __shared__ double st[5];
    const int q = blockIdx.x;
    const int W = plan->off[kUnitWalker][q + 1] - plan->off[kUnitWalker][q];
    double* row = hist + ((size_t)plan->step * plan->n_sys + q) * stride;
    const BatchSys& b = sys[q];
    const double et = ctl[q].e_trial, cut = ctl[q].e_cut;
    if (W == 0) {   // stopped system (uniform for the CTA)
        if (threadIdx.x == 0) {
            for (int k = 0; k < kHistHead; ++k) row[k] = 0.0;
            row[6] = et;
            ctl[q].sweep += 1u;
        }
        return;
    }
    const int fixed = ctl[q].fixed_pop;
    const double uc = fixed ? draw_uniform(b.key, ctl[q].sweep, 0xFFFFFFFFu, 0xFFFFFFFFu, 2u) : 0.5;
    branch_scan_block(W, b.copies, b.wts, b.eloc_new, et - cut, et + cut, b.cap, b.offsets, st, fixed, uc);
    if (threadIdx.x == 0) {
        BatchCtl& c = ctl[q];
        const int Wn = (int)st[2];
        row[0] = st[0];
        row[1] = st[1];
        row[2] = st[2];
        row[3] = st[3];
        row[4] = st[4];
        row[7] = (double)W;
        if (st[3] != 0.0) {
            c.status = 1;
        } else if (Wn == 0) {
            c.status = 2;
        } else {
            c.pop = Wn;
            c.hist[c.head] = st[4] / st[0];
            c.head = (c.head + 1) % kBatchHist;
            if (c.n_hist < kBatchHist) ++c.n_hist;
            double est = 0.0;
            for (int k = 0; k < c.n_hist; ++k) est += c.hist[(c.head - c.n_hist + k + kBatchHist) % kBatchHist];
            est /= (double)c.n_hist;
            c.e_trial = c.fixed_pop ? est : est - c.feedback * log((double)Wn / c.W0);
        }
        row[6] = c.e_trial;
        c.sweep += 1u;
    }
}

// Walker copies of every system into the other buffer: items are (source
// walker, array) pairs, one CTA each (batches hold no determinant
// expansions: five arrays per walker).  The descriptor is read in place.
__global__ void k_branch_copy_batch(const BatchSys* __restrict__ sys, const BatchPlan* plan,
                                    const BatchCtl* __restrict__ ctl, int parity) {
    constexpr int kSegs = 5;
    const int total = plan->total[kUnitWalker] * kSegs;
    for (int it = blockIdx.x; it < total; it += gridDim.x) {
        const int t = it / kSegs, seg = it - t * kSegs;
        const int q = batch_find(plan, kUnitWalker, t);
        const int w = t - plan->off[kUnitWalker][q];
        if (ctl[q].status) continue;   // uniform for the CTA
        const BatchSys& b = sys[q];
        copy_walker_seg(b.s, b.wk[parity], b.wk[1 - parity], w, seg, b.copies, b.offsets, b.eloc_new, b.elem);
    }
}

// One CTA per system: sum w E^2 and, with forces, the weighted force sums of
// the walkers before branching (the layout of the single-system estimator).
__global__ void k_batch_reduce(const BatchSys* __restrict__ sys, const BatchPlan* plan, double* hist, int stride,
                               int forces) {
    __shared__ double scratch[kMaxWarps];
    const int q = blockIdx.x;
    const int W = plan->off[kUnitWalker][q + 1] - plan->off[kUnitWalker][q];
    double* row = hist + ((size_t)plan->step * plan->n_sys + q) * stride;
    const BatchSys& b = sys[q];
    double v[1] = {0.0};
    for (int w = threadIdx.x; w < W; w += blockDim.x) v[0] += b.wts[w] * b.eloc_new[w] * b.eloc_new[w];
    block_sum<1>(v, scratch);
    if (threadIdx.x == 0) row[5] = v[0];
    if (!forces) return;
    const int K = 3 * b.s.n_nuc;
    double* f = row + kHistHead;
    for (int k = threadIdx.x; k < 2 + 3 * K; k += blockDim.x) {
        double a = 0.0;
        if (k == 0) {
            for (int w = 0; w < W; ++w) a += b.wts[w];
        } else if (k == 1) {
            for (int w = 0; w < W; ++w) a += b.wts[w] * b.eloc_new[w];
        } else if (k < 2 + K) {
            const int c = k - 2;
            for (int w = 0; w < W; ++w) a += b.wts[w] * b.dEL[(size_t)w * K + c];
        } else if (k < 2 + 2 * K) {
            const int c = k - 2 - K;
            for (int w = 0; w < W; ++w) a += b.wts[w] * b.eloc_new[w] * b.dlog[(size_t)w * K + c];
        } else {
            const int c = k - 2 - 2 * K;
            for (int w = 0; w < W; ++w) a += b.wts[w] * b.dlog[(size_t)w * K + c];
        }
        f[k] = a;
    }
}

// Next RNG sweep of every system (after a sweep without branching).
__global__ void k_batch_advance(BatchCtl* ctl, int n_sys) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q < n_sys) ctl[q].sweep += 1u;
}

cudaError_t launch_batch_advance(BatchCtl* ctl, int n_sys, cudaStream_t st) {
    k_batch_advance<<<(n_sys + 127) / 128, 128, 0, st>>>(ctl, n_sys);
    return cudaGetLastError();
}

cudaError_t launch_batch_plan(BatchPlan* plan, const BatchCtl* ctl, const BatchSys* sys, int n_sys, cudaStream_t st) {
    k_batch_plan<<<1, 32, 0, st>>>(plan, ctl, sys, n_sys);
    return cudaGetLastError();
}

cudaError_t launch_branch_batch(const BatchSys* sys, BatchPlan* plan, BatchCtl* ctl, int n_sys, int parity,
                                double tau, double* hist, int hist_stride, int forces, int copy_grid,
                                cudaStream_t st) {
    k_branch_weights_batch<<<copy_grid, 256, 0, st>>>(sys, plan, ctl, parity, tau);
    k_batch_reduce<<<n_sys, 256, 0, st>>>(sys, plan, hist, hist_stride, forces);
    k_branch_scan_batch<<<n_sys, 1024, 0, st>>>(sys, plan, ctl, hist, hist_stride);
    k_branch_copy_batch<<<copy_grid, 256, 0, st>>>(sys, plan, ctl, parity);
    return cudaGetLastError();
}

}  // namespace qmc

// ---------------------------------------------------------------------
// Allocation-free population control (qmc_branch_noalloc in qmc.h).
//
// Callers that cannot allocate device memory (for example a host framework
// that owns every device buffer itself and hands the library only pointers
// into its own pool) still need the branching step.  This variant runs the
// same weight and scan kernels as the DMC driver but keeps their per-walker
// scratch (copies, offsets, weights) in the file-scope array below instead
// of handle-owned cudaMalloc memory, and returns a parent map so that the
// caller gathers its own walker arrays.  Every GPU that loads the library
// holds this array until the process exits.
// ---------------------------------------------------------------------

#include <mutex>

#include "qmc.h"

namespace {

constexpr int kNoAllocMaxWalkers = 65536;
constexpr size_t kNoAllocScratchBytes = (size_t)kNoAllocMaxWalkers * (2 * sizeof(int) + sizeof(double));
constexpr int kNoAllocMaxDevices = 64;

std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kNoAllocMaxDevices] = {};

}  // namespace

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

namespace qmc {

__global__ void k_branch_parent(int W, const int* copies, const int* offsets, const double* stats, int* parent) {
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= W || stats[3] != 0.0) return;
    const int m = copies[w], off = offsets[w];
    for (int t = 0; t < m; ++t) parent[off + t] = w;
}

}  // namespace qmc

// Device address of the scratch array on the current device.  The host-side
// name of a __device__ array is only a stand-in, so the address is looked up
// with cudaGetSymbolAddress.  Outside stream capture it is looked up on every
// call (the lookup follows the current context, so a context that was reset
// or replaced gets the array's new address); a call made while its stream is
// capturing may not trigger module loading and uses the address the last
// uncaptured call on this device found (QMC_ERR_STATE if there was none).
static int noalloc_scratch(cudaStream_t s, void** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return QMC_ERR_CUDA;
    }
    if (dev < 0 || dev >= kNoAllocMaxDevices) return QMC_ERR_UNSUPPORTED;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) {
        cudaGetLastError();
        return QMC_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (cap == cudaStreamCaptureStatusNone) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) {
            cudaGetLastError();
            return QMC_ERR_CUDA;
        }
        g_noalloc_ptr[dev] = p;
    } else if (!g_noalloc_ptr[dev]) {
        return QMC_ERR_STATE;
    }
    *out = g_noalloc_ptr[dev];
    return QMC_OK;
}

extern "C" int qmc_branch_noalloc(int n_walkers, const double* eloc_old, const double* eloc_new, double tau,
                                  double e_trial, double e_cut, uint64_t seed, uint32_t sweep, int capacity,
                                  int* parent, double* stats, void* cuda_stream) {
    if (n_walkers > kNoAllocMaxWalkers) return QMC_ERR_UNSUPPORTED;
    if (n_walkers < 1 || capacity < 1 || !eloc_old || !eloc_new || !parent || !stats) return QMC_ERR_ARG;
    if (!(tau > 0.0) || !(e_cut > 0.0) || !isfinite(tau) || !isfinite(e_trial) || !isfinite(e_cut))
        return QMC_ERR_ARG;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    // an error left pending by the caller's earlier work is not ours to
    // report (or to clear)
    if (cudaPeekAtLastError() != cudaSuccess) return QMC_ERR_CUDA;
    void* scr = nullptr;
    const int st = noalloc_scratch(s, &scr);
    if (st != QMC_OK) return st;
    int* copies = (int*)scr;
    int* offsets = copies + kNoAllocMaxWalkers;
    double* wts = (double*)(offsets + kNoAllocMaxWalkers);
    qmc::DevWalkers src{};
    src.eloc = const_cast<double*>(eloc_old);
    qmc::BranchParams p{};
    p.tau = tau;
    p.e_trial = e_trial;
    p.e_cut = e_cut;
    p.key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
    p.sweep = sweep;
    p.cap = capacity;
    const int W = n_walkers;
    qmc::k_branch_weights<<<(W + 255) / 256, 256, 0, s>>>(src, W, eloc_new, p, copies, wts);
    if (cudaGetLastError() != cudaSuccess) return QMC_ERR_CUDA;
    qmc::k_branch_scan<<<1, 1024, 0, s>>>(W, copies, wts, eloc_new, e_trial - e_cut, e_trial + e_cut, capacity,
                                          offsets, stats, 0, p.key, p.sweep);
    if (cudaGetLastError() != cudaSuccess) return QMC_ERR_CUDA;
    qmc::k_branch_parent<<<(W + 255) / 256, 256, 0, s>>>(W, copies, offsets, stats, parent);
    if (cudaGetLastError() != cudaSuccess) return QMC_ERR_CUDA;
    return QMC_OK;
}
