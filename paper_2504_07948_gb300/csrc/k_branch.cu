// Branching step of diffusion Monte Carlo (the projection of Eq. 1 with
// population control, following Reynolds et al. 1982).
//
//   w = exp(-tau [ (E_old + E_new)/2 - E_T ]),  E clipped to E_T +- e_cut,
//   copies = min(floor(w + u), 3), each copy restarts with weight 1.
// Walkers are compacted into a second buffer in source order: the copies of
// walker w occupy slots offsets[w] .. offsets[w] + copies[w] - 1.
#include "qmc_internal.cuh"

namespace qmc {

__global__ void k_branch_weights(DevWalkers src, int W, const double* eloc_new, BranchParams p, int* copies,
                                 double* wts) {
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= W) return;
    const double lo = p.e_trial - p.e_cut, hi = p.e_trial + p.e_cut;
    const double eo = fmin(fmax(src.eloc[w], lo), hi);
    const double en = fmin(fmax(eloc_new[w], lo), hi);
    double wt = exp(-p.tau * (0.5 * (eo + en) - p.e_trial));
    if (!isfinite(eloc_new[w])) wt = 0.0;  // a broken walker is dropped
    const double u = draw_uniform(p.key, p.sweep, 0xFFFFFFFFu, (uint32_t)w, 2u);
    int m = (int)floor(wt + u);
    copies[w] = m > 3 ? 3 : m;
    wts[w] = wt;
}

// Single CTA: exclusive scan of copies, ordered sums of w, w E_new and
// w clip(E_new) (the clipped energy drives the trial-energy feedback).
__global__ void k_branch_scan(int W, const int* copies, const double* wts, const double* eloc_new, double lo,
                              double hi, int cap, int* offsets, double* stats) {
    __shared__ int s_cnt[1024];
    __shared__ double s_w[1024], s_we[1024], s_wc[1024];
    const int t = threadIdx.x, nt = blockDim.x;
    const int chunk = (W + nt - 1) / nt;
    const int b = t * chunk, e = min(W, b + chunk);
    int c = 0;
    double sw = 0.0, swe = 0.0, swc = 0.0;
    for (int w = b; w < e; ++w) {
        c += copies[w];
        sw += wts[w];
        if (wts[w] != 0.0) {
            swe += wts[w] * eloc_new[w];
            swc += wts[w] * fmin(fmax(eloc_new[w], lo), hi);
        }
    }
    s_cnt[t] = c;
    s_w[t] = sw;
    s_we[t] = swe;
    s_wc[t] = swc;
    __syncthreads();
    if (t == 0) {
        int run = 0;
        double a = 0.0, ae = 0.0, ac = 0.0;
        for (int q = 0; q < nt; ++q) {
            const int v = s_cnt[q];
            s_cnt[q] = run;
            run += v;
            a += s_w[q];
            ae += s_we[q];
            ac += s_wc[q];
        }
        stats[0] = a;
        stats[1] = ae;
        stats[2] = (double)run;
        stats[3] = run > cap ? 1.0 : 0.0;
        stats[4] = ac;
    }
    __syncthreads();
    int run = s_cnt[t];
    for (int w = b; w < e; ++w) {
        offsets[w] = run;
        run += copies[w];
    }
}

__device__ __forceinline__ void cta_copy(void* dst, const void* src, size_t bytes) {
    if ((((uintptr_t)dst | (uintptr_t)src | bytes) & 15) == 0) {
        uint4* d = (uint4*)dst;
        const uint4* s = (const uint4*)src;
        for (size_t q = threadIdx.x; q < bytes / 16; q += blockDim.x) d[q] = s[q];
    } else {
        uint32_t* d = (uint32_t*)dst;
        const uint32_t* s = (const uint32_t*)src;
        for (size_t q = threadIdx.x; q < bytes / 4; q += blockDim.x) d[q] = s[q];
    }
}

__global__ void k_branch_copy(DevSys s, DevWalkers src, DevWalkers dst, int W, const int* copies,
                              const int* offsets, const double* eloc_new, const double* stats, int elem) {
    const int w = blockIdx.x;
    if (w >= W || stats[3] != 0.0) return;
    const int m = copies[w], off = offsets[w];
    const int N = s.N, nu = s.n_up, nd = s.n_dn;
    const size_t a0 = (size_t)nu * nu * elem, a1 = (size_t)nd * nd * elem;
    for (int t = 0; t < m; ++t) {
        const int d = off + t;
        cta_copy(dst.R + (size_t)d * 3 * N, src.R + (size_t)w * 3 * N, sizeof(double) * 3 * N);
        cta_copy((char*)dst.Ainv[0] + d * a0, (const char*)src.Ainv[0] + w * a0, a0);
        cta_copy((char*)dst.Ainv[1] + d * a1, (const char*)src.Ainv[1] + w * a1, a1);
        cta_copy((char*)dst.G[0] + d * 4 * a0, (const char*)src.G[0] + w * 4 * a0, 4 * a0);
        cta_copy((char*)dst.G[1] + d * 4 * a1, (const char*)src.G[1] + w * 4 * a1, 4 * a1);
        if (s.msd) {
            for (int spin = 0; spin < 2; ++spin) {
                const size_t n = spin ? nd : nu, nv = s.n_vir[spin], ns = s.n_str[spin];
                const size_t ta = n * nv * elem, tr = ns * elem;
                cta_copy((char*)dst.Av[spin] + d * ta, (const char*)src.Av[spin] + w * ta, ta);
                cta_copy((char*)dst.Gv[spin] + d * 4 * ta, (const char*)src.Gv[spin] + w * 4 * ta, 4 * ta);
                cta_copy((char*)dst.Tt[spin] + d * ta, (const char*)src.Tt[spin] + w * ta, ta);
                cta_copy((char*)dst.Rs[spin] + d * tr, (const char*)src.Rs[spin] + w * tr, tr);
                cta_copy((char*)dst.Cd[spin] + d * tr, (const char*)src.Cd[spin] + w * tr, tr);
            }
            if (threadIdx.x == 0) dst.Ssum[d] = src.Ssum[w];
        }
        if (threadIdx.x == 0) {
            dst.logdet[2 * d] = src.logdet[2 * w];
            dst.logdet[2 * d + 1] = src.logdet[2 * w + 1];
            dst.sgn[2 * d] = src.sgn[2 * w];
            dst.sgn[2 * d + 1] = src.sgn[2 * w + 1];
            dst.eloc[d] = eloc_new[w];
            dst.weight[d] = 1.0;
        }
    }
}

cudaError_t launch_branch(const DevSys& s, const DevWalkers& src, const DevWalkers& dst, int W,
                          const double* eloc_new, const BranchParams& p, int* copies, int* offsets, double* wts,
                          double* stats, int elem_bytes, cudaStream_t st) {
    if (W == 0) return cudaSuccess;
    k_branch_weights<<<(W + 255) / 256, 256, 0, st>>>(src, W, eloc_new, p, copies, wts);
    k_branch_scan<<<1, 1024, 0, st>>>(W, copies, wts, eloc_new, p.e_trial - p.e_cut, p.e_trial + p.e_cut, p.cap,
                                      offsets, stats);
    k_branch_copy<<<W, 256, 0, st>>>(s, src, dst, W, copies, offsets, eloc_new, stats, elem_bytes);
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

// Device address of the scratch array on the current device, looked up once
// per device (the host-side name of a __device__ array is only a stand-in).
static int noalloc_scratch(void** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return QMC_ERR_CUDA;
    }
    if (dev < 0 || dev >= kNoAllocMaxDevices) return QMC_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) {
            cudaGetLastError();
            return QMC_ERR_CUDA;
        }
        g_noalloc_ptr[dev] = p;
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
    void* scr = nullptr;
    const int st = noalloc_scratch(&scr);
    if (st != QMC_OK) return st;
    int* copies = (int*)scr;
    int* offsets = copies + kNoAllocMaxWalkers;
    double* wts = (double*)(offsets + kNoAllocMaxWalkers);
    cudaStream_t s = (cudaStream_t)cuda_stream;
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
    qmc::k_branch_scan<<<1, 1024, 0, s>>>(W, copies, wts, eloc_new, e_trial - e_cut, e_trial + e_cut, capacity,
                                          offsets, stats);
    qmc::k_branch_parent<<<(W + 255) / 256, 256, 0, s>>>(W, copies, offsets, stats, parent);
    if (cudaGetLastError() != cudaSuccess) return QMC_ERR_CUDA;
    return QMC_OK;
}
