// Host side of the C ABI declared in include/qmc.h: handle, input
// validation, device uploads, walker buffers and the VMC / DMC drivers.
#include <cublas_v2.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <limits>
#include <random>
#include <string>
#include <vector>

#include "batch.cuh"
#include "qmc.h"
#include "qmc_internal.cuh"
#include "sweep_tiled.cuh"

using namespace qmc;

namespace {

struct QmcError {
    int code;
    std::string msg;
};

// cudaErrorNotSupported from a launcher of this library means a size its
// kernel does not take (e.g. shared memory beyond a CTA's): QMC_ERR_UNSUPPORTED.
#define QMC_CK(call)                                                                                  \
    do {                                                                                              \
        cudaError_t e_ = (call);                                                                      \
        if (e_ != cudaSuccess)                                                                        \
            throw QmcError{e_ == cudaErrorNotSupported ? QMC_ERR_UNSUPPORTED : QMC_ERR_CUDA,          \
                           std::string(#call) + ": " + cudaGetErrorString(e_)};                       \
    } while (0)

void require(bool ok, int code, const std::string& msg) {
    if (!ok) throw QmcError{code, msg};
}

// Limits of the kernels (shared-memory Gauss-Jordan inverse in FP64, pivot
// table of 256 entries).
constexpr int kMaxSpinElectrons = 160;

double dfact(int n) {
    double r = 1.0;
    while (n > 1) {
        r *= n;
        n -= 2;
    }
    return r;
}

// Normalised contraction coefficients of one shell.  A primitive of angular
// momentum l is scaled to unit norm by (2a/pi)^(3/4) (4a)^(l/2) /
// sqrt((2l-1)!!); the contraction then by 1/sqrt(sum_pq d_p d_q S_pq) with
// S_pq = (2 sqrt(a_p a_q) / (a_p + a_q))^(l + 3/2), the overlap of two such
// normalised primitives.  Shells with a zero exponent are not normalisable
// and keep their raw weights.
std::vector<double> contraction(int l, const double* a, const double* d, int np) {
    std::vector<double> c(d, d + np);
    for (int p = 0; p < np; ++p)
        if (a[p] == 0.0) return c;
    double norm2 = 0.0;
    for (int p = 0; p < np; ++p)
        for (int q = 0; q < np; ++q) {
            const double g = 2.0 * std::sqrt(a[p] * a[q]) / (a[p] + a[q]);
            norm2 += d[p] * d[q] * std::pow(g, l + 1.5);
        }
    const double inv = 1.0 / std::sqrt(norm2);
    for (int p = 0; p < np; ++p)
        c[p] = d[p] * inv * std::pow(2.0 * a[p] / M_PI, 0.75) * std::pow(4.0 * a[p], 0.5 * l) / std::sqrt(dfact(2 * l - 1));
    return c;
}

// Blocking analysis of a serially correlated series: the largest naive
// standard error over successive pair-averagings (Flyvbjerg-Petersen).
double blocked_error(std::vector<double> x) {
    if (x.size() < 2) return 0.0;
    auto se = [](const std::vector<double>& v) {
        double m = 0.0;
        for (double t : v) m += t;
        m /= v.size();
        double s = 0.0;
        for (double t : v) s += (t - m) * (t - m);
        return std::sqrt(s / (v.size() - 1) / v.size());
    };
    double best = se(x);
    while (x.size() >= 16) {
        std::vector<double> y(x.size() / 2);
        for (size_t i = 0; i < y.size(); ++i) y[i] = 0.5 * (x[2 * i] + x[2 * i + 1]);
        x.swap(y);
        best = std::max(best, se(x));
    }
    return best;
}

}  // namespace

// Tiny device helpers used only by the drivers.
namespace qmc {
__global__ void k_moments(const double* x, int W, double* out /*[2]*/) {
    __shared__ double scratch[kMaxWarps * 2];
    double v[2] = {0.0, 0.0};
    for (int w = threadIdx.x; w < W; w += blockDim.x) {
        v[0] += x[w];
        v[1] += x[w] * x[w];
    }
    block_sum<2>(v, scratch);
    if (threadIdx.x == 0) {
        out[0] = v[0];
        out[1] = v[1];
    }
}
__global__ void k_fill(double* x, int n, double v) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) x[i] = v;
}
__global__ void k_mul(const double* a, const double* b, int n, double* out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = a[i] * b[i];
}
// Initial walkers: electron e of walker w at R_nuc[owner[e]] + sigma chi,
// chi three normals from the counter-based stream (counter = (0xFFFFFFFE,
// electron, walker, 3), Box-Muller of words (0, 1) and (2, 3), keeping three).
__global__ void k_init_walkers(double* R, int W, int N, const int* owner, const double* Rn, uint2 key, double sigma) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= W * N) return;
    const int w = i / N, e = i - w * N;
    const uint4 x = philox4x32_10(make_uint4(0xFFFFFFFEu, (uint32_t)e, (uint32_t)w, 3u), key);
    const double r1 = sqrt(-2.0 * log(u01(x.x))), r2 = sqrt(-2.0 * log(u01(x.z)));
    double s1, c1, s2, c2;
    sincospi(2.0 * u01(x.y), &s1, &c1);
    sincospi(2.0 * u01(x.w), &s2, &c2);
    const double chi[3] = {r1 * c1, r1 * s1, r2 * c2};
    const int a = owner[e];
    for (int c = 0; c < 3; ++c) R[(size_t)i * 3 + c] = Rn[3 * a + c] + sigma * chi[c];
}
__global__ void k_pack_per_walker(const double* dEL, const double* dlog, int W, int K, double* out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= W * K) return;
    const int w = i / K, k = i - w * K;
    out[(size_t)w * 2 * K + k] = dEL[i];
    out[(size_t)w * 2 * K + K + k] = dlog[i];
}
}  // namespace qmc

// Per-family kernel timing with CUDA events on the handle's stream.
enum { F_SWEEP = 0, F_ELOC, F_FORCE, F_BRANCH, F_RECOMPUTE, F_REDUCE, F_SWEEP_GEMM, F_NLPP, F_COUNT };
constexpr int kTiledMaxGroups = 4;   // walker groups of the tiled sweep run side by side
static const char* kFamily[F_COUNT] = {"sweep", "eloc", "force", "branch", "recompute", "reduce", "sweep_gemm",
                                       "nlpp"};

struct KernelTimer {
    bool on = false;
    struct Pending {
        int fam;
        cudaEvent_t a, b;
    };
    std::vector<Pending> pend;
    std::vector<cudaEvent_t> pool;
    cudaEvent_t open_ev = nullptr;
    double ms[F_COUNT] = {0};
    long long n[F_COUNT] = {0};

    cudaEvent_t take() {
        if (pool.empty()) {
            cudaEvent_t e;
            QMC_CK(cudaEventCreate(&e));
            return e;
        }
        cudaEvent_t e = pool.back();
        pool.pop_back();
        return e;
    }
    void begin(cudaStream_t st) {
        if (!on) return;
        open_ev = take();
        QMC_CK(cudaEventRecord(open_ev, st));
    }
    void end(int fam, int kernels, cudaStream_t st) {
        n[fam] += kernels;
        if (!on || !open_ev) return;
        cudaEvent_t b = take();
        QMC_CK(cudaEventRecord(b, st));
        pend.push_back({fam, open_ev, b});
        open_ev = nullptr;
    }
    // Spans that overlap others (work on several streams): an explicit start
    // event (nullptr when timing is off) closed on the same stream.
    cudaEvent_t mark(cudaStream_t st) {
        if (!on) return nullptr;
        cudaEvent_t a = take();
        QMC_CK(cudaEventRecord(a, st));
        return a;
    }
    void span(int fam, int kernels, cudaEvent_t a, cudaStream_t st) {
        n[fam] += kernels;
        if (!on || !a) return;
        cudaEvent_t b = take();
        QMC_CK(cudaEventRecord(b, st));
        pend.push_back({fam, a, b});
    }
    void collect() {  // after the stream has been synchronised
        for (const Pending& p : pend) {
            float t = 0.f;
            QMC_CK(cudaEventElapsedTime(&t, p.a, p.b));
            ms[p.fam] += t;
            pool.push_back(p.a);
            pool.push_back(p.b);
        }
        pend.clear();
    }
    void reset() {
        for (int f = 0; f < F_COUNT; ++f) {
            ms[f] = 0.0;
            n[f] = 0;
        }
    }
    void release() {
        for (const Pending& p : pend) {
            cudaEventDestroy(p.a);
            cudaEventDestroy(p.b);
        }
        for (cudaEvent_t e : pool) cudaEventDestroy(e);
        if (open_ev) cudaEventDestroy(open_ev);
        pend.clear();
        pool.clear();
    }
};

struct ForceSample {
    // sums over one sweep/step: w, w E, w dE (K), w E dlog (K), w dlog (K)
    std::vector<double> v;
};

struct qmc_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::string err;

    bool have_sys = false, have_basis = false, have_mos = false, have_jas = false;
    int n_nuc = 0, n_up = 0, n_dn = 0;
    std::vector<double> Z, Rn, a_en;
    double a_anti = 0, a_par = 0, b_ee = 0, b_en = 0;
    // three-body Jastrow (n3 terms; 0 = none)
    int n3 = 0;
    std::vector<int> e3;
    std::vector<double> c3;
    double b3 = 1.0;
    // semi-local pseudopotential (n_pp radial terms; 0 = none)
    int n_pp = 0;
    std::vector<int> pp_nuc, pp_l, pp_n;
    std::vector<double> pp_alpha, pp_beta, pp_rcut, pp_quad, pp_qw;
    int pp_rotate = 1;
    std::vector<int> sh_center, sh_l, sh_pure, sh_nprim;
    std::vector<double> alpha, coef;
    int n_basis = 0;
    int n_mo = 0, n_basis_C = 0;
    std::vector<double> C;
    std::vector<int> occ_up, occ_dn;
    int mode = QMC_FP64, delay_rank = 1, recompute_period = 0;
    // multi-determinant expansion (bit strings over orbital index)
    bool have_msd = false;
    int msd_words = 0;
    std::vector<uint64_t> det_up, det_dn;
    std::vector<double> ci;
    uint64_t seed = 1005;
    uint32_t sweep = 0;
    int cap_factor = 2;
    int pop_mode = QMC_POP_BRANCH;
    uint64_t gen = 0;   // changes whenever the system or wavefunction changes

    // device copy of the system
    bool sys_dirty = true;
    std::vector<void*> sys_allocs;
    DevSys ds{};
    double* d_dvnn = nullptr;

    // walkers
    std::vector<void*> wk_allocs;
    DevWalkers wk[2]{};
    int cur = 0, W = 0, cap = 0, W0 = 0;
    bool walkers_valid = false;
    int sweeps_since_recompute = 0;
    double *d_eloc_new = nullptr, *d_wts = nullptr, *d_stats = nullptr, *d_tmp = nullptr, *d_wE = nullptr;
    int *d_copies = nullptr, *d_offsets = nullptr;
    double *d_dEL = nullptr, *d_dlog = nullptr, *d_Bscr = nullptr, *d_Pscr = nullptr, *d_ones = nullptr;
    double* d_facc = nullptr;
    double* d_sign = nullptr;
    int* d_refresh = nullptr;   // per-walker "rebuild in FP64" flags (determinant expansions)
    double* d_fmsd = nullptr;   // per-walker scratch of the multi-determinant force kernel
    void* d_nlB = nullptr;      // per-walker non-local matrix rows of both spins (force pass)
    double* d_nlF = nullptr;    // per-walker direct non-local derivative terms
    // u_k = C_s A^-1 e_k of the non-local kernel from the tensor cores (mixed
    // form): rows of a slice of nlU_W walkers, [slice][n_s][ldu] per spin
    float* d_nlU = nullptr;
    int nlU_W = 0;
    int nlpp_tc = 1;
    int nlpp_tc_min_n = 64;   // electrons per spin from which the GEMMs pay for their launches and traffic
    // space warp of the ionic derivatives (off by default): per-walker
    // electron gradients [cap][N][3], allocated on first use
    int space_warp = 0;
    double *d_gEdet = nullptr, *d_gtot = nullptr;
    // large-determinant force path (batched GEMMs)
    cublasHandle_t blas = nullptr;
    int force_gemm_min_n = 65;  // spins with more electrons use the GEMM path
    int force_gemm_cublas = 0;  // FP32 GEMMs on cuBLAS instead of the tensor-core kernel
    int fchunk = 0;
    void *d_fB = nullptr, *d_fPT = nullptr, *d_fQ = nullptr, *d_fM = nullptr, *d_fY = nullptr;
    double *d_fgJ = nullptr, *d_faccw = nullptr;
    unsigned* d_err = nullptr;
    unsigned long long* d_nacc = nullptr;
    // sharded DMC: a caller-supplied sum over ranks of each step's sums, and
    // the reference population of the trial-energy feedback (0 = W0)
    qmc_reduce_fn reduce_fn = nullptr;
    void* reduce_ctx = nullptr;
    double pop_ref = 0.0;
    // walker-tiled mixed sweep (tensor-core orbital contraction) for large
    // determinants with delayed updates; scratch sized for tiled_W walkers
    int tiled_min_n = 96;   // electrons per spin from which the tiled sweep runs
    int tiled_enable = 1;
    std::vector<void*> tiled_allocs;
    TiledState tiled{};
    int tiled_W = 0;
    // walker groups of the tiled sweep: group 0 on the handle's stream, the
    // others on streams of their own, forked from it and joined back
    int tiled_groups = 2;
    cudaStream_t tiled_side[kTiledMaxGroups - 1] = {};
    cudaEvent_t tiled_ev[kTiledMaxGroups] = {};   // the fork, then one join per side stream

    // estimators
    std::vector<double> vmc_e, vmc_e2, dmc_e, dmc_e2;
    std::vector<ForceSample> vmc_f, dmc_f;
    unsigned long long acc_base = 0;
    long long n_prop = 0;
    KernelTimer tm;

    int N() const { return n_up + n_dn; }
    int elem() const { return mode == QMC_MIXED ? 4 : 8; }

    template <typename T>
    T* dalloc(std::vector<void*>& list, size_t count) {
        void* p = nullptr;
        if (count == 0) count = 1;
        cudaError_t e = cudaMalloc(&p, sizeof(T) * count);
        if (e != cudaSuccess) {
            cudaGetLastError();
            throw QmcError{QMC_ERR_OOM, "cudaMalloc of " + std::to_string(sizeof(T) * count) + " bytes failed"};
        }
        list.push_back(p);
        return (T*)p;
    }
    template <typename T>
    T* upload(std::vector<void*>& list, const std::vector<T>& v) {
        T* p = dalloc<T>(list, v.size());
        if (!v.empty()) QMC_CK(cudaMemcpyAsync(p, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice, stream));
        return p;
    }
    void free_list(std::vector<void*>& list) {
        for (void* p : list) cudaFree(p);
        list.clear();
    }
    void sync() {
        QMC_CK(cudaStreamSynchronize(stream));
        tm.collect();
    }

    void check_device_errors() {
        unsigned e = 0;
        QMC_CK(cudaMemcpyAsync(&e, d_err, sizeof(unsigned), cudaMemcpyDeviceToHost, stream));
        sync();
        if (e) {
            QMC_CK(cudaMemsetAsync(d_err, 0, sizeof(unsigned), stream));
            if (e & kErrSingular) throw QmcError{QMC_ERR_SINGULAR, "a Slater matrix is singular"};
            if (e & kErrNonFinite) throw QmcError{QMC_ERR_NONFINITE, "non-finite local energy"};
            if (e & kErrTimeout) throw QmcError{QMC_ERR_TIMEOUT, "a bounded device wait gave up"};
            throw QmcError{QMC_ERR_CUDA, "device error flag " + std::to_string(e)};
        }
    }

    void build_system() {
        require(have_sys && have_basis && have_mos && have_jas, QMC_ERR_STATE,
                "system, basis, orbitals and Jastrow must all be set");
        require(n_basis_C == n_basis, QMC_ERR_ARG,
                "orbital coefficients have " + std::to_string(n_basis_C) + " columns but the basis has " +
                    std::to_string(n_basis) + " functions");
        for (int c : sh_center) require(c >= 0 && c < n_nuc, QMC_ERR_ARG, "shell centre out of range");
        require(!(have_msd && n_pp), QMC_ERR_UNSUPPORTED,
                "the non-local pseudopotential is evaluated for single-determinant trial functions only");
        if (!sys_dirty) return;
        free_list(sys_allocs);
        if (have_msd) {
            // the reference determinant (first of the expansion) defines the
            // occupied columns, in ascending orbital order
            occ_up = string_orbitals(&det_up[0]);
            occ_dn = string_orbitals(&det_dn[0]);
            for (int o : occ_up) require(o < n_mo, QMC_ERR_ARG, "reference orbital beyond n_mo");
            for (int o : occ_dn) require(o < n_mo, QMC_ERR_ARG, "reference orbital beyond n_mo");
        }
        DevSys s{};
        s.n_nuc = n_nuc;
        s.n_up = n_up;
        s.n_dn = n_dn;
        s.N = n_up + n_dn;
        s.n_shell = (int)sh_l.size();
        s.n_basis = n_basis;
        s.n_prim = (int)alpha.size();
        s.a_anti = a_anti;
        s.a_par = a_par;
        s.b_ee = b_ee;
        s.b_en = b_en;
        double vnn = 0.0;
        std::vector<double> dv(3 * n_nuc, 0.0);
        for (int a = 0; a < n_nuc; ++a)
            for (int b = 0; b < n_nuc; ++b) {
                if (a == b) continue;
                double d[3], r2 = 0.0;
                for (int c = 0; c < 3; ++c) {
                    d[c] = Rn[3 * a + c] - Rn[3 * b + c];
                    r2 += d[c] * d[c];
                }
                const double r = std::sqrt(r2);
                if (b > a) vnn += Z[a] * Z[b] / r;
                for (int c = 0; c < 3; ++c) dv[3 * a + c] -= Z[a] * Z[b] * d[c] / (r2 * r);
            }
        s.vnn = vnn;
        s.Z = upload(sys_allocs, Z);
        s.Rn = upload(sys_allocs, Rn);
        {
            std::vector<float> hi(Rn.size()), lo(Rn.size());
            for (size_t q = 0; q < Rn.size(); ++q) {
                hi[q] = (float)Rn[q];
                lo[q] = (float)(Rn[q] - (double)hi[q]);
            }
            s.Rn_hi = upload(sys_allocs, hi);
            s.Rn_lo = upload(sys_allocs, lo);
        }
        s.a_en = upload(sys_allocs, a_en);
        s.n3 = n3;
        s.b3 = b3;
        s.e3 = n3 ? upload(sys_allocs, e3) : nullptr;
        s.c3 = n3 ? upload(sys_allocs, c3) : nullptr;
        if (n_pp) {
            // terms grouped by nucleus (stable), the nuclei with a non-local
            // channel and a positive cutoff
            std::vector<int> order(n_pp);
            for (int t = 0; t < n_pp; ++t) order[t] = t;
            std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return pp_nuc[x] < pp_nuc[y]; });
            std::vector<int> off(n_nuc + 1, 0);
            std::vector<int2> ln(n_pp);
            std::vector<double2> ab(n_pp);
            std::vector<float2> abf(n_pp);
            std::vector<int> nonlocal(n_nuc, 0);
            for (int q = 0; q < n_pp; ++q) {
                const int t = order[q];
                ++off[pp_nuc[t] + 1];
                ln[q] = make_int2(pp_l[t], pp_n[t]);
                ab[q] = make_double2(pp_alpha[t], pp_beta[t]);
                abf[q] = make_float2((float)pp_alpha[t], (float)pp_beta[t]);
                if (pp_l[t] >= 0) nonlocal[pp_nuc[t]] = 1;
            }
            for (int a = 0; a < n_nuc; ++a) off[a + 1] += off[a];
            std::vector<int> ecp;
            for (int a = 0; a < n_nuc; ++a)
                if (nonlocal[a] && pp_rcut[a] > 0.0) ecp.push_back(a);
            s.npp = n_pp;
            s.pp_off = upload(sys_allocs, off);
            s.pp_ln = upload(sys_allocs, ln);
            s.pp_ab = upload(sys_allocs, ab);
            s.pp_ab_f = upload(sys_allocs, abf);
            s.pp_rcut = upload(sys_allocs, pp_rcut);
            s.n_ecp = (int)ecp.size();
            s.ecp_nuc = upload(sys_allocs, ecp);
            s.pp_nq = (int)pp_qw.size();
            s.pp_rotate = pp_rotate;
            s.pp_quad = upload(sys_allocs, pp_quad);
            s.pp_qw = upload(sys_allocs, pp_qw);
            for (int spin = 0; spin < 2; ++spin) {
                const std::vector<int>& occ = spin ? occ_dn : occ_up;
                const int n = (int)occ.size();
                std::vector<double> ct((size_t)n * n_basis);
                for (int j = 0; j < n; ++j)
                    for (int l = 0; l < n_basis; ++l) ct[(size_t)j * n_basis + l] = C[(size_t)occ[j] * n_basis + l];
                s.CT[spin] = upload(sys_allocs, ct);
                s.CT_f[spin] = upload(sys_allocs, std::vector<float>(ct.begin(), ct.end()));
            }
            s.a_en_f = upload(sys_allocs, std::vector<float>(a_en.begin(), a_en.end()));
            std::vector<int> bytype((size_t)s.n_shell);
            for (int q = 0; q < s.n_shell; ++q) bytype[q] = q;
            std::stable_sort(bytype.begin(), bytype.end(), [&](int x, int y) {
                return (sh_l[x] << 1 | sh_pure[x]) < (sh_l[y] << 1 | sh_pure[y]);
            });
            s.shell_by_type = upload(sys_allocs, bytype);
        }
        d_dvnn = upload(sys_allocs, dv);
        std::vector<int4> sh(s.n_shell);
        std::vector<int> fn(s.n_shell + 1);
        std::vector<double> cn(alpha.size());
        int p0 = 0, f0 = 0;
        for (int q = 0; q < s.n_shell; ++q) {
            sh[q] = make_int4(sh_center[q], sh_l[q] | (sh_pure[q] << 8), p0, sh_nprim[q]);
            fn[q] = f0;
            std::vector<double> c = contraction(sh_l[q], &alpha[p0], &coef[p0], sh_nprim[q]);
            std::copy(c.begin(), c.end(), cn.begin() + p0);
            p0 += sh_nprim[q];
            f0 += shell_nfn(sh_l[q], sh_pure[q]);
        }
        fn[s.n_shell] = f0;
        s.shell = upload(sys_allocs, sh);
        s.shell_fn = upload(sys_allocs, fn);
        std::vector<int> runs;
        for (int q = 0; q < s.n_shell; ++q)
            if (q == 0 || sh_center[q] != sh_center[q - 1]) runs.push_back(q);
        runs.push_back(s.n_shell);
        s.n_run = (int)runs.size() - 1;
        s.run_sh = upload(sys_allocs, runs);
        s.alpha = upload(sys_allocs, alpha);
        s.cn = upload(sys_allocs, cn);
        {
            // smallest exponent per shell (the screening test of the live-shell basis)
            std::vector<double> am(s.n_shell, std::numeric_limits<double>::infinity());
            std::vector<float> amf(s.n_shell, std::numeric_limits<float>::infinity());
            for (int q = 0; q < s.n_shell; ++q)
                for (int p = sh[q].z; p < sh[q].z + sh[q].w; ++p) {
                    am[q] = std::min(am[q], alpha[p]);
                    amf[q] = std::min(amf[q], (float)alpha[p]);
                }
            s.shell_amin = upload(sys_allocs, am);
            s.shell_amin_f = upload(sys_allocs, amf);
        }
        s.alpha_f = upload(sys_allocs, std::vector<float>(alpha.begin(), alpha.end()));
        s.cn_f = upload(sys_allocs, std::vector<float>(cn.begin(), cn.end()));
        for (int spin = 0; spin < 2; ++spin) {
            const std::vector<int>& occ = spin ? occ_dn : occ_up;
            const int n = (int)occ.size();
            std::vector<double> Cs((size_t)n_basis * n);
            for (int l = 0; l < n_basis; ++l)
                for (int j = 0; j < n; ++j) Cs[(size_t)l * n + j] = C[(size_t)occ[j] * n_basis + l];
            s.C[spin] = upload(sys_allocs, Cs);
            s.C_f[spin] = upload(sys_allocs, std::vector<float>(Cs.begin(), Cs.end()));
        }
        if (have_msd) build_multidet(s);
        ds = s;
        sync();
        sys_dirty = false;
    }

    std::vector<int> string_orbitals(const uint64_t* w) const {
        std::vector<int> o;
        for (int b = 0; b < 64 * msd_words; ++b)
            if ((w[b / 64] >> (b % 64)) & 1ULL) o.push_back(b);
        return o;
    }

    // Unique spin strings of the expansion relative to the reference:
    // holes, particles and the sign of the sorting permutation, plus the
    // determinant lists of each string (for S = sum_k c_k R_up R_dn).
    void build_multidet(DevSys& s) {
        const int n_det = (int)ci.size();
        s.msd = 1;
        std::vector<int> sid[2];
        for (int spin = 0; spin < 2; ++spin) {
            const std::vector<uint64_t>& bits = spin ? det_dn : det_up;
            const std::vector<int> ref = spin ? occ_dn : occ_up;
            const int n = (int)ref.size();
            std::vector<char> in_ref(64 * msd_words, 0);
            for (int o : ref) in_ref[o] = 1;
            // active virtual orbitals: every orbital some determinant adds
            std::vector<int> vir;
            for (int k = 0; k < n_det; ++k)
                for (int o : string_orbitals(&bits[(size_t)k * msd_words]))
                    if (!in_ref[o]) vir.push_back(o);
            std::sort(vir.begin(), vir.end());
            vir.erase(std::unique(vir.begin(), vir.end()), vir.end());
            require((int)vir.size() <= kMaxVirtual, QMC_ERR_UNSUPPORTED,
                    "at most " + std::to_string(kMaxVirtual) + " active virtual orbitals per spin");
            for (int o : vir) require(o < n_mo, QMC_ERR_ARG, "determinant uses an orbital beyond n_mo");
            std::vector<int> vpos(64 * msd_words, -1);
            for (size_t q = 0; q < vir.size(); ++q) vpos[vir[q]] = (int)q;
            // unique strings (the reference first)
            std::vector<std::vector<uint64_t>> uniq;
            std::vector<int4> packed;
            sid[spin].resize(n_det);
            auto key_of = [&](int k) {
                return std::vector<uint64_t>(bits.begin() + (size_t)k * msd_words,
                                             bits.begin() + (size_t)(k + 1) * msd_words);
            };
            std::vector<std::pair<std::vector<uint64_t>, int>> index;
            for (int k = 0; k < n_det; ++k) {
                std::vector<uint64_t> key = key_of(k);
                auto it = std::lower_bound(index.begin(), index.end(), std::make_pair(key, -1));
                if (it != index.end() && it->first == key) {
                    sid[spin][k] = it->second;
                    continue;
                }
                const int id = (int)uniq.size();
                index.insert(it, std::make_pair(key, id));
                uniq.push_back(key);
                sid[spin][k] = id;
                const std::vector<int> orb = string_orbitals(key.data());
                require((int)orb.size() == n, QMC_ERR_ARG, "a determinant string has the wrong electron count");
                std::vector<int> holes, parts;
                std::vector<char> in_s(64 * msd_words, 0);
                for (int o : orb) in_s[o] = 1;
                for (int a = 0; a < n; ++a)
                    if (!in_s[ref[a]]) holes.push_back(a);
                for (int o : orb)
                    if (!in_ref[o]) parts.push_back(vpos[o]);
                const int e = (int)holes.size();
                require(e <= kMaxExcitation, QMC_ERR_UNSUPPORTED,
                        "excitations above " + std::to_string(kMaxExcitation) + "-fold are not supported");
                // in-place replacement, then the parity of sorting it
                std::vector<int> lst(ref);
                for (int a = 0; a < e; ++a) lst[holes[a]] = vir[parts[a]];
                int inv = 0;
                for (int x = 0; x < n; ++x)
                    for (int y = x + 1; y < n; ++y)
                        if (lst[x] > lst[y]) ++inv;
                int hw = 0, pw = 0;
                for (int a = 0; a < e; ++a) {
                    require(holes[a] < 256, QMC_ERR_UNSUPPORTED, "hole position beyond 255");
                    hw |= holes[a] << (8 * a);
                    pw |= parts[a] << (8 * a);
                }
                packed.push_back(make_int4(e | ((inv & 1) << 8), hw, pw, 0));
            }
            require(sid[spin][0] == 0, QMC_ERR_ARG, "internal: reference string must come first");
            // group strings by excitation level (reference first) so that
            // neighbouring threads evaluate minors of the same size, and
            // within a level by holes, then particles: neighbouring threads
            // then gather their minors mostly from the same rows of the
            // table T in shared memory (distinct banks within a row, one
            // broadcast where the entry is the same)
            std::vector<int> order(packed.size());
            for (size_t q = 0; q < order.size(); ++q) order[q] = (int)q;
            auto str_key = [&](int u) {
                const int4 v = packed[u];
                std::array<int, 9> k{};
                k[0] = v.x & 0xff;
                for (int a = 0; a < 4; ++a) {
                    k[1 + a] = (v.y >> (8 * a)) & 0xff;
                    k[5 + a] = (v.z >> (8 * a)) & 0xff;
                }
                return k;
            };
            std::stable_sort(order.begin() + 1, order.end(), [&](int a, int b) { return str_key(a) < str_key(b); });
            std::vector<int> newid(order.size());
            std::vector<int4> sorted(packed.size());
            for (size_t q = 0; q < order.size(); ++q) {
                newid[order[q]] = (int)q;
                sorted[q] = packed[order[q]];
            }
            packed.swap(sorted);
            for (int k = 0; k < n_det; ++k) sid[spin][k] = newid[sid[spin][k]];
            s.n_vir[spin] = (int)vir.size();
            s.n_str[spin] = (int)uniq.size();
            s.str[spin] = upload(sys_allocs, packed);
            std::vector<double> Cv((size_t)n_basis * vir.size());
            for (int l = 0; l < n_basis; ++l)
                for (size_t q = 0; q < vir.size(); ++q) Cv[l * vir.size() + q] = C[(size_t)vir[q] * n_basis + l];
            s.Cv[spin] = upload(sys_allocs, Cv);
            s.Cv_f[spin] = upload(sys_allocs, std::vector<float>(Cv.begin(), Cv.end()));
        }
        for (int spin = 0; spin < 2; ++spin) {
            const int ns = s.n_str[spin];
            std::vector<int> off(ns + 1, 0), other(n_det);
            std::vector<double> cc(n_det);
            for (int k = 0; k < n_det; ++k) ++off[sid[spin][k] + 1];
            for (int u = 0; u < ns; ++u) off[u + 1] += off[u];
            std::vector<int> fill(off.begin(), off.end() - 1);
            for (int k = 0; k < n_det; ++k) {
                const int q = fill[sid[spin][k]]++;
                other[q] = sid[1 - spin][k];
                cc[q] = ci[k];
            }
            s.csr_off[spin] = upload(sys_allocs, off);
            s.csr_other[spin] = upload(sys_allocs, other);
            s.csr_c[spin] = upload(sys_allocs, cc);
        }
    }

    void alloc_walkers(int Wn) {
        free_list(wk_allocs);
        free_list(tiled_allocs);
        tiled_W = 0;
        d_fmsd = nullptr;
        d_nlB = nullptr;
        d_nlF = nullptr;
        d_nlU = nullptr;
        nlU_W = 0;
        d_gEdet = nullptr;
        d_gtot = nullptr;
        fchunk = 0;
        cap = std::max(Wn, cap_factor * Wn);
        const int N3 = 3 * N();
        const size_t a0 = (size_t)n_up * n_up, a1 = (size_t)n_dn * n_dn;
        const int nmax = std::max(n_up, n_dn);
        d_nacc = dalloc<unsigned long long>(wk_allocs, 1);
        QMC_CK(cudaMemsetAsync(d_nacc, 0, sizeof(unsigned long long), stream));
        for (int b = 0; b < 2; ++b) {
            DevWalkers& k = wk[b];
            k.cap = cap;
            k.R = dalloc<double>(wk_allocs, (size_t)cap * N3);
            k.Ainv[0] = dalloc<char>(wk_allocs, (size_t)cap * a0 * elem());
            k.Ainv[1] = dalloc<char>(wk_allocs, (size_t)cap * a1 * elem());
            k.G[0] = dalloc<char>(wk_allocs, (size_t)cap * 4 * a0 * elem());
            k.G[1] = dalloc<char>(wk_allocs, (size_t)cap * 4 * a1 * elem());
            k.logdet = dalloc<double>(wk_allocs, 2 * (size_t)cap);
            k.sgn = dalloc<double>(wk_allocs, 2 * (size_t)cap);
            k.eloc = dalloc<double>(wk_allocs, cap);
            k.weight = dalloc<double>(wk_allocs, cap);
            k.n_acc = d_nacc;
        }
        if (ds.msd) {
            for (int b = 0; b < 2; ++b) {
                DevWalkers& k = wk[b];
                for (int spin = 0; spin < 2; ++spin) {
                    const size_t n = spin ? n_dn : n_up, nv = ds.n_vir[spin], ns = ds.n_str[spin];
                    k.Av[spin] = dalloc<char>(wk_allocs, (size_t)cap * n * nv * elem());
                    k.Gv[spin] = dalloc<char>(wk_allocs, (size_t)cap * 4 * n * nv * elem());
                    k.Tt[spin] = dalloc<char>(wk_allocs, (size_t)cap * n * nv * elem());
                    k.Rs[spin] = dalloc<char>(wk_allocs, (size_t)cap * ns * elem());
                    k.Rn[spin] = dalloc<char>(wk_allocs, (size_t)cap * ns * elem());
                    k.Cd[spin] = dalloc<char>(wk_allocs, (size_t)cap * ns * elem());
                }
                k.Ssum = dalloc<double>(wk_allocs, cap);
            }
        }
        d_sign = dalloc<double>(wk_allocs, cap);
        d_refresh = dalloc<int>(wk_allocs, cap);
        QMC_CK(cudaMemsetAsync(d_refresh, 0, sizeof(int) * cap, stream));
        wk[0].refresh = d_refresh;
        wk[1].refresh = d_refresh;
        double* s0 = dalloc<double>(wk_allocs, (size_t)cap * a0);
        double* s1 = dalloc<double>(wk_allocs, (size_t)cap * a1);
        for (int b = 0; b < 2; ++b) {
            wk[b].Ascr[0] = s0;
            wk[b].Ascr[1] = s1;
        }
        d_eloc_new = dalloc<double>(wk_allocs, cap);
        d_wts = dalloc<double>(wk_allocs, cap);
        d_wE = dalloc<double>(wk_allocs, cap);
        d_ones = dalloc<double>(wk_allocs, cap);
        d_stats = dalloc<double>(wk_allocs, 8);
        d_tmp = dalloc<double>(wk_allocs, 8);
        d_copies = dalloc<int>(wk_allocs, cap);
        d_offsets = dalloc<int>(wk_allocs, cap);
        const int K = 3 * n_nuc;
        d_dEL = dalloc<double>(wk_allocs, (size_t)cap * K);
        d_dlog = dalloc<double>(wk_allocs, (size_t)cap * K);
        d_Bscr = dalloc<double>(wk_allocs, (size_t)cap * nmax * nmax);
        d_Pscr = dalloc<double>(wk_allocs, (size_t)cap * nmax * nmax);
        d_facc = dalloc<double>(wk_allocs, 2 + 3 * (size_t)K);
        d_err = dalloc<unsigned>(wk_allocs, 1);
        QMC_CK(cudaMemsetAsync(d_err, 0, sizeof(unsigned), stream));
        wk[0].err = d_err;
        wk[1].err = d_err;
        k_fill<<<(cap + 255) / 256, 256, 0, stream>>>(d_ones, cap, 1.0);
        QMC_CK(cudaGetLastError());
        cur = 0;
    }

    // FP64 recompute of every walker's inverse, log-determinant and
    // orbital-gradient cache from its positions.
    void recompute(int which) {
        const DevWalkers& k = wk[which];
        tm.begin(stream);
        if (mode == QMC_MIXED) {
            QMC_CK(launch_orbitals_all<float>(ds, k, W, stream));
        } else {
            QMC_CK(launch_orbitals_all<double>(ds, k, W, stream));
        }
        QMC_CK(launch_invert(ds, k, W, mode == QMC_MIXED, d_err, stream));
        int nk = 2;
        if (ds.msd) {
            if (mode == QMC_MIXED) {
                QMC_CK(launch_msd_table<float>(ds, k, W, stream));
            } else {
                QMC_CK(launch_msd_table<double>(ds, k, W, stream));
            }
            ++nk;
        }
        tm.end(F_RECOMPUTE, nk, stream);
        sweeps_since_recompute = 0;
    }

    // Runs pass(w0, w1, U0, U1) of the non-local kernel over slices of the
    // walkers.  In the mixed form with spin blocks of 4k electrons, u_k =
    // C_s A^-1 e_k of every electron of a slice is formed first as batched
    // tensor-core GEMMs, U_s[w][k][l] = sum_j A^-T_w[k][j] C_s[l][j] (three-way
    // split TF32, N_b in column blocks of 256), slices holding at most
    // kNlUBytes of rows.  Below nlpp_tc_min_n electrons per spin (where the
    // GEMM launches and the rows' traffic cost more than the kernel's own
    // product: measured on the 6-water cluster), or where TMA cannot address
    // the operands, one slice without rows and the kernel forms u_k itself.
    // Returns the number of kernels launched.
    template <class F>
    int nl_passes(const DevWalkers& k, F pass) {
        constexpr size_t kNlUBytes = (size_t)2 << 30;
        const int ldu = (n_basis + 3) & ~3;
        if (!(nlpp_tc && mode == QMC_MIXED && n_up % 4 == 0 && n_dn % 4 == 0 &&
              std::max(n_up, n_dn) >= nlpp_tc_min_n)) {
            pass(0, W, nullptr, nullptr);
            return 1;
        }
        const size_t per_w = (size_t)(n_up + n_dn) * ldu * sizeof(float);
        if (nlU_W == 0) {
            // sized once for the capacity (no regrowth as the population moves)
            nlU_W = (int)std::max<size_t>(1, std::min<size_t>((size_t)cap, kNlUBytes / per_w));
            d_nlU = dalloc<float>(wk_allocs, (size_t)nlU_W * (n_up + n_dn) * ldu);
            QMC_CK(cudaMemsetAsync(d_nlU, 0, (size_t)nlU_W * per_w, stream));
        }
        const int smax = std::min(W, nlU_W);
        const int ns = (W + smax - 1) / smax, S = (W + ns - 1) / ns;
        float* U[2] = {d_nlU, d_nlU + (size_t)nlU_W * n_up * ldu};
        int launches = 0;
        for (int w0 = 0; w0 < W; w0 += S) {
            const int nw = std::min(S, W - w0);
            bool ok = true;
            for (int spin = 0; spin < 2 && ok; ++spin) {
                const int n = spin ? n_dn : n_up;
                if (n == 0) continue;
                const float* A = (const float*)k.Ainv[spin] + (size_t)w0 * n * n;
                for (int c0 = 0; c0 < n_basis && ok; c0 += 256) {
                    const cudaError_t e = launch_tc_gemm_ab(nw, n, std::min(256, n_basis - c0), n, 1.f, A,
                                                            (long long)n * n, n, ds.C_f[spin] + (size_t)c0 * n, 0, n,
                                                            0, 0.f, U[spin] + c0, (long long)n * ldu, ldu, d_err,
                                                            stream);
                    if (e == cudaErrorNotSupported) {
                        ok = false;   // refused before any launch: TMA cannot address the operands
                    } else {
                        QMC_CK(e);
                        ++launches;
                    }
                }
            }
            pass(w0, w0 + nw, ok ? U[0] : nullptr, ok ? U[1] : nullptr);
            ++launches;
        }
        return launches;
    }

    // E_L of every walker; with a pseudopotential the non-local term is
    // added with quadrature rotations drawn at the current sweep counter
    // (after a sweep: the counter of the next one).
    void eloc(int which, double* out, double* logpsi, double* grad, double* lap) {
        tm.begin(stream);
        if (mode == QMC_MIXED) {
            QMC_CK(launch_eloc<float>(ds, wk[which], W, out, logpsi, grad, lap, d_err, stream));
            if (ds.msd) QMC_CK(launch_msd_eloc<float>(ds, wk[which], W, out, logpsi, d_sign, grad, stream));
        } else {
            QMC_CK(launch_eloc<double>(ds, wk[which], W, out, logpsi, grad, lap, d_err, stream));
            if (ds.msd) QMC_CK(launch_msd_eloc<double>(ds, wk[which], W, out, logpsi, d_sign, grad, stream));
        }
        tm.end(F_ELOC, ds.msd ? 2 : 1, stream);
        if (ds.npp && ds.n_ecp) {
            const uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
            tm.begin(stream);
            const int nl = nl_passes(wk[which], [&](int w0, int w1, const void* U0, const void* U1) {
                if (mode == QMC_MIXED) {
                    QMC_CK(launch_nlpp<float>(ds, wk[which], w0, w1, out, key, sweep, U0, U1, stream));
                } else {
                    QMC_CK(launch_nlpp<double>(ds, wk[which], w0, w1, out, key, sweep, U0, U1, stream));
                }
            });
            tm.end(F_NLPP, nl, stream);
        }
    }

    // The walker-tiled sweep takes mixed-precision single determinants with
    // delayed updates of a rank divisible by 4 and spin blocks of 4k
    // electrons (row strides TMA can address), from tiled_min_n electrons of
    // one spin up to the tensor-core GEMM's 256 columns.
    bool tiled_eligible() const {
        const int nmax = std::max(n_up, n_dn);
        return tiled_enable && n3 == 0 && mode == QMC_MIXED && !ds.msd && delay_rank > 1 && delay_rank % 4 == 0 &&
               n_up % 4 == 0 && n_dn % 4 == 0 && nmax >= tiled_min_n && nmax <= 256 &&
               (int)sh_l.size() <= kTiledMaxShells;
    }

    void ensure_tiled() {
        if (tiled_W >= W && tiled_W > 0) return;
        free_list(tiled_allocs);
        const int Wt = std::max(W, 1);
        const int nmax = std::max(n_up, n_dn), kmax = delay_rank;
        TiledState t{};
        t.kmax = kmax;
        t.ldv = (nmax + 3) & ~3;
        t.nbp = (n_basis + 3) & ~3;
        t.Bh = dalloc<float>(tiled_allocs, (size_t)Wt * 5 * t.nbp);
        t.Bl = dalloc<float>(tiled_allocs, (size_t)Wt * 5 * t.nbp);
        t.Phi = dalloc<float>(tiled_allocs, (size_t)Wt * 5 * nmax);
        for (int spin = 0; spin < 2; ++spin) {
            t.Cth[spin] = dalloc<float>(tiled_allocs, (size_t)std::max(spin ? n_dn : n_up, 1) * t.nbp);
            t.Ctl[spin] = dalloc<float>(tiled_allocs, (size_t)std::max(spin ? n_dn : n_up, 1) * t.nbp);
        }
        t.ce = dalloc<float>(tiled_allocs, (size_t)Wt * t.ldv);
        t.V = dalloc<float>(tiled_allocs, (size_t)Wt * kmax * t.ldv);
        t.P = dalloc<float>(tiled_allocs, (size_t)Wt * kmax * t.ldv);
        t.Zt = dalloc<float>(tiled_allocs, (size_t)Wt * nmax * kmax);
        t.Xt = dalloc<float>(tiled_allocs, (size_t)Wt * nmax * kmax);
        t.KinvT = dalloc<float2>(tiled_allocs, (size_t)Wt * kmax * kmax);
        t.tv = dalloc<float2>(tiled_allocs, (size_t)Wt * kmax);
        t.rows = dalloc<int>(tiled_allocs, (size_t)Wt * kmax);
        t.dq = dalloc<int>(tiled_allocs, Wt);
        t.acc = dalloc<unsigned>(tiled_allocs, Wt);
        t.mv = dalloc<float>(tiled_allocs, (size_t)Wt * kTiledMv);
        t.rn = dalloc<double>(tiled_allocs, (size_t)Wt * 3);
        t.Rp = dalloc<float2>(tiled_allocs, (size_t)Wt * 3 * N());
        {
            std::vector<int> fs;
            for (int q = 0; q < (int)sh_l.size(); ++q) {
                const int nf = sh_l[q] == 0 ? 1 : sh_l[q] == 1 ? 3 : (sh_pure[q] ? 5 : 6);
                for (int f = 0; f < nf; ++f) fs.push_back(q);
            }
            t.fn_shell = upload(tiled_allocs, fs);
        }
        // the padding columns of B' and the queue rows are read by the GEMMs
        // before anything is written there: start from zeros
        QMC_CK(cudaMemsetAsync(t.Bh, 0, sizeof(float) * (size_t)Wt * 5 * t.nbp, stream));
        QMC_CK(cudaMemsetAsync(t.Bl, 0, sizeof(float) * (size_t)Wt * 5 * t.nbp, stream));
        QMC_CK(cudaMemsetAsync(t.V, 0, sizeof(float) * (size_t)Wt * kmax * t.ldv, stream));
        QMC_CK(launch_tiled_coeffs(ds, t, stream));
        tiled = t;
        tiled_W = Wt;
    }

    // Walker-tiled sweep: per electron a propose launch, the orbital GEMM on
    // the tensor cores and an accept launch; the queues are flushed every
    // delay_rank electrons and at the end of each spin block.  The walkers
    // are split into groups (whole 128-row tiles of the GEMM, at least 256
    // walkers each) whose chains of launches run on separate streams: the
    // groups share no state, so one group's GEMM fills the SMs that the
    // other's latency-bound accept/propose leaves idle, and the GEMM of a
    // group is under one wave of tiles.  Timed as one span ("sweep"), the
    // GEMM launches inside it also as their own family ("sweep_gemm").
    void sweep_tiled(const SweepParams& p) {
        ensure_tiled();
        const DevWalkers& k = wk[cur];
        const int groups_max = std::max(1, std::min(tiled_groups, W / 256));
        const int per = ((W + groups_max - 1) / groups_max + 127) / 128 * 128;
        const int ng = std::max(1, (W + per - 1) / per);
        int gw0[kTiledMaxGroups + 1];
        for (int g = 0; g <= ng; ++g) gw0[g] = std::min(W, g * per);
        cudaStream_t st[kTiledMaxGroups];
        st[0] = stream;
        for (int g = 1; g < ng; ++g) {
            if (!tiled_side[g - 1]) QMC_CK(cudaStreamCreateWithFlags(&tiled_side[g - 1], cudaStreamNonBlocking));
            st[g] = tiled_side[g - 1];
        }
        for (int g = 0; g < ng; ++g)
            if (!tiled_ev[g]) QMC_CK(cudaEventCreateWithFlags(&tiled_ev[g], cudaEventDisableTiming));
        TcSplitPlan plan[kTiledMaxGroups][2];
        for (int g = 0; g < ng; ++g)
            for (int spin = 0; spin < 2; ++spin) {
                const int n = spin ? n_dn : n_up;
                if (n == 0) continue;
                const size_t off = (size_t)gw0[g] * 5 * tiled.nbp;
                require(tc_split_plan(&plan[g][spin], 5 * (gw0[g + 1] - gw0[g]), n, tiled.nbp, tiled.Bh + off,
                                      tiled.Bl + off, tiled.nbp, tiled.Cth[spin], tiled.Ctl[spin], tiled.nbp),
                        QMC_ERR_UNSUPPORTED, "tensor maps of the tiled sweep's orbital GEMM could not be encoded");
            }
        for (int spin = 0; spin < 2; ++spin)
            if ((spin ? n_dn : n_up) > 0) QMC_CK(tc_split_prepare(spin ? n_dn : n_up));
        cudaEvent_t t0 = tm.mark(stream);
        int launches = 1;
        QMC_CK(tiled_begin(k, W, N(), tiled, stream));
        if (ng > 1) {
            QMC_CK(cudaEventRecord(tiled_ev[0], stream));
            for (int g = 1; g < ng; ++g) QMC_CK(cudaStreamWaitEvent(st[g], tiled_ev[0], 0));
        }
        auto chains = [&] {
            for (int g = 0; g < ng; ++g)
                QMC_CK(tiled_propose(ds, k, tiled, gw0[g], gw0[g + 1] - gw0[g], 0, p, st[g]));
            launches += ng;
            for (int e = 0; e < N(); ++e) {
                const int spin = e >= n_up, n = spin ? n_dn : n_up, kk = spin ? e - n_up : e;
                const bool flush = (kk + 1) % tiled.kmax == 0 || e == n_up - 1 || e == N() - 1;
                for (int g = 0; g < ng; ++g) {
                    const int w0 = gw0[g], nw = gw0[g + 1] - gw0[g];
                    cudaEvent_t a = tm.mark(st[g]);
                    QMC_CK(launch_tc_gemm_split(plan[g][spin], tiled.Phi + (size_t)w0 * 5 * n, n, d_err, st[g]));
                    tm.span(F_SWEEP_GEMM, 1, a, st[g]);
                    if (flush) {
                        // accept, flush the queues, then (unless it was the
                        // last electron) propose the next electron's move
                        QMC_CK(tiled_accept(ds, k, tiled, w0, nw, e, p, st[g]));
                        QMC_CK(tiled_flush(k, tiled, w0, nw, spin, n, d_err, st[g]));
                        if (e + 1 < N()) QMC_CK(tiled_propose(ds, k, tiled, w0, nw, e + 1, p, st[g]));
                        launches += e + 1 < N() ? 6 : 5;
                    } else {
                        QMC_CK(tiled_accept_propose(ds, k, tiled, w0, nw, e, p, st[g]));
                        launches += 1;
                    }
                }
            }
        };
        // the handle's stream waits for every side stream again, also when a
        // launch fails part-way (no work of the sweep left unordered)
        auto join = [&] {
            for (int g = 1; g < ng; ++g) {
                const cudaError_t e1 = cudaEventRecord(tiled_ev[g], st[g]);
                const cudaError_t e2 = cudaStreamWaitEvent(stream, tiled_ev[g], 0);
                if (e1 != cudaSuccess || e2 != cudaSuccess) return e1 != cudaSuccess ? e1 : e2;
            }
            return cudaSuccess;
        };
        try {
            chains();
        } catch (...) {
            join();
            throw;
        }
        QMC_CK(join());
        QMC_CK(tiled_end(tiled, W, d_nacc, stream));
        tm.span(F_SWEEP, launches + 1, t0, stream);
    }

    void sweep_once(double tau) {
        require(n3 == 0 || (!ds.msd && delay_rank == 1), QMC_ERR_UNSUPPORTED,
                "the three-body Jastrow is carried by the Sherman-Morrison sweep of a single determinant only "
                "(delay rank 1)");
        SweepParams p{};
        p.tau = tau;
        p.key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
        p.sweep = sweep;
        if (ds.msd) {
            const size_t need = mode == QMC_MIXED ? msd_sweep_smem_bytes<float>(ds) : msd_sweep_smem_bytes<double>(ds);
            require(need <= 227 * 1024, QMC_ERR_UNSUPPORTED,
                    "determinant-expansion sweep needs " + std::to_string(need) + " bytes of shared memory");
            tm.begin(stream);
            if (mode == QMC_MIXED) {
                QMC_CK(launch_sweep_msd<float>(ds, wk[cur], W, p, stream));
            } else {
                QMC_CK(launch_sweep_msd<double>(ds, wk[cur], W, p, stream));
            }
            tm.end(F_SWEEP, 1, stream);
            // walkers flagged by the sweep (reference determinant near its
            // node on an accepted move): FP64 rebuild of their state only
            tm.begin(stream);
            const DevWalkers& k = wk[cur];
            if (mode == QMC_MIXED) {
                QMC_CK(launch_orbitals_all<float>(ds, k, W, stream, d_refresh));
            } else {
                QMC_CK(launch_orbitals_all<double>(ds, k, W, stream, d_refresh));
            }
            QMC_CK(launch_invert(ds, k, W, mode == QMC_MIXED, d_err, stream, d_refresh));
            if (mode == QMC_MIXED) {
                QMC_CK(launch_msd_table<float>(ds, k, W, stream, d_refresh));
            } else {
                QMC_CK(launch_msd_table<double>(ds, k, W, stream, d_refresh));
            }
            QMC_CK(cudaMemsetAsync(d_refresh, 0, sizeof(int) * W, stream));
            tm.end(F_RECOMPUTE, 3, stream);
            n_prop += (long long)W * N();
            ++sweep;
            ++sweeps_since_recompute;
            return;
        }
        // A^-1 is read and rewritten on every accepted move and stays in
        // shared memory; the gradient cache is touched once per move (one
        // row) and lives in global memory so that more walkers fit per SM.
        p.ainv_smem = 1;
        p.g_smem = 0;
        const size_t limit = 227 * 1024;
        if (tiled_eligible()) {
            sweep_tiled(p);
            n_prop += (long long)W * N();
            ++sweep;
            ++sweeps_since_recompute;
            return;
        }
        if (delay_rank > 1) {
            const size_t need =
                mode == QMC_MIXED ? delayed_smem_bytes<float>(ds, delay_rank) : delayed_smem_bytes<double>(ds, delay_rank);
            require(need <= limit, QMC_ERR_UNSUPPORTED,
                    "delayed-update sweep needs " + std::to_string(need) + " bytes of shared memory");
            tm.begin(stream);
            if (mode == QMC_MIXED) {
                QMC_CK(launch_sweep_delayed<float>(ds, wk[cur], W, p, delay_rank, stream));
            } else {
                QMC_CK(launch_sweep_delayed<double>(ds, wk[cur], W, p, delay_rank, stream));
            }
            tm.end(F_SWEEP, 1, stream);
            n_prop += (long long)W * N();
            ++sweep;
            ++sweeps_since_recompute;
            return;
        }
        tm.begin(stream);
        if (mode == QMC_MIXED) {
            if (sweep_smem_bytes<float>(ds, 1, p.g_smem) > limit) p.ainv_smem = 0;
            QMC_CK(launch_sweep<float>(ds, wk[cur], W, p, nullptr, stream));
        } else {
            if (sweep_smem_bytes<double>(ds, 1, p.g_smem) > limit) p.ainv_smem = 0;
            QMC_CK(launch_sweep<double>(ds, wk[cur], W, p, nullptr, stream));
        }
        tm.end(F_SWEEP, 1, stream);
        n_prop += (long long)W * N();
        ++sweep;
        ++sweeps_since_recompute;
    }

    template <typename T>
    void gemm_sb(cublasOperation_t ta, cublasOperation_t tb, int m, int n, int k, const T* A, int lda, long long sA,
                 const T* B, int ldb, long long sB, T* Cm, int ldc, long long sC, int batch);

    // Adjoint forces with the dense products as batched GEMMs, in walker
    // chunks: prep (B, grad J, Jastrow terms) -> PT = AT B^T, Q = PT AT,
    // M = C AT^T, Y = C Q^T per spin -> third-order basis contraction.
    template <typename T>
    void forces_gemm(const DevWalkers& kw) {
        const int nmax = std::max(n_up, n_dn), nb = n_basis, N3 = 3 * N(), nn = n_nuc;
        const int Wc = std::min(W, 512);
        if (fchunk < Wc) {
            fchunk = std::max(Wc, std::min(cap, 512));
            d_fB = dalloc<T>(wk_allocs, 2 * (size_t)fchunk * nmax * nmax);
            d_fPT = dalloc<T>(wk_allocs, 2 * (size_t)fchunk * nmax * nmax);
            d_fQ = dalloc<T>(wk_allocs, 2 * (size_t)fchunk * nmax * nmax);
            d_fM = dalloc<T>(wk_allocs, 2 * (size_t)fchunk * nb * nmax);
            d_fY = dalloc<T>(wk_allocs, 2 * (size_t)fchunk * nb * nmax);
            d_fgJ = dalloc<double>(wk_allocs, (size_t)fchunk * N3);
            d_faccw = dalloc<double>(wk_allocs, (size_t)fchunk * 6 * nn);
        }
        if (!blas) {
            require(cublasCreate(&blas) == CUBLAS_STATUS_SUCCESS, QMC_ERR_CUDA, "cublasCreate failed");
        }
        require(cublasSetStream(blas, stream) == CUBLAS_STATUS_SUCCESS, QMC_ERR_CUDA, "cublasSetStream failed");
        const DevWalkers& k = kw;
        for (int w0 = 0; w0 < W; w0 += Wc) {
            const int wc = std::min(Wc, W - w0);
            QMC_CK(launch_force_prep<T>(ds, k, w0, wc, d_dvnn, d_fB, d_fgJ, d_faccw, d_gtot, stream));
            for (int spin = 0; spin < 2; ++spin) {
                const int n = spin ? n_dn : n_up;
                if (n == 0) continue;
                const T* AT = (const T*)k.Ainv[spin] + (size_t)w0 * n * n;
                const T* Bm = (const T*)d_fB + (size_t)spin * wc * nmax * nmax;
                T* PT = (T*)d_fPT + (size_t)spin * wc * nmax * nmax;
                T* Q = (T*)d_fQ + (size_t)spin * wc * nmax * nmax;
                T* M = (T*)d_fM + (size_t)spin * wc * nb * n;
                T* Y = (T*)d_fY + (size_t)spin * wc * nb * n;
                const T* Cs = sizeof(T) == 8 ? (const T*)(const void*)ds.C[spin] : (const T*)(const void*)ds.C_f[spin];
                const long long nn2 = (long long)nmax * nmax, n2 = (long long)n * n;
                if (sizeof(T) == 4 && !force_gemm_cublas) {
                    // tensor cores (3xTF32): D_b = A_b B_b^T (B_b when transposed)
                    const float* ATf = (const float*)(const void*)AT;
                    const float* Bf = (const float*)(const void*)Bm;
                    const float* Cf = (const float*)(const void*)Cs;
                    float* PTf = (float*)(void*)PT;
                    float* Qf = (float*)(void*)Q;
                    QMC_CK(launch_tc_gemm(wc, n, n, n, ATf, n2, n, Bf, nn2, n, 0, PTf, nn2, n, d_err, stream));
                    QMC_CK(launch_tc_gemm(wc, n, n, n, PTf, nn2, n, ATf, n2, n, 1, Qf, nn2, n, d_err, stream));
                    QMC_CK(launch_tc_gemm(wc, nb, n, n, Cf, 0, n, ATf, n2, n, 0, (float*)(void*)M, (long long)nb * n, n,
                                          d_err, stream));
                    QMC_CK(launch_tc_gemm(wc, nb, n, n, Cf, 0, n, Qf, nn2, n, 0, (float*)(void*)Y, (long long)nb * n, n,
                                          d_err, stream));
                    continue;
                }
                // column-major views of row-major matrices are their transposes
                gemm_sb<T>(CUBLAS_OP_T, CUBLAS_OP_N, n, n, n, Bm, n, nn2, AT, n, n2, PT, n, nn2, wc);   // PT = AT B^T
                gemm_sb<T>(CUBLAS_OP_N, CUBLAS_OP_N, n, n, n, AT, n, n2, PT, n, nn2, Q, n, nn2, wc);    // Q = PT AT
                gemm_sb<T>(CUBLAS_OP_T, CUBLAS_OP_N, n, nb, n, AT, n, n2, Cs, n, 0, M, n, (long long)nb * n, wc);
                gemm_sb<T>(CUBLAS_OP_T, CUBLAS_OP_N, n, nb, n, Q, n, nn2, Cs, n, 0, Y, n, (long long)nb * n, wc);
            }
            QMC_CK(launch_force_contract<T>(ds, k, w0, wc, d_fM, d_fY, d_fgJ, d_faccw, d_dEL, d_dlog, d_gEdet,
                                            stream));
        }
    }

    void forces_per_walker(int which) {
        require(n3 == 0, QMC_ERR_UNSUPPORTED, "no ionic derivatives of the three-body Jastrow");
        require(n_pp == 0 || (!ds.msd && !space_warp), QMC_ERR_UNSUPPORTED,
                "the pseudopotential's ionic derivatives are carried for single determinants without space warp");
        if (space_warp && !d_gEdet) {
            d_gEdet = dalloc<double>(wk_allocs, (size_t)cap * 3 * N());
            d_gtot = dalloc<double>(wk_allocs, (size_t)cap * 3 * N());
        }
        double* gE = space_warp ? d_gEdet : nullptr;
        double* gt = space_warp ? d_gtot : nullptr;
        // non-local pseudopotential: its rows of the B matrix (so that
        // X = A^-1 B A^-1 of Eq. 4 carries them) and its direct terms, by a
        // force pass of the non-local kernel ahead of either force path
        DevWalkers k = wk[which];
        if (ds.npp && ds.n_ecp) {
            const size_t nB = (size_t)n_up * n_up + (size_t)n_dn * n_dn;
            if (!d_nlB) {
                d_nlB = dalloc<double>(wk_allocs, (size_t)cap * nB);
                d_nlF = dalloc<double>(wk_allocs, (size_t)cap * 3 * n_nuc);
            }
            void* b0 = d_nlB;
            void* b1 = (unsigned char*)d_nlB + (size_t)cap * n_up * n_up * elem();
            tm.begin(stream);
            // rows of electrons out of every cutoff stay zero: clear the live walkers' blocks
            QMC_CK(cudaMemsetAsync(b0, 0, (size_t)W * n_up * n_up * elem(), stream));
            QMC_CK(cudaMemsetAsync(b1, 0, (size_t)W * n_dn * n_dn * elem(), stream));
            const uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
            const int nl = nl_passes(k, [&](int w0, int w1, const void* U0, const void* U1) {
                if (mode == QMC_MIXED) {
                    QMC_CK(launch_nlpp_force<float>(ds, k, w0, w1, b0, b1, d_nlF, key, sweep, U0, U1, stream));
                } else {
                    QMC_CK(launch_nlpp_force<double>(ds, k, w0, w1, b0, b1, d_nlF, key, sweep, U0, U1, stream));
                }
            });
            tm.end(F_FORCE, nl, stream);
            k.nlB[0] = b0;
            k.nlB[1] = b1;
            k.nlF = d_nlF;
        }
        if (!ds.msd && std::max(n_up, n_dn) >= force_gemm_min_n) {
            tm.begin(stream);
            if (mode == QMC_MIXED)
                forces_gemm<float>(k);
            else
                forces_gemm<double>(k);
            tm.end(F_FORCE, 2, stream);
        } else if (ds.msd) {
            if (!d_fmsd) d_fmsd = dalloc<double>(wk_allocs, (size_t)cap * force_msd_scratch_words(ds));
            tm.begin(stream);
            if (mode == QMC_MIXED) {
                QMC_CK(launch_force_msd<float>(ds, wk[which], W, d_dvnn, d_fmsd, d_dEL, d_dlog, gE, gt, stream));
            } else {
                QMC_CK(launch_force_msd<double>(ds, wk[which], W, d_dvnn, d_fmsd, d_dEL, d_dlog, gE, gt, stream));
            }
            tm.end(F_FORCE, 1, stream);
        } else {
            tm.begin(stream);
            if (mode == QMC_MIXED) {
                QMC_CK(launch_force<float>(ds, k, W, d_dvnn, d_Bscr, d_Pscr, d_dEL, d_dlog, gE, gt, stream));
            } else {
                QMC_CK(launch_force<double>(ds, k, W, d_dvnn, d_Bscr, d_Pscr, d_dEL, d_dlog, gE, gt, stream));
            }
            tm.end(F_FORCE, 1, stream);
        }
        if (space_warp) {
            tm.begin(stream);
            if (mode == QMC_MIXED) {
                QMC_CK(launch_space_warp<float>(ds, wk[which], W, d_gEdet, d_gtot, d_dEL, d_dlog, stream));
            } else {
                QMC_CK(launch_space_warp<double>(ds, wk[which], W, d_gEdet, d_gtot, d_dEL, d_dlog, stream));
            }
            tm.end(F_FORCE, 1, stream);
        }
    }

    // Weighted force sums of the walkers currently in d_dEL / d_dlog with
    // weights wts[W] and energies E[W].
    ForceSample force_sample(const double* wts, const double* E) {
        const int K = 3 * n_nuc;
        tm.begin(stream);
        k_mul<<<(W + 255) / 256, 256, 0, stream>>>(wts, E, W, d_wE);
        QMC_CK(cudaGetLastError());
        QMC_CK(launch_weighted_sum(wts, nullptr, W, 1, d_facc, 0, stream));
        QMC_CK(launch_weighted_sum(d_wE, nullptr, W, 1, d_facc + 1, 0, stream));
        QMC_CK(launch_weighted_sum(d_dEL, wts, W, K, d_facc + 2, 0, stream));
        QMC_CK(launch_weighted_sum(d_dlog, d_wE, W, K, d_facc + 2 + K, 0, stream));
        QMC_CK(launch_weighted_sum(d_dlog, wts, W, K, d_facc + 2 + 2 * K, 0, stream));
        tm.end(F_REDUCE, 6, stream);
        ForceSample fs;
        fs.v.resize(2 + 3 * K);
        QMC_CK(cudaMemcpyAsync(fs.v.data(), d_facc, sizeof(double) * fs.v.size(), cudaMemcpyDeviceToHost, stream));
        sync();
        return fs;
    }

    void invalidate() {
        walkers_valid = false;
        sys_dirty = true;
        ++gen;
    }
};

template <>
void qmc_ctx::gemm_sb<double>(cublasOperation_t ta, cublasOperation_t tb, int m, int n, int k, const double* A, int lda,
                              long long sA, const double* B, int ldb, long long sB, double* Cm, int ldc, long long sC,
                              int batch) {
    const double one = 1.0, zero = 0.0;
    const cublasStatus_t st =
        cublasDgemmStridedBatched(blas, ta, tb, m, n, k, &one, A, lda, sA, B, ldb, sB, &zero, Cm, ldc, sC, batch);
    require(st == CUBLAS_STATUS_SUCCESS, QMC_ERR_CUDA, "cublasDgemmStridedBatched failed: " + std::to_string((int)st));
}

template <>
void qmc_ctx::gemm_sb<float>(cublasOperation_t ta, cublasOperation_t tb, int m, int n, int k, const float* A, int lda,
                             long long sA, const float* B, int ldb, long long sB, float* Cm, int ldc, long long sC,
                             int batch) {
    const float one = 1.f, zero = 0.f;
    const cublasStatus_t st =
        cublasSgemmStridedBatched(blas, ta, tb, m, n, k, &one, A, lda, sA, B, ldb, sB, &zero, Cm, ldc, sC, batch);
    require(st == CUBLAS_STATUS_SUCCESS, QMC_ERR_CUDA, "cublasSgemmStridedBatched failed: " + std::to_string((int)st));
}

namespace {

thread_local std::string g_create_error;

template <typename F>
int guarded(qmc_t h, F&& f) {
    try {
        f();
        if (h) h->err.clear();
        return QMC_OK;
    } catch (const QmcError& e) {
        if (h) h->err = e.msg;
        return e.code;
    } catch (const std::bad_alloc&) {
        if (h) h->err = "host allocation failed";
        return QMC_ERR_OOM;
    } catch (...) {
        if (h) h->err = "unexpected exception";
        return QMC_ERR_ARG;
    }
}

void need_walkers(qmc_t h) {
    require(h->walkers_valid && h->W > 0, QMC_ERR_STATE, "no walkers: call qmc_set_walkers first");
}

void copy_out(qmc_t h, void* dst, const void* src_dev, size_t bytes, int on_device) {
    if (!dst || bytes == 0) return;
    QMC_CK(cudaMemcpyAsync(dst, src_dev, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                           h->stream));
}

}  // namespace

extern "C" {

int qmc_create(qmc_t* out, int device, void* cuda_stream) {
    if (!out) return QMC_ERR_ARG;
    *out = nullptr;
    qmc_ctx* h = nullptr;
    try {
        h = new qmc_ctx();
    } catch (...) {
        g_create_error = "host allocation failed";
        return QMC_ERR_OOM;
    }
    int n_dev = 0;
    cudaError_t e = cudaGetDeviceCount(&n_dev);
    if (e != cudaSuccess || device < 0 || device >= n_dev) {
        g_create_error = e != cudaSuccess ? cudaGetErrorString(e) : "device index out of range";
        cudaGetLastError();
        delete h;
        return e != cudaSuccess ? QMC_ERR_CUDA : QMC_ERR_ARG;
    }
    h->device = device;
    if (const char* env = std::getenv("QMC_FORCE_GEMM_MIN_N")) h->force_gemm_min_n = std::max(1, std::atoi(env));
    if (const char* env = std::getenv("QMC_FORCE_GEMM_CUBLAS")) h->force_gemm_cublas = std::atoi(env) != 0;
    if (const char* env = std::getenv("QMC_SWEEP_TILED")) h->tiled_enable = std::atoi(env) != 0;
    if (const char* env = std::getenv("QMC_SWEEP_TILED_MIN_N")) h->tiled_min_n = std::max(4, std::atoi(env));
    if (const char* env = std::getenv("QMC_NLPP_TC")) h->nlpp_tc = std::atoi(env) != 0;
    if (const char* env = std::getenv("QMC_NLPP_TC_MIN_N")) h->nlpp_tc_min_n = std::max(1, std::atoi(env));
    if (const char* env = std::getenv("QMC_SWEEP_TILED_GROUPS"))
        h->tiled_groups = std::max(1, std::min(kTiledMaxGroups, std::atoi(env)));
    if (cudaSetDevice(device) != cudaSuccess) {
        g_create_error = "cudaSetDevice failed";
        delete h;
        return QMC_ERR_CUDA;
    }
    if (cuda_stream) {
        h->stream = (cudaStream_t)cuda_stream;
    } else {
        if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) {
            g_create_error = "cudaStreamCreate failed";
            delete h;
            return QMC_ERR_CUDA;
        }
        h->own_stream = true;
    }
    *out = h;
    return QMC_OK;
}

int qmc_destroy(qmc_t h) {
    if (!h) return QMC_ERR_ARG;
    cudaSetDevice(h->device);
    cudaStreamSynchronize(h->stream);
    h->tm.release();
    if (h->blas) cublasDestroy(h->blas);
    for (cudaStream_t t : h->tiled_side)
        if (t) {
            cudaStreamSynchronize(t);
            cudaStreamDestroy(t);
        }
    for (cudaEvent_t e : h->tiled_ev)
        if (e) cudaEventDestroy(e);
    h->free_list(h->wk_allocs);
    h->free_list(h->tiled_allocs);
    h->free_list(h->sys_allocs);
    if (h->own_stream) cudaStreamDestroy(h->stream);
    delete h;
    return QMC_OK;
}

const char* qmc_last_error(qmc_t h) { return h ? h->err.c_str() : g_create_error.c_str(); }

int qmc_set_system(qmc_t h, int n_nuc, const double* Z, const double* R, int n_up, int n_dn) {
    if (!h) return QMC_ERR_ARG;
    return guarded(h, [&] {
        require(n_nuc >= 1 && Z && R, QMC_ERR_ARG, "need at least one nucleus and non-null Z, R");
        require(n_up >= 0 && n_dn >= 0 && n_up + n_dn >= 1, QMC_ERR_ARG, "need at least one electron");
        require(n_up <= kMaxSpinElectrons && n_dn <= kMaxSpinElectrons, QMC_ERR_UNSUPPORTED,
                "at most " + std::to_string(kMaxSpinElectrons) + " electrons per spin");
        for (int a = 0; a < n_nuc; ++a)
            for (int c = 0; c < 3; ++c) require(std::isfinite(R[3 * a + c]), QMC_ERR_ARG, "non-finite nuclear position");
        h->n_nuc = n_nuc;
        h->Z.assign(Z, Z + n_nuc);
        h->Rn.assign(R, R + 3 * n_nuc);
        h->n_up = n_up;
        h->n_dn = n_dn;
        if ((int)h->a_en.size() != n_nuc) h->have_jas = false;
        if ((int)h->pp_rcut.size() != n_nuc) {   // per-nucleus data of another system
            h->n_pp = 0;
            h->pp_rcut.clear();
        }
        if ((int)h->c3.size() != n_nuc * h->n3) h->n3 = 0;
        h->have_sys = true;
        h->invalidate();
    });
}

int qmc_set_nuclei(qmc_t h, const double* R) {
    if (!h) return QMC_ERR_ARG;
    return guarded(h, [&] {
        require(h->have_sys && R, QMC_ERR_STATE, "call qmc_set_system first");
        for (int q = 0; q < 3 * h->n_nuc; ++q) require(std::isfinite(R[q]), QMC_ERR_ARG, "non-finite nuclear position");
        h->Rn.assign(R, R + 3 * h->n_nuc);
        h->sys_dirty = true;
        if (h->walkers_valid) {
            QMC_CK(cudaSetDevice(h->device));
            h->build_system();
            h->recompute(h->cur);
            h->eloc(h->cur, h->wk[h->cur].eloc, nullptr, nullptr, nullptr);
            h->check_device_errors();
        }
    });
}

int qmc_set_basis(qmc_t h, int n_shell, const int* center, const int* l, const int* pure, const int* nprim,
                  const double* alpha, const double* coef) {
    if (!h) return QMC_ERR_ARG;
    return guarded(h, [&] {
        require(n_shell >= 1 && center && l && pure && nprim && alpha && coef, QMC_ERR_ARG, "bad basis arrays");
        int np = 0, nb = 0;
        for (int q = 0; q < n_shell; ++q) {
            require(l[q] >= 0 && l[q] <= 2, QMC_ERR_UNSUPPORTED, "only s, p and d shells are supported");
            require(nprim[q] >= 1, QMC_ERR_ARG, "a shell needs at least one primitive");
            np += nprim[q];
            nb += shell_nfn(l[q], pure[q] ? 1 : 0);
        }
        for (int p = 0; p < np; ++p)
            require(alpha[p] >= 0.0 && std::isfinite(alpha[p]) && std::isfinite(coef[p]), QMC_ERR_ARG,
                    "exponents must be finite and >= 0");
        h->sh_center.assign(center, center + n_shell);
        h->sh_l.assign(l, l + n_shell);
        h->sh_pure.resize(n_shell);
        for (int q = 0; q < n_shell; ++q) h->sh_pure[q] = pure[q] ? 1 : 0;
        h->sh_nprim.assign(nprim, nprim + n_shell);
        h->alpha.assign(alpha, alpha + np);
        h->coef.assign(coef, coef + np);
        h->n_basis = nb;
        h->have_basis = true;
        h->invalidate();
    });
}

int qmc_set_mos(qmc_t h, int n_mo, int n_basis, const double* C, const int* occ_up, const int* occ_dn) {
    if (!h) return QMC_ERR_ARG;
    return guarded(h, [&] {
        require(h->have_sys, QMC_ERR_STATE, "call qmc_set_system first");
        require(n_mo >= 1 && n_basis >= 1 && C, QMC_ERR_ARG, "bad orbital matrix");
        require((h->n_up == 0 || occ_up) && (h->n_dn == 0 || occ_dn), QMC_ERR_ARG, "missing occupation list");
        for (int j = 0; j < h->n_up; ++j) require(occ_up[j] >= 0 && occ_up[j] < n_mo, QMC_ERR_ARG, "occ_up out of range");
        for (int j = 0; j < h->n_dn; ++j) require(occ_dn[j] >= 0 && occ_dn[j] < n_mo, QMC_ERR_ARG, "occ_dn out of range");
        h->n_mo = n_mo;
        h->n_basis_C = n_basis;
        h->C.assign(C, C + (size_t)n_mo * n_basis);
        h->occ_up.assign(occ_up ? occ_up : nullptr, occ_up ? occ_up + h->n_up : nullptr);
        h->occ_dn.assign(occ_dn ? occ_dn : nullptr, occ_dn ? occ_dn + h->n_dn : nullptr);
        h->have_mos = true;
        h->invalidate();
    });
}

int qmc_set_multidet(qmc_t h, int n_det, int n_words, const uint64_t* det_up, const uint64_t* det_dn,
                     const double* ci) {
    if (!h) return QMC_ERR_ARG;
    return guarded(h, [&] {
        require(h->have_sys, QMC_ERR_STATE, "call qmc_set_system first");
        if (n_det == 0) {
            h->have_msd = false;
            h->invalidate();
            return;
        }
        require(n_det >= 1 && n_words >= 1 && n_words <= 64 && det_up && det_dn && ci, QMC_ERR_ARG,
                "bad determinant expansion");
        for (int k = 0; k < n_det; ++k) require(std::isfinite(ci[k]), QMC_ERR_ARG, "non-finite CI coefficient");
        require(ci[0] != 0.0, QMC_ERR_ARG, "the reference determinant (first) needs a nonzero coefficient");
        h->msd_words = n_words;
        h->det_up.assign(det_up, det_up + (size_t)n_det * n_words);
        h->det_dn.assign(det_dn, det_dn + (size_t)n_det * n_words);
        h->ci.assign(ci, ci + n_det);
        for (int spin = 0; spin < 2; ++spin) {
            const std::vector<int> o = h->string_orbitals(spin ? &h->det_dn[0] : &h->det_up[0]);
            require((int)o.size() == (spin ? h->n_dn : h->n_up), QMC_ERR_ARG,
                    "reference string has the wrong electron count");
        }
        h->have_msd = true;
        h->invalidate();
    });
}

int qmc_set_jastrow(qmc_t h, double a_anti, double a_par, double b_ee, const double* a_en, double b_en) {
    if (!h) return QMC_ERR_ARG;
    return guarded(h, [&] {
        require(h->have_sys, QMC_ERR_STATE, "call qmc_set_system first");
        require(a_en != nullptr, QMC_ERR_ARG, "a_en must hold one value per nucleus");
        require(b_ee >= 0.0 && b_en >= 0.0, QMC_ERR_ARG, "Pade b parameters must be >= 0");
        h->a_anti = a_anti;
        h->a_par = a_par;
        h->b_ee = b_ee;
        h->b_en = b_en;
        h->a_en.assign(a_en, a_en + h->n_nuc);
        h->have_jas = true;
        h->invalidate();
    });
}

int qmc_set_jastrow3(qmc_t h, int n_terms, const int* exponents, const double* coef, double b3) {
    if (!h) return QMC_ERR_ARG;
    return guarded(h, [&] {
        require(h->have_sys, QMC_ERR_STATE, "call qmc_set_system first");
        require(n_terms >= 0 && n_terms <= 64, QMC_ERR_ARG, "0 <= n_terms <= 64");
        require(n_terms == 0 || (exponents && coef), QMC_ERR_ARG, "null exponents or coefficients");
        require(n_terms == 0 || (b3 > 0.0 && std::isfinite(b3)), QMC_ERR_ARG, "b3 must be positive");
        for (int q = 0; q < 3 * n_terms; ++q)
            require(exponents[q] == 0 || (exponents[q] >= 2 && exponents[q] <= 8), QMC_ERR_ARG,
                    "three-body exponents must be 0 or 2..8 (powers 1 would change the cusps)");
        for (int q = 0; q < h->n_nuc * n_terms; ++q)
            require(std::isfinite(coef[q]), QMC_ERR_ARG, "non-finite three-body coefficient");
        h->n3 = n_terms;
        h->e3.assign(exponents, exponents + 3 * n_terms);
        h->c3.assign(coef, coef + (size_t)h->n_nuc * n_terms);
        h->b3 = n_terms ? b3 : 1.0;
        h->invalidate();
    });
}

int qmc_set_pseudopotential(qmc_t h, int n_terms, const int* nucleus, const int* l, const int* n,
                            const double* alpha, const double* beta, const double* rcut, int n_quad,
                            const double* quad, const double* weights, int rotate) {
    if (!h) return QMC_ERR_ARG;
    return guarded(h, [&] {
        require(h->have_sys, QMC_ERR_STATE, "call qmc_set_system first");
        require(n_terms >= 0 && n_terms <= 4096, QMC_ERR_ARG, "0 <= n_terms <= 4096");
        if (n_terms > 0) {
            require(nucleus && l && n && alpha && beta && rcut, QMC_ERR_ARG, "null term array");
            require(n_quad >= 1 && n_quad <= 192 && quad && weights, QMC_ERR_ARG,
                    "a quadrature rule of 1..192 points is required");
            for (int t = 0; t < n_terms; ++t) {
                require(nucleus[t] >= 0 && nucleus[t] < h->n_nuc, QMC_ERR_ARG, "term nucleus out of range");
                require(l[t] >= -1 && l[t] <= 3, QMC_ERR_ARG, "channel l must be -1 (local) or 0..3");
                require(n[t] >= 0 && n[t] <= 8, QMC_ERR_ARG, "power n must be 0..8 (r^(n-2))");
                require(alpha[t] > 0.0 && std::isfinite(alpha[t]) && std::isfinite(beta[t]), QMC_ERR_ARG,
                        "term exponents must be positive and coefficients finite");
            }
            for (int a = 0; a < h->n_nuc; ++a)
                require(rcut[a] >= 0.0 && std::isfinite(rcut[a]), QMC_ERR_ARG, "cutoff radii must be finite, >= 0");
            for (int q = 0; q < n_quad; ++q) {
                const double* d = quad + 3 * q;
                const double nn = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                require(std::fabs(nn - 1.0) < 1e-12 && std::isfinite(weights[q]), QMC_ERR_ARG,
                        "quadrature points must be unit vectors with finite weights");
            }
        }
        h->n_pp = n_terms;
        h->pp_nuc.assign(nucleus, nucleus + n_terms);
        h->pp_l.assign(l, l + n_terms);
        h->pp_n.assign(n, n + n_terms);
        h->pp_alpha.assign(alpha, alpha + n_terms);
        h->pp_beta.assign(beta, beta + n_terms);
        h->pp_rcut.assign(n_terms ? rcut : nullptr, n_terms ? rcut + h->n_nuc : nullptr);
        h->pp_quad.assign(n_terms ? quad : nullptr, n_terms ? quad + 3 * n_quad : nullptr);
        h->pp_qw.assign(n_terms ? weights : nullptr, n_terms ? weights + n_quad : nullptr);
        h->pp_rotate = rotate ? 1 : 0;
        h->invalidate();
    });
}

int qmc_jastrow_derivs(qmc_t h, double* dlog, double* deloc, int on_device) {
    if (!h) return QMC_ERR_ARG;
    return guarded(h, [&] {
        need_walkers(h);
        require(dlog && deloc, QMC_ERR_ARG, "null output");
        QMC_CK(cudaSetDevice(h->device));
        const int W = h->W, N = h->N(), P = 4 + h->n_nuc + h->n_nuc * h->n3;
        h->recompute(h->cur);
        std::vector<void*> tmp;
        double* d_g = h->dalloc<double>(tmp, (size_t)W * N * 3);
        h->eloc(h->cur, h->wk[h->cur].eloc, nullptr, d_g, nullptr);
        double* d_l = on_device ? dlog : h->dalloc<double>(tmp, (size_t)W * P);
        double* d_e = on_device ? deloc : h->dalloc<double>(tmp, (size_t)W * P);
        h->tm.begin(h->stream);
        QMC_CK(launch_jastrow_derivs(h->ds, h->wk[h->cur].R, d_g, W, d_l, d_e, h->stream));
        h->tm.end(F_ELOC, 1, h->stream);
        if (h->ds.npp && h->ds.n_ecp) {
            // the non-local term's ratios carry the Jastrow: its part of dE_L/dp,
            // with the rotations of the E_L evaluated above
            const uint2 key = make_uint2((uint32_t)h->seed, (uint32_t)(h->seed >> 32));
            h->tm.begin(h->stream);
            const int nl = h->nl_passes(h->wk[h->cur], [&](int w0, int w1, const void* U0, const void* U1) {
                if (h->mode == QMC_MIXED) {
                    QMC_CK(launch_nlpp_param<float>(h->ds, h->wk[h->cur], w0, w1, d_e, key, h->sweep, U0, U1,
                                                    h->stream));
                } else {
                    QMC_CK(launch_nlpp_param<double>(h->ds, h->wk[h->cur], w0, w1, d_e, key, h->sweep, U0, U1,
                                                     h->stream));
                }
            });
            h->tm.end(F_NLPP, nl, h->stream);
        }
        if (!on_device) {
            copy_out(h, dlog, d_l, sizeof(double) * W * P, 0);
            copy_out(h, deloc, d_e, sizeof(double) * W * P, 0);
        }
        h->sync();
        h->free_list(tmp);
        h->check_device_errors();
    });
}

int qmc_set_precision(qmc_t h, int mode, int delay_rank, int recompute_period) {
    if (!h) return QMC_ERR_ARG;
    return guarded(h, [&] {
        require(mode == QMC_FP64 || mode == QMC_MIXED, QMC_ERR_ARG, "mode must be QMC_FP64 or QMC_MIXED");
        require(delay_rank >= 1 && delay_rank <= kMaxDelayRank, QMC_ERR_UNSUPPORTED,
                "delay_rank must be in [1, " + std::to_string(kMaxDelayRank) + "]");
        require(recompute_period >= 0, QMC_ERR_ARG, "recompute_period must be >= 0");
        if (mode != h->mode) h->invalidate();
        h->mode = mode;
        h->delay_rank = delay_rank;
        h->recompute_period = recompute_period;
    });
}

int qmc_set_population_control(qmc_t h, int mode) {
    if (!h) return QMC_ERR_ARG;
    return guarded(h, [&] {
        require(mode == QMC_POP_BRANCH || mode == QMC_POP_FIXED, QMC_ERR_ARG, "unknown population control");
        h->pop_mode = mode;
    });
}

int qmc_set_space_warp(qmc_t h, int enable) {
    if (!h) return QMC_ERR_ARG;
    return guarded(h, [&] {
        require(enable == 0 || enable == 1, QMC_ERR_ARG, "space warp flag must be 0 or 1");
        h->space_warp = enable;
    });
}

int qmc_set_rng(qmc_t h, uint64_t seed, uint32_t sweep) {
    if (!h) return QMC_ERR_ARG;
    h->seed = seed;
    h->sweep = sweep;
    return QMC_OK;
}

int qmc_set_capacity_factor(qmc_t h, int cap_factor) {
    if (!h) return QMC_ERR_ARG;
    return guarded(h, [&] {
        require(cap_factor >= 1 && cap_factor <= 16, QMC_ERR_ARG, "cap_factor must be in [1, 16]");
        h->cap_factor = cap_factor;
    });
}

int qmc_set_walkers(qmc_t h, int n_walkers, const double* R, int on_device) {
    if (!h) return QMC_ERR_ARG;
    return guarded(h, [&] {
        require(n_walkers >= 1 && R, QMC_ERR_ARG, "need at least one walker and non-null R");
        QMC_CK(cudaSetDevice(h->device));
        h->build_system();
        const size_t N3 = 3 * (size_t)h->N();
        if (!on_device) {
            for (size_t q = 0; q < (size_t)n_walkers * N3; ++q)
                require(std::isfinite(R[q]), QMC_ERR_ARG, "non-finite electron coordinate");
        }
        h->alloc_walkers(n_walkers);
        h->W = n_walkers;
        h->W0 = n_walkers;
        QMC_CK(cudaMemcpyAsync(h->wk[0].R, R, sizeof(double) * n_walkers * N3,
                               on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->stream));
        k_fill<<<(n_walkers + 255) / 256, 256, 0, h->stream>>>(h->wk[0].weight, n_walkers, 1.0);
        QMC_CK(cudaGetLastError());
        h->recompute(0);
        h->eloc(0, h->wk[0].eloc, nullptr, nullptr, nullptr);
        h->check_device_errors();
        h->walkers_valid = true;
        QMC_CK(cudaMemcpyAsync(&h->acc_base, h->d_nacc, sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                               h->stream));
        h->sync();
        h->n_prop = 0;
    });
}

int qmc_init_walkers(qmc_t h, int n_walkers, uint64_t seed) {
    if (!h) return QMC_ERR_ARG;
    return guarded(h, [&] {
        require(n_walkers >= 1, QMC_ERR_ARG, "need at least one walker");
        QMC_CK(cudaSetDevice(h->device));
        h->build_system();
        const int N = h->N();
        // round(Z_a) electrons per nucleus in nucleus order (extra electrons of
        // an anion on nucleus 0); spin up takes the even entries of that list,
        // spin down the odd ones (in order if one spin runs short)
        std::vector<int> owners;
        for (int a = 0; a < h->n_nuc; ++a)
            for (int q = 0; q < (int)std::lround(h->Z[a]); ++q) owners.push_back(a);
        while ((int)owners.size() < N) owners.push_back(0);
        owners.resize(N);
        std::vector<int> up, dn;
        for (int k = 0; k < N; ++k) (k % 2 == 0 ? up : dn).push_back(k);
        if ((int)up.size() < h->n_up || (int)dn.size() < h->n_dn) {
            up.clear();
            dn.clear();
            for (int k = 0; k < N; ++k) (k < h->n_up ? up : dn).push_back(k);
        }
        up.resize(h->n_up);
        dn.resize(h->n_dn);
        std::vector<int> owner;
        for (int k : up) owner.push_back(owners[k]);
        for (int k : dn) owner.push_back(owners[k]);
        h->alloc_walkers(n_walkers);
        h->W = n_walkers;
        h->W0 = n_walkers;
        const int* d_owner = h->upload(h->wk_allocs, owner);
        const uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
        const long long tot = (long long)n_walkers * N;
        k_init_walkers<<<(unsigned)((tot + 255) / 256), 256, 0, h->stream>>>(h->wk[0].R, n_walkers, N, d_owner,
                                                                             h->ds.Rn, key, 0.5);
        QMC_CK(cudaGetLastError());
        k_fill<<<(n_walkers + 255) / 256, 256, 0, h->stream>>>(h->wk[0].weight, n_walkers, 1.0);
        QMC_CK(cudaGetLastError());
        h->recompute(0);
        h->eloc(0, h->wk[0].eloc, nullptr, nullptr, nullptr);
        h->check_device_errors();
        h->walkers_valid = true;
        QMC_CK(cudaMemcpyAsync(&h->acc_base, h->d_nacc, sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                               h->stream));
        h->sync();
        h->n_prop = 0;
    });
}

int qmc_get_walkers(qmc_t h, double* R, double* weight, int on_device) {
    if (!h) return QMC_ERR_ARG;
    return guarded(h, [&] {
        need_walkers(h);
        copy_out(h, R, h->wk[h->cur].R, sizeof(double) * 3 * h->N() * h->W, on_device);
        copy_out(h, weight, h->wk[h->cur].weight, sizeof(double) * h->W, on_device);
        h->sync();
    });
}

int qmc_n_walkers(qmc_t h) {
    if (!h) return QMC_ERR_ARG;
    if (!h->walkers_valid) return QMC_ERR_STATE;
    return h->W;
}

static void evaluate_impl(qmc_t h, double* logpsi, double* sign, double* eloc, double* grad, int on_device,
                          bool recompute);

int qmc_evaluate(qmc_t h, double* logpsi, double* sign, double* eloc, double* grad, int on_device) {
    if (!h) return QMC_ERR_ARG;
    return guarded(h, [&] { evaluate_impl(h, logpsi, sign, eloc, grad, on_device, true); });
}

int qmc_eval_cached(qmc_t h, double* logpsi, double* sign, double* eloc, double* grad, int on_device) {
    if (!h) return QMC_ERR_ARG;
    return guarded(h, [&] { evaluate_impl(h, logpsi, sign, eloc, grad, on_device, false); });
}

static void evaluate_impl(qmc_t h, double* logpsi, double* sign, double* eloc, double* grad, int on_device,
                          bool recompute) {
    {
        need_walkers(h);
        QMC_CK(cudaSetDevice(h->device));
        const int W = h->W, N = h->N();
        if (recompute) h->recompute(h->cur);
        std::vector<void*> tmp;
        double* d_lp2 = nullptr;
        double* d_g = nullptr;
        if (logpsi && !on_device) d_lp2 = h->dalloc<double>(tmp, W);
        if (grad) d_g = on_device ? grad : h->dalloc<double>(tmp, (size_t)W * N * 3);
        h->eloc(h->cur, h->wk[h->cur].eloc, logpsi ? (on_device ? logpsi : d_lp2) : nullptr, d_g, nullptr);
        copy_out(h, eloc, h->wk[h->cur].eloc, sizeof(double) * W, on_device);
        if (logpsi && !on_device) copy_out(h, logpsi, d_lp2, sizeof(double) * W, 0);
        if (grad && !on_device) copy_out(h, grad, d_g, sizeof(double) * W * N * 3, 0);
        if (sign) {
            std::vector<double> sg(2 * (size_t)W);
            QMC_CK(cudaMemcpyAsync(sg.data(), h->wk[h->cur].sgn, sizeof(double) * 2 * W, cudaMemcpyDeviceToHost,
                                   h->stream));
            h->sync();
            std::vector<double> s1(W);
            for (int w = 0; w < W; ++w) s1[w] = sg[2 * w] * sg[2 * w + 1];
            if (h->ds.msd) {
                QMC_CK(cudaMemcpyAsync(s1.data(), h->d_sign, sizeof(double) * W, cudaMemcpyDeviceToHost, h->stream));
                h->sync();
            }
            QMC_CK(cudaMemcpyAsync(sign, s1.data(), sizeof(double) * W,
                                   on_device ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost, h->stream));
        }
        h->sync();
        h->free_list(tmp);
        h->check_device_errors();
    }
}

int qmc_force_vjp(qmc_t h, const double* g_eloc, const double* g_logpsi, double* dR, double* per_walker,
                  int on_device) {
    if (!h) return QMC_ERR_ARG;
    return guarded(h, [&] {
        need_walkers(h);
        QMC_CK(cudaSetDevice(h->device));
        const int W = h->W, K = 3 * h->n_nuc;
        h->forces_per_walker(h->cur);
        std::vector<void*> tmp;
        const double* gE = nullptr;
        const double* gL = nullptr;
        if (g_eloc) {
            if (on_device) {
                gE = g_eloc;
            } else {
                double* p = h->dalloc<double>(tmp, W);
                QMC_CK(cudaMemcpyAsync(p, g_eloc, sizeof(double) * W, cudaMemcpyHostToDevice, h->stream));
                gE = p;
            }
        }
        if (g_logpsi) {
            if (on_device) {
                gL = g_logpsi;
            } else {
                double* p = h->dalloc<double>(tmp, W);
                QMC_CK(cudaMemcpyAsync(p, g_logpsi, sizeof(double) * W, cudaMemcpyHostToDevice, h->stream));
                gL = p;
            }
        }
        if (dR) {
            double* d_out = on_device ? dR : h->dalloc<double>(tmp, K);
            QMC_CK(cudaMemsetAsync(d_out, 0, sizeof(double) * K, h->stream));
            if (gE) QMC_CK(launch_weighted_sum(h->d_dEL, gE, W, K, d_out, 1, h->stream));
            if (gL) QMC_CK(launch_weighted_sum(h->d_dlog, gL, W, K, d_out, 1, h->stream));
            if (!on_device) copy_out(h, dR, d_out, sizeof(double) * K, 0);
        }
        if (per_walker) {
            double* d_pw = on_device ? per_walker : h->dalloc<double>(tmp, (size_t)W * 2 * K);
            k_pack_per_walker<<<(W * K + 255) / 256, 256, 0, h->stream>>>(h->d_dEL, h->d_dlog, W, K, d_pw);
            QMC_CK(cudaGetLastError());
            if (!on_device) copy_out(h, per_walker, d_pw, sizeof(double) * W * 2 * K, 0);
        }
        h->sync();
        h->free_list(tmp);
    });
}

int qmc_vmc(qmc_t h, int n_sweeps, double tau, int forces_every, double* eloc_trace, int on_device) {
    if (!h) return QMC_ERR_ARG;
    return guarded(h, [&] {
        need_walkers(h);
        require(n_sweeps >= 0 && tau > 0.0 && std::isfinite(tau), QMC_ERR_ARG, "need n_sweeps >= 0 and tau > 0");
        QMC_CK(cudaSetDevice(h->device));
        const int W = h->W;
        for (int k = 0; k < n_sweeps; ++k) {
            h->sweep_once(tau);
            if (h->recompute_period > 0 && h->sweeps_since_recompute >= h->recompute_period) h->recompute(h->cur);
            h->eloc(h->cur, h->wk[h->cur].eloc, nullptr, nullptr, nullptr);
            if (eloc_trace)
                copy_out(h, eloc_trace + (size_t)k * W, h->wk[h->cur].eloc, sizeof(double) * W, on_device);
            h->tm.begin(h->stream);
            k_moments<<<1, 256, 0, h->stream>>>(h->wk[h->cur].eloc, W, h->d_tmp);
            QMC_CK(cudaGetLastError());
            h->tm.end(F_REDUCE, 1, h->stream);
            double m[2];
            QMC_CK(cudaMemcpyAsync(m, h->d_tmp, sizeof(m), cudaMemcpyDeviceToHost, h->stream));
            if (forces_every > 0 && k % forces_every == 0) {
                h->forces_per_walker(h->cur);
                h->vmc_f.push_back(h->force_sample(h->d_ones, h->wk[h->cur].eloc));
            }
            h->sync();
            h->vmc_e.push_back(m[0] / W);
            h->vmc_e2.push_back(m[1] / W);
        }
        h->check_device_errors();
    });
}

int qmc_trial_energy(const double* hist, int n_hist, double pop, double pop0, double tau, int fixed_pop,
                     double* e_trial) {
    if (!hist || !e_trial || n_hist < 1 || !(tau > 0.0) || (!fixed_pop && !(pop > 0.0 && pop0 > 0.0)))
        return QMC_ERR_ARG;
    const int k0 = n_hist > 20 ? n_hist - 20 : 0;
    double est = 0.0;
    for (int q = k0; q < n_hist; ++q) est += hist[q];
    est /= (double)(n_hist - k0);
    *e_trial = fixed_pop ? est : est - std::log(pop / pop0) / (10.0 * tau);
    return std::isfinite(*e_trial) ? QMC_OK : QMC_ERR_NONFINITE;
}

int qmc_set_step_reduce(qmc_t h, qmc_reduce_fn fn, void* ctx) {
    if (!h) return QMC_ERR_ARG;
    return guarded(h, [&] {
        h->reduce_fn = fn;
        h->reduce_ctx = ctx;
    });
}

int qmc_set_population_reference(qmc_t h, double pop0) {
    if (!h) return QMC_ERR_ARG;
    return guarded(h, [&] {
        require(pop0 >= 0.0 && std::isfinite(pop0), QMC_ERR_ARG, "the reference population must be >= 0");
        h->pop_ref = pop0;
    });
}

int qmc_dmc(qmc_t h, int n_steps, double tau, double e_trial, int n_equil, int forces_every, double* e_step,
            int* pop, double* e_trial_out) {
    if (!h) return QMC_ERR_ARG;
    return guarded(h, [&] {
        need_walkers(h);
        require(n_steps >= 0 && tau > 0.0 && std::isfinite(tau) && std::isfinite(e_trial), QMC_ERR_ARG,
                "need n_steps >= 0, tau > 0 and a finite trial energy");
        QMC_CK(cudaSetDevice(h->device));
        const double e_cut = 0.2 * std::sqrt((double)h->N() / tau);
        double ET = e_trial;
        std::vector<double> hist;
        for (int k = 0; k < n_steps; ++k) {
            const int W = h->W;
            const uint32_t sw = h->sweep;
            h->sweep_once(tau);
            if (h->recompute_period > 0 && h->sweeps_since_recompute >= h->recompute_period) h->recompute(h->cur);
            h->eloc(h->cur, h->d_eloc_new, nullptr, nullptr, nullptr);
            const bool do_f = forces_every > 0 && k >= n_equil && (k % forces_every) == 0;
            if (do_f) h->forces_per_walker(h->cur);
            BranchParams bp{};
            bp.tau = tau;
            bp.e_trial = ET;
            bp.e_cut = e_cut;
            bp.key = make_uint2((uint32_t)h->seed, (uint32_t)(h->seed >> 32));
            bp.sweep = sw;
            bp.cap = h->cap;
            bp.fixed_pop = h->pop_mode == QMC_POP_FIXED ? h->W0 : 0;
            h->tm.begin(h->stream);
            QMC_CK(launch_branch(h->ds, h->wk[h->cur], h->wk[1 - h->cur], W, h->d_eloc_new, bp, h->d_copies,
                                 h->d_offsets, h->d_wts, h->d_stats, h->elem(), h->stream));
            h->tm.end(F_BRANCH, 3, h->stream);
            // second moment of E_L under the branching weights
            h->tm.begin(h->stream);
            k_mul<<<(W + 255) / 256, 256, 0, h->stream>>>(h->d_wts, h->d_eloc_new, W, h->d_wE);
            QMC_CK(cudaGetLastError());
            QMC_CK(launch_weighted_sum(h->d_wE, h->d_eloc_new, W, 1, h->d_tmp, 0, h->stream));
            h->tm.end(F_REDUCE, 2, h->stream);
            ForceSample fs;
            if (do_f) fs = h->force_sample(h->d_wts, h->d_eloc_new);
            double st[5], m2 = 0.0;
            QMC_CK(cudaMemcpyAsync(st, h->d_stats, sizeof(st), cudaMemcpyDeviceToHost, h->stream));
            QMC_CK(cudaMemcpyAsync(&m2, h->d_tmp, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
            h->sync();
            const int Wn = (int)st[2];
            if (st[3] != 0.0 || Wn == 0)
                throw QmcError{QMC_ERR_POPULATION, Wn == 0 ? "population died out"
                                                           : "population " + std::to_string(Wn) +
                                                                 " exceeds capacity " + std::to_string(h->cap)};
            // this rank's step sums; with a reduce callback, the sums over all
            // ranks (every rank then sets the same trial energy and records
            // the same estimator samples)
            double sum_w = st[0], swe = st[1], swc = st[4], m2w = m2, Wtot = (double)Wn;
            double Wref = h->pop_ref > 0.0 ? h->pop_ref : (double)h->W0;
            if (h->reduce_fn) {
                std::vector<double> buf = {sum_w, swe, Wtot, swc, m2w, Wref};
                if (do_f) buf.insert(buf.end(), fs.v.begin(), fs.v.end());
                require(h->reduce_fn(buf.data(), (int)buf.size(), h->reduce_ctx) == 0, QMC_ERR_STATE,
                        "the step reduction callback failed");
                sum_w = buf[0];
                swe = buf[1];
                Wtot = buf[2];
                swc = buf[3];
                m2w = buf[4];
                Wref = buf[5];
                if (do_f) std::copy(buf.begin() + 6, buf.end(), fs.v.begin());
            }
            const double Ek = swe / sum_w;
            if (!std::isfinite(Ek)) throw QmcError{QMC_ERR_NONFINITE, "non-finite DMC step energy"};
            if (e_step) e_step[k] = Ek;
            if (k >= n_equil) {
                h->dmc_e.push_back(Ek);
                h->dmc_e2.push_back(m2w / sum_w);
                if (do_f) h->dmc_f.push_back(fs);
            }
            h->cur = 1 - h->cur;
            h->W = Wn;
            if (pop) pop[k] = Wn;
            hist.push_back(swc / sum_w);   // clipped energies set the growth rate
            const int st_et = qmc_trial_energy(hist.data(), (int)hist.size(), Wtot, Wref, tau,
                                               h->pop_mode == QMC_POP_FIXED, &ET);
            require(st_et == QMC_OK, st_et, "trial energy update failed");
            if (e_trial_out) e_trial_out[k] = ET;
        }
        h->check_device_errors();
    });
}

int qmc_get_energy(qmc_t h, int estimator, double* mean, double* stderr_blocked, double* variance,
                   double* acceptance) {
    if (!h) return QMC_ERR_ARG;
    return guarded(h, [&] {
        require(estimator == QMC_EST_VMC || estimator == QMC_EST_DMC || estimator == QMC_EST_MIXED, QMC_ERR_ARG,
                "unknown estimator");
        const std::vector<double>& e = estimator == QMC_EST_VMC ? h->vmc_e : h->dmc_e;
        const std::vector<double>& e2 = estimator == QMC_EST_VMC ? h->vmc_e2 : h->dmc_e2;
        require(!e.empty(), QMC_ERR_STATE, "no samples for this estimator");
        double m = 0.0, m2 = 0.0;
        for (size_t q = 0; q < e.size(); ++q) {
            m += e[q];
            m2 += e2[q];
        }
        m /= e.size();
        m2 /= e.size();
        if (mean) *mean = m;
        if (stderr_blocked) *stderr_blocked = blocked_error(e);
        if (variance) *variance = m2 - m * m;
        if (acceptance) {
            unsigned long long a = 0;
            if (h->d_nacc) {
                QMC_CK(cudaMemcpyAsync(&a, h->d_nacc, sizeof(a), cudaMemcpyDeviceToHost, h->stream));
                h->sync();
            }
            *acceptance = h->n_prop > 0 ? (double)(a - h->acc_base) / (double)h->n_prop : 0.0;
        }
    });
}

static void force_from_samples(const std::vector<ForceSample>& f, int K, std::vector<double>& F,
                               std::vector<double>& Ferr) {
    F.assign(K, 0.0);
    Ferr.assign(K, 0.0);
    if (f.empty()) return;
    std::vector<double> tot(2 + 3 * K, 0.0);
    for (const ForceSample& s : f)
        for (size_t q = 0; q < tot.size(); ++q) tot[q] += s.v[q];
    auto est = [K](const std::vector<double>& t, int k) {
        const double sw = t[0], E = t[1] / sw;
        return -(t[2 + k] / sw + 2.0 * (t[2 + K + k] / sw - E * t[2 + 2 * K + k] / sw));
    };
    for (int k = 0; k < K; ++k) {
        F[k] = est(tot, k);
        std::vector<double> series(f.size());
        for (size_t q = 0; q < f.size(); ++q) series[q] = est(f[q].v, k);
        Ferr[k] = blocked_error(series);
    }
}

int qmc_get_forces(qmc_t h, int estimator, double* F, double* F_err) {
    if (!h) return QMC_ERR_ARG;
    return guarded(h, [&] {
        const int K = 3 * h->n_nuc;
        std::vector<double> fv, ev, fd, ed;
        force_from_samples(h->vmc_f, K, fv, ev);
        force_from_samples(h->dmc_f, K, fd, ed);
        if (estimator == QMC_EST_VMC) {
            require(!h->vmc_f.empty(), QMC_ERR_STATE, "no VMC force samples");
        } else if (estimator == QMC_EST_DMC) {
            require(!h->dmc_f.empty(), QMC_ERR_STATE, "no DMC force samples");
        } else {
            require(estimator == QMC_EST_MIXED, QMC_ERR_ARG, "unknown estimator");
            require(!h->vmc_f.empty() && !h->dmc_f.empty(), QMC_ERR_STATE, "mixed estimator needs VMC and DMC samples");
        }
        for (int k = 0; k < K; ++k) {
            double v, e;
            if (estimator == QMC_EST_VMC) {
                v = fv[k];
                e = ev[k];
            } else if (estimator == QMC_EST_DMC) {
                v = fd[k];
                e = ed[k];
            } else {
                v = 2.0 * fd[k] - fv[k];
                e = std::sqrt(4.0 * ed[k] * ed[k] + ev[k] * ev[k]);
            }
            if (F) F[k] = v;
            if (F_err) F_err[k] = e;
        }
    });
}

int qmc_force_estimate(qmc_t h, const double* weights, double* F, int on_device) {
    if (!h) return QMC_ERR_ARG;
    return guarded(h, [&] {
        need_walkers(h);
        require(F != nullptr, QMC_ERR_ARG, "F is null");
        QMC_CK(cudaSetDevice(h->device));
        const int W = h->W, K = 3 * h->n_nuc;
        h->forces_per_walker(h->cur);
        std::vector<void*> tmp;
        const double* wts = h->d_ones;
        if (weights) {
            if (on_device) {
                wts = weights;
            } else {
                for (int w = 0; w < W; ++w)
                    require(std::isfinite(weights[w]) && weights[w] >= 0.0, QMC_ERR_ARG,
                            "weights must be finite and non-negative");
                double* p = h->dalloc<double>(tmp, W);
                QMC_CK(cudaMemcpyAsync(p, weights, sizeof(double) * W, cudaMemcpyHostToDevice, h->stream));
                wts = p;
            }
        }
        ForceSample fs = h->force_sample(wts, h->wk[h->cur].eloc);
        h->free_list(tmp);
        require(fs.v[0] > 0.0, QMC_ERR_ARG, "the weights sum to zero");
        std::vector<double> Fv, Fe;
        force_from_samples(std::vector<ForceSample>{fs}, K, Fv, Fe);
        if (on_device) {
            QMC_CK(cudaMemcpyAsync(F, Fv.data(), sizeof(double) * K, cudaMemcpyHostToDevice, h->stream));
            h->sync();
        } else {
            std::copy(Fv.begin(), Fv.end(), F);
        }
    });
}

int qmc_reset_estimators(qmc_t h) {
    if (!h) return QMC_ERR_ARG;
    return guarded(h, [&] {
        h->vmc_e.clear();
        h->vmc_e2.clear();
        h->dmc_e.clear();
        h->dmc_e2.clear();
        h->vmc_f.clear();
        h->dmc_f.clear();
        if (h->d_nacc) {
            QMC_CK(cudaMemcpyAsync(&h->acc_base, h->d_nacc, sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                                   h->stream));
            h->sync();
        }
        h->n_prop = 0;
    });
}

int qmc_set_timing(qmc_t h, int enable) {
    if (!h) return QMC_ERR_ARG;
    return guarded(h, [&] {
        h->sync();
        h->tm.on = enable != 0;
        h->tm.reset();
    });
}

int qmc_get_timing(qmc_t h, const char* family, double* total_ms, long long* launches) {
    if (!h) return QMC_ERR_ARG;
    return guarded(h, [&] {
        require(family != nullptr, QMC_ERR_ARG, "null family");
        h->sync();
        const std::string f(family);
        double ms = 0.0;
        long long n = 0;
        bool found = false;
        for (int q = 0; q < F_COUNT; ++q)
            if (f == "all" || f == kFamily[q]) {
                // the tiled sweep's GEMMs run inside its "sweep" span: "all"
                // counts their launches but not their time a second time
                if (!(f == "all" && q == F_SWEEP_GEMM)) ms += h->tm.ms[q];
                n += h->tm.n[q];
                found = true;
            }
        require(found, QMC_ERR_ARG, "unknown kernel family " + f);
        if (total_ms) *total_ms = ms;
        if (launches) *launches = n;
    });
}

static const uint64_t kCheckpointMagic = 0x314B504351424D47ULL;  // "GMBQCPK1"

int qmc_checkpoint(qmc_t h, const char* path) {
    if (!h) return QMC_ERR_ARG;
    return guarded(h, [&] {
        need_walkers(h);
        require(path != nullptr, QMC_ERR_ARG, "null path");
        const int W = h->W, N = h->N();
        std::vector<double> R((size_t)W * N * 3), wt(W);
        QMC_CK(cudaMemcpyAsync(R.data(), h->wk[h->cur].R, sizeof(double) * R.size(), cudaMemcpyDeviceToHost, h->stream));
        QMC_CK(cudaMemcpyAsync(wt.data(), h->wk[h->cur].weight, sizeof(double) * W, cudaMemcpyDeviceToHost, h->stream));
        h->sync();
        FILE* f = std::fopen(path, "wb");
        require(f != nullptr, QMC_ERR_ARG, std::string("cannot open ") + path);
        const uint64_t hdr[6] = {kCheckpointMagic, 1u, (uint64_t)W, (uint64_t)N, h->seed, h->sweep};
        const int64_t w0 = h->W0;
        bool ok = std::fwrite(hdr, sizeof(hdr), 1, f) == 1 && std::fwrite(&w0, sizeof(w0), 1, f) == 1 &&
                  std::fwrite(R.data(), sizeof(double), R.size(), f) == R.size() &&
                  std::fwrite(wt.data(), sizeof(double), W, f) == (size_t)W;
        ok = (std::fclose(f) == 0) && ok;
        require(ok, QMC_ERR_ARG, "checkpoint write failed");
    });
}

int qmc_restore(qmc_t h, const char* path) {
    if (!h) return QMC_ERR_ARG;
    uint64_t hdr[6];
    int64_t w0 = 0;
    std::vector<double> R, wt;
    int st = guarded(h, [&] {
        require(path != nullptr, QMC_ERR_ARG, "null path");
        FILE* f = std::fopen(path, "rb");
        require(f != nullptr, QMC_ERR_ARG, std::string("cannot open ") + path);
        bool ok = std::fread(hdr, sizeof(hdr), 1, f) == 1 && std::fread(&w0, sizeof(w0), 1, f) == 1;
        if (ok) ok = hdr[0] == kCheckpointMagic && hdr[1] == 1u && (int)hdr[3] == h->N() && hdr[2] > 0;
        if (ok) {
            R.resize(hdr[2] * hdr[3] * 3);
            wt.resize(hdr[2]);
            ok = std::fread(R.data(), sizeof(double), R.size(), f) == R.size() &&
                 std::fread(wt.data(), sizeof(double), wt.size(), f) == wt.size();
        }
        std::fclose(f);
        require(ok, QMC_ERR_ARG, "not a compatible checkpoint file");
    });
    if (st != QMC_OK) return st;
    st = qmc_set_walkers(h, (int)hdr[2], R.data(), 0);
    if (st != QMC_OK) return st;
    h->seed = hdr[4];
    h->sweep = (uint32_t)hdr[5];
    h->W0 = (int)w0;
    return guarded(h, [&] {
        QMC_CK(cudaMemcpyAsync(h->wk[h->cur].weight, wt.data(), sizeof(double) * wt.size(), cudaMemcpyHostToDevice,
                               h->stream));
        h->sync();
    });
}

}  // extern "C"

// ---------------------------------------------------------------------
// Batches of independent systems (qmc_batch_* in qmc.h).  Every kernel
// family of a DMC step is one persistent launch over the work items of all
// systems; the launches of one step (plan, sweep, optional recompute, E_L,
// optional forces, branching and estimator sums) are captured once per
// (buffer parity, recompute, forces) variant in a CUDA graph and replayed.
// Trial energies and populations evolve on the device; the per-step
// estimator sums go to a device history that the host reads once per chunk
// of steps.
// ---------------------------------------------------------------------
struct qmc_batch {
    int device = 0;
    cudaStream_t stream = nullptr;
    std::string err;
    std::vector<qmc_t> sys;       // descriptor order (decreasing cost per walker)
    std::vector<int> caller;      // descriptor index -> caller index
    std::vector<uint64_t> gen;
    int mode = QMC_FP64;
    int n = 0;
    int n_sm = 0;
    BatchSys* d_sys = nullptr;
    BatchPlan* d_plan = nullptr;
    BatchCtl* d_ctl = nullptr;
    double* d_hist = nullptr;
    int hist_stride = 0;
    int chunk = 64;
    std::vector<BatchSys> h_sys;
    // launch configuration
    int sweep_block = 128;
    size_t sweep_smem = 0;
    int sweep_grid = 0;
    int any_delay = 0;             // some member uses delayed updates
    std::vector<int> delay, ainv;  // per descriptor
    size_t orb_smem = 0, inv_smem = 0, eloc_smem = 0, force_smem = 0;
    int orb_grid = 0, inv_grid = 0, eloc_grid = 0, force_grid = 0, copy_grid = 0;
    std::vector<int> warp;         // per descriptor: space warp on (read at creation)
    int any_warp = 0;
    size_t warp_smem = 0;
    int warp_grid = 0;
    int recompute_period = 0, steps_since = 0;
    int tuned = 0;
    int use_graph = 1;
    cudaGraphExec_t graph[8] = {};
    double graph_tau[8] = {};
    long long graph_launches[8] = {};
    KernelTimer tm;
    long long launches = 0;       // kernel launches enqueued by the last run

    int elem() const { return mode == QMC_MIXED ? 4 : 8; }
    void sync() {
        QMC_CK(cudaStreamSynchronize(stream));
        tm.collect();
    }
    void drop_graphs() {
        for (int k = 0; k < 8; ++k)
            if (graph[k]) {
                cudaGraphExecDestroy(graph[k]);
                graph[k] = nullptr;
            }
    }

    // Rebuilds the descriptors from the handles (walker buffers may have been
    // reallocated) with every handle's current buffer in slot 0.
    void refresh_descriptors() {
        for (int q = 0; q < n; ++q) {
            qmc_t h = sys[q];
            require(h->gen == gen[q], QMC_ERR_STATE,
                    "a system of the batch changed after qmc_batch_create; create the batch again");
            need_walkers(h);
            if (h->cur == 1) {   // make buffer 0 the current one
                std::swap(h->wk[0], h->wk[1]);
                h->cur = 0;
            }
            BatchSys& b = h_sys[q];
            b.s = h->ds;
            b.wk[0] = h->wk[0];
            b.wk[1] = h->wk[1];
            b.key = make_uint2((uint32_t)h->seed, (uint32_t)(h->seed >> 32));
            b.cap = h->cap;
            b.delay_rank = delay[q];
            b.ainv_smem = ainv[q];
            b.elem = elem();
            b.eloc_new = h->d_eloc_new;
            b.wts = h->d_wts;
            b.copies = h->d_copies;
            b.offsets = h->d_offsets;
            b.dEL = h->d_dEL;
            b.dlog = h->d_dlog;
            b.Bscr = h->d_Bscr;
            b.Pscr = h->d_Pscr;
            b.dvnn = h->d_dvnn;
            b.err = h->d_err;
            require(h->space_warp == warp[q], QMC_ERR_STATE,
                    "a system's space-warp setting changed after qmc_batch_create; create the batch again");
            b.space_warp = warp[q];
            if (warp[q] && !h->d_gEdet) {
                h->d_gEdet = h->template dalloc<double>(h->wk_allocs, (size_t)h->cap * 3 * h->N());
                h->d_gtot = h->template dalloc<double>(h->wk_allocs, (size_t)h->cap * 3 * h->N());
            }
            b.gEdet = warp[q] ? h->d_gEdet : nullptr;
            b.gtot = warp[q] ? h->d_gtot : nullptr;
        }
        QMC_CK(cudaMemcpyAsync(d_sys, h_sys.data(), sizeof(BatchSys) * n, cudaMemcpyHostToDevice, stream));
    }

    // Launch configuration for a sweep policy: systems with at least
    // delay_min electrons of one spin use delayed updates of rank k (k = 1:
    // none); a Sherman-Morrison system keeps A^-1 in shared memory when its
    // sweep then needs at most budget bytes.
    void configure(int block, size_t budget, int k, int delay_min) {
        size_t smem = 0;
        for (int q = 0; q < n; ++q) {
            const DevSys& s = sys[q]->ds;
            const int nmax = std::max(s.n_up, s.n_dn);
            delay[q] = (k > 1 && nmax >= delay_min) ? k : 1;
            if (delay[q] > 1) {
                ainv[q] = 0;
                smem = std::max(smem, mode == QMC_MIXED ? sweep_batch_smem<float>(s, delay[q], 0)
                                                        : sweep_batch_smem<double>(s, delay[q], 0));
                continue;
            }
            const size_t with = mode == QMC_MIXED ? sweep_batch_smem<float>(s, 1, 1) : sweep_batch_smem<double>(s, 1, 1);
            const size_t without =
                mode == QMC_MIXED ? sweep_batch_smem<float>(s, 1, 0) : sweep_batch_smem<double>(s, 1, 0);
            ainv[q] = with <= budget ? 1 : 0;
            smem = std::max(smem, ainv[q] ? with : without);
        }
        require(smem <= 227 * 1024, QMC_ERR_UNSUPPORTED,
                "the batched sweep needs " + std::to_string(smem) + " bytes of shared memory");
        int dl = 0;
        for (int q = 0; q < n; ++q) dl |= delay[q] > 1;
        const int occ = mode == QMC_MIXED ? sweep_batch_prepare<float>(block, smem, dl)
                                          : sweep_batch_prepare<double>(block, smem, dl);
        require(occ > 0, QMC_ERR_UNSUPPORTED, "batched sweep configuration cannot run");
        sweep_block = block;
        sweep_smem = smem;
        sweep_grid = occ * n_sm;
        any_delay = dl;
        drop_graphs();
    }

    void configure_other() {
        size_t orb = 0, inv = 0, el = 0, fo = 0;
        for (int q = 0; q < n; ++q) {
            const DevSys& s = sys[q]->ds;
            const int nmax = std::max(s.n_up, s.n_dn);
            orb = std::max(orb, sizeof(double) * 5 * (size_t)s.n_basis);
            inv = std::max(inv, sizeof(double) * ((size_t)nmax * nmax + nmax + 1));
            el = std::max(el, (sizeof(double) + sizeof(float)) * 3 * (size_t)s.N);
            fo = std::max(fo, force_batch_smem_bytes(s, elem(), warp[q]));
        }
        const bool mx = mode == QMC_MIXED;
        const int o_orb = wf_batch_prepare(mx ? 3 : 0, 128, orb);
        const int o_inv = wf_batch_prepare(1, 256, inv);
        const int o_el = wf_batch_prepare(mx ? 4 : 2, 128, el);
        int aw = 0;
        for (int q = 0; q < n; ++q) aw |= warp[q];
        const int o_fo = mx ? force_batch_prepare<float>(fo, aw) : force_batch_prepare<double>(fo, aw);
        require(o_orb > 0 && o_inv > 0 && o_el > 0 && o_fo > 0, QMC_ERR_UNSUPPORTED,
                "a batched kernel does not fit the largest system");
        orb_smem = orb;
        inv_smem = inv;
        eloc_smem = el;
        force_smem = fo;
        orb_grid = o_orb * n_sm;
        inv_grid = o_inv * n_sm;
        eloc_grid = o_el * n_sm;
        force_grid = o_fo * n_sm;
        copy_grid = 8 * n_sm;
        size_t wsm = 0;
        any_warp = 0;
        for (int q = 0; q < n; ++q)
            if (warp[q]) {
                any_warp = 1;
                wsm = std::max(wsm, space_warp_batch_smem_bytes(sys[q]->ds, elem()));
            }
        if (any_warp) {
            const int o_w = mx ? space_warp_batch_prepare<float>(wsm) : space_warp_batch_prepare<double>(wsm);
            require(o_w > 0, QMC_ERR_UNSUPPORTED, "the batched space warp does not fit the largest system");
            warp_smem = wsm;
            warp_grid = o_w * n_sm;
        }
    }

    void launch_sweep(int parity, double tau, int ctr) {
        if (mode == QMC_MIXED)
            QMC_CK(launch_sweep_batch<float>(d_sys, d_plan, d_ctl, parity, tau, ctr, sweep_grid, sweep_block,
                                             sweep_smem, any_delay, stream));
        else
            QMC_CK(launch_sweep_batch<double>(d_sys, d_plan, d_ctl, parity, tau, ctr, sweep_grid, sweep_block,
                                              sweep_smem, any_delay, stream));
        ++launches;
    }

    void launch_eloc(int parity, int into_walker, int ctr) {
        if (mode == QMC_MIXED)
            QMC_CK(launch_eloc_batch<float>(d_sys, d_plan, parity, into_walker, ctr, eloc_grid, eloc_smem, stream));
        else
            QMC_CK(launch_eloc_batch<double>(d_sys, d_plan, parity, into_walker, ctr, eloc_grid, eloc_smem, stream));
        ++launches;
    }

    // One DMC step of every system (kernel launches only: capturable).
    void enqueue_step(int parity, bool rec, bool forces, double tau) {
        const bool mx = mode == QMC_MIXED;
        QMC_CK(launch_batch_plan(d_plan, d_ctl, d_sys, n, stream));
        ++launches;
        tm.begin(stream);
        launch_sweep(parity, tau, 0);
        tm.end(F_SWEEP, 1, stream);
        if (rec) {
            tm.begin(stream);
            if (mx)
                QMC_CK(launch_orbitals_batch<float>(d_sys, d_plan, parity, 1, orb_grid, orb_smem, stream));
            else
                QMC_CK(launch_orbitals_batch<double>(d_sys, d_plan, parity, 1, orb_grid, orb_smem, stream));
            QMC_CK(launch_invert_batch(d_sys, d_plan, parity, mx ? 1 : 0, 2, inv_grid, inv_smem, stream));
            launches += 2;
            tm.end(F_RECOMPUTE, 2, stream);
        }
        tm.begin(stream);
        launch_eloc(parity, 0, 3);
        tm.end(F_ELOC, 1, stream);
        if (forces) {
            tm.begin(stream);
            if (mx)
                QMC_CK(launch_force_batch<float>(d_sys, d_plan, parity, 4, force_grid, force_smem, any_warp, stream));
            else
                QMC_CK(launch_force_batch<double>(d_sys, d_plan, parity, 4, force_grid, force_smem, any_warp, stream));
            ++launches;
            if (any_warp) {
                if (mx)
                    QMC_CK(launch_space_warp_batch<float>(d_sys, d_plan, parity, 5, warp_grid, warp_smem, stream));
                else
                    QMC_CK(launch_space_warp_batch<double>(d_sys, d_plan, parity, 5, warp_grid, warp_smem, stream));
                ++launches;
            }
            tm.end(F_FORCE, any_warp ? 2 : 1, stream);
        }
        tm.begin(stream);
        QMC_CK(launch_branch_batch(d_sys, d_plan, d_ctl, n, parity, tau, d_hist, hist_stride, forces ? 1 : 0,
                                   copy_grid, stream));
        launches += 4;
        tm.end(F_BRANCH, 4, stream);
    }

    void run_step(int parity, bool rec, bool forces, double tau) {
        const int key = parity | (rec ? 2 : 0) | (forces ? 4 : 0);
        if (!use_graph || tm.on) {
            enqueue_step(parity, rec, forces, tau);
            return;
        }
        if (graph[key] && graph_tau[key] != tau) {
            cudaGraphExecDestroy(graph[key]);
            graph[key] = nullptr;
        }
        if (!graph[key]) {
            const long long l0 = launches;
            graph_launches[key] = 0;
            QMC_CK(cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal));
            try {
                enqueue_step(parity, rec, forces, tau);
            } catch (...) {
                cudaGraph_t g = nullptr;
                cudaStreamEndCapture(stream, &g);
                if (g) cudaGraphDestroy(g);
                cudaGetLastError();
                throw;
            }
            cudaGraph_t g = nullptr;
            QMC_CK(cudaStreamEndCapture(stream, &g));
            const cudaError_t e = cudaGraphInstantiate(&graph[key], g, 0);
            cudaGraphDestroy(g);
            QMC_CK(e);
            graph_tau[key] = tau;
            graph_launches[key] = launches - l0;
            launches = l0;   // counted when replayed
        }
        QMC_CK(cudaGraphLaunch(graph[key], stream));
        launches += graph_launches[key];
    }

    void upload_ctl(const double* e_trial, double tau) {
        std::vector<BatchCtl> c(n);
        for (int q = 0; q < n; ++q) {
            qmc_t h = sys[q];
            BatchCtl& x = c[q];
            std::memset(&x, 0, sizeof(x));
            x.e_trial = e_trial ? e_trial[caller[q]] : 0.0;
            x.e_cut = 0.2 * std::sqrt((double)h->N() / tau);
            x.feedback = 1.0 / (10.0 * tau);
            x.W0 = (double)h->W0;
            x.pop = h->W;
            x.sweep = h->sweep;
            x.fixed_pop = h->pop_mode == QMC_POP_FIXED ? h->W0 : 0;
        }
        QMC_CK(cudaMemcpyAsync(d_ctl, c.data(), sizeof(BatchCtl) * n, cudaMemcpyHostToDevice, stream));
    }

    // After a run: populations, RNG counters and buffer parity back into
    // the handles; the device status of every system checked.
    void finish(int parity) {
        std::vector<BatchCtl> c(n);
        QMC_CK(cudaMemcpyAsync(c.data(), d_ctl, sizeof(BatchCtl) * n, cudaMemcpyDeviceToHost, stream));
        sync();
        std::string bad;
        int code = QMC_OK;
        for (int q = 0; q < n; ++q) {
            qmc_t h = sys[q];
            h->cur = parity;
            h->sweep = c[q].sweep;
            if (c[q].status == 0) {
                h->W = c[q].pop;
            } else {
                h->walkers_valid = false;
                code = QMC_ERR_POPULATION;
                bad = "system " + std::to_string(caller[q]) +
                      (c[q].status == 1 ? ": population exceeds capacity " + std::to_string(h->cap)
                                        : ": population died out");
            }
        }
        for (int q = 0; q < n; ++q) {
            qmc_t h = sys[q];
            unsigned e = 0;
            QMC_CK(cudaMemcpy(&e, h->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost));
            if (e) {
                QMC_CK(cudaMemset(h->d_err, 0, sizeof(unsigned)));
                if (code == QMC_OK) {
                    code = (e & kErrSingular) ? QMC_ERR_SINGULAR : QMC_ERR_NONFINITE;
                    bad = "system " + std::to_string(caller[q]) +
                          ((e & kErrSingular) ? ": a Slater matrix is singular" : ": non-finite local energy");
                }
            }
        }
        if (code != QMC_OK) throw QmcError{code, bad};
    }
};

namespace {

template <typename F>
int guarded_b(qmc_batch_t b, F&& f) {
    try {
        f();
        if (b) b->err.clear();
        return QMC_OK;
    } catch (const QmcError& e) {
        if (b) b->err = e.msg;
        return e.code;
    } catch (const std::bad_alloc&) {
        if (b) b->err = "host allocation failed";
        return QMC_ERR_OOM;
    } catch (...) {
        if (b) b->err = "unexpected exception";
        return QMC_ERR_ARG;
    }
}

thread_local std::string g_batch_error;

}  // namespace

extern "C" {

int qmc_batch_create(qmc_batch_t* out, int n_systems, qmc_t const* systems) {
    if (!out) return QMC_ERR_ARG;
    *out = nullptr;
    qmc_batch* b = new (std::nothrow) qmc_batch();
    if (!b) return QMC_ERR_OOM;
    const int st = guarded_b(b, [&] {
        require(n_systems >= 1 && n_systems <= kMaxBatchSystems && systems, QMC_ERR_ARG,
                "need 1.." + std::to_string(kMaxBatchSystems) + " systems");
        for (int i = 0; i < n_systems; ++i) {
            require(systems[i] != nullptr, QMC_ERR_ARG, "null system handle");
            for (int j = 0; j < i; ++j) require(systems[j] != systems[i], QMC_ERR_ARG, "a system appears twice");
            need_walkers(systems[i]);
            require(systems[i]->device == systems[0]->device, QMC_ERR_ARG, "all systems must be on one device");
            require(systems[i]->mode == systems[0]->mode, QMC_ERR_ARG, "all systems must use one precision mode");
            require(systems[i]->n3 == 0, QMC_ERR_UNSUPPORTED, "batches carry no three-body Jastrow");
            require(systems[i]->n_pp == 0, QMC_ERR_UNSUPPORTED, "batches carry no pseudopotential");
            require(!systems[i]->ds.msd, QMC_ERR_UNSUPPORTED,
                    "batches hold single-determinant systems (expansions run per handle)");
        }
        b->device = systems[0]->device;
        b->mode = systems[0]->mode;
        b->n = n_systems;
        QMC_CK(cudaSetDevice(b->device));
        QMC_CK(cudaDeviceGetAttribute(&b->n_sm, cudaDevAttrMultiProcessorCount, b->device));
        QMC_CK(cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking));
        // largest cost per walker first (N * n * N_b ~ the sweep's work)
        std::vector<int> idx(n_systems);
        for (int i = 0; i < n_systems; ++i) idx[i] = i;
        auto cost = [&](int i) {
            const qmc_t h = systems[i];
            return (double)h->N() * std::max(h->n_up, h->n_dn) * h->n_basis;
        };
        std::stable_sort(idx.begin(), idx.end(), [&](int x, int y) { return cost(x) > cost(y); });
        int kmax = 0;
        for (int q = 0; q < n_systems; ++q) {
            b->sys.push_back(systems[idx[q]]);
            b->caller.push_back(idx[q]);
            b->gen.push_back(systems[idx[q]]->gen);
            kmax = std::max(kmax, 3 * systems[idx[q]]->n_nuc);
        }
        b->hist_stride = kHistHead + 2 + 3 * kmax;
        b->h_sys.resize(n_systems);
        b->delay.assign(n_systems, 1);
        b->ainv.assign(n_systems, 0);
        for (qmc_t h : b->sys) b->warp.push_back(h->space_warp);
        for (qmc_t h : b->sys)
            if (h->recompute_period > 0)
                b->recompute_period =
                    b->recompute_period ? std::min(b->recompute_period, h->recompute_period) : h->recompute_period;
        auto alloc = [&](void** p, size_t bytes) {
            const cudaError_t e = cudaMalloc(p, bytes);
            if (e != cudaSuccess) {
                cudaGetLastError();
                throw QmcError{QMC_ERR_OOM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed"};
            }
        };
        alloc((void**)&b->d_sys, sizeof(BatchSys) * n_systems);
        alloc((void**)&b->d_plan, sizeof(BatchPlan));
        alloc((void**)&b->d_ctl, sizeof(BatchCtl) * n_systems);
        alloc((void**)&b->d_hist, sizeof(double) * (size_t)b->chunk * n_systems * b->hist_stride);
        QMC_CK(cudaMemsetAsync(b->d_plan, 0, sizeof(BatchPlan), b->stream));
        // default configuration: Sherman-Morrison everywhere, A^-1 in shared
        // memory for every system that fits 100 KB
        b->configure(128, 100 * 1024, 1, 0);
        b->configure_other();
        b->sync();
    });
    if (st != QMC_OK) {
        g_batch_error = b->err;
        qmc_batch_destroy(b);
        return st;
    }
    *out = b;
    return QMC_OK;
}

int qmc_batch_destroy(qmc_batch_t b) {
    if (!b) return QMC_ERR_ARG;
    cudaSetDevice(b->device);
    if (b->stream) cudaStreamSynchronize(b->stream);
    b->drop_graphs();
    b->tm.release();
    cudaFree(b->d_sys);
    cudaFree(b->d_plan);
    cudaFree(b->d_ctl);
    cudaFree(b->d_hist);
    if (b->stream) cudaStreamDestroy(b->stream);
    delete b;
    return QMC_OK;
}

const char* qmc_batch_last_error(qmc_batch_t b) { return b ? b->err.c_str() : g_batch_error.c_str(); }

int qmc_batch_set_options(qmc_batch_t b, int use_graph, int sweep_block, int delay_rank, int delay_min_electrons,
                          int smem_budget) {
    if (!b) return QMC_ERR_ARG;
    return guarded_b(b, [&] {
        require(sweep_block == 64 || sweep_block == 128 || sweep_block == 256, QMC_ERR_ARG,
                "sweep block must be 64, 128 or 256 threads");
        require(delay_rank >= 1 && delay_rank <= kMaxDelayRank, QMC_ERR_UNSUPPORTED,
                "delay rank must be 1.." + std::to_string(kMaxDelayRank));
        require(smem_budget >= 0 && delay_min_electrons >= 0, QMC_ERR_ARG, "negative option");
        QMC_CK(cudaSetDevice(b->device));
        b->use_graph = use_graph ? 1 : 0;
        b->configure(sweep_block, (size_t)smem_budget, delay_rank, delay_min_electrons);
        b->tuned = 0;
    });
}

// Times one batched sweep per candidate configuration and keeps the fastest.
// The trial sweeps are ordinary Metropolis sweeps of every system at time
// step tau (without branching), so they also equilibrate.
int qmc_batch_autotune(qmc_batch_t b, double tau, int* chosen) {
    if (!b) return QMC_ERR_ARG;
    return guarded_b(b, [&] {
        require(tau > 0.0 && std::isfinite(tau), QMC_ERR_ARG, "need tau > 0");
        QMC_CK(cudaSetDevice(b->device));
        for (qmc_t h : b->sys) QMC_CK(cudaStreamSynchronize(h->stream));
        b->refresh_descriptors();
        b->upload_ctl(nullptr, tau);
        // candidate shared-memory budgets: every system's need with A^-1 in
        // shared memory, plus none
        std::vector<size_t> budgets{0};
        for (qmc_t h : b->sys) {
            const size_t with =
                b->mode == QMC_MIXED ? sweep_batch_smem<float>(h->ds, 1, 1) : sweep_batch_smem<double>(h->ds, 1, 1);
            if (with <= 227 * 1024) budgets.push_back(with);
        }
        std::sort(budgets.begin(), budgets.end());
        budgets.erase(std::unique(budgets.begin(), budgets.end()), budgets.end());
        if (budgets.size() > 6) {   // keep none, four quantiles and the largest
            std::vector<size_t> pick{budgets[0]};
            for (int k = 1; k <= 4; ++k) pick.push_back(budgets[budgets.size() * k / 5]);
            pick.push_back(budgets.back());
            std::sort(pick.begin(), pick.end());
            pick.erase(std::unique(pick.begin(), pick.end()), pick.end());
            budgets.swap(pick);
        }
        struct Cand {
            int block;
            size_t budget;
            int k, kmin;
        };
        std::vector<Cand> cands;
        for (int block : {128, 256}) {
            for (size_t bud : budgets) cands.push_back({block, bud, 1, 0});
            for (int k : {8, 16, 32}) cands.push_back({block, 0, k, 32});
        }
        cudaEvent_t e0, e1;
        QMC_CK(cudaEventCreate(&e0));
        QMC_CK(cudaEventCreate(&e1));
        double best = 1e300;
        Cand pick = cands[0];
        try {
            for (const Cand& c : cands) {
                try {
                    b->configure(c.block, c.budget, c.k, c.kmin);
                } catch (const QmcError&) {
                    continue;   // does not fit
                }
                b->refresh_descriptors();
                float t_min = 1e30f;
                for (int rep = 0; rep < 2; ++rep) {
                    QMC_CK(launch_batch_plan(b->d_plan, b->d_ctl, b->d_sys, b->n, b->stream));
                    QMC_CK(cudaEventRecord(e0, b->stream));
                    b->launch_sweep(0, tau, 0);
                    QMC_CK(cudaEventRecord(e1, b->stream));
                    QMC_CK(launch_batch_advance(b->d_ctl, b->n, b->stream));
                    QMC_CK(cudaEventSynchronize(e1));
                    float t = 0.f;
                    QMC_CK(cudaEventElapsedTime(&t, e0, e1));
                    t_min = std::min(t_min, t);
                }
                if (t_min < best) {
                    best = t_min;
                    pick = c;
                }
            }
        } catch (...) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            throw;
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        b->configure(pick.block, pick.budget, pick.k, pick.kmin);
        b->refresh_descriptors();
        // the trial sweeps moved the walkers: E_L of the current positions
        QMC_CK(launch_batch_plan(b->d_plan, b->d_ctl, b->d_sys, b->n, b->stream));
        b->launch_eloc(0, 1, 3);
        b->tuned = 1;
        b->finish(0);
        if (chosen) {
            chosen[0] = b->sweep_block;
            chosen[1] = (int)b->sweep_smem;
            chosen[2] = b->sweep_grid;
            chosen[3] = (int)(best * 1000.0);   // microseconds of the fastest sweep
            for (int q = 0; q < b->n; ++q) chosen[4 + b->caller[q]] = b->delay[q] * 2 + b->ainv[q];
        }
    });
}

int qmc_batch_vmc(qmc_batch_t b, int n_sweeps, double tau) {
    if (!b) return QMC_ERR_ARG;
    return guarded_b(b, [&] {
        require(n_sweeps >= 0 && tau > 0.0 && std::isfinite(tau), QMC_ERR_ARG, "need n_sweeps >= 0 and tau > 0");
        QMC_CK(cudaSetDevice(b->device));
        for (qmc_t h : b->sys) QMC_CK(cudaStreamSynchronize(h->stream));
        b->refresh_descriptors();
        b->upload_ctl(nullptr, tau);
        b->launches = 0;
        for (int k = 0; k < n_sweeps; ++k) {
            QMC_CK(launch_batch_plan(b->d_plan, b->d_ctl, b->d_sys, b->n, b->stream));
            b->tm.begin(b->stream);
            b->launch_sweep(0, tau, 0);
            b->tm.end(F_SWEEP, 1, b->stream);
            b->tm.begin(b->stream);
            b->launch_eloc(0, 1, 3);
            b->tm.end(F_ELOC, 1, b->stream);
            QMC_CK(launch_batch_advance(b->d_ctl, b->n, b->stream));
            b->launches += 3;
            for (qmc_t h : b->sys) h->n_prop += (long long)h->W * h->N();
        }
        b->finish(0);
    });
}

int qmc_batch_dmc(qmc_batch_t b, int n_steps, double tau, const double* e_trial, int n_equil, int forces_every,
                  double* e_step, int* pop) {
    if (!b) return QMC_ERR_ARG;
    return guarded_b(b, [&] {
        require(n_steps >= 0 && tau > 0.0 && std::isfinite(tau) && e_trial, QMC_ERR_ARG,
                "need n_steps >= 0, tau > 0 and one trial energy per system");
        for (int i = 0; i < b->n; ++i) require(std::isfinite(e_trial[i]), QMC_ERR_ARG, "non-finite trial energy");
        QMC_CK(cudaSetDevice(b->device));
        for (qmc_t h : b->sys) QMC_CK(cudaStreamSynchronize(h->stream));
        b->refresh_descriptors();
        b->upload_ctl(e_trial, tau);
        b->launches = 0;
        const int n = b->n;
        std::vector<double> rows;
        std::vector<std::pair<int, bool>> meta;   // (step, forces) of each history row
        int parity = 0;
        auto flush = [&]() {
            if (meta.empty()) return;
            rows.resize((size_t)meta.size() * n * b->hist_stride);
            QMC_CK(cudaMemcpyAsync(rows.data(), b->d_hist, sizeof(double) * rows.size(), cudaMemcpyDeviceToHost,
                                   b->stream));
            b->sync();
            for (size_t r = 0; r < meta.size(); ++r) {
                const int k = meta[r].first;
                const bool f = meta[r].second;
                for (int q = 0; q < n; ++q) {
                    const double* row = &rows[((size_t)r * n + q) * b->hist_stride];
                    qmc_t h = b->sys[q];
                    const int ci = b->caller[q];
                    h->n_prop += (long long)row[7] * h->N();
                    const double Ek = row[0] > 0.0 ? row[1] / row[0] : 0.0;
                    if (e_step) e_step[(size_t)k * n + ci] = Ek;
                    if (pop) pop[(size_t)k * n + ci] = (int)row[2];
                    if (row[0] <= 0.0 || row[3] != 0.0) continue;   // stopped system
                    if (k >= n_equil) {
                        h->dmc_e.push_back(Ek);
                        h->dmc_e2.push_back(row[5] / row[0]);
                        if (f) {
                            ForceSample fs;
                            const int K = 3 * h->n_nuc;
                            fs.v.assign(row + kHistHead, row + kHistHead + 2 + 3 * K);
                            h->dmc_f.push_back(fs);
                        }
                    }
                }
            }
            meta.clear();
            // the next chunk starts at history row 0
            const int minus_one = -1;
            QMC_CK(cudaMemcpyAsync(&b->d_plan->step, &minus_one, sizeof(int), cudaMemcpyHostToDevice, b->stream));
            b->sync();
        };
        {
            const int minus_one = -1;
            QMC_CK(cudaMemcpyAsync(&b->d_plan->step, &minus_one, sizeof(int), cudaMemcpyHostToDevice, b->stream));
        }
        try {
            for (int k = 0; k < n_steps; ++k) {
                const bool rec = b->recompute_period > 0 && (b->steps_since + 1) >= b->recompute_period;
                const bool f = forces_every > 0 && k >= n_equil && (k % forces_every) == 0;
                b->run_step(parity, rec, f, tau);
                b->steps_since = rec ? 0 : b->steps_since + 1;
                meta.push_back({k, f});
                parity ^= 1;
                if ((int)meta.size() == b->chunk) flush();
            }
            flush();
        } catch (...) {
            cudaStreamSynchronize(b->stream);
            cudaGetLastError();
            throw;
        }
        b->finish(parity);
    });
}

int qmc_tc_gemm(int batch, int M, int N, int K, const float* A, long long strideA, int lda, const float* B,
                long long strideB, int ldb, int b_trans, float* D, long long strideD, int ldd, void* cuda_stream) {
    if (batch < 0 || M < 0 || N < 0 || K < 0 || N > 256 || !A || !B || !D) return QMC_ERR_ARG;
    if (lda < K || ldd < N || ldb < (b_trans ? N : K)) return QMC_ERR_ARG;
    if (batch == 0 || M == 0 || N == 0) return QMC_OK;
    static unsigned* d_flag[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return QMC_ERR_CUDA;
    if (!d_flag[dev]) {
        if (cudaMalloc(&d_flag[dev], sizeof(unsigned)) != cudaSuccess) return QMC_ERR_OOM;
        if (cudaMemset(d_flag[dev], 0, sizeof(unsigned)) != cudaSuccess) return QMC_ERR_CUDA;
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    if (launch_tc_gemm(batch, M, N, K, A, strideA, lda, B, strideB, ldb, b_trans, D, strideD, ldd, d_flag[dev], st) !=
        cudaSuccess)
        return QMC_ERR_CUDA;
    unsigned f = 0;
    if (cudaMemcpyAsync(&f, d_flag[dev], sizeof(unsigned), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return QMC_ERR_CUDA;
    if (f) {
        cudaMemset(d_flag[dev], 0, sizeof(unsigned));
        return QMC_ERR_TIMEOUT;
    }
    return QMC_OK;
}

int qmc_tc_gemm_split(int M, int N, int K, const float* A_hi, const float* A_lo, int lda, const float* B_hi,
                      const float* B_lo, int ldb, float* D, int ldd, void* cuda_stream) {
    if (M < 0 || N < 0 || K < 1 || N > 256 || !A_hi || !A_lo || !B_hi || !B_lo || !D) return QMC_ERR_ARG;
    if (lda < K || ldb < K || ldd < N) return QMC_ERR_ARG;
    if (M == 0 || N == 0) return QMC_OK;
    static unsigned* d_flag[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return QMC_ERR_CUDA;
    if (!d_flag[dev]) {
        if (cudaMalloc(&d_flag[dev], sizeof(unsigned)) != cudaSuccess) return QMC_ERR_OOM;
        if (cudaMemset(d_flag[dev], 0, sizeof(unsigned)) != cudaSuccess) return QMC_ERR_CUDA;
    }
    TcSplitPlan plan;
    if (!tc_split_plan(&plan, M, N, K, A_hi, A_lo, lda, B_hi, B_lo, ldb)) return QMC_ERR_UNSUPPORTED;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    if (tc_split_prepare(N) != cudaSuccess || launch_tc_gemm_split(plan, D, ldd, d_flag[dev], st) != cudaSuccess)
        return QMC_ERR_CUDA;
    unsigned f = 0;
    if (cudaMemcpyAsync(&f, d_flag[dev], sizeof(unsigned), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return QMC_ERR_CUDA;
    if (f) {
        cudaMemset(d_flag[dev], 0, sizeof(unsigned));
        return QMC_ERR_TIMEOUT;
    }
    return QMC_OK;
}

int qmc_batch_set_timing(qmc_batch_t b, int enable) {
    if (!b) return QMC_ERR_ARG;
    return guarded_b(b, [&] {
        b->tm.on = enable != 0;
        b->tm.reset();
    });
}

int qmc_batch_get_timing(qmc_batch_t b, const char* family, double* total_ms, long long* launches) {
    if (!b) return QMC_ERR_ARG;
    return guarded_b(b, [&] {
        require(family != nullptr, QMC_ERR_ARG, "null family");
        if (std::strcmp(family, "all") == 0) {
            double t = 0.0;
            long long c = 0;
            for (int f = 0; f < F_COUNT; ++f) {
                t += b->tm.ms[f];
                c += b->tm.n[f];
            }
            if (total_ms) *total_ms = t;
            if (launches) *launches = b->launches;
            return;
        }
        for (int f = 0; f < F_COUNT; ++f)
            if (std::strcmp(family, kFamily[f]) == 0) {
                if (total_ms) *total_ms = b->tm.ms[f];
                if (launches) *launches = b->tm.n[f];
                return;
            }
        throw QmcError{QMC_ERR_ARG, std::string("unknown kernel family ") + family};
    });
}

}  // extern "C"
