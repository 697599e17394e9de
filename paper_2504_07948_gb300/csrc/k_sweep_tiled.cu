// Walker-tiled particle-by-particle sweep of the mixed form with delayed
// (Woodbury) inverse updates, for large determinants.
//
// The one-CTA-per-walker sweeps contract the basis of one proposed move with
// the orbital coefficients as a matrix-vector product ([5 x N_b] x [N_b x n]
// per walker-move), re-reading the coefficient rows for every walker.  Here
// every walker proposes a move of the same electron e at the same time, so
// the contraction of Eq. 2 for all walkers is one dense GEMM,
//   Phi'[5W x n] = B'[5W x N_b] C^T,   rows (walker, value / d/dx / d/dy /
//   d/dz / Laplacian),
// on the tensor cores (tcgen05, 3xTF32, TMA-fed; launch_tc_gemm_ab).  A
// move of electron e is three launches:
//   propose  (one CTA per walker) the column c_e of the current inverse
//            from the queue, the drift at r_e, the proposal r', and the
//            basis at r' written as the walker's five rows of B';
//   GEMM     Phi' = B' C^T;
//   accept   (one CTA per walker) ratio, drift at r', Jastrow change,
//            fixed-node Metropolis test; an accepted move borders K^-1 and
//            appends its orbital row to the queue.
// The queue of accepted rows is flushed for all walkers together every kmax
// electrons and at the end of each spin block (at most one accepted move
// per electron, so the queue never holds more than kmax rows):
//   P      = rows r_m of A0^-T                       (gather),
//   Z^T    = A0^-T V^T                              (batched GEMM, tensor cores),
//   X^T    = (K^-1 (Z - E^T))^T                     (FP64, the bordered K^-1),
//   A0^-T <- A0^-T - X^T P                          (batched GEMM, tensor cores),
// the same algebra as the fused delayed sweep (k_sweep_delayed.cu): with
// rows r_1..r_d replaced by phi'_1..phi'_d, A^-1 = A0^-1 - A0^-1 E K^-1 (V^T
// A0^-1 - E^T), K_mm' = phi'_m . A0^-1[:, r_m'], and the column a move needs
// is c_e = A0^-1[:, e] - sum_m (K^-1 y)_m A0^-1[:, r_m], y_m = phi'_m .
// A0^-1[:, e].  The move arithmetic (drift, Green's function, acceptance,
// Jastrow pair terms with hi/lo float offsets) is the mixed form's
// (propose_move_mixed / accept_move_mixed); K^-1, its bordering and the
// product K^-1 Z are carried in double-float arithmetic (two floats per
// value, ~44 bits) on the FP32 pipe where the fused sweep uses FP64.
#include "qmc_internal.cuh"
#include "sweep_tiled.cuh"

namespace qmc {

namespace {

constexpr int kTb = 128;   // threads per walker (one CTA per walker)

__device__ __forceinline__ float wsum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ float tf32_rna(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// Sums of K values over the CTA, delivered to thread 0 (scratch: 4 x K).
template <int K>
__device__ __forceinline__ void cta_sum_to0(float (&v)[K], float* scratch) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int c = 0; c < K; ++c) v[c] = wsum(v[c]);
    if (lane == 0)
#pragma unroll
        for (int c = 0; c < K; ++c) scratch[wid * K + c] = v[c];
    __syncthreads();
    if (threadIdx.x == 0)
#pragma unroll
        for (int c = 0; c < K; ++c) v[c] = scratch[c] + scratch[K + c] + scratch[2 * K + c] + scratch[3 * K + c];
}

// Jastrow pair sums of electron e at (rh, rl) (hi/lo floats) over the other
// electrons and the nuclei, threads over partners: u = sum a r / (1 + b r)
// and its gradient; thread-partial values.
__device__ __forceinline__ void jastrow_at(const DevSys& s, const float2* Rp, int e, const float rh[3],
                                           const float rl[3], float& u, float g[3]) {
    const int N = s.N, nu = s.n_up;
    u = 0.f;
    g[0] = g[1] = g[2] = 0.f;
    for (int q = threadIdx.x; q < N + s.n_nuc; q += kTb) {
        float x, y, z, a, b;
        if (q < N) {
            if (q == e) continue;
            const float2 q0 = Rp[3 * q], q1 = Rp[3 * q + 1], q2 = Rp[3 * q + 2];
            x = diff_f2(rh[0], rl[0], q0.x, q0.y);
            y = diff_f2(rh[1], rl[1], q1.x, q1.y);
            z = diff_f2(rh[2], rl[2], q2.x, q2.y);
            a = (float)(((q < nu) == (e < nu)) ? s.a_par : s.a_anti);
            b = (float)s.b_ee;
        } else {
            const int c = q - N;
            x = diff_f2(rh[0], rl[0], s.Rn_hi[3 * c], s.Rn_lo[3 * c]);
            y = diff_f2(rh[1], rl[1], s.Rn_hi[3 * c + 1], s.Rn_lo[3 * c + 1]);
            z = diff_f2(rh[2], rl[2], s.Rn_hi[3 * c + 2], s.Rn_lo[3 * c + 2]);
            a = (float)s.a_en[c];
            b = (float)s.b_en;
        }
        const float ir = rsqrtf(x * x + y * y + z * z);
        const float r = (x * x + y * y + z * z) * ir;
        const float qd = 1.f / (1.f + b * r);
        u += a * r * qd;
        const float gg = a * qd * qd * ir;
        g[0] += gg * x;
        g[1] += gg * y;
        g[2] += gg * z;
    }
}

__global__ void k_tiled_begin(const double* R, int W, int N, TiledState ts) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < W) {
        ts.dq[i] = 0;
        ts.acc[i] = 0u;
    }
    if (i >= W * 3 * N) return;
    const double r = R[i];
    const float hi = (float)r;
    ts.Rp[i] = make_float2(hi, (float)(r - (double)hi));
}

// ---------------------------------------------------------------------
// Double-float arithmetic (a value as an unevaluated sum hi + lo of two
// floats; Dekker 1971, Knuth's two-sum): the bordered K^-1 and its products
// keep ~44 significant bits on the FP32 pipe, where FP64 instructions issue
// at 1/64 of the FP32 rate on this GPU.
// ---------------------------------------------------------------------
__device__ __forceinline__ float2 df_quick(float a, float b) {   // |a| >= |b|
    const float s = a + b;
    return make_float2(s, b - (s - a));
}
__device__ __forceinline__ float2 df_add(float2 x, float2 y) {
    const float s = x.x + y.x;
    const float bp = s - x.x;
    const float e = (x.x - (s - bp)) + (y.x - bp) + x.y + y.y;
    return df_quick(s, e);
}
__device__ __forceinline__ float2 df_mul(float2 x, float2 y) {
    const float p = x.x * y.x;
    const float e = fmaf(x.x, y.x, -p) + (x.x * y.y + x.y * y.x);
    return df_quick(p, e);
}
__device__ __forceinline__ float2 df_mulf(float2 x, float y) {
    const float p = x.x * y;
    const float e = fmaf(x.x, y, -p) + x.y * y;
    return df_quick(p, e);
}
__device__ __forceinline__ float2 df_neg(float2 x) { return make_float2(-x.x, -x.y); }
// 1 / r for a float r, to double-float accuracy (one Newton correction).
__device__ __forceinline__ float2 df_rcp(float r) {
    const float q = 1.f / r;
    const float res = fmaf(-r, q, 1.f);   // exact residual
    return df_quick(q, q * res);
}

struct ProposeSmem {
    float y[32], tf[32], red[4 * 7], fs[6];
    int rows[32];
    float rad[3 * kTiledMaxShells];   // f, f', f'' of every shell at r' (zeros where screened)
};
struct AcceptSmem {
    float red[4 * 8];
    float c[32];
    float2 u[32], t[32];
    int rows[32], acc;
    float rho;
};

// Column e of the current inverse, drift, proposal and the basis at r' as
// TF32 hi / lo rows of B', for walker w (the whole CTA).
__device__ __forceinline__ void propose_body(const DevSys& s, const DevWalkers& wk, const TiledState& ts, int w,
                                             int e, const SweepParams& p, ProposeSmem& S) {
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int nu = s.n_up, N = s.N, spin = e >= nu, n = spin ? s.n_dn : nu, k = spin ? e - nu : e;
    const int kmax = ts.kmax, ldv = ts.ldv, nbp = ts.nbp;
    const float* AT = (const float*)wk.Ainv[spin] + (size_t)w * n * n;
    const float* V = ts.V + (size_t)w * kmax * ldv;
    const int dq = ts.dq[w];
    if (tid < dq) S.rows[tid] = ts.rows[(size_t)w * kmax + tid];
    // y_m = phi'_m . A0^-1[:, e] (row k of A0^-T): a warp per m
    for (int m = wid; m < dq; m += kTb / 32) {
        float a = 0.f;
        for (int j = lane; j < n; j += 32) a += V[(size_t)m * ldv + j] * AT[(size_t)k * n + j];
        a = wsum(a);
        if (lane == 0) S.y[m] = a;
    }
    __syncthreads();
    // t = K^-1 y in double-float (KinvT[q][m] = (K^-1)_{mq}), thread m
    if (tid < dq) {
        const float2* KT = ts.KinvT + (size_t)w * kmax * kmax;
        float2 t = make_float2(0.f, 0.f);
        for (int q = 0; q < dq; ++q) t = df_add(t, df_mulf(KT[(size_t)q * kmax + tid], S.y[q]));
        ts.tv[(size_t)w * kmax + tid] = t;
        S.tf[tid] = t.x + t.y;
    }
    __syncthreads();
    // c_e = A0^-1[:, e] - sum_m t_m A0^-1[:, r_m] and the determinant drift
    const float* Gk = (const float*)wk.G[spin] + ((size_t)w * n + k) * 4 * n;
    float* ce = ts.ce + (size_t)w * ldv;
    float v7[7] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int j = tid; j < n; j += kTb) {
        float a = AT[(size_t)k * n + j];
        for (int m = 0; m < dq; ++m) a -= S.tf[m] * AT[(size_t)S.rows[m] * n + j];
        ce[j] = a;
        v7[0] += Gk[j] * a;
        v7[1] += Gk[n + j] * a;
        v7[2] += Gk[2 * n + j] * a;
    }
    // Jastrow value and gradient at r_e
    const float2* Rp = ts.Rp + (size_t)w * 3 * N;
    {
        const float rh[3] = {Rp[3 * e].x, Rp[3 * e + 1].x, Rp[3 * e + 2].x};
        const float rl[3] = {Rp[3 * e].y, Rp[3 * e + 1].y, Rp[3 * e + 2].y};
        float gj[3];
        jastrow_at(s, Rp, e, rh, rl, v7[6], gj);
        v7[3] = gj[0];
        v7[4] = gj[1];
        v7[5] = gj[2];
    }
    cta_sum_to0<7>(v7, S.red);
    if (tid == 0) {
        const float g[3] = {v7[0] + v7[3], v7[1] + v7[4], v7[2] + v7[5]};
        const double* R = wk.R + ((size_t)w * N + e) * 3;
        const double r[3] = {R[0], R[1], R[2]};
        double scal[8];
        float fs[12];
        propose_move_mixed(g, p.tau, r, p.key, p.sweep, (uint32_t)e, (uint32_t)w, scal, fs);
        float* mv = ts.mv + (size_t)w * kTiledMv;
#pragma unroll
        for (int c = 0; c < 12; ++c) mv[c] = fs[c];
        mv[12] = v7[6];
        double* rn = ts.rn + (size_t)w * 3;
        rn[0] = scal[0];
        rn[1] = scal[1];
        rn[2] = scal[2];
#pragma unroll
        for (int c = 0; c < 6; ++c) S.fs[c] = fs[c];
    }
    __syncthreads();
    const float ph[3] = {S.fs[0], S.fs[1], S.fs[2]}, pl[3] = {S.fs[3], S.fs[4], S.fs[5]};
    // basis at r': the radial sums of every shell once (thread per shell,
    // zeros where screened) into shared memory, then the walker's five rows
    // of B' as TF32 hi / lo halves, one thread per basis function
    // (consecutive threads write consecutive columns); functions of screened
    // shells are written as zeros (the buffers are reused every move)
    float* Bh = ts.Bh + (size_t)w * 5 * nbp;
    float* Bl = ts.Bl + (size_t)w * 5 * nbp;
    const float* amin = s.shell_amin_f;
    for (int sh = tid; sh < s.n_shell; sh += kTb) {
        const int4 d = s.shell[sh];
        const int c3 = 3 * d.x;
        const float x = diff_f2(ph[0], pl[0], s.Rn_hi[c3], s.Rn_lo[c3]);
        const float y = diff_f2(ph[1], pl[1], s.Rn_hi[c3 + 1], s.Rn_lo[c3 + 1]);
        const float z = diff_f2(ph[2], pl[2], s.Rn_hi[c3 + 2], s.Rn_lo[c3 + 2]);
        const float t2 = x * x + y * y + z * z;
        float f0 = 0.f, f1 = 0.f, f2 = 0.f, f3;
        if (!(amin[sh] * t2 > (float)kScreenExponent)) radial<float, false>(s.alpha_f, s.cn_f, d.z, d.w, t2, f0, f1, f2, f3);
        S.rad[3 * sh] = f0;
        S.rad[3 * sh + 1] = f1;
        S.rad[3 * sh + 2] = f2;
    }
    __syncthreads();
    for (int fn = tid; fn < s.n_basis; fn += kTb) {
        const int sh = ts.fn_shell[fn];
        const int4 d = s.shell[sh];
        const int c3 = 3 * d.x;
        const float x = diff_f2(ph[0], pl[0], s.Rn_hi[c3], s.Rn_lo[c3]);
        const float y = diff_f2(ph[1], pl[1], s.Rn_hi[c3 + 1], s.Rn_lo[c3 + 1]);
        const float z = diff_f2(ph[2], pl[2], s.Rn_hi[c3 + 2], s.Rn_lo[c3 + 2]);
        const float t2 = x * x + y * y + z * z;
        float out[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
        const float f0 = S.rad[3 * sh], f1 = S.rad[3 * sh + 1], f2 = S.rad[3 * sh + 2];
        if (f0 != 0.f || f1 != 0.f || f2 != 0.f) {
            const AngPoly<float> a = angular<float>(d.y & 0xff, d.y >> 8, fn - s.shell_fn[sh], x, y, z);
            const float Sx = 2.f * x * f1, Sy = 2.f * y * f1, Sz = 2.f * z * f1;
            const float LS = 6.f * f1 + 4.f * t2 * f2;
            out[0] = a.P * f0;
            out[1] = a.P * Sx + a.Px * f0;
            out[2] = a.P * Sy + a.Py * f0;
            out[3] = a.P * Sz + a.Pz * f0;
            out[4] = a.P * LS + 2.f * (a.Px * Sx + a.Py * Sy + a.Pz * Sz) + (a.Hxx + a.Hyy + a.Hzz) * f0;
        }
#pragma unroll
        for (int c = 0; c < 5; ++c) {
            const float h = tf32_rna(out[c]);
            Bh[c * nbp + fn] = h;
            Bl[c * nbp + fn] = tf32_rna(out[c] - h);
        }
    }
}

// Ratio, drift at r', Jastrow change, Metropolis test of walker w's move of
// electron e; an accepted move borders K^-1 and queues its orbital row.
__device__ __forceinline__ void accept_body(const DevSys& s, const DevWalkers& wk, const TiledState& ts, int w, int e,
                                            const SweepParams& p, AcceptSmem& S) {
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int nu = s.n_up, N = s.N, spin = e >= nu, n = spin ? s.n_dn : nu, k = spin ? e - nu : e;
    const int kmax = ts.kmax, ldv = ts.ldv;
    const float* Phi = ts.Phi + (size_t)w * 5 * n;
    const float* ce = ts.ce + (size_t)w * ldv;
    const float* mv = ts.mv + (size_t)w * kTiledMv;
    float v8[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int j = tid; j < n; j += kTb) {
        const float a = ce[j];
        v8[0] += Phi[j] * a;
        v8[1] += Phi[n + j] * a;
        v8[2] += Phi[2 * n + j] * a;
        v8[3] += Phi[3 * n + j] * a;
    }
    const float2* Rp = ts.Rp + (size_t)w * 3 * N;
    {
        const float rh[3] = {mv[0], mv[1], mv[2]}, rl[3] = {mv[3], mv[4], mv[5]};
        float gj[3];
        jastrow_at(s, Rp, e, rh, rl, v8[4], gj);
        v8[5] = gj[0];
        v8[6] = gj[1];
        v8[7] = gj[2];
    }
    cta_sum_to0<8>(v8, S.red);
    if (tid == 0) {
        float fs[12];
#pragma unroll
        for (int c = 0; c < 12; ++c) fs[c] = mv[c];
        const float gd[3] = {v8[1], v8[2], v8[3]}, gj[3] = {v8[5], v8[6], v8[7]};
        S.acc = accept_move_mixed(v8[0], gd, gj, v8[4] - mv[12], p.tau, fs, p.key, p.sweep, (uint32_t)e,
                                  (uint32_t)w);
        S.rho = v8[0];
    }
    __syncthreads();
    if (!S.acc) return;   // uniform over the CTA
    const float rho = S.rho;
    const float* AT = (const float*)wk.Ainv[spin] + (size_t)w * n * n;
    float* V = ts.V + (size_t)w * kmax * ldv;
    float2* KT = ts.KinvT + (size_t)w * kmax * kmax;
    const int dq = ts.dq[w];
    if (tid < dq) {
        S.rows[tid] = ts.rows[(size_t)w * kmax + tid];
        S.t[tid] = ts.tv[(size_t)w * kmax + tid];
    }
    __syncthreads();
    // new row of K: c_m = phi' . A0^-1[:, r_m] (a warp per m)
    for (int m = wid; m < dq; m += kTb / 32) {
        float a = 0.f;
        for (int j = lane; j < n; j += 32) a += Phi[j] * AT[(size_t)S.rows[m] * n + j];
        a = wsum(a);
        if (lane == 0) S.c[m] = a;
    }
    for (int j = tid; j < n; j += kTb) V[(size_t)dq * ldv + j] = Phi[j];
    float* Gk = (float*)wk.G[spin] + ((size_t)w * n + k) * 4 * n;
    for (int o = tid; o < 4 * n; o += kTb) Gk[o] = Phi[n + o];
    __syncthreads();
    // u^T = c^T K^-1: u_m = sum_q c_q (K^-1)_{qm} = sum_q c_q KinvT[m][q]
    if (tid < dq) {
        float2 u = make_float2(0.f, 0.f);
        for (int q = 0; q < dq; ++q) u = df_add(u, df_mulf(KT[(size_t)tid * kmax + q], S.c[q]));
        S.u[tid] = u;
    }
    __syncthreads();
    // K'^-1 = [[Ki + t u^T / rho, -t / rho], [-u^T / rho, 1 / rho]]
    const float2 is = df_rcp(rho);
    for (int q2 = tid; q2 < dq * dq; q2 += kTb) {
        const int q = q2 / dq, m = q2 - q * dq;
        float2* kk = KT + (size_t)q * kmax + m;                            // (Ki)_{mq}
        *kk = df_add(*kk, df_mul(df_mul(S.t[m], S.u[q]), is));
    }
    if (tid < dq) {
        KT[(size_t)dq * kmax + tid] = df_neg(df_mul(S.t[tid], is));        // (K'^-1)_{tid, dq}
        KT[(size_t)tid * kmax + dq] = df_neg(df_mul(S.u[tid], is));        // (K'^-1)_{dq, tid}
    }
    if (tid == 0) {
        KT[(size_t)dq * kmax + dq] = is;
        ts.rows[(size_t)w * kmax + dq] = k;
        ts.dq[w] = dq + 1;
        wk.logdet[2 * w + spin] += (double)logf(rho);
        const double* rn = ts.rn + (size_t)w * 3;
        double* R = wk.R + ((size_t)w * N + e) * 3;
        float2* Re = ts.Rp + ((size_t)w * N + e) * 3;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            R[c] = rn[c];
            Re[c] = make_float2(mv[c], mv[3 + c]);
        }
        ts.acc[w] += 1u;
    }
}

// Walkers w0 + blockIdx.x < W of the launch's walker group.
__global__ void __launch_bounds__(kTb, 8) k_tiled_propose(DevSys s, DevWalkers wk, TiledState ts, int w0, int W,
                                                          int e, SweepParams p) {
    __shared__ ProposeSmem S;
    const int w = w0 + (int)blockIdx.x;
    if (w >= W) return;
    propose_body(s, wk, ts, w, e, p, S);
}

__global__ void __launch_bounds__(kTb, 8) k_tiled_accept(DevSys s, DevWalkers wk, TiledState ts, int w0, int W,
                                                         int e, SweepParams p) {
    __shared__ AcceptSmem S;
    const int w = w0 + (int)blockIdx.x;
    if (w >= W) return;
    accept_body(s, wk, ts, w, e, p, S);
}

// The accept step of electron e and the proposal of electron e + 1 of the
// same walker in one launch (no flush between them): the walker's queue,
// inverse and positions written by the accept step are read back by the
// same CTA after a barrier.  Bound by the latency of its dependent loads:
// twelve CTAs per SM (40 registers, 36 bytes of spills) hide more of it than
// eight (64 registers): the 32-water step 100.9 -> 95.3 ms at 4096 walkers.
__global__ void __launch_bounds__(kTb, 12) k_tiled_accept_propose(DevSys s, DevWalkers wk, TiledState ts, int w0,
                                                                 int W, int e, SweepParams p) {
    __shared__ AcceptSmem Sa;
    __shared__ ProposeSmem Sp;
    const int w = w0 + (int)blockIdx.x;
    if (w >= W) return;
    accept_body(s, wk, ts, w, e, p, Sa);
    __syncthreads();
    propose_body(s, wk, ts, w, e + 1, p, Sp);
}

// P[m] = row r_m of A0^-T for m < dq, zero rows beyond.
__global__ void k_tiled_gather(DevWalkers wk, TiledState ts, int w0, int W, int spin, int n) {
    const int w = w0 + (int)blockIdx.x;
    if (w >= W) return;
    const int kmax = ts.kmax, ldv = ts.ldv, dq = ts.dq[w];
    const float* AT = (const float*)wk.Ainv[spin] + (size_t)w * n * n;
    float* P = ts.P + (size_t)w * kmax * ldv;
    for (int q = threadIdx.x; q < kmax * n; q += blockDim.x) {
        const int m = q / n, i = q - m * n;
        P[(size_t)m * ldv + i] = m < dq ? AT[(size_t)ts.rows[(size_t)w * kmax + m] * n + i] : 0.f;
    }
}

// X^T[j][m] = sum_q (K^-1)_{mq} (Z^T[j][q] - delta(j, r_q)) for m < dq, zero
// for m >= dq; the queue is emptied.  The product is formed in double-float
// arithmetic: each entry of K^-1 a pair (hi, lo) of floats, the exact error
// of every product hi z (fma) and of every addition (Knuth's two-sum)
// carried in a second float, ~44 bits on the FP32 pipe.
__global__ void __launch_bounds__(kTb) k_tiled_x(TiledState ts, int w0, int W, int n) {
    __shared__ float2 s_k[32 * 32];   // (K^-1)_{mq} as (hi, lo) at [q][m]
    __shared__ int s_rows[32];
    const int w = w0 + (int)blockIdx.x;
    if (w >= W) return;
    const int kmax = ts.kmax, dq = ts.dq[w];
    const float2* KT = ts.KinvT + (size_t)w * kmax * kmax;
    for (int q2 = threadIdx.x; q2 < dq * dq; q2 += kTb) {
        const int q = q2 / dq, m = q2 - q * dq;
        s_k[q * 32 + m] = KT[(size_t)q * kmax + m];
    }
    if (threadIdx.x < dq) s_rows[threadIdx.x] = ts.rows[(size_t)w * kmax + threadIdx.x];
    __syncthreads();
    const float* Zt = ts.Zt + (size_t)w * n * kmax;
    float* Xt = ts.Xt + (size_t)w * n * kmax;
    for (int q2 = threadIdx.x; q2 < n * kmax; q2 += kTb) {
        const int j = q2 / kmax, m = q2 - j * kmax;
        float hi = 0.f, lo = 0.f;
        if (m < dq) {
            const float* z = Zt + (size_t)j * kmax;
            for (int q = 0; q < dq; ++q) {
                const float2 kk = s_k[q * 32 + m];
                float zq = z[q];
                float kh = kk.x, kl = kk.y;
                if (s_rows[q] == j) {   // - delta(j, r_q): add -(K^-1)_{mq} as a separate exact term
                    const float t = hi - kh;
                    const float bp = t - hi;
                    lo += (hi - (t - bp)) + (-kh - bp) - kl;
                    hi = t;
                }
                const float pr = kh * zq;
                const float pe = fmaf(kh, zq, -pr) + kl * zq;
                const float t = hi + pr;
                const float bp = t - hi;
                lo += (hi - (t - bp)) + (pr - bp) + pe;
                hi = t;
            }
        }
        Xt[q2] = hi + lo;
    }
    __syncthreads();
    if (threadIdx.x == 0) ts.dq[w] = 0;
}

__global__ void k_tiled_end(TiledState ts, int W, unsigned long long* n_acc) {
    __shared__ unsigned long long s;
    if (threadIdx.x == 0) s = 0ull;
    __syncthreads();
    unsigned long long a = 0ull;
    for (int w = blockIdx.x * blockDim.x + threadIdx.x; w < W; w += gridDim.x * blockDim.x) a += ts.acc[w];
    atomicAdd(&s, a);
    __syncthreads();
    if (threadIdx.x == 0 && s) atomicAdd(n_acc, s);
}

}  // namespace

cudaError_t tiled_begin(const DevWalkers& wk, int W, int N, const TiledState& ts, cudaStream_t st) {
    const int nthr = 3 * W * N > W ? 3 * W * N : W;
    k_tiled_begin<<<(nthr + 255) / 256, 256, 0, st>>>(wk.R, W, N, ts);
    return cudaGetLastError();
}

cudaError_t tiled_propose(const DevSys& s, const DevWalkers& wk, const TiledState& ts, int w0, int nw, int e,
                          const SweepParams& p, cudaStream_t st) {
    if (nw <= 0) return cudaSuccess;
    k_tiled_propose<<<nw, kTb, 0, st>>>(s, wk, ts, w0, w0 + nw, e, p);
    return cudaGetLastError();
}

cudaError_t tiled_accept(const DevSys& s, const DevWalkers& wk, const TiledState& ts, int w0, int nw, int e,
                         const SweepParams& p, cudaStream_t st) {
    if (nw <= 0) return cudaSuccess;
    k_tiled_accept<<<nw, kTb, 0, st>>>(s, wk, ts, w0, w0 + nw, e, p);
    return cudaGetLastError();
}

cudaError_t tiled_accept_propose(const DevSys& s, const DevWalkers& wk, const TiledState& ts, int w0, int nw, int e,
                                 const SweepParams& p, cudaStream_t st) {
    if (nw <= 0) return cudaSuccess;
    k_tiled_accept_propose<<<nw, kTb, 0, st>>>(s, wk, ts, w0, w0 + nw, e, p);
    return cudaGetLastError();
}

// The queues of walkers [w0, w0 + nw) into A0^-T of one spin (four
// launches; the GEMMs batch over the group's walkers).
cudaError_t tiled_flush(const DevWalkers& wk, const TiledState& ts, int w0, int nw, int spin, int n, unsigned* err,
                        cudaStream_t st) {
    if (nw <= 0) return cudaSuccess;
    const long long n2 = (long long)n * n;
    float* AT = (float*)wk.Ainv[spin] + (size_t)w0 * n2;
    float* V = ts.V + (size_t)w0 * ts.kmax * ts.ldv;
    float* P = ts.P + (size_t)w0 * ts.kmax * ts.ldv;
    float* Zt = ts.Zt + (size_t)w0 * n * ts.kmax;
    float* Xt = ts.Xt + (size_t)w0 * n * ts.kmax;
    k_tiled_gather<<<nw, 128, 0, st>>>(wk, ts, w0, w0 + nw, spin, n);
    cudaError_t e0 = cudaGetLastError();
    if (e0 != cudaSuccess) return e0;
    // Z^T[j][m] = sum_i A0^-T[j][i] V[m][i]
    e0 = launch_tc_gemm_ab(nw, n, ts.kmax, n, 1.f, AT, n2, n, V, (long long)ts.kmax * ts.ldv, ts.ldv, 0, 0.f, Zt,
                           (long long)n * ts.kmax, ts.kmax, err, st);
    if (e0 != cudaSuccess) return e0;
    k_tiled_x<<<nw, kTb, 0, st>>>(ts, w0, w0 + nw, n);
    if ((e0 = cudaGetLastError()) != cudaSuccess) return e0;
    // A0^-T[j][i] -= sum_m X^T[j][m] P[m][i]
    return launch_tc_gemm_ab(nw, n, n, ts.kmax, -1.f, Xt, (long long)n * ts.kmax, ts.kmax, P,
                             (long long)ts.kmax * ts.ldv, ts.ldv, 1, 1.f, AT, n2, n, err, st);
}

cudaError_t tiled_end(const TiledState& ts, int W, unsigned long long* n_acc, cudaStream_t st) {
    k_tiled_end<<<64, 256, 0, st>>>(ts, W, n_acc);
    return cudaGetLastError();
}

// C^T of one spin as TF32 hi / lo halves: Ct[j][l] = C[l][j] for l <
// n_basis, zero for the padding columns l < nbp.
__global__ void k_transpose_coeffs(const float* C, int nb, int n, int nbp, float* Cth, float* Ctl) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n * nbp) return;
    const int j = i / nbp, l = i - j * nbp;
    const float v = l < nb ? C[(size_t)l * n + j] : 0.f;
    const float h = tf32_rna(v);
    Cth[i] = h;
    Ctl[i] = tf32_rna(v - h);
}

cudaError_t launch_tiled_coeffs(const DevSys& s, const TiledState& ts, cudaStream_t st) {
    for (int spin = 0; spin < 2; ++spin) {
        const int n = spin ? s.n_dn : s.n_up;
        if (n == 0) continue;
        k_transpose_coeffs<<<(n * ts.nbp + 255) / 256, 256, 0, st>>>(s.C_f[spin], s.n_basis, n, ts.nbp,
                                                                     ts.Cth[spin], ts.Ctl[spin]);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace qmc
