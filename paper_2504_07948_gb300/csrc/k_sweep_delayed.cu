// Particle-by-particle sweep with delayed (Woodbury) inverse updates.
//
// For large determinants the Sherman-Morrison update reads and rewrites the
// whole n x n inverse on every accepted move.  Here accepted moves are
// queued: after d accepted moves of distinct rows r_1..r_d with new orbital
// rows phi'_1..phi'_d since the last flush, the current inverse is
//   A^-1 = A0^-1 - A0^-1 E K^-1 (V^T A0^-1 - E^T),
//   E = [e_{r_1} .. e_{r_d}],  V = [phi'_1 .. phi'_d],
//   K_{m m'} = phi'_m . A0^-1[:, r_{m'}]          (d x d),
// (the identity and the old rows cancel because the rows are distinct), so
// the column a move needs is
//   c_e = A0^-1[:, e] - sum_m (K^-1 y)_m A0^-1[:, r_m],  y_m = phi'_m . A0^-1[:, e],
// at O(n d) cost.  Accepting a move borders K (its new row are d dots, its
// new column is y, and the Schur complement is the ratio itself), and every
// k accepted moves (and at the end of each spin block) a rank-d flush
//   A0^-1 <- A0^-1 - P K^-1 Z,  P = A0^-1 E,  Z = V^T A0^-1 - E^T,
// touches the inverse once.  A0^-1 is kept transposed (row e = column e) in
// global memory; the queue lives in shared memory.  K^-1, its bordering and
// the flush product K^-1 Z are FP64 in both forms (the flush carries every
// queued move into A0^-1); the mixed form's per-move column update applies
// a float copy of K^-1 y.
#include "batch.cuh"
#include "qmc_internal.cuh"
#include "sweep_sm.cuh"

namespace qmc {

template <typename T>
__host__ __device__ inline size_t delayed_smem_layout(int N, int nb, int nmax, int kmax, size_t* o_bas, size_t* o_phi,
                                                      size_t* o_ce, size_t* o_V, size_t* o_P, size_t* o_K,
                                                      size_t* o_small) {
    // positions (double), reductions, scalars, positions as (hi, lo) float
    // pairs (FP32 offsets of the mixed form)
    size_t o = sizeof(double) * (3 * (size_t)N + kMaxWarps * 8 + 16) + sizeof(float2) * 3 * (size_t)N;
    o = (o + 15) & ~(size_t)15;
    *o_bas = o;
    o += basis_live_bytes<T, false>(nb);   // no shell list: the queue fills the shared memory
    *o_phi = o;
    o += sizeof(T) * 5 * (size_t)nmax;
    *o_ce = o;
    o += sizeof(T) * (size_t)nmax;
    o = (o + 15) & ~(size_t)15;
    *o_V = o;
    o += sizeof(T) * (size_t)kmax * nmax;  // queued rows phi'_m (later Z)
    *o_P = o;
    o += sizeof(T) * 2 * (size_t)kmax * nmax;  // rows r_m of A0^-T and Z (flush)
    *o_K = o;
    o += sizeof(double) * (size_t)kmax * kmax;
    *o_small = o;
    o += sizeof(double) * 3 * (size_t)kmax + sizeof(int) * (size_t)kmax + sizeof(float) * (size_t)kmax;
    return o;
}

template <typename T>
size_t delayed_smem_bytes(const DevSys& s, int kmax) {
    size_t a, b, c, d, e, f, g;
    const int nmax = s.n_up > s.n_dn ? s.n_up : s.n_dn;
    return delayed_smem_layout<T>(s.N, s.n_basis, nmax, kmax, &a, &b, &c, &d, &e, &f, &g);
}

// Lane m of the warp ends with the warp-wide sum of v[m] (m < 32): a
// transposing butterfly, 31 shuffles and adds per lane for 32 values.
template <typename T>
__device__ __forceinline__ T warp_transpose_sum32(T (&v)[32]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int half = 16; half >= 1; half >>= 1) {
        const bool up = lane & half;
#pragma unroll
        for (int i = 0; i < half; ++i) {
            const T send = up ? v[i] : v[i + half];
            const T keep = up ? v[i + half] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, half);
        }
    }
    // each step keeps the upper half of the values on lanes whose bit
    // `half` is set, so lane L ends with the total of value L
    return v[0];
}

// Rank-d flush of the queue into A0^-T (AT, row-major n x n, global).
template <typename T>
__device__ void flush_queue(T* AT, int n, int d, T* Vq, T* Pq, const double* Kinv, int kmax, const int* rows,
                            T* Zs) {
    if (d == 0) return;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    // P: rows r_m of A0^-T (columns r_m of A0^-1), copied before AT changes
    for (int q = threadIdx.x; q < d * n; q += blockDim.x) {
        const int m = q / n, i = q - m * n;
        Pq[q] = AT[(size_t)rows[m] * n + i];
    }
    // Z[m][j] = phi'_m . A0^-1[:, j] - delta(j, r_m) = sum_i phi'_m[i] AT[j][i] - delta:
    // a warp per row j of AT, lanes over i (coalesced), then the 32 partial
    // sums are transposed so that lane m holds Z[m][j].
    for (int j = wid; j < n; j += nw) {
        T part[32];
#pragma unroll
        for (int m = 0; m < 32; ++m) part[m] = T(0);
        const T* ATj = AT + (size_t)j * n;
        for (int i = lane; i < n; i += 32) {
            const T a = ATj[i];
#pragma unroll
            for (int m = 0; m < 32; ++m)
                if (m < d) part[m] += Vq[m * n + i] * a;
        }
        const T z = warp_transpose_sum32<T>(part);
        const int m = lane;
        if (m < d) Zs[m * n + j] = z - (rows[m] == j ? T(1) : T(0));
    }
    __syncthreads();
    // X = K^-1 Z (d x n), into Vq (the queued rows are no longer needed).  In
    // FP64 in both forms: with K^-1 rounded to FP32 and an FP32 product the
    // mixed form's propagated gradients reached 0.2 relative error on the
    // 32-water cluster after 12 sweeps (1e-3 with this product in FP64).
    for (int q = threadIdx.x; q < d * n; q += blockDim.x) {
        const int m = q / n, j = q - m * n;
        double a = 0.0;
        for (int r = 0; r < d; ++r) a += Kinv[m * kmax + r] * (double)Zs[r * n + j];
        Vq[q] = T(a);
    }
    __syncthreads();
    // AT[j][i] -= sum_m X[m][j] P[m][i]
    for (int q = threadIdx.x; q < n * n; q += blockDim.x) {
        const int j = q / n, i = q - j * n;
        T a = T(0);
        for (int m = 0; m < d; ++m) a += Vq[m * n + j] * Pq[m * n + i];
        AT[q] -= a;
    }
    __syncthreads();
}

// One CTA sweeps walker w with delayed updates of rank kmax.  smem: the
// dynamic shared memory laid out by delayed_smem_layout.
template <typename T>
__device__ __forceinline__ void sweep_delayed_walker(const DevSys& s, const DevWalkers& wk, int w,
                                                     const SweepParams& p, int kmax, unsigned char* smem) {
    const int N = s.N, nu = s.n_up, nd = s.n_dn, nb = s.n_basis, nn = s.n_nuc;
    const int nmax = nu > nd ? nu : nd;
    size_t ob, oph, oce, oV, oP, oK, osm;
    delayed_smem_layout<T>(N, nb, nmax, kmax, &ob, &oph, &oce, &oV, &oP, &oK, &osm);
    double* sR = (double*)smem;
    double* red = sR + 3 * N;
    double* scal = red + kMaxWarps * 8;
    float2* sRp = (float2*)(scal + 16);
    // mixed form: thread 0's move results as floats (layout of
    // propose_move_mixed: r' hi/lo, step, drift; [12] ratio, [13] accept)
    float* fs = (float*)(scal + 8);
    constexpr bool kMixed = sizeof(T) == 4;
    T* bas = (T*)(smem + ob);
    T* phi = (T*)(smem + oph);
    T* ce = (T*)(smem + oce);
    T* Vq = (T*)(smem + oV);
    T* Pq = (T*)(smem + oP);
    const bool lst_fits = (size_t)2 * kmax * nmax * sizeof(T) >= sizeof(int2) * (size_t)s.n_shell &&
                          (((uintptr_t)Pq) & 7) == 0;
    // K^-1 and its vectors in FP64 (the bordering recursion), with a float
    // copy of t = K^-1 y for the mixed form's column update
    double* Kinv = (double*)(smem + oK);
    double* yv = (double*)(smem + osm);
    double* tv = yv + kmax;
    double* cv = tv + kmax;
    int* rows = (int*)(cv + kmax);
    float* tvf = (float*)(rows + kmax);
    for (int q = threadIdx.x; q < 3 * N; q += blockDim.x) {
        const double r = wk.R[(size_t)w * 3 * N + q];
        sR[q] = r;
        if constexpr (kMixed) {
            const float hi = (float)r;
            sRp[q] = make_float2(hi, (float)(r - (double)hi));
        }
    }
    double ld0 = 0.0, ld1 = 0.0;
    if (threadIdx.x == 0) {
        ld0 = wk.logdet[2 * w];
        ld1 = wk.logdet[2 * w + 1];
    }
    unsigned long long acc = 0;
    int dq = 0;  // queued accepted moves of the current spin block
    __syncthreads();
    const double tau = p.tau;
    T* redT = (T*)red;

    for (int e = 0; e < N; ++e) {
        const int spin = e >= nu;
        const int n = spin ? nd : nu;
        const int k = spin ? e - nu : e;
        T* AT = (T*)wk.Ainv[spin] + (size_t)w * n * n;
        T* Gk = (T*)wk.G[spin] + ((size_t)w * n + k) * 4 * n;
        const double re0 = sR[3 * e], re1 = sR[3 * e + 1], re2 = sR[3 * e + 2];

        // -- column e of the current inverse -------------------------------
        // y_m = phi'_m . AT[k]  (warp per m)
        {
            const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
            const T* ATk = AT + (size_t)k * n;
            for (int m = wid; m < dq; m += nw) {
                T a = T(0);
                for (int j = lane; j < n; j += 32) a += Vq[m * n + j] * ATk[j];
                a = warp_sum(a);
                if (lane == 0) yv[m] = (double)a;
            }
        }
        __syncthreads();
        for (int m = threadIdx.x; m < dq; m += blockDim.x) {
            double a = 0.0;
            for (int q = 0; q < dq; ++q) a += Kinv[m * kmax + q] * yv[q];
            tv[m] = a;
            tvf[m] = (float)a;
        }
        __syncthreads();
        for (int j = threadIdx.x; j < n; j += blockDim.x) {
            T a = AT[(size_t)k * n + j];
            if constexpr (kMixed)
                for (int m = 0; m < dq; ++m) a -= tvf[m] * AT[(size_t)rows[m] * n + j];
            else
                for (int m = 0; m < dq; ++m) a -= T(tv[m]) * AT[(size_t)rows[m] * n + j];
            ce[j] = a;
        }
        __syncthreads();

        // -- drift at the current position ---------------------------------
        T va[8] = {T(0), T(0), T(0), T(0), T(0), T(0), T(0), T(0)};
        T u_old = T(0);
        for (int j = threadIdx.x; j < n; j += blockDim.x) {
            const T a = ce[j];
            va[0] += Gk[j] * a;
            va[1] += Gk[n + j] * a;
            va[2] += Gk[2 * n + j] * a;
        }
        float2 ep[3];
        if constexpr (kMixed) {
            ep[0] = sRp[3 * e];
            ep[1] = sRp[3 * e + 1];
            ep[2] = sRp[3 * e + 2];
        }
        for (int q = threadIdx.x; q < N + nn; q += blockDim.x) {
            T x, y, z, a, b;
            if (q < N) {
                if (q == e) continue;
                if constexpr (kMixed) {
                    const float2 q0 = sRp[3 * q], q1 = sRp[3 * q + 1], q2 = sRp[3 * q + 2];
                    x = diff_f2(ep[0].x, ep[0].y, q0.x, q0.y);
                    y = diff_f2(ep[1].x, ep[1].y, q1.x, q1.y);
                    z = diff_f2(ep[2].x, ep[2].y, q2.x, q2.y);
                } else {
                    x = T(re0 - sR[3 * q]); y = T(re1 - sR[3 * q + 1]); z = T(re2 - sR[3 * q + 2]);
                }
                a = T(((q < nu) == (e < nu)) ? s.a_par : s.a_anti);
                b = T(s.b_ee);
            } else {
                const int c = q - N;
                if constexpr (kMixed) {
                    x = diff_f2(ep[0].x, ep[0].y, s.Rn_hi[3 * c], s.Rn_lo[3 * c]);
                    y = diff_f2(ep[1].x, ep[1].y, s.Rn_hi[3 * c + 1], s.Rn_lo[3 * c + 1]);
                    z = diff_f2(ep[2].x, ep[2].y, s.Rn_hi[3 * c + 2], s.Rn_lo[3 * c + 2]);
                } else {
                    x = T(re0 - s.Rn[3 * c]); y = T(re1 - s.Rn[3 * c + 1]); z = T(re2 - s.Rn[3 * c + 2]);
                }
                a = T(s.a_en[c]);
                b = T(s.b_en);
            }
            const T ir = rsqrt_t(x * x + y * y + z * z);
            const T r = (x * x + y * y + z * z) * ir;
            const T qd = T(1) / (T(1) + b * r);
            u_old += a * r * qd;
            const T g = a * qd * qd * ir;
            va[3] += g * x;
            va[4] += g * y;
            va[5] += g * z;
        }
        block_sum8_to0<T>(va, redT);
        if (threadIdx.x < 2) {
            const T g[3] = {va[0] + va[3], va[1] + va[4], va[2] + va[5]};
            const double r[3] = {re0, re1, re2};
            if constexpr (kMixed) {
                if (threadIdx.x == 0) propose_move_mixed(g, tau, r, p.key, p.sweep, (uint32_t)e, (uint32_t)w, scal, fs);
            } else {
                const double gd[3] = {g[0], g[1], g[2]};
                propose_move_fp64_pair(gd, tau, r, p.key, p.sweep, (uint32_t)e, (uint32_t)w, scal);
            }
        }
        __syncthreads();
        double rn[3];
        if constexpr (!kMixed) {
            rn[0] = scal[0]; rn[1] = scal[1]; rn[2] = scal[2];
        }

        // -- basis (live shells, packed) and orbitals at r' -------------------
        const int ldb = basis_live_ld(nb);
        int* brows = (int*)(bas + 5 * ldb);   // packed basis rows (basis_live)
        // the live shells are compacted onto consecutive threads when the
        // flush buffer (idle until the queue is flushed) can hold their list
        int nrow;
        const double* rd = kMixed ? nullptr : rn;
        if (lst_fits)
            nrow = basis_live<T, true>(s, rd, fs, fs + 3, bas, ldb, brows, brows + ldb, reinterpret_cast<int2*>(Pq));
        else
            nrow = basis_live<T, false>(s, rd, fs, fs + 3, bas, ldb, brows, brows + ldb);
        const T* C = sys_C<T>(s, spin);
        contract5<T>(C, n, nrow, ldb, brows, bas, phi, nmax);
        __syncthreads();

        // -- ratio, new determinant gradient, Jastrow change -----------------
        T vb2[8] = {T(0), T(0), T(0), T(0), -u_old, T(0), T(0), T(0)};
        for (int j = threadIdx.x; j < n; j += blockDim.x) {
            const T a = ce[j];
            vb2[0] += phi[j] * a;
            vb2[1] += phi[nmax + j] * a;
            vb2[2] += phi[2 * nmax + j] * a;
            vb2[3] += phi[3 * nmax + j] * a;
        }
        for (int q = threadIdx.x; q < N + nn; q += blockDim.x) {
            T x, y, z, a, b;
            if (q < N) {
                if (q == e) continue;
                if constexpr (kMixed) {
                    const float2 q0 = sRp[3 * q], q1 = sRp[3 * q + 1], q2 = sRp[3 * q + 2];
                    x = diff_f2(fs[0], fs[3], q0.x, q0.y);
                    y = diff_f2(fs[1], fs[4], q1.x, q1.y);
                    z = diff_f2(fs[2], fs[5], q2.x, q2.y);
                } else {
                    x = T(rn[0] - sR[3 * q]); y = T(rn[1] - sR[3 * q + 1]); z = T(rn[2] - sR[3 * q + 2]);
                }
                a = T(((q < nu) == (e < nu)) ? s.a_par : s.a_anti);
                b = T(s.b_ee);
            } else {
                const int c = q - N;
                if constexpr (kMixed) {
                    x = diff_f2(fs[0], fs[3], s.Rn_hi[3 * c], s.Rn_lo[3 * c]);
                    y = diff_f2(fs[1], fs[4], s.Rn_hi[3 * c + 1], s.Rn_lo[3 * c + 1]);
                    z = diff_f2(fs[2], fs[5], s.Rn_hi[3 * c + 2], s.Rn_lo[3 * c + 2]);
                } else {
                    x = T(rn[0] - s.Rn[3 * c]); y = T(rn[1] - s.Rn[3 * c + 1]); z = T(rn[2] - s.Rn[3 * c + 2]);
                }
                a = T(s.a_en[c]);
                b = T(s.b_en);
            }
            const T ir = rsqrt_t(x * x + y * y + z * z);
            const T r = (x * x + y * y + z * z) * ir;
            const T qd = T(1) / (T(1) + b * r);
            vb2[4] += a * r * qd;
            const T g = a * qd * qd * ir;
            vb2[5] += g * x;
            vb2[6] += g * y;
            vb2[7] += g * z;
        }
        block_sum8_to0<T>(vb2, redT);
        if (threadIdx.x == 0) {
            const T gd[3] = {vb2[1], vb2[2], vb2[3]}, gj[3] = {vb2[5], vb2[6], vb2[7]};
            int accept;
            if constexpr (kMixed) {
                accept = accept_move_mixed(vb2[0], gd, gj, vb2[4], tau, fs, p.key, p.sweep, (uint32_t)e,
                                           (uint32_t)w);
                ((int*)fs)[13] = accept;
            } else {
                const double ro3[3] = {re0, re1, re2};
                accept = accept_move<T>(vb2[0], gd, gj, vb2[4], tau, ro3, rn, scal + 3, p.key, p.sweep,
                                        (uint32_t)e, (uint32_t)w);
                scal[7] = accept ? 1.0 : 0.0;
            }
            scal[6] = double(vb2[0]);
            scal[15] = 1.0 / scal[6];   // one FP64 division for the CTA
        }
        __syncthreads();
        if (kMixed ? ((const int*)fs)[13] != 0 : scal[7] != 0.0) {
            // border K: new row c_m' = phi' . A0^-1[:, r_m'] (warp per m'), new column y
            {
                const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
                for (int m = wid; m < dq; m += nw) {
                    const T* ATr = AT + (size_t)rows[m] * n;
                    T a = T(0);
                    for (int j = lane; j < n; j += 32) a += phi[j] * ATr[j];
                    a = warp_sum(a);
                    if (lane == 0) cv[m] = (double)a;
                }
            }
            for (int j = threadIdx.x; j < n; j += blockDim.x) Vq[dq * n + j] = phi[j];
            __syncthreads();
            // K' = [[K, y], [c^T, kappa]], s = kappa - c^T K^-1 y = rho
            // K'^-1 = [[Ki + t u^T / s, -t / s], [-u^T / s, 1 / s]], t = Ki y, u^T = c^T Ki
            double* uu = yv;  // y is not needed any more
            for (int m = threadIdx.x; m < dq; m += blockDim.x) {
                double a = 0.0;
                for (int q = 0; q < dq; ++q) a += cv[q] * Kinv[q * kmax + m];
                uu[m] = a;
            }
            __syncthreads();
            const double is = scal[15];
            for (int q2 = threadIdx.x; q2 < dq * dq; q2 += blockDim.x) {
                const int m = q2 / dq, q = q2 - m * dq;
                Kinv[m * kmax + q] += tv[m] * uu[q] * is;
            }
            for (int m = threadIdx.x; m < dq; m += blockDim.x) {
                Kinv[m * kmax + dq] = -tv[m] * is;
                Kinv[dq * kmax + m] = -uu[m] * is;
            }
            if (threadIdx.x == 0) {
                Kinv[dq * kmax + dq] = is;
                rows[dq] = k;
                // the mixed form's ratio is an FP32 number: its log in FP32
                const double lr = kMixed ? (double)logf((float)scal[6]) : log(scal[6]);
                if (spin)
                    ld1 += lr;
                else
                    ld0 += lr;
                for (int c = 0; c < 3; ++c) {
                    sR[3 * e + c] = scal[c];
                    if constexpr (kMixed) sRp[3 * e + c] = make_float2(fs[c], fs[3 + c]);
                }
                ++acc;
            }
            for (int o = threadIdx.x; o < 4 * n; o += blockDim.x) {
                const int c = o / n, j = o - c * n;
                Gk[o] = phi[(c + 1) * nmax + j];
            }
            ++dq;
            __syncthreads();
        }
        const bool block_end = (e == nu - 1) || (e == N - 1);
        if (dq == kmax || (block_end && dq > 0)) {
            flush_queue<T>(AT, n, dq, Vq, Pq, Kinv, kmax, rows, Pq + (size_t)kmax * nmax);
            dq = 0;
        }
    }
    __syncthreads();
    for (int q = threadIdx.x; q < 3 * N; q += blockDim.x) wk.R[(size_t)w * 3 * N + q] = sR[q];
    if (threadIdx.x == 0) {
        wk.logdet[2 * w] = ld0;
        wk.logdet[2 * w + 1] = ld1;
        if (acc) atomicAdd(wk.n_acc, acc);
    }
}

template <typename T>
__global__ void __launch_bounds__(256, 2) k_sweep_delayed(DevSys s, DevWalkers wk, int W, SweepParams p, int kmax) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int w = blockIdx.x;
    if (w >= W) return;
    sweep_delayed_walker<T>(s, wk, w, p, kmax, smem);
}

template <typename T>
cudaError_t launch_sweep_delayed(const DevSys& s, const DevWalkers& wk, int W, const SweepParams& p, int kmax,
                                 cudaStream_t st) {
    if (W == 0 || s.N == 0) return cudaSuccess;
    const size_t smem = delayed_smem_bytes<T>(s, kmax);
    cudaError_t e = cudaFuncSetAttribute(k_sweep_delayed<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_sweep_delayed<T><<<W, 256, smem, st>>>(s, wk, W, p, kmax);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------
// Batched sweep: one persistent launch over the walkers of every system of
// a batch; each walker is swept with its system's update scheme (Sherman-
// Morrison or delayed, rank chosen per system).  The dynamic shared memory
// is the largest any system needs.  kDelayed = false compiles the Sherman-
// Morrison body alone (fewer registers, more resident CTAs) for batches in
// which no system uses delayed updates.
// ---------------------------------------------------------------------
template <typename T, bool kDelayed>
__global__ void __launch_bounds__(256, 3)
    k_sweep_batch(const BatchSys* __restrict__ sys, BatchPlan* plan, const BatchCtl* __restrict__ ctl, int parity,
                  double tau, int ctr) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ BatchSys bs;
    __shared__ int s_sys, s_idx;
    for (;;) {
        if (threadIdx.x == 0) batch_next(plan, kUnitWalker, ctr, &s_sys, &s_idx);
        __syncthreads();
        const int q = s_sys;
        if (q < 0) break;
        batch_load(&bs, sys + q);
        __syncthreads();
        SweepParams p{};
        p.tau = tau;
        p.key = bs.key;
        p.sweep = ctl[q].sweep;
        p.ainv_smem = bs.ainv_smem;
        p.g_smem = 0;
        if (kDelayed && bs.delay_rank > 1)
            sweep_delayed_walker<T>(bs.s, bs.wk[parity], s_idx, p, bs.delay_rank, smem);
        else
            sweep_walker<T>(bs.s, bs.wk[parity], s_idx, p, smem);
        __syncthreads();
    }
}

template <typename T>
size_t sweep_batch_smem(const DevSys& s, int delay_rank, int ainv_smem) {
    if (delay_rank > 1) return delayed_smem_bytes<T>(s, delay_rank);
    return sweep_smem_bytes<T>(s, ainv_smem, 0);
}

// Sets the kernel's dynamic shared memory limit (before any launch or graph
// capture) and returns its resident CTAs per SM (0 if it cannot run).
template <typename T>
int sweep_batch_prepare(int block, size_t smem, int delayed) {
    int nb = 0;
    const void* f = delayed ? (const void*)k_sweep_batch<T, true> : (const void*)k_sweep_batch<T, false>;
    if (cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, f, block, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return nb;
}

template <typename T>
cudaError_t launch_sweep_batch(const BatchSys* sys, BatchPlan* plan, const BatchCtl* ctl, int parity, double tau,
                               int ctr, int grid, int block, size_t smem, int delayed, cudaStream_t st) {
    if (delayed)
        k_sweep_batch<T, true><<<grid, block, smem, st>>>(sys, plan, ctl, parity, tau, ctr);
    else
        k_sweep_batch<T, false><<<grid, block, smem, st>>>(sys, plan, ctl, parity, tau, ctr);
    return cudaGetLastError();
}

template size_t sweep_batch_smem<double>(const DevSys&, int, int);
template size_t sweep_batch_smem<float>(const DevSys&, int, int);
template int sweep_batch_prepare<double>(int, size_t, int);
template int sweep_batch_prepare<float>(int, size_t, int);
template cudaError_t launch_sweep_batch<double>(const BatchSys*, BatchPlan*, const BatchCtl*, int, double, int, int,
                                                int, size_t, int, cudaStream_t);
template cudaError_t launch_sweep_batch<float>(const BatchSys*, BatchPlan*, const BatchCtl*, int, double, int, int,
                                               int, size_t, int, cudaStream_t);

template size_t delayed_smem_bytes<double>(const DevSys&, int);
template size_t delayed_smem_bytes<float>(const DevSys&, int);
template cudaError_t launch_sweep_delayed<double>(const DevSys&, const DevWalkers&, int, const SweepParams&, int,
                                                  cudaStream_t);
template cudaError_t launch_sweep_delayed<float>(const DevSys&, const DevWalkers&, int, const SweepParams&, int,
                                                 cudaStream_t);

}  // namespace qmc
