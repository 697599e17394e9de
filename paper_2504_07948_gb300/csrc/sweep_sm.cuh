// Body of the Sherman-Morrison sweep of one walker (see k_sweep.cu), shared
// by the single-system kernel and the batched persistent kernel.
#pragma once

#include "qmc_internal.cuh"

namespace qmc {

template <typename T>
__host__ __device__ inline size_t sweep_smem_layout(int N, int nb, int nu, int nd, int ainv_smem, int g_smem,
                                                    size_t* off_bas, size_t* off_phi, size_t* off_cold,
                                                    size_t* off_A, size_t* off_G) {
    const int nmax = nu > nd ? nu : nd;
    // positions (double), reductions, scalars, then the positions split as
    // hi + lo floats for the FP32 offsets of the mixed form
    size_t o = sizeof(double) * (3 * (size_t)N + kMaxWarps * 8 + 16) + sizeof(float) * 6 * (size_t)N;
    o = (o + 15) & ~(size_t)15;
    *off_bas = o;
    o += basis_live_bytes<T>(nb);
    *off_phi = o;
    o += sizeof(T) * 5 * (size_t)nmax;
    *off_cold = o;
    o += sizeof(T) * (size_t)nmax;
    o = (o + 15) & ~(size_t)15;
    *off_A = o;
    if (ainv_smem) o += sizeof(T) * ((size_t)nu * nu + (size_t)nd * nd);
    *off_G = o;
    if (g_smem) o += sizeof(T) * 4 * ((size_t)nu * nu + (size_t)nd * nd);
    return o;
}

// Three-body Jastrow terms of electron e placed at (x0, x1, x2) with the
// partner and nucleus of item q = a N + j (j != e; the item is skipped when
// j == e): value and gradient in r_e, summed over the terms.
__device__ __forceinline__ void j3_of_electron_pair(const DevSys& s, const double* sR, int e, double x0, double x1,
                                                    double x2, int q, double& uv, double gg[3]) {
    uv = 0.0;
    gg[0] = gg[1] = gg[2] = 0.0;
    const int a = q / s.N, j = q - a * s.N;
    if (j == e) return;
    const double* ra = s.Rn + 3 * a;
    const double* rj = sR + 3 * j;
    const SDist xe = sdist(s.b3, x0 - ra[0], x1 - ra[1], x2 - ra[2]);
    const SDist xj = sdist(s.b3, rj[0] - ra[0], rj[1] - ra[1], rj[2] - ra[2]);
    const SDist y = sdist(s.b3, x0 - rj[0], x1 - rj[1], x2 - rj[2]);
    const double* c = s.c3 + (size_t)a * s.n3;
    for (int k = 0; k < s.n3; ++k) {
        if (c[k] == 0.0) continue;
        double v, g[3], l;
        j3_term(s.e3[3 * k], s.e3[3 * k + 1], s.e3[3 * k + 2], xe, xj, y, v, g, l);
        uv += c[k] * v;
        gg[0] += c[k] * g[0];
        gg[1] += c[k] * g[1];
        gg[2] += c[k] * g[2];
    }
}

// One CTA sweeps walker w of the system (every electron once).  smem: the
// dynamic shared memory laid out by sweep_smem_layout.  kSliced: see
// contract5.  kJ3: the trial function carries the three-body Jastrow
// (separate instantiation, so the code of the two-body sweep is unchanged).
template <typename T, bool kSliced = true, bool kJ3 = false>
__device__ __forceinline__ void sweep_walker(const DevSys& s, const DevWalkers& wk, int w, const SweepParams& p,
                                             unsigned char* smem) {
    const int N = s.N, nu = s.n_up, nd = s.n_dn, nb = s.n_basis, nn = s.n_nuc;
    const int nmax = nu > nd ? nu : nd;
    size_t ob, oph, oc, oA, oG;
    sweep_smem_layout<T>(N, nb, nu, nd, p.ainv_smem, p.g_smem, &ob, &oph, &oc, &oA, &oG);
    double* sR = (double*)smem;
    double* red = sR + 3 * N;
    double* scal = red + kMaxWarps * 8;
    float* sRf = (float*)(scal + 16);
    float* sRl = sRf + 3 * N;
    // Mixed form: thread 0's move results as floats, read by every thread
    // without an FP64 instruction: [0..2] r' hi, [3..5] r' lo, [6..8] the
    // step r' - r, [9..11] the drift at r, [12] ratio, [13] accept (int).
    float* fs = (float*)(scal + 8);
    constexpr bool kMixed = sizeof(T) == 4;
    // positions in the precision of the pair terms
    T* sRt = sizeof(T) == 8 ? (T*)(void*)sR : (T*)(void*)sRf;
    T* bas = (T*)(smem + ob);
    T* phi = (T*)(smem + oph);
    T* cold = (T*)(smem + oc);

    T* gA[2] = {(T*)wk.Ainv[0] + (size_t)w * nu * nu, (T*)wk.Ainv[1] + (size_t)w * nd * nd};
    T* gG[2] = {(T*)wk.G[0] + (size_t)w * 4 * nu * nu, (T*)wk.G[1] + (size_t)w * 4 * nd * nd};
    T* Ainv[2];
    T* Gc[2];
    if (p.ainv_smem) {
        Ainv[0] = (T*)(smem + oA);
        Ainv[1] = Ainv[0] + nu * nu;
        for (int q = threadIdx.x; q < nu * nu; q += blockDim.x) Ainv[0][q] = gA[0][q];
        for (int q = threadIdx.x; q < nd * nd; q += blockDim.x) Ainv[1][q] = gA[1][q];
    } else {
        Ainv[0] = gA[0];
        Ainv[1] = gA[1];
    }
    if (p.g_smem) {
        Gc[0] = (T*)(smem + oG);
        Gc[1] = Gc[0] + 4 * nu * nu;
        for (int q = threadIdx.x; q < 4 * nu * nu; q += blockDim.x) Gc[0][q] = gG[0][q];
        for (int q = threadIdx.x; q < 4 * nd * nd; q += blockDim.x) Gc[1][q] = gG[1][q];
    } else {
        Gc[0] = gG[0];
        Gc[1] = gG[1];
    }
    for (int q = threadIdx.x; q < 3 * N; q += blockDim.x) {
        sR[q] = wk.R[(size_t)w * 3 * N + q];
        sRf[q] = (float)sR[q];
        if constexpr (kMixed) sRl[q] = (float)(sR[q] - (double)sRf[q]);
    }
    double ld0 = 0.0, ld1 = 0.0;
    if (threadIdx.x == 0) {
        ld0 = wk.logdet[2 * w];
        ld1 = wk.logdet[2 * w + 1];
    }
    unsigned long long acc = 0;
    __syncthreads();

    const double tau = p.tau;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    T* redT = (T*)red;

    for (int e = 0; e < N; ++e) {
        const int spin = e >= nu;
        const int n = spin ? nd : nu;
        const int k = spin ? e - nu : e;
        T* A = Ainv[spin];
        T* Gs = Gc[spin];
        const T* Ae = A + (size_t)k * n;
        const T* Ge = Gs + (size_t)k * 4 * n;
        const double re0 = sR[3 * e], re1 = sR[3 * e + 1], re2 = sR[3 * e + 2];
        const T et0 = sRt[3 * e], et1 = sRt[3 * e + 1], et2 = sRt[3 * e + 2];

        // -- drift at the current position: grad_e ln|D| + grad_e J --------
        // Each thread keeps its share of sum_q u(r_eq) at the old position for
        // the Jastrow change of phase B (same q loop in both phases).
        T va[8] = {T(0), T(0), T(0), T(0), T(0), T(0), T(0), T(0)};
        T u_old = T(0);
        for (int j = threadIdx.x; j < n; j += blockDim.x) {
            const T a = Ae[j];
            va[0] += Ge[j] * a;
            va[1] += Ge[n + j] * a;
            va[2] += Ge[2 * n + j] * a;
        }
        for (int q = threadIdx.x; q < N + nn; q += blockDim.x) {
            T x, y, z, a, b;
            if (q < N) {
                if (q == e) continue;
                x = et0 - sRt[3 * q]; y = et1 - sRt[3 * q + 1]; z = et2 - sRt[3 * q + 2];
                a = T(((q < nu) == (e < nu)) ? s.a_par : s.a_anti);
                b = T(s.b_ee);
            } else {
                const int c = q - N;
                if constexpr (kMixed) {
                    x = diff_f2(sRf[3 * e], sRl[3 * e], s.Rn_hi[3 * c], s.Rn_lo[3 * c]);
                    y = diff_f2(sRf[3 * e + 1], sRl[3 * e + 1], s.Rn_hi[3 * c + 1], s.Rn_lo[3 * c + 1]);
                    z = diff_f2(sRf[3 * e + 2], sRl[3 * e + 2], s.Rn_hi[3 * c + 2], s.Rn_lo[3 * c + 2]);
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
            const T g = a * qd * qd * ir;   // u'(r) / r
            va[3] += g * x;
            va[4] += g * y;
            va[5] += g * z;
        }
        if constexpr (kJ3) {
            // three-body terms of electron e: every (nucleus, partner) pair
            for (int q = threadIdx.x; q < nn * N; q += blockDim.x) {
                double uv, gg[3];
                j3_of_electron_pair(s, sR, e, re0, re1, re2, q, uv, gg);
                u_old += T(uv);
                va[3] += T(gg[0]);
                va[4] += T(gg[1]);
                va[5] += T(gg[2]);
            }
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
        T rt0, rt1, rt2;
        if constexpr (kMixed) {
            rt0 = fs[0]; rt1 = fs[1]; rt2 = fs[2];
        } else {
            rn[0] = scal[0]; rn[1] = scal[1]; rn[2] = scal[2];
            rt0 = T(rn[0]); rt1 = T(rn[1]); rt2 = T(rn[2]);
        }

        // -- basis (live shells, packed) and orbitals at the proposed position
        const int ldb = basis_live_ld(nb);
        int* brows = (int*)(bas + 5 * ldb);   // packed basis rows (basis_live)
        int nrow;
        if constexpr (kMixed)
            nrow = basis_live<T>(s, nullptr, fs, fs + 3, bas, ldb, brows, brows + ldb);
        else
            nrow = basis_live<T>(s, rn, nullptr, nullptr, bas, ldb, brows, brows + ldb);
        const T* C = sys_C<T>(s, spin);
        contract5<T, kSliced>(C, n, nrow, ldb, brows, bas, phi, nmax);
        __syncthreads();

        // -- ratio, new determinant gradient, Jastrow change ----------------
        T vb2[8] = {T(0), T(0), T(0), T(0), -u_old, T(0), T(0), T(0)};
        for (int j = threadIdx.x; j < n; j += blockDim.x) {
            const T a = Ae[j];
            vb2[0] += phi[j] * a;
            vb2[1] += phi[nmax + j] * a;
            vb2[2] += phi[2 * nmax + j] * a;
            vb2[3] += phi[3 * nmax + j] * a;
        }
        for (int q = threadIdx.x; q < N + nn; q += blockDim.x) {
            T x, y, z, a, b;
            if (q < N) {
                if (q == e) continue;
                x = rt0 - sRt[3 * q]; y = rt1 - sRt[3 * q + 1]; z = rt2 - sRt[3 * q + 2];
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
        if constexpr (kJ3) {
            for (int q = threadIdx.x; q < nn * N; q += blockDim.x) {
                double uv, gg[3];
                j3_of_electron_pair(s, sR, e, scal[0], scal[1], scal[2], q, uv, gg);
                vb2[4] += T(uv);
                vb2[5] += T(gg[0]);
                vb2[6] += T(gg[1]);
                vb2[7] += T(gg[2]);
            }
        }
        block_sum8_to0<T>(vb2, redT);
        if (threadIdx.x == 0) {
            const T gd[3] = {vb2[1], vb2[2], vb2[3]}, gj[3] = {vb2[5], vb2[6], vb2[7]};
            if constexpr (kMixed) {
                const int accept = accept_move_mixed(vb2[0], gd, gj, vb2[4], tau, fs, p.key, p.sweep, (uint32_t)e,
                                                     (uint32_t)w);
                fs[12] = vb2[0];
                ((int*)fs)[13] = accept;
            } else {
                const double ro3[3] = {re0, re1, re2};
                const int accept = accept_move<T>(vb2[0], gd, gj, vb2[4], tau, ro3, rn, scal + 3, p.key, p.sweep,
                                                  (uint32_t)e, (uint32_t)w);
                scal[6] = double(vb2[0]);
                scal[7] = accept ? 1.0 : 0.0;
            }
        }
        __syncthreads();
        const bool accepted = kMixed ? ((const int*)fs)[13] != 0 : scal[7] != 0.0;
        if (accepted) {
            for (int j = threadIdx.x; j < n; j += blockDim.x) cold[j] = A[(size_t)k * n + j];
            __syncthreads();
            const T rinv = kMixed ? T(1) / T(fs[12]) : T(1.0 / scal[6]);
            if (!kMixed && p.ainv_smem && n <= kMaxWarps * 8) {
                // FP64 form, A^-1 in shared memory: each row's dot product on
                // its own thread (n FMAs, no warp reduction: a warp-wide sum
                // costs five FP64 adds per row on every warp), the factors
                // through the block scratch, then the rank-1 update
                double* fq = red;
                for (int q = threadIdx.x; q < n; q += blockDim.x) {
                    const T* Aq = A + (size_t)q * n;
                    T t = T(0);
                    for (int j = 0; j < n; ++j) t += phi[j] * Aq[j];
                    if (q == k) t -= T(1);
                    fq[q] = double(t * rinv);
                }
                __syncthreads();
                for (int o = threadIdx.x; o < n * n; o += blockDim.x) {
                    const int q = o / n, j = o - q * n;
                    A[o] -= T(fq[q]) * cold[j];
                }
            } else {
                for (int q = wid; q < n; q += nw) {
                    T* Aq = A + (size_t)q * n;
                    T t = T(0);
                    for (int j = lane; j < n; j += 32) t += phi[j] * Aq[j];
                    t = warp_sum(t);
                    if (q == k) t -= T(1);
                    const T f = t * rinv;
                    for (int j = lane; j < n; j += 32) Aq[j] -= f * cold[j];
                }
            }
            T* Gk = Gs + (size_t)k * 4 * n;
            for (int o = threadIdx.x; o < 4 * n; o += blockDim.x) {
                const int c = o / n, j = o - c * n;
                Gk[o] = phi[(c + 1) * nmax + j];
            }
            if (threadIdx.x == 0) {
                // the mixed form's ratio is an FP32 number: its log in FP32
                const double lr = kMixed ? (double)logf(fs[12]) : log(scal[6]);
                if (spin)
                    ld1 += lr;
                else
                    ld0 += lr;
                for (int c = 0; c < 3; ++c) {
                    sR[3 * e + c] = scal[c];
                    if constexpr (kMixed) {
                        sRf[3 * e + c] = fs[c];
                        sRl[3 * e + c] = fs[3 + c];
                    } else {
                        sRf[3 * e + c] = (float)scal[c];
                    }
                }
                ++acc;
            }
            __syncthreads();
        }
    }

    __syncthreads();
    for (int q = threadIdx.x; q < 3 * N; q += blockDim.x) wk.R[(size_t)w * 3 * N + q] = sR[q];
    if (p.ainv_smem) {
        for (int q = threadIdx.x; q < nu * nu; q += blockDim.x) gA[0][q] = Ainv[0][q];
        for (int q = threadIdx.x; q < nd * nd; q += blockDim.x) gA[1][q] = Ainv[1][q];
    }
    if (p.g_smem) {
        for (int q = threadIdx.x; q < 4 * nu * nu; q += blockDim.x) gG[0][q] = Gc[0][q];
        for (int q = threadIdx.x; q < 4 * nd * nd; q += blockDim.x) gG[1][q] = Gc[1][q];
    }
    if (threadIdx.x == 0) {
        wk.logdet[2 * w] = ld0;
        wk.logdet[2 * w + 1] = ld1;
        if (acc) atomicAdd(wk.n_acc, acc);
    }
}

}  // namespace qmc
