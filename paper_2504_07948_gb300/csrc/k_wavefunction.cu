// Full (non-incremental) wavefunction evaluation at fixed walker
// configurations: basis -> orbitals for every electron, FP64 inversion of
// the Slater matrices, and the local energy.  These kernels serve the
// parity entry point and the periodic FP64 recompute of the incremental
// inverse.
#include "batch.cuh"
#include "qmc_internal.cuh"

namespace qmc {

// One CTA per (walker, electron).  Basis value/gradient/Laplacian of every
// shell at r_i in FP64 (one thread per shell, the "multi-center" flattening
// of {centres x electrons} onto the grid), then the LCAO contraction
// phi_j = sum_l C_l^j Phi_l (Eq. 2) for the occupied orbitals of the
// electron's spin.  A goes to FP64 scratch, the gradient/Laplacian rows to
// the walker cache in the storage type T.
// Orbitals of electron i of walker w (body of k_orbitals_all).  sh_bas:
// 5 n_basis doubles of shared memory.  live (optional, n_shell bytes of
// shared memory): shells whose values and derivatives are all exactly zero
// (screened) are left out of the occupied-orbital contraction; the terms
// that remain are added in the same order, so the result is unchanged.
template <typename T>
__device__ __forceinline__ void orbitals_item(const DevSys& s, const DevWalkers& wk, int w, int i, double* sh_bas,
                                              unsigned char* live = nullptr) {
    const int nb = s.n_basis;
    double r[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) r[c] = wk.R[((size_t)w * s.N + i) * 3 + c];
    for (int sh = threadIdx.x; sh < s.n_shell; sh += blockDim.x) shell_vgl<double>(s, sh, r, sh_bas, nb);
    __syncthreads();
    if (live) {
        for (int sh = threadIdx.x; sh < s.n_shell; sh += blockDim.x) {
            const int f0 = s.shell_fn[sh], f1 = s.shell_fn[sh + 1];
            bool nz = false;
            for (int c = 0; c < 5 && !nz; ++c)
                for (int f = f0; f < f1 && !nz; ++f) nz = sh_bas[c * nb + f] != 0.0;
            live[sh] = nz ? 1 : 0;
        }
        __syncthreads();
    }
    const int spin = i < s.n_up ? 0 : 1;
    const int n = spin ? s.n_dn : s.n_up;
    const int k = spin ? i - s.n_up : i;
    const double* C = s.C[spin];
    T* G = (T*)wk.G[spin] + ((size_t)w * n + k) * 4 * n;
    double* A = wk.Ascr[spin] + ((size_t)w * n + k) * n;
    for (int o = threadIdx.x; o < 5 * n; o += blockDim.x) {
        const int c = o / n, j = o - c * n;
        const double* b = sh_bas + c * nb;
        double acc = 0.0;
        if (live) {
            for (int sh = 0; sh < s.n_shell; ++sh) {
                if (!live[sh]) continue;
                for (int l = s.shell_fn[sh]; l < s.shell_fn[sh + 1]; ++l) acc += C[(size_t)l * n + j] * b[l];
            }
        } else {
            for (int l = 0; l < nb; ++l) acc += C[(size_t)l * n + j] * b[l];
        }
        if (c == 0)
            A[j] = acc;
        else
            G[(c - 1) * n + j] = (T)acc;
    }
    if (s.msd) {  // active virtual orbitals of a determinant expansion
        const int nv = s.n_vir[spin];
        const double* Cv = s.Cv[spin];
        T* Av = (T*)wk.Av[spin] + ((size_t)w * n + k) * nv;
        T* Gv = (T*)wk.Gv[spin] + ((size_t)w * n + k) * 4 * nv;
        for (int o = threadIdx.x; o < 5 * nv; o += blockDim.x) {
            const int c = o / nv, p = o - c * nv;
            const double* b = sh_bas + c * nb;
            double acc = 0.0;
            for (int l = 0; l < nb; ++l) acc += Cv[(size_t)l * nv + p] * b[l];
            if (c == 0)
                Av[p] = (T)acc;
            else
                Gv[(c - 1) * nv + p] = (T)acc;
        }
    }
}

template <typename T>
__global__ void k_orbitals_all(DevSys s, DevWalkers wk, int W, const int* only) {
    extern __shared__ double sh_bas[];  // [5][n_basis], then one live flag per shell
    const int w = blockIdx.x, i = blockIdx.y;
    if (w >= W || (only && !only[w])) return;
    orbitals_item<T>(s, wk, w, i, sh_bas, reinterpret_cast<unsigned char*>(sh_bas + 5 * s.n_basis));
}

// In-place Gauss-Jordan inversion with partial (row) pivoting, FP64, one
// CTA per (walker, spin), the n x n matrix in shared memory.  Produces
// ln|det A|, sign(det A) and the transposed inverse in the storage type.
// Inversion of one (walker, spin) matrix (body of k_invert).  M: n^2 + n
// doubles of shared memory.
__device__ __forceinline__ void invert_item(const DevSys& s, const DevWalkers& wk, int w, int spin, int store_fp32, unsigned* err, double* M) {
    __shared__ int s_piv;
    __shared__ int s_ipiv[256];
    __shared__ double s_ld, s_sg;
    __shared__ int s_sing;
    const int n = spin ? s.n_dn : s.n_up;
    if (n == 0) {
        if (threadIdx.x == 0) {
            wk.logdet[2 * w + spin] = 0.0;
            wk.sgn[2 * w + spin] = 1.0;
        }
        return;
    }
    double* fcol = M + n * n;
    const double* A = wk.Ascr[spin] + (size_t)w * n * n;
    for (int q = threadIdx.x; q < n * n; q += blockDim.x) M[q] = A[q];
    if (threadIdx.x == 0) {
        s_ld = 0.0;
        s_sg = 1.0;
        s_sing = 0;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int k = 0; k < n; ++k) {
        if (wid == 0) {
            double best = -1.0;
            int bi = k;
            for (int i = k + lane; i < n; i += 32) {
                const double v = fabs(M[i * n + k]);
                if (v > best) {
                    best = v;
                    bi = i;
                }
            }
            for (int o = 16; o > 0; o >>= 1) {
                const double ob = __shfl_xor_sync(0xffffffffu, best, o);
                const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                if (ob > best || (ob == best && oi < bi)) {
                    best = ob;
                    bi = oi;
                }
            }
            if (lane == 0) s_piv = bi;
        }
        __syncthreads();
        const int p = s_piv;
        if (p != k)
            for (int j = threadIdx.x; j < n; j += blockDim.x) {
                const double t = M[k * n + j];
                M[k * n + j] = M[p * n + j];
                M[p * n + j] = t;
            }
        __syncthreads();
        const double piv = M[k * n + k];
        if (piv == 0.0 || !isfinite(piv)) {
            if (threadIdx.x == 0) s_sing = 1;
            break;  // uniform: every thread read the same pivot
        }
        if (threadIdx.x == 0) {
            s_ipiv[k] = p;
            s_ld += log(fabs(piv));
            s_sg *= (piv < 0.0 ? -1.0 : 1.0) * (p != k ? -1.0 : 1.0);
        }
        const double pinv = 1.0 / piv;
        __syncthreads();
        for (int j = threadIdx.x; j < n; j += blockDim.x) {
            fcol[j] = (j == k) ? 0.0 : M[j * n + k];
            M[k * n + j] = (j == k) ? pinv : M[k * n + j] * pinv;
        }
        __syncthreads();
        for (int q = threadIdx.x; q < n * n; q += blockDim.x) {
            const int i = q / n, j = q - i * n;
            if (i == k) continue;
            const double base = (j == k) ? 0.0 : M[q];
            M[q] = base - fcol[i] * M[k * n + j];
        }
        __syncthreads();
    }
    __syncthreads();
    if (s_sing) {
        if (threadIdx.x == 0) {
            wk.logdet[2 * w + spin] = -INFINITY;
            wk.sgn[2 * w + spin] = 0.0;
            atomicOr(err, kErrSingular);
        }
        return;
    }
    // undo the row interchanges as column interchanges, last first
    for (int k = n - 1; k >= 0; --k) {
        const int p = s_ipiv[k];
        if (p != k)
            for (int i = threadIdx.x; i < n; i += blockDim.x) {
                const double t = M[i * n + k];
                M[i * n + k] = M[i * n + p];
                M[i * n + p] = t;
            }
        __syncthreads();
    }
    // AinvT[e][j] = (A^-1)[j][e]
    if (store_fp32) {
        float* out = (float*)wk.Ainv[spin] + (size_t)w * n * n;
        for (int q = threadIdx.x; q < n * n; q += blockDim.x) {
            const int e = q / n, j = q - e * n;
            out[q] = (float)M[j * n + e];
        }
    } else {
        double* out = (double*)wk.Ainv[spin] + (size_t)w * n * n;
        for (int q = threadIdx.x; q < n * n; q += blockDim.x) {
            const int e = q / n, j = q - e * n;
            out[q] = M[j * n + e];
        }
    }
    if (threadIdx.x == 0) {
        wk.logdet[2 * w + spin] = s_ld;
        wk.sgn[2 * w + spin] = s_sg;
    }
}

__global__ void k_invert(DevSys s, DevWalkers wk, int W, int store_fp32, unsigned* err, const int* only) {
    extern __shared__ double M[];  // [n][n], then fcol[n]
    const int w = blockIdx.x, spin = blockIdx.y;
    if (w >= W || (only && !only[w])) return;
    invert_item(s, wk, w, spin, store_fp32, err, M);
}

// Local energy, ln|psi| and (optionally) grad / Laplacian of ln|psi| from
// the cached inverse and orbital gradient/Laplacian rows.  One CTA per
// walker, one thread per electron; sums in FP64.
//   E_L = sum_i -1/2 [lap_i D/D + lap_i J + 2 grad_i J . grad_i D/D
//         + |grad_i J|^2] + V_ee + V_en + V_nn.
// Local energy of walker w (body of k_eloc).  sR: 3 N doubles of shared
// memory.
// J3 seen from electron i: the value of the pairs (i, j > i) and the
// gradient and Laplacian in r_i of every pair (i, j != i).
__device__ void j3_electron(const DevSys& s, const double* sR, int i, double& val, double g[3], double& lap) {
    val = 0.0;
    g[0] = g[1] = g[2] = 0.0;
    lap = 0.0;
    const double* ri = sR + 3 * i;
    for (int a = 0; a < s.n_nuc; ++a) {
        const double* ra = s.Rn + 3 * a;
        const SDist xi = sdist(s.b3, ri[0] - ra[0], ri[1] - ra[1], ri[2] - ra[2]);
        const double* c = s.c3 + (size_t)a * s.n3;
        for (int j = 0; j < s.N; ++j) {
            if (j == i) continue;
            const double* rj = sR + 3 * j;
            const SDist xj = sdist(s.b3, rj[0] - ra[0], rj[1] - ra[1], rj[2] - ra[2]);
            const SDist y = sdist(s.b3, ri[0] - rj[0], ri[1] - rj[1], ri[2] - rj[2]);
            for (int k = 0; k < s.n3; ++k) {
                if (c[k] == 0.0) continue;
                double v, gg[3], l;
                j3_term(s.e3[3 * k], s.e3[3 * k + 1], s.e3[3 * k + 2], xi, xj, y, v, gg, l);
                if (j > i) val += c[k] * v;
                g[0] += c[k] * gg[0];
                g[1] += c[k] * gg[1];
                g[2] += c[k] * gg[2];
                lap += c[k] * l;
            }
        }
    }
}

template <typename T>
__device__ __forceinline__ void eloc_walker(const DevSys& s, const DevWalkers& wk, int w, double* eloc_out, double* logpsi, double* grad,
                                            double* lap, unsigned* err, double* sR) {
    __shared__ double scratch[kMaxWarps * 2];
    const int N = s.N, nu = s.n_up;
    float* sRf = (float*)(sR + 3 * N);   // float copy for the pair terms of the mixed form
    for (int q = threadIdx.x; q < 3 * N; q += blockDim.x) {
        sR[q] = wk.R[(size_t)w * 3 * N + q];
        sRf[q] = (float)sR[q];
    }
    __syncthreads();
    double v[2] = {0.0, 0.0};
    if constexpr (sizeof(T) == 4) {
        // Mixed form: pair terms and dot products in FP32 with compensated
        // per-electron sums, assembled in FP64.
        for (int i = threadIdx.x; i < N; i += blockDim.x) {
            const int spin = i >= nu;
            const int n = spin ? s.n_dn : nu;
            const int k = spin ? i - nu : i;
            const float* Ai = (const float*)wk.Ainv[spin] + ((size_t)w * n + k) * n;
            const float* Gi = (const float*)wk.G[spin] + ((size_t)w * n + k) * 4 * n;
            Acc<float> dd[4];
            for (int j = 0; j < n; ++j) {
                const float a = Ai[j];
                dd[0].add(Gi[j] * a);
                dd[1].add(Gi[n + j] * a);
                dd[2].add(Gi[2 * n + j] * a);
                dd[3].add(Gi[3 * n + j] * a);
            }
            const float xi = sRf[3 * i], yi = sRf[3 * i + 1], zi = sRf[3 * i + 2];
            const float bee = (float)s.b_ee, ben = (float)s.b_en;
            float gx = 0.f, gy = 0.f, gz = 0.f;
            Acc<float> lJ, Ji, V;
            for (int j = 0; j < N; ++j) {
                if (j == i) continue;
                const float x = xi - sRf[3 * j], y = yi - sRf[3 * j + 1], z = zi - sRf[3 * j + 2];
                const float r2 = x * x + y * y + z * z;
                const float ir = rsqrtf(r2), r = r2 * ir;
                const float a = (float)(((i < nu) == (j < nu)) ? s.a_par : s.a_anti);
                const float q = 1.0f / (1.0f + bee * r);
                const float du = a * q * q, g = du * ir;
                gx += g * x;
                gy += g * y;
                gz += g * z;
                lJ.add(-2.0f * bee * du * q + 2.0f * g);
                if (j > i) {
                    Ji.add(a * r * q);
                    V.add(ir);
                }
            }
            for (int a = 0; a < s.n_nuc; ++a) {
                const float x = (float)(sR[3 * i] - s.Rn[3 * a]), y = (float)(sR[3 * i + 1] - s.Rn[3 * a + 1]),
                            z = (float)(sR[3 * i + 2] - s.Rn[3 * a + 2]);
                const float r2 = x * x + y * y + z * z;
                const float ir = rsqrtf(r2), r = r2 * ir;
                const float ae = (float)s.a_en[a];
                const float q = 1.0f / (1.0f + ben * r);
                const float du = ae * q * q, g = du * ir;
                gx += g * x;
                gy += g * y;
                gz += g * z;
                lJ.add(-2.0f * ben * du * q + 2.0f * g);
                Ji.add(ae * r * q);
                V.add(-(float)s.Z[a] * ir);
                if (s.npp) V.add(pp_local<float>(s, a, r));
            }
            const double d0 = (double)dd[0].h + dd[0].l, d1 = (double)dd[1].h + dd[1].l;
            const double d2 = (double)dd[2].h + dd[2].l, dl = (double)dd[3].h + dd[3].l;
            double lj = (double)lJ.h + lJ.l;
            if (s.n3 > 0) {
                double v3, g3[3], l3;
                j3_electron(s, sR, i, v3, g3, l3);
                gx = (float)((double)gx + g3[0]);
                gy = (float)((double)gy + g3[1]);
                gz = (float)((double)gz + g3[2]);
                lj += l3;
                v[1] += v3;
            }
            const double Ti = -0.5 * (dl + lj + 2.0 * (gx * d0 + gy * d1 + gz * d2) + (double)gx * gx +
                                      (double)gy * gy + (double)gz * gz);
            v[0] += Ti + ((double)V.h + V.l);
            v[1] += (double)Ji.h + Ji.l;
            if (grad) {
                double* g = grad + ((size_t)w * N + i) * 3;
                g[0] = gx + d0;
                g[1] = gy + d1;
                g[2] = gz + d2;
            }
            if (lap) lap[(size_t)w * N + i] = lj + dl - (d0 * d0 + d1 * d1 + d2 * d2);
        }
    } else
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        const int spin = i >= nu;
        const int n = spin ? s.n_dn : nu;
        const int k = spin ? i - nu : i;
        const T* Ai = (const T*)wk.Ainv[spin] + ((size_t)w * n + k) * n;
        const T* Gi = (const T*)wk.G[spin] + ((size_t)w * n + k) * 4 * n;
        double d0 = 0, d1 = 0, d2 = 0, dl = 0;
        for (int j = 0; j < n; ++j) {
            const double a = (double)Ai[j];
            d0 += (double)Gi[j] * a;
            d1 += (double)Gi[n + j] * a;
            d2 += (double)Gi[2 * n + j] * a;
            dl += (double)Gi[3 * n + j] * a;
        }
        const double xi = sR[3 * i], yi = sR[3 * i + 1], zi = sR[3 * i + 2];
        double gx = 0, gy = 0, gz = 0, lJ = 0, Ji = 0, V = 0;
        // pair terms with one reciprocal square root and one division each:
        // u = a r q, u' = a q^2, u'' = -2 a b q^3 with q = 1 / (1 + b r)
        for (int j = 0; j < N; ++j) {
            if (j == i) continue;
            const double x = xi - sR[3 * j], y = yi - sR[3 * j + 1], z = zi - sR[3 * j + 2];
            const double r2 = x * x + y * y + z * z;
            const double ir = rsqrt(r2), r = r2 * ir;
            const double a = ((i < nu) == (j < nu)) ? s.a_par : s.a_anti;
            const double q = 1.0 / (1.0 + s.b_ee * r);
            const double du = a * q * q, g = du * ir;
            gx += g * x;
            gy += g * y;
            gz += g * z;
            lJ += -2.0 * s.b_ee * du * q + 2.0 * g;
            if (j > i) {
                Ji += a * r * q;
                V += ir;
            }
        }
        for (int a = 0; a < s.n_nuc; ++a) {
            const double x = xi - s.Rn[3 * a], y = yi - s.Rn[3 * a + 1], z = zi - s.Rn[3 * a + 2];
            const double r2 = x * x + y * y + z * z;
            const double ir = rsqrt(r2), r = r2 * ir;
            const double q = 1.0 / (1.0 + s.b_en * r);
            const double du = s.a_en[a] * q * q, g = du * ir;
            gx += g * x;
            gy += g * y;
            gz += g * z;
            lJ += -2.0 * s.b_en * du * q + 2.0 * g;
            Ji += s.a_en[a] * r * q;
            V -= s.Z[a] * ir;
            if (s.npp) V += pp_local<double>(s, a, r);
        }
        if (s.n3 > 0) {
            double v3, g3[3], l3;
            j3_electron(s, sR, i, v3, g3, l3);
            gx += g3[0];
            gy += g3[1];
            gz += g3[2];
            lJ += l3;
            Ji += v3;
        }
        const double Ti = -0.5 * (dl + lJ + 2.0 * (gx * d0 + gy * d1 + gz * d2) + gx * gx + gy * gy + gz * gz);
        v[0] += Ti + V;
        v[1] += Ji;
        if (grad) {
            double* g = grad + ((size_t)w * N + i) * 3;
            g[0] = gx + d0;
            g[1] = gy + d1;
            g[2] = gz + d2;
        }
        if (lap) lap[(size_t)w * N + i] = lJ + dl - (d0 * d0 + d1 * d1 + d2 * d2);
    }
    block_sum<2>(v, scratch);
    if (threadIdx.x == 0) {
        const double el = v[0] + s.vnn;
        eloc_out[w] = el;
        if (logpsi) logpsi[w] = v[1] + wk.logdet[2 * w] + wk.logdet[2 * w + 1];
        if (!isfinite(el) && err) atomicOr(err, kErrNonFinite);
    }
}

template <typename T>
__global__ void k_eloc(DevSys s, DevWalkers wk, int W, double* eloc_out, double* logpsi,
                       double* grad, double* lap, unsigned* err) {
    extern __shared__ double sR[];  // [N][3]
    const int w = blockIdx.x;
    if (w >= W) return;
    eloc_walker<T>(s, wk, w, eloc_out, logpsi, grad, lap, err, sR);
}

// Jastrow parameter derivatives of walker w (one CTA): d ln|psi| / dp is
// the derivative of J alone, B_p = dJ/dp, and dE_L / dp = -1/2 sum_i
// (lap_i B_p + 2 grad_i ln|psi| . grad_i B_p) (the determinant and the
// potential do not depend on the Jastrow).  Linear parameters give B_p as
// their own term with unit coefficient; for b of u = a r / (1 + b r),
// dB/db = -a r^2 / (1 + b r)^2 with radial derivatives -2 a r / (1 + b r)^3
// and -2 a (1 - 2 b r) / (1 + b r)^4.
__global__ void k_jastrow_derivs(DevSys s, const double* __restrict__ R, const double* __restrict__ G, int W,
                                 double* dlog, double* deloc) {
    extern __shared__ double jsm[];   // positions [3N], gradients [3N], per-nucleus b_en parts [2 n_nuc]
    __shared__ double scratch[kMaxWarps * 8];
    const int w = blockIdx.x;
    if (w >= W) return;
    const int N = s.N, nu = s.n_up, nn = s.n_nuc, P = 4 + nn + nn * s.n3;
    double* sR = jsm;
    double* sG = sR + 3 * N;
    double* bpart = sG + 3 * N;
    for (int q = threadIdx.x; q < 3 * N; q += blockDim.x) {
        sR[q] = R[(size_t)w * 3 * N + q];
        sG[q] = G[(size_t)w * 3 * N + q];
    }
    __syncthreads();
    double* out_l = dlog + (size_t)w * P;
    double* out_e = deloc + (size_t)w * P;
    // electron pairs: a_anti, a_par, b_ee
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int i = wid; i < N; i += nw)
        for (int j = i + 1 + lane; j < N; j += 32) {
            double x[3], r2 = 0.0;
            for (int c = 0; c < 3; ++c) {
                x[c] = sR[3 * i + c] - sR[3 * j + c];
                r2 += x[c] * x[c];
            }
            const double ir = rsqrt(r2), r = r2 * ir;
            const bool like = (i < nu) == (j < nu);
            const double a = like ? s.a_par : s.a_anti, b = s.b_ee;
            const double q = 1.0 / (1.0 + b * r);
            double gdot = 0.0;   // (G_i - G_j) . u
            for (int c = 0; c < 3; ++c) gdot += (sG[3 * i + c] - sG[3 * j + c]) * x[c] * ir;
            // linear: B = r q, B' = q^2, B'' = -2 b q^3
            const double B = r * q, B1 = q * q, B2 = -2.0 * b * q * q * q;
            const double dEa = -0.5 * (2.0 * (B2 + 2.0 * B1 * ir) + 2.0 * B1 * gdot);
            acc[like ? 2 : 0] += B;
            acc[like ? 3 : 1] += dEa;
            // b_ee
            const double g = -a * r * r * q * q, g1 = -2.0 * a * r * q * q * q, g2 = -2.0 * a * (1.0 - 2.0 * b * r) * q * q * q * q;
            acc[4] += g;
            acc[5] += -0.5 * (2.0 * (g2 + 2.0 * g1 * ir) + 2.0 * g1 * gdot);
        }
    // electron-nucleus: a_en[a] (direct), b_en (per nucleus, summed below)
    for (int a = threadIdx.x; a < nn; a += blockDim.x) {
        double Bl = 0.0, Be = 0.0, bl = 0.0, be = 0.0;
        const double ae = s.a_en[a], b = s.b_en;
        for (int i = 0; i < N; ++i) {
            double x[3], r2 = 0.0;
            for (int c = 0; c < 3; ++c) {
                x[c] = sR[3 * i + c] - s.Rn[3 * a + c];
                r2 += x[c] * x[c];
            }
            const double ir = rsqrt(r2), r = r2 * ir;
            const double q = 1.0 / (1.0 + b * r);
            double gdot = 0.0;
            for (int c = 0; c < 3; ++c) gdot += sG[3 * i + c] * x[c] * ir;
            const double B = r * q, B1 = q * q, B2 = -2.0 * b * q * q * q;
            Bl += B;
            Be += -0.5 * ((B2 + 2.0 * B1 * ir) + 2.0 * B1 * gdot);
            const double g = -ae * r * r * q * q, g1 = -2.0 * ae * r * q * q * q,
                         g2 = -2.0 * ae * (1.0 - 2.0 * b * r) * q * q * q * q;
            bl += g;
            be += -0.5 * ((g2 + 2.0 * g1 * ir) + 2.0 * g1 * gdot);
        }
        out_l[4 + a] = Bl;
        out_e[4 + a] = Be;
        bpart[2 * a] = bl;
        bpart[2 * a + 1] = be;
    }
    // three-body terms: one thread per (nucleus, term), pairs in a fixed order
    for (int pk = threadIdx.x; pk < nn * s.n3; pk += blockDim.x) {
        const int a = pk / s.n3, k = pk - a * s.n3;
        const int m = s.e3[3 * k], n = s.e3[3 * k + 1], o = s.e3[3 * k + 2];
        const double* ra = s.Rn + 3 * a;
        double Bv = 0.0, Bt = 0.0;
        for (int i = 0; i < N; ++i) {
            const double* ri = sR + 3 * i;
            const SDist xi = sdist(s.b3, ri[0] - ra[0], ri[1] - ra[1], ri[2] - ra[2]);
            for (int j = 0; j < N; ++j) {
                if (j == i) continue;
                const double* rj = sR + 3 * j;
                const SDist xj = sdist(s.b3, rj[0] - ra[0], rj[1] - ra[1], rj[2] - ra[2]);
                const SDist y = sdist(s.b3, ri[0] - rj[0], ri[1] - rj[1], ri[2] - rj[2]);
                double v, g[3], l;
                j3_term(m, n, o, xi, xj, y, v, g, l);
                if (j > i) Bv += v;
                Bt += l + 2.0 * (sG[3 * i] * g[0] + sG[3 * i + 1] * g[1] + sG[3 * i + 2] * g[2]);
            }
        }
        out_l[4 + nn + pk] = Bv;
        out_e[4 + nn + pk] = -0.5 * Bt;
    }
    block_sum<6>(*reinterpret_cast<double(*)[6]>(acc), scratch);
    if (threadIdx.x == 0) {
        double bl = 0.0, be = 0.0;
        for (int a = 0; a < nn; ++a) {
            bl += bpart[2 * a];
            be += bpart[2 * a + 1];
        }
        out_l[0] = acc[0];
        out_e[0] = acc[1];
        out_l[1] = acc[2];
        out_e[1] = acc[3];
        out_l[2] = acc[4];
        out_e[2] = acc[5];
        out_l[3] = bl;
        out_e[3] = be;
    }
}

cudaError_t launch_jastrow_derivs(const DevSys& s, const double* R, const double* G, int W, double* dlog,
                                  double* deloc, cudaStream_t st) {
    if (W == 0) return cudaSuccess;
    const size_t smem = sizeof(double) * (6 * (size_t)s.N + 2 * (size_t)s.n_nuc);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_jastrow_derivs, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    k_jastrow_derivs<<<W, 256, smem, st>>>(s, R, G, W, dlog, deloc);
    return cudaGetLastError();
}

// out[k] (+)= sum_w g[w] x[w][k]  (g == nullptr: plain sum).  One CTA per
// k, threads over walkers, deterministic order.
__global__ void k_weighted_sum(const double* x, const double* g, int W, int K, double* out, int accumulate) {
    __shared__ double scratch[kMaxWarps];
    const int k = blockIdx.x;
    double v[1] = {0.0};
    for (int w = threadIdx.x; w < W; w += blockDim.x) v[0] += (g ? g[w] : 1.0) * x[(size_t)w * K + k];
    block_sum<1>(v, scratch);
    if (threadIdx.x == 0) out[k] = (accumulate ? out[k] : 0.0) + v[0];
}

template <typename T>
cudaError_t launch_orbitals_all(const DevSys& s, const DevWalkers& wk, int W, cudaStream_t st, const int* only) {
    if (W == 0 || s.N == 0) return cudaSuccess;
    const size_t smem = sizeof(double) * 5 * s.n_basis + (size_t)s.n_shell;
    const int nt = s.n_up > 32 ? 256 : 128;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_orbitals_all<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
    }
    k_orbitals_all<T><<<dim3(W, s.N), nt, smem, st>>>(s, wk, W, only);
    return cudaGetLastError();
}

cudaError_t launch_invert(const DevSys& s, const DevWalkers& wk, int W, int store_fp32, unsigned* err,
                          cudaStream_t st, const int* only) {
    if (W == 0) return cudaSuccess;
    const int nmax = s.n_up > s.n_dn ? s.n_up : s.n_dn;
    const size_t smem = sizeof(double) * ((size_t)nmax * nmax + nmax + 1);
    cudaError_t e = cudaFuncSetAttribute(k_invert, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int nt = nmax > 64 ? 512 : (nmax > 16 ? 256 : 64);
    k_invert<<<dim3(W, 2), nt, smem, st>>>(s, wk, W, store_fp32, err, only);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_eloc(const DevSys& s, const DevWalkers& wk, int W, double* eloc_out, double* logpsi,
                        double* grad, double* lap, unsigned* err, cudaStream_t st) {
    if (W == 0) return cudaSuccess;
    const size_t smem = (sizeof(double) + sizeof(float)) * 3 * s.N;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_eloc<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    const int nt = s.N > 128 ? 256 : (s.N > 32 ? 128 : 32);
    k_eloc<T><<<W, nt, smem, st>>>(s, wk, W, eloc_out, logpsi, grad, lap, err);
    return cudaGetLastError();
}

cudaError_t launch_weighted_sum(const double* x, const double* g, int W, int K, double* out, int accumulate,
                                cudaStream_t st) {
    if (K == 0) return cudaSuccess;
    k_weighted_sum<<<K, 256, 0, st>>>(x, g, W, K, out, accumulate);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------
// Batched forms: persistent CTAs over the items of every system.
// ---------------------------------------------------------------------
template <typename T>
__global__ void k_orbitals_batch(const BatchSys* __restrict__ sys, BatchPlan* plan, int parity, int ctr) {
    extern __shared__ double sh_bas[];
    __shared__ BatchSys bs;
    __shared__ int s_sys, s_idx;
    for (;;) {
        if (threadIdx.x == 0) batch_next(plan, kUnitElectron, ctr, &s_sys, &s_idx);
        __syncthreads();
        const int q = s_sys;
        if (q < 0) break;
        batch_load(&bs, sys + q);
        __syncthreads();
        const int N = bs.s.N;
        orbitals_item<T>(bs.s, bs.wk[parity], s_idx / N, s_idx % N, sh_bas);
        __syncthreads();
    }
}

__global__ void k_invert_batch(const BatchSys* __restrict__ sys, BatchPlan* plan, int parity, int store_fp32,
                               int ctr) {
    extern __shared__ double M[];
    __shared__ BatchSys bs;
    __shared__ int s_sys, s_idx;
    for (;;) {
        if (threadIdx.x == 0) batch_next(plan, kUnitSpin, ctr, &s_sys, &s_idx);
        __syncthreads();
        const int q = s_sys;
        if (q < 0) break;
        batch_load(&bs, sys + q);
        __syncthreads();
        invert_item(bs.s, bs.wk[parity], s_idx >> 1, s_idx & 1, store_fp32, bs.err, M);
        __syncthreads();
    }
}

template <typename T>
__global__ void k_eloc_batch(const BatchSys* __restrict__ sys, BatchPlan* plan, int parity, int into_walker, int ctr) {
    extern __shared__ double sR[];
    __shared__ BatchSys bs;
    __shared__ int s_sys, s_idx;
    for (;;) {
        if (threadIdx.x == 0) batch_next(plan, kUnitWalker, ctr, &s_sys, &s_idx);
        __syncthreads();
        const int q = s_sys;
        if (q < 0) break;
        batch_load(&bs, sys + q);
        __syncthreads();
        eloc_walker<T>(bs.s, bs.wk[parity], s_idx, into_walker ? bs.wk[parity].eloc : bs.eloc_new, nullptr, nullptr,
                       nullptr, bs.err, sR);
        __syncthreads();
    }
}

template <typename T>
cudaError_t launch_orbitals_batch(const BatchSys* sys, BatchPlan* plan, int parity, int ctr, int grid, size_t smem,
                                  cudaStream_t st) {
    k_orbitals_batch<T><<<grid, 128, smem, st>>>(sys, plan, parity, ctr);
    return cudaGetLastError();
}

cudaError_t launch_invert_batch(const BatchSys* sys, BatchPlan* plan, int parity, int store_fp32, int ctr, int grid,
                                size_t smem, cudaStream_t st) {
    k_invert_batch<<<grid, 256, smem, st>>>(sys, plan, parity, store_fp32, ctr);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_eloc_batch(const BatchSys* sys, BatchPlan* plan, int parity, int into_walker, int ctr, int grid,
                              size_t smem, cudaStream_t st) {
    k_eloc_batch<T><<<grid, 128, smem, st>>>(sys, plan, parity, into_walker, ctr);
    return cudaGetLastError();
}

// Sets the dynamic shared memory limit of a batched family (0 orbitals,
// 1 inversion, 2 local energy; 3 and 4: the FP32-storage forms of 0 and 2)
// before any launch or graph capture; returns its resident CTAs per SM.
int wf_batch_prepare(int family, int block, size_t smem) {
    int nb = 0;
    const void* f = nullptr;
    switch (family) {
        case 0: f = (const void*)k_orbitals_batch<double>; break;
        case 1: f = (const void*)k_invert_batch; break;
        case 2: f = (const void*)k_eloc_batch<double>; break;
        case 3: f = (const void*)k_orbitals_batch<float>; break;
        case 4: f = (const void*)k_eloc_batch<float>; break;
        default: return 0;
    }
    if (cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, f, block, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return nb;
}

template cudaError_t launch_orbitals_batch<double>(const BatchSys*, BatchPlan*, int, int, int, size_t, cudaStream_t);
template cudaError_t launch_orbitals_batch<float>(const BatchSys*, BatchPlan*, int, int, int, size_t, cudaStream_t);
template cudaError_t launch_eloc_batch<double>(const BatchSys*, BatchPlan*, int, int, int, int, size_t,
                                               cudaStream_t);
template cudaError_t launch_eloc_batch<float>(const BatchSys*, BatchPlan*, int, int, int, int, size_t, cudaStream_t);

template cudaError_t launch_orbitals_all<double>(const DevSys&, const DevWalkers&, int, cudaStream_t, const int*);
template cudaError_t launch_orbitals_all<float>(const DevSys&, const DevWalkers&, int, cudaStream_t, const int*);
template cudaError_t launch_eloc<double>(const DevSys&, const DevWalkers&, int, double*, double*, double*,
                                         double*, unsigned*, cudaStream_t);
template cudaError_t launch_eloc<float>(const DevSys&, const DevWalkers&, int, double*, double*, double*,
                                        double*, unsigned*, cudaStream_t);

}  // namespace qmc
