// Ionic derivatives of E_L and ln|psi| for a multi-determinant wavefunction
// (Sec. "Multideterminant QMC Forces": derivatives of ratios of sums of
// determinants, with the single-determinant quantities reused).
//
// Per spin, with X = A0^-1, the table T = X A_v, the kinetic operator B
// (= -1/2 lap phi - grad J . grad phi, occupied block B0, virtual block Bv),
// Theta = X (Bv - B0 T), and per string u: M = T[H,P], N = Theta[H,P],
// R_u = ph det M, D_u = ph d/de det(M + e N) at e = 0,
//   ln psi_D = ln D0_up + ln D0_dn + ln S,      S  = sum_k c_k R_up R_dn,
//   E_L      = E_L(reference) + Sd / S,        Sd = sum_k c_k (D_up R_dn + R_up D_dn).
// Their changes under a nuclear displacement are linear in the changes of
// A0, A_v, B0, Bv (every change of T and Theta is), so one adjoint pass per
// walker collects the weights of those four matrices:
//   d ln S   = sum Ybar dT,                Ybar[h_a][p_c] += (Cd_u / S) ph cof(M)_ac
//   d(Sd/S)  = sum Yt dT + sum Ytheta dTheta,
//              Yt[h_a][p_c]     += alpha_u dD_u/dM_ac + beta_u ph cof(M)_ac
//              Ytheta[h_a][p_c] += alpha_u ph cof(M)_ac
//   alpha_u = Cd_u / S, beta_u = (CdD_u - (Sd/S) Cd_u) / S, CdD_u = sum over
//   the string's determinants of c_k D_other.  With dT = X (dA_v - dA0 T) and
//   dTheta = -X dA0 Theta + X (dBv - dB0 T) - X B0 dT the weights become
//   coefficient matrices on the occupied and virtual orbital blocks, which
//   are pulled back to basis space and contracted with the third-order basis
//   derivatives exactly as for one determinant (k_force.cu), plus a change of
//   the Jastrow-gradient weight (B depends on grad J).
#include "msd_small.cuh"
#include "qmc_internal.cuh"

namespace qmc {

constexpr int kFmTile = 32;

// First derivatives, derivatives of the Laplacian and the Hessian applied
// to g of one function of a shell (the same decomposition as the
// single-determinant force kernel: Phi = P S; the Hessian itself is never
// formed).
template <typename F>
struct D3 {
    F d1[3], hg[3], dl[3];
};

__device__ __forceinline__ int hix(int a, int b) {
    const int lo = a < b ? a : b, hi = a < b ? b : a;
    return lo == 0 ? hi : (lo == 1 ? 2 + hi : 5);
}

template <typename F>
__device__ __forceinline__ void shell_d3m(int l, int pure, const F x[3], const F g[3], int fi, F f0, F f1, F f2,
                                          F f3, D3<F>& out) {
    const F t = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
    const AngPoly<F> a = angular<F>(l, pure, fi, x[0], x[1], x[2]);
    const F Pk[3] = {a.Px, a.Py, a.Pz};
    const F HP[6] = {a.Hxx, a.Hxy, a.Hxz, a.Hyy, a.Hyz, a.Hzz};
    const F LP = a.Hxx + a.Hyy + a.Hzz;
    F Sk[3];
    for (int k = 0; k < 3; ++k) Sk[k] = F(2) * x[k] * f1;
    const F LS = F(6) * f1 + F(4) * t * f2;
    const F Px = Pk[0] * x[0] + Pk[1] * x[1] + Pk[2] * x[2];
    const F Pg = Pk[0] * g[0] + Pk[1] * g[1] + Pk[2] * g[2];
    const F xg = x[0] * g[0] + x[1] * g[1] + x[2] * g[2];
    const F c3 = F(20) * f2 + F(8) * t * f3;
    for (int q = 0; q < 3; ++q) {
        const F HSk = HP[hix(0, q)] * Sk[0] + HP[hix(1, q)] * Sk[1] + HP[hix(2, q)] * Sk[2];
        const F Hg = HP[hix(0, q)] * g[0] + HP[hix(1, q)] * g[1] + HP[hix(2, q)] * g[2];
        out.d1[q] = a.P * Sk[q] + Pk[q] * f0;
        const F acc = HSk + F(4) * x[q] * f2 * Px + F(2) * f1 * Pk[q];
        out.dl[q] = Pk[q] * LS + a.P * x[q] * c3 + F(2) * acc + Sk[q] * LP;
        out.hg[q] = a.P * (F(4) * x[q] * f2 * xg + F(2) * f1 * g[q]) + Sk[q] * Pg + Pk[q] * (F(2) * f1 * xg) +
                    f0 * Hg;
    }
}

template <typename F>
__device__ __forceinline__ F det4(int e, const F m[4][4]) {
    switch (e) {
        case 0:
            return F(1);
        case 1:
            return m[0][0];
        case 2:
            return m[0][0] * m[1][1] - m[0][1] * m[1][0];
        case 3:
            return m[0][0] * (m[1][1] * m[2][2] - m[1][2] * m[2][1]) - m[0][1] * (m[1][0] * m[2][2] - m[1][2] * m[2][0]) +
                   m[0][2] * (m[1][0] * m[2][1] - m[1][1] * m[2][0]);
        default: {
            const F a01 = m[0][0] * m[1][1] - m[0][1] * m[1][0], a02 = m[0][0] * m[1][2] - m[0][2] * m[1][0];
            const F a03 = m[0][0] * m[1][3] - m[0][3] * m[1][0], a12 = m[0][1] * m[1][2] - m[0][2] * m[1][1];
            const F a13 = m[0][1] * m[1][3] - m[0][3] * m[1][1], a23 = m[0][2] * m[1][3] - m[0][3] * m[1][2];
            const F b01 = m[2][0] * m[3][1] - m[2][1] * m[3][0], b02 = m[2][0] * m[3][2] - m[2][2] * m[3][0];
            const F b03 = m[2][0] * m[3][3] - m[2][3] * m[3][0], b12 = m[2][1] * m[3][2] - m[2][2] * m[3][1];
            const F b13 = m[2][1] * m[3][3] - m[2][3] * m[3][1], b23 = m[2][2] * m[3][3] - m[2][3] * m[3][2];
            return a01 * b23 - a02 * b13 + a03 * b12 + a12 * b03 - a13 * b02 + a23 * b01;
        }
    }
}

struct SDesc {
    int e;
    double ph;
    int h[4], p[4];
};

__device__ __forceinline__ SDesc sdecode(int4 v) {
    SDesc d;
    d.e = v.x & 0xff;
    d.ph = ((v.x >> 8) & 1) ? -1.0 : 1.0;
    for (int a = 0; a < 4; ++a) {
        d.h[a] = (v.y >> (8 * a)) & 0xff;
        d.p[a] = (v.z >> (8 * a)) & 0xff;
    }
    return d;
}

// Terms of the functions of one shell at one electron with the weights
// ME, YE, ML of their rows (stride ld): vt[q] += me (lap/2 + gj.grad) terms
// + ye d_q Phi, vt[3 + q] += ml d_q Phi.  L = 0 or 1 fixes the angular
// momentum at compile time (constant angular factors fold); L = -1 takes
// l, pure, nf at run time.
template <typename T, int L>
__device__ __forceinline__ void shell_terms_m(int l, int pure, int nf, const T x[3], T f0, T f1, T f2, T f3,
                                              const T gj[3], const T* MEr, const T* YEr, const T* MLr, int ld,
                                              T (&vt)[6]) {
    auto body = [&](int fi) {
        D3<T> D;
        shell_d3m<T>(L >= 0 ? L : l, pure, x, gj, fi, f0, f1, f2, f3, D);
        const T me = MEr[fi * ld], ye = YEr[fi * ld], ml = MLr[fi * ld];
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            vt[q] += me * (T(0.5) * D.dl[q] + D.hg[q]) + ye * D.d1[q];
            vt[3 + q] += ml * D.d1[q];
        }
    };
    if constexpr (L >= 0) {
#pragma unroll
        for (int fi = 0; fi < (L == 0 ? 1 : 3); ++fi) body(fi);
    } else {
        for (int fi = 0; fi < nf; ++fi) body(fi);
    }
}

// Per-walker scratch layout (doubles), per spin s with n = n_s, v = n_vir[s]:
//   B0 n*n, Bv n*v, Th n*v, Q n*v, Z n*v, ZT n*v, Zh n*v, V n*v, BX n*n,
//   Ew n*(n+v), Yw n*(n+v), Lw n*(n+v), then D[n_str], CdD[n_str].
__host__ __device__ inline size_t fm_spin_words(int n, int v, int ns) {
    return (size_t)2 * n * n + (size_t)7 * n * v + (size_t)3 * n * (n + v) + 2 * (size_t)ns;
}

// kE: also the determinant part of dE_L/dr_i into gEdet [W][N][3] and
// grad_i ln|psi| into gtot [W][N][3] (space-warp form; see k_force.cu).
template <typename T, bool kE>
__global__ void __launch_bounds__(256) k_force_msd(DevSys s, DevWalkers wk, int W, const double* dvnn,
                                                   double* scr, size_t stride, double* dEL, double* dlog,
                                                   double* gEdet, double* gtot) {
    extern __shared__ double sm[];
    __shared__ double red[kMaxWarps * 4];
    const int w = blockIdx.x;
    if (w >= W) return;
    const int N = s.N, nu = s.n_up, nd = s.n_dn, nn = s.n_nuc;
    const int nmax = nu > nd ? nu : nd;
    const int nvmax = s.n_vir[0] > s.n_vir[1] ? s.n_vir[0] : s.n_vir[1];
    double* sR = sm;
    double* gJ = sR + 3 * N;
    double* gt = gJ + 3 * N;
    double* kap = gt + 3 * N;
    double* acc = kap + 3 * N;                  // [nn][6]
    T* Yb = (T*)(acc + 6 * nn);                 // [3][nmax][nvmax]: Ybar, Yt, Ytheta
    double* tiles = acc + 6 * nn + 3 * nmax * nvmax;   // [3][kFmTile][nmax]: ME, YE, ML
    double* gEs = tiles + 3 * kFmTile * nmax;          // [N][3] (kE only)
    double* base = scr + (size_t)w * stride;
    double* sp[2];
    sp[0] = base;
    sp[1] = base + fm_spin_words(nu, s.n_vir[0], s.n_str[0]);

    for (int q = threadIdx.x; q < 3 * N; q += blockDim.x) {
        sR[q] = wk.R[(size_t)w * 3 * N + q];
        kap[q] = 0.0;
        if constexpr (kE) gEs[q] = 0.0;
    }
    __syncthreads();
    // grad J, grad ln D0 per electron
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        const int spin = i >= nu;
        const int n = spin ? nd : nu, k = spin ? i - nu : i;
        const T* Ai = (const T*)wk.Ainv[spin] + ((size_t)w * n + k) * n;
        const T* Gi = (const T*)wk.G[spin] + ((size_t)w * n + k) * 4 * n;
        double d[3] = {0, 0, 0}, g[3] = {0, 0, 0};
        for (int j = 0; j < n; ++j)
            for (int c = 0; c < 3; ++c) d[c] += (double)Gi[c * n + j] * (double)Ai[j];
        for (int j = 0; j < N + nn; ++j) {
            double x[3], a, b;
            if (j < N) {
                if (j == i) continue;
                for (int c = 0; c < 3; ++c) x[c] = sR[3 * i + c] - sR[3 * j + c];
                a = ((i < nu) == (j < nu)) ? s.a_par : s.a_anti;
                b = s.b_ee;
            } else {
                for (int c = 0; c < 3; ++c) x[c] = sR[3 * i + c] - s.Rn[3 * (j - N) + c];
                a = s.a_en[j - N];
                b = s.b_en;
            }
            const double r2 = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
            const double ir = rsqrt(r2);
            const double qd = 1.0 / (1.0 + b * r2 * ir);
            for (int c = 0; c < 3; ++c) g[c] += a * qd * qd * ir * x[c];
        }
        for (int c = 0; c < 3; ++c) {
            gJ[3 * i + c] = g[c];
            gt[3 * i + c] = g[c] + d[c];
        }
    }
    __syncthreads();

    // ---- B, Theta and the string quantities D_u -------------------------
    for (int spin = 0; spin < 2; ++spin) {
        const int n = spin ? nd : nu, v = s.n_vir[spin], i0 = spin ? nu : 0, ns = s.n_str[spin];
        double* B0 = sp[spin];
        double* Bv = B0 + n * n;
        double* Th = Bv + n * v;
        double* Q = Th + n * v;
        double* Dd = sp[spin] + fm_spin_words(n, v, ns) - 2 * ns;
        const T* AT = (const T*)wk.Ainv[spin] + (size_t)w * n * n;
        const T* G = (const T*)wk.G[spin] + (size_t)w * 4 * n * n;
        const T* Gv = (const T*)wk.Gv[spin] + (size_t)w * 4 * n * v;
        const T* Tt = (const T*)wk.Tt[spin] + (size_t)w * n * v;
        for (int q = threadIdx.x; q < n * (n + v); q += blockDim.x) {
            const int i = q / (n + v), j = q - i * (n + v);
            const double* gj = gJ + 3 * (i0 + i);
            if (j < n) {
                const T* Gi = G + (size_t)i * 4 * n;
                B0[i * n + j] = -0.5 * (double)Gi[3 * n + j] - gj[0] * (double)Gi[j] - gj[1] * (double)Gi[n + j] -
                                gj[2] * (double)Gi[2 * n + j];
            } else {
                const int p = j - n;
                const T* Gi = Gv + (size_t)i * 4 * v;
                Bv[i * v + p] = -0.5 * (double)Gi[3 * v + p] - gj[0] * (double)Gi[p] - gj[1] * (double)Gi[v + p] -
                                gj[2] * (double)Gi[2 * v + p];
            }
        }
        __syncthreads();
        for (int q = threadIdx.x; q < n * v; q += blockDim.x) {
            const int i = q / v, p = q - i * v;
            double a = Bv[q];
            for (int j = 0; j < n; ++j) a -= B0[i * n + j] * (double)Tt[(size_t)j * v + p];
            Q[q] = a;
        }
        __syncthreads();
        for (int q = threadIdx.x; q < n * v; q += blockDim.x) {
            const int h = q / v, p = q - h * v;
            double a = 0.0;
            for (int i = 0; i < n; ++i) a += (double)AT[(size_t)i * n + h] * Q[i * v + p];
            Th[q] = a;
        }
        __syncthreads();
        for (int u = threadIdx.x; u < ns; u += blockDim.x) {
            const SDesc d = sdecode(s.str[spin][u]);
            T acc2 = T(0);
            if (d.e > 0) {
                T m[4][4], nm[4][4];
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        const bool in = a < d.e && c < d.e;
                        m[a][c] = in ? Tt[(size_t)d.h[a] * v + d.p[c]] : T(0);
                        nm[a][c] = in ? T(Th[d.h[a] * v + d.p[c]]) : T(0);
                    }
                for (int b = 0; b < d.e; ++b) {
                    T t[4][4];
#pragma unroll
                    for (int a = 0; a < 4; ++a)
#pragma unroll
                        for (int c = 0; c < 4; ++c) t[a][c] = (c == b) ? nm[a][c] : m[a][c];
                    acc2 += det4<T>(d.e, t);
                }
            }
            Dd[u] = d.ph * (double)acc2;
        }
        __syncthreads();
    }
    // CdD per spin and Sd
    double sdv[1] = {0.0};
    for (int spin = 0; spin < 2; ++spin) {
        const int n = spin ? nd : nu, v = s.n_vir[spin], ns = s.n_str[spin];
        const int no = spin ? nu : nd, vo = s.n_vir[1 - spin], nso = s.n_str[1 - spin];
        double* Dd = sp[spin] + fm_spin_words(n, v, ns) - 2 * ns;
        double* CdD = Dd + ns;
        const double* Do = sp[1 - spin] + fm_spin_words(no, vo, nso) - 2 * nso;
        const T* R = (const T*)wk.Rs[spin] + (size_t)w * ns;
        const T* Cd = (const T*)wk.Cd[spin] + (size_t)w * ns;
        for (int u = threadIdx.x; u < ns; u += blockDim.x) {
            double a = 0.0;
            for (int q = s.csr_off[spin][u]; q < s.csr_off[spin][u + 1]; ++q)
                a += s.csr_c[spin][q] * Do[s.csr_other[spin][q]];
            CdD[u] = a;
            if (spin == 0) sdv[0] += Dd[u] * (double)Cd[u] + (double)R[u] * a;
        }
    }
    block_sum<1>(sdv, red);
    const double S = wk.Ssum[w], Sd = sdv[0];

    // ---- adjoint weights per spin ----------------------------------------
    for (int spin = 0; spin < 2; ++spin) {
        const int n = spin ? nd : nu, v = s.n_vir[spin], i0 = spin ? nu : 0, ns = s.n_str[spin];
        if (n == 0) continue;
        double* B0 = sp[spin];
        double* Bv = B0 + n * n;
        double* Th = Bv + n * v;
        double* Z = Th + 2 * n * v;  // after Q
        double* ZT = Z + n * v;
        double* Zh = ZT + n * v;
        double* V = Zh + n * v;
        double* BX = V + n * v;
        // adjoint weights in the precision of the form (read by the tile
        // products below); T occupies at most the double slots
        T* Ew = (T*)(BX + n * n);
        T* Yw = (T*)(BX + n * n + n * (n + v));
        T* Lw = (T*)(BX + n * n + 2 * n * (n + v));
        double* Dd = sp[spin] + fm_spin_words(n, v, ns) - 2 * ns;
        double* CdD = Dd + ns;
        const T* AT = (const T*)wk.Ainv[spin] + (size_t)w * n * n;
        const T* G = (const T*)wk.G[spin] + (size_t)w * 4 * n * n;
        const T* Gv = (const T*)wk.Gv[spin] + (size_t)w * 4 * n * v;
        const T* Tt = (const T*)wk.Tt[spin] + (size_t)w * n * v;
        const T* R = (const T*)wk.Rs[spin] + (size_t)w * ns;
        const T* Cd = (const T*)wk.Cd[spin] + (size_t)w * ns;
        T* Ybar = Yb;
        T* Ytt = Yb + nmax * nvmax;
        T* Yth = Yb + 2 * nmax * nvmax;
        for (int q = threadIdx.x; q < 3 * nmax * nvmax; q += blockDim.x) Yb[q] = T(0);
        __syncthreads();
        // string weights in the precision of the form (the inverse of S and
        // Sd / S once per walker)
        const T invS = T(1.0 / S), sdS = T(Sd / S);
        for (int u = threadIdx.x; u < ns; u += blockDim.x) {
            const SDesc d = sdecode(s.str[spin][u]);
            if (d.e == 0) continue;
            T m[4][4], nm[4][4], cof[4][4], dDdM[4][4];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const bool in = a < d.e && c < d.e;
                    m[a][c] = in ? Tt[(size_t)d.h[a] * v + d.p[c]] : T(0);
                    nm[a][c] = in ? T(Th[d.h[a] * v + d.p[c]]) : T(0);
                    dDdM[a][c] = T(0);
                }
            cofactors<T>(d.e, m, cof);
            for (int b = 0; b < d.e; ++b) {  // d/dM of det(M with column b <- N)
                T t[4][4], cb[4][4];
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int c = 0; c < 4; ++c) t[a][c] = (c == b) ? nm[a][c] : m[a][c];
                cofactors<T>(d.e, t, cb);
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int c = 0; c < 4; ++c)
                        if (c != b) dDdM[a][c] += cb[a][c];
            }
            const T cdu = Cd[u];
            const T ph = T(d.ph);
            const T al = ph * cdu * invS, be = ph * (T(CdD[u]) - sdS * cdu) * invS;
            for (int a = 0; a < d.e; ++a)
                for (int c = 0; c < d.e; ++c) {
                    const int o = d.h[a] * nvmax + d.p[c];
                    atomicAdd(&Ybar[o], al * cof[a][c]);
                    atomicAdd(&Ytt[o], al * dDdM[a][c] + be * cof[a][c]);
                    atomicAdd(&Yth[o], al * cof[a][c]);
                }
            (void)R;
        }
        __syncthreads();
        // Z = X^T Ybar, ZT = X^T Yt, Zh = X^T Ytheta   (X^T[i][h] = AT[i][h])
        for (int q = threadIdx.x; q < n * v; q += blockDim.x) {
            const int i = q / v, p = q - i * v;
            double a0 = 0.0, a1 = 0.0, a2 = 0.0;
            for (int h = 0; h < n; ++h) {
                const double x = (double)AT[(size_t)i * n + h];
                a0 += x * (double)Ybar[h * nvmax + p];
                a1 += x * (double)Ytt[h * nvmax + p];
                a2 += x * (double)Yth[h * nvmax + p];
            }
            Z[q] = a0;
            ZT[q] = a1;
            Zh[q] = a2;
        }
        // BX[i][m] = sum_j B0[i][j] X[j][m] = sum_j B0[i][j] AT[m][j]
        for (int q = threadIdx.x; q < n * n; q += blockDim.x) {
            const int i = q / n, mm = q - i * n;
            double a = 0.0;
            for (int j = 0; j < n; ++j) a += B0[i * n + j] * (double)AT[(size_t)mm * n + j];
            BX[q] = a;
        }
        __syncthreads();
        // V[m][p] = sum_i BX[i][m] Zh[i][p]
        for (int q = threadIdx.x; q < n * v; q += blockDim.x) {
            const int mm = q / v, p = q - mm * v;
            double a = 0.0;
            for (int i = 0; i < n; ++i) a += BX[i * n + mm] * Zh[i * v + p];
            V[q] = a;
        }
        __syncthreads();
        // weights on the occupied (j < n) and virtual (p) blocks:
        //   Ew = [X^T + wB0 | wBv], Yw = [Y_SD - wA0 | -wAv], Lw = [X^T - W0 | Z]
        //   wBv = Zh, wB0 = -Zh T^T, wAv = ZT - V, wA0 = -ZT T^T - Zh Th^T + V T^T,
        //   W0 = Z T^T, Y_SD[i][j] = (X B0 X)[j][i] = sum_p AT[p][j] BX[p][i]... (see k_force)
        for (int q = threadIdx.x; q < n * (n + v); q += blockDim.x) {
            const int i = q / (n + v), j = q - i * (n + v);
            if (j < n) {
                double zt = 0.0, zh = 0.0, vt = 0.0, zz = 0.0, zth = 0.0;
                for (int p = 0; p < v; ++p) {
                    const double tjp = (double)Tt[(size_t)j * v + p];
                    zt += ZT[i * v + p] * tjp;
                    zh += Zh[i * v + p] * tjp;
                    vt += V[i * v + p] * tjp;
                    zz += Z[i * v + p] * tjp;
                    zth += Zh[i * v + p] * Th[j * v + p];
                }
                // X B0 X: (X B0 X)[j][i] = sum_m X[j][m] (B0 X)[m][i] = sum_m AT[m][j] BX[m][i]
                double ysd = 0.0;
                for (int mm = 0; mm < n; ++mm) ysd += (double)AT[(size_t)mm * n + j] * BX[mm * n + i];
                const double wB0 = -zh, wA0 = -zt - zth + vt;
                const double xt = (double)AT[(size_t)i * n + j];
                Ew[q] = T(xt + wB0);
                Yw[q] = T(ysd - wA0);
                Lw[q] = T(xt - zz);
            } else {
                const int p = j - n;
                Ew[q] = T(Zh[i * v + p]);
                Yw[q] = T(-(ZT[i * v + p] - V[i * v + p]));
                Lw[q] = T(Z[i * v + p]);
            }
        }
        __syncthreads();
        // Jastrow-gradient weight: kappa_i = sum_j wB0[i][j] grad phi_j + sum_p wBv[i][p] grad phi_p
        for (int q = threadIdx.x; q < 3 * n; q += blockDim.x) {
            const int i = q / 3, c = q - 3 * i;
            const T* Gi = G + (size_t)i * 4 * n;
            const T* Gvi = Gv + (size_t)i * 4 * v;
            double a = 0.0;
            for (int j = 0; j < n; ++j)
                a += ((double)Ew[i * (n + v) + j] - (double)AT[(size_t)i * n + j]) * (double)Gi[c * n + j];
            for (int p = 0; p < v; ++p) a += (double)Ew[i * (n + v) + n + p] * (double)Gvi[c * v + p];
            kap[3 * (i0 + i) + c] = a;
        }
        __syncthreads();
    }

    // ---- e-n Jastrow, V_en, V_nn ------------------------------------------
    for (int a = threadIdx.x; a < nn; a += blockDim.x) {
        double dT[3] = {0, 0, 0}, dJ[3] = {0, 0, 0};
        for (int i = 0; i < N; ++i) {
            double x[3];
            for (int c = 0; c < 3; ++c) x[c] = sR[3 * i + c] - s.Rn[3 * a + c];
            const double r2 = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
            const double r = sqrt(r2);
            double u, du, d2u, d3u;
            pade3<double>(s.a_en[a], s.b_en, r, u, du, d2u, d3u);
            const double cl = 0.5 * (d3u + 2.0 * d2u / r - 2.0 * du / r2) / r;
            const double hx = (d2u - du / r) / r2;
            double g[3];
            for (int c = 0; c < 3; ++c) g[c] = gt[3 * i + c] + kap[3 * i + c];
            const double gdot = g[0] * x[0] + g[1] * x[1] + g[2] * x[2];
            for (int q = 0; q < 3; ++q) {
                dT[q] += cl * x[q] + hx * x[q] * gdot + (du / r) * g[q] - s.Z[a] * x[q] / (r2 * r);
                dJ[q] += -du * x[q] / r;
            }
        }
        for (int q = 0; q < 3; ++q) {
            acc[6 * a + q] = dT[q] + dvnn[3 * a + q];
            acc[6 * a + 3 + q] = dJ[q];
        }
    }
    __syncthreads();

    // ---- pull back to basis space and contract -----------------------------
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    T* ME = (T*)tiles;
    T* YE = ME + kFmTile * nmax;
    T* ML = ME + 2 * kFmTile * nmax;
    for (int spin = 0; spin < 2; ++spin) {
        const int n = spin ? nd : nu, v = s.n_vir[spin], i0 = spin ? nu : 0;
        if (n == 0) continue;
        const double* wbase = sp[spin] + 2 * n * n + 7 * (size_t)n * v;  // after B0,Bv,Th,Q,Z,ZT,Zh,V,BX
        const T* Ew = (const T*)wbase;
        const T* Yw = (const T*)(wbase + n * (n + v));
        const T* Lw = (const T*)(wbase + 2 * n * (n + v));
        const T* C0 = sys_C<T>(s, spin);
        const T* Cv = sys_Cv<T>(s, spin);
        int sh0 = 0;
        while (sh0 < s.n_shell) {
            const int fl0 = s.shell_fn[sh0];
            int sh1 = sh0 + 1;
            while (sh1 < s.n_shell && s.shell_fn[sh1 + 1] - fl0 <= kFmTile) ++sh1;
            const int nfl = s.shell_fn[sh1] - fl0;
            for (int q = threadIdx.x; q < nfl * n; q += blockDim.x) {
                const int l = q / n, i = q - l * n;
                const T* c0 = C0 + (size_t)(fl0 + l) * n;
                const T* cv = Cv + (size_t)(fl0 + l) * v;
                const T* e = Ew + (size_t)i * (n + v);
                const T* y = Yw + (size_t)i * (n + v);
                const T* lw = Lw + (size_t)i * (n + v);
                T me = T(0), ye = T(0), ml = T(0);
                for (int j = 0; j < n; ++j) {
                    me += c0[j] * e[j];
                    ye += c0[j] * y[j];
                    ml += c0[j] * lw[j];
                }
                for (int p = 0; p < v; ++p) {
                    me += cv[p] * e[n + p];
                    ye += cv[p] * y[n + p];
                    ml += cv[p] * lw[n + p];
                }
                ME[l * nmax + i] = me;
                YE[l * nmax + i] = ye;
                ML[l * nmax + i] = ml;
            }
            __syncthreads();
            for (int sh = sh0 + wid; sh < sh1; sh += nw) {
                const int4 d = s.shell[sh];
                const int l = d.y & 0xff, pure = d.y >> 8;
                const int nf = shell_nfn(l, pure);
                const int lb = s.shell_fn[sh] - fl0;
                T vv[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
                for (int i = lane; i < n; i += 32) {
                    const T x[3] = {T(sR[3 * (i0 + i)] - s.Rn[3 * d.x]), T(sR[3 * (i0 + i) + 1] - s.Rn[3 * d.x + 1]),
                                    T(sR[3 * (i0 + i) + 2] - s.Rn[3 * d.x + 2])};
                    T f0, f1, f2, f3;
                    radial<T, true>(sys_alpha<T>(s), sys_cn<T>(s), d.z, d.w, x[0] * x[0] + x[1] * x[1] + x[2] * x[2],
                                    f0, f1, f2, f3);
                    if (f0 == T(0) && f1 == T(0) && f2 == T(0) && f3 == T(0)) continue;
                    const T gj[3] = {T(gJ[3 * (i0 + i)]), T(gJ[3 * (i0 + i) + 1]), T(gJ[3 * (i0 + i) + 2])};
                    T vt[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
                    const int o = lb * nmax + i;
                    if (l == 0)
                        shell_terms_m<T, 0>(l, pure, nf, x, f0, f1, f2, f3, gj, ME + o, YE + o, ML + o, nmax, vt);
                    else if (l == 1)
                        shell_terms_m<T, 1>(l, pure, nf, x, f0, f1, f2, f3, gj, ME + o, YE + o, ML + o, nmax, vt);
                    else
                        shell_terms_m<T, -1>(l, pure, nf, x, f0, f1, f2, f3, gj, ME + o, YE + o, ML + o, nmax, vt);
                    for (int q = 0; q < 6; ++q) vv[q] += vt[q];
                    if constexpr (kE)
                        for (int q = 0; q < 3; ++q) atomicAdd(&gEs[3 * (i0 + i) + q], -double(vt[q]));
                }
                // one shell's sum over this spin's electrons; shells add in FP64
                for (int q = 0; q < 6; ++q) vv[q] = warp_sum(vv[q]);
                if (lane == 0)
                    for (int q = 0; q < 6; ++q) atomicAdd(&acc[6 * d.x + q], q < 3 ? double(vv[q]) : -double(vv[q]));
            }
            __syncthreads();
            sh0 = sh1;
        }
    }
    __syncthreads();
    for (int q = threadIdx.x; q < 3 * nn; q += blockDim.x) {
        const int a = q / 3, c = q - 3 * a;
        dEL[(size_t)w * 3 * nn + q] = acc[6 * a + c];
        dlog[(size_t)w * 3 * nn + q] = acc[6 * a + 3 + c];
    }
    if constexpr (kE)
        for (int q = threadIdx.x; q < 3 * N; q += blockDim.x) {
            gEdet[(size_t)w * 3 * N + q] = gEs[q];
            gtot[(size_t)w * 3 * N + q] = gt[q] + kap[q];
        }
}

size_t force_msd_scratch_words(const DevSys& s) {
    return fm_spin_words(s.n_up, s.n_vir[0], s.n_str[0]) + fm_spin_words(s.n_dn, s.n_vir[1], s.n_str[1]);
}

// gEdet, gtot (both null, or both [W][N][3]): the space-warp form's
// per-electron outputs.
template <typename T>
cudaError_t launch_force_msd(const DevSys& s, const DevWalkers& wk, int W, const double* dvnn, double* scr,
                             double* dEL, double* dlog, double* gEdet, double* gtot, cudaStream_t st) {
    if (W == 0) return cudaSuccess;
    const int nmax = s.n_up > s.n_dn ? s.n_up : s.n_dn;
    const int nvmax = s.n_vir[0] > s.n_vir[1] ? s.n_vir[0] : s.n_vir[1];
    const size_t smem =
        sizeof(double) * (12 * (size_t)s.N + 6 * (size_t)s.n_nuc + 3 * (size_t)nmax * nvmax + 3 * (size_t)kFmTile * nmax);
    if (gEdet) {
        const size_t smem_e = smem + sizeof(double) * 3 * (size_t)s.N;
        cudaError_t e =
            cudaFuncSetAttribute(k_force_msd<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_e);
        if (e != cudaSuccess) return e;
        k_force_msd<T, true><<<W, 256, smem_e, st>>>(s, wk, W, dvnn, scr, force_msd_scratch_words(s), dEL, dlog,
                                                     gEdet, gtot);
        return cudaGetLastError();
    }
    cudaError_t e = cudaFuncSetAttribute(k_force_msd<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_force_msd<T, false><<<W, 256, smem, st>>>(s, wk, W, dvnn, scr, force_msd_scratch_words(s), dEL, dlog, nullptr,
                                                nullptr);
    return cudaGetLastError();
}

template cudaError_t launch_force_msd<double>(const DevSys&, const DevWalkers&, int, const double*, double*, double*,
                                              double*, double*, double*, cudaStream_t);
template cudaError_t launch_force_msd<float>(const DevSys&, const DevWalkers&, int, const double*, double*, double*,
                                             double*, double*, double*, cudaStream_t);

}  // namespace qmc
