// Multi-determinant expansions by the table method (Sec. "Multideterminant
// QMC Forces": excited determinants from small determinants of a table,
// determinants grouped by excitation level).
//
// With the reference Slater matrix A0 (n x n) of a spin and the values of
// the active virtual orbitals at the same electrons, A_v (n x n_vir), the
// table T = A0^-1 A_v gives every excited determinant of that spin as
//   D_u / D_0 = phase_u det(T[H_u, P_u])          (e_u <= 4 rows/columns),
// H_u the replaced reference positions, P_u the replacing virtuals, and
// phase_u the sign of sorting the replaced orbital list.  The expansion is
//   psi_D / (D0_up D0_dn) = S = sum_k c_k R_up[u(k)] R_dn[d(k)].
// For any operator B applied to the orbital matrix one electron row at a
// time (a derivative in that electron's coordinates), the change of ln D_u
// relative to ln D_0 is tr(M^-1 Theta[H,P]) with M = T[H,P] and
//   Theta = A0^-1 (B_v - B_0 T),
// i.e. the first-order change of det(M) along Theta; used here for the
// kinetic operator of the local energy and for electron gradients.
#include "msd_small.cuh"
#include "qmc_internal.cuh"

namespace qmc {

template <typename F>
__device__ __forceinline__ F det_small(int e, const F m[4][4]) {
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
            // Laplace expansion along the first two rows (2x2 minors)
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

struct StrDesc {
    int e;
    float phase;
    int h[4], p[4];
};

__device__ __forceinline__ StrDesc decode(int4 v) {
    StrDesc d;
    d.e = v.x & 0xff;
    d.phase = ((v.x >> 8) & 1) ? -1.f : 1.f;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        d.h[a] = (v.y >> (8 * a)) & 0xff;
        d.p[a] = (v.z >> (8 * a)) & 0xff;
    }
    return d;
}

// M = T[H,P] from a row-major table with leading dimension ld.
template <typename F, typename TT>
__device__ __forceinline__ void gather_minor(const StrDesc& d, const TT* T, int ld, F m[4][4]) {
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) m[a][b] = (a < d.e && b < d.e) ? F(T[d.h[a] * ld + d.p[b]]) : F(0);
}

// det(M with column b replaced by the vector u), b = 0..e-1.
template <typename F>
__device__ __forceinline__ void col_replaced_dets(int e, const F m[4][4], const F u[4], F out[4]) {
    for (int b = 0; b < 4; ++b) {
        if (b >= e) {
            out[b] = F(0);
            continue;
        }
        F t[4][4];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int c = 0; c < 4; ++c) t[a][c] = (c == b) ? u[a] : m[a][c];
        out[b] = det_small<F>(e, t);
    }
}

// Table, string ratios, CI partial sums and S for every walker (after an
// FP64 recompute of the reference inverse and the virtual orbital values).
template <typename T>
__global__ void k_msd_table(DevSys s, DevWalkers wk, int W, const int* only) {
    __shared__ double scratch[kMaxWarps];
    const int w = blockIdx.x;
    if (w >= W || (only && !only[w])) return;
    for (int spin = 0; spin < 2; ++spin) {
        const int n = spin ? s.n_dn : s.n_up, nv = s.n_vir[spin];
        const T* AT = (const T*)wk.Ainv[spin] + (size_t)w * n * n;
        const T* Av = (const T*)wk.Av[spin] + (size_t)w * n * nv;
        T* Tt = (T*)wk.Tt[spin] + (size_t)w * n * nv;
        for (int q = threadIdx.x; q < n * nv; q += blockDim.x) {
            const int h = q / nv, p = q - h * nv;
            T acc = T(0);
            for (int i = 0; i < n; ++i) acc += AT[(size_t)i * n + h] * Av[(size_t)i * nv + p];
            Tt[q] = acc;
        }
        __syncthreads();
        T* R = (T*)wk.Rs[spin] + (size_t)w * s.n_str[spin];
        for (int u = threadIdx.x; u < s.n_str[spin]; u += blockDim.x) {
            const StrDesc d = decode(s.str[spin][u]);
            T m[4][4];
            gather_minor<T>(d, Tt, nv, m);
            R[u] = T(d.phase) * det_small<T>(d.e, m);
        }
        __syncthreads();
    }
    for (int spin = 0; spin < 2; ++spin) {
        const T* Ro = (const T*)wk.Rs[1 - spin] + (size_t)w * s.n_str[1 - spin];
        T* Cd = (T*)wk.Cd[spin] + (size_t)w * s.n_str[spin];
        for (int u = threadIdx.x; u < s.n_str[spin]; u += blockDim.x) {
            double acc = 0.0;
            for (int q = s.csr_off[spin][u]; q < s.csr_off[spin][u + 1]; ++q)
                acc += s.csr_c[spin][q] * (double)Ro[s.csr_other[spin][q]];
            Cd[u] = (T)acc;
        }
    }
    __syncthreads();
    double v[1] = {0.0};
    const T* R0 = (const T*)wk.Rs[0] + (size_t)w * s.n_str[0];
    const T* C0 = (const T*)wk.Cd[0] + (size_t)w * s.n_str[0];
    for (int u = threadIdx.x; u < s.n_str[0]; u += blockDim.x) v[0] += (double)R0[u] * (double)C0[u];
    block_sum<1>(v, scratch);
    if (threadIdx.x == 0) wk.Ssum[w] = v[0];
}

// Adds the multi-determinant part to E_L, ln|psi|, the sign and (when grad
// is given) the electron gradients of ln|psi| computed for the reference
// determinant by k_eloc.
template <typename T>
__global__ void k_msd_eloc(DevSys s, DevWalkers wk, int W, double* eloc, double* logpsi, double* sign,
                           double* grad) {
    extern __shared__ double sm[];
    __shared__ double scratch[kMaxWarps * 4];
    const int w = blockIdx.x;
    if (w >= W) return;
    const int N = s.N, nu = s.n_up, nn = s.n_nuc;
    const int nmax = nu > s.n_dn ? nu : s.n_dn;
    const int nvmax = s.n_vir[0] > s.n_vir[1] ? s.n_vir[0] : s.n_vir[1];
    double* sR = sm;
    double* gJ = sR + 3 * N;
    double* Q = gJ + 3 * N;              // [nmax][nvmax]
    double* Th = Q + nmax * nvmax;       // [nmax][nvmax]
    double* Wg = Th + nmax * nvmax;      // [3][nvmax]
    for (int q = threadIdx.x; q < 3 * N; q += blockDim.x) sR[q] = wk.R[(size_t)w * 3 * N + q];
    __syncthreads();
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        double g[3] = {0, 0, 0};
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
            const double gr = a * qd * qd * ir;
            for (int c = 0; c < 3; ++c) g[c] += gr * x[c];
        }
        for (int c = 0; c < 3; ++c) gJ[3 * i + c] = g[c];
    }
    __syncthreads();
    const double S = wk.Ssum[w];
    // per string: tr(adj(M) Theta[H,P]) with the cofactors of the table minor
    // in the storage type and the contraction with Theta in FP64
    Acc<double> sd[1];
    for (int spin = 0; spin < 2; ++spin) {
        const int n = spin ? s.n_dn : nu, nv = s.n_vir[spin], i0 = spin ? nu : 0;
        if (n == 0) continue;
        const T* AT = (const T*)wk.Ainv[spin] + (size_t)w * n * n;
        const T* G = (const T*)wk.G[spin] + (size_t)w * 4 * n * n;
        const T* Gv = (const T*)wk.Gv[spin] + (size_t)w * 4 * n * nv;
        const T* Tt = (const T*)wk.Tt[spin] + (size_t)w * n * nv;
        // Q = B_v - B_0 T with B = -1/2 lap phi - grad J . grad phi per row
        for (int q = threadIdx.x; q < n * nv; q += blockDim.x) {
            const int i = q / nv, p = q - i * nv;
            const double* gj = gJ + 3 * (i0 + i);
            const T* Gi = G + (size_t)i * 4 * n;
            const T* Gvi = Gv + (size_t)i * 4 * nv;
            double acc = -0.5 * (double)Gvi[3 * nv + p] - gj[0] * (double)Gvi[p] - gj[1] * (double)Gvi[nv + p] -
                         gj[2] * (double)Gvi[2 * nv + p];
            for (int j = 0; j < n; ++j) {
                const double b0 = -0.5 * (double)Gi[3 * n + j] - gj[0] * (double)Gi[j] - gj[1] * (double)Gi[n + j] -
                                  gj[2] * (double)Gi[2 * n + j];
                acc -= b0 * (double)Tt[(size_t)j * nv + p];
            }
            Q[i * nvmax + p] = acc;
        }
        __syncthreads();
        // Theta = A0^-1 Q
        for (int q = threadIdx.x; q < n * nv; q += blockDim.x) {
            const int h = q / nv, p = q - h * nv;
            double acc = 0.0;
            for (int i = 0; i < n; ++i) acc += (double)AT[(size_t)i * n + h] * Q[i * nvmax + p];
            Th[h * nvmax + p] = acc;
        }
        __syncthreads();
        const T* Cd = (const T*)wk.Cd[spin] + (size_t)w * s.n_str[spin];
        for (int u = threadIdx.x; u < s.n_str[spin]; u += blockDim.x) {
            const StrDesc d = decode(s.str[spin][u]);
            if (d.e == 0) continue;
            T m[4][4], cof[4][4];
            gather_minor<T>(d, Tt, nv, m);
            cofactors<T>(d.e, m, cof);
            double tr = 0.0;
            for (int a = 0; a < d.e; ++a)
                for (int c = 0; c < d.e; ++c) tr += (double)cof[a][c] * Th[d.h[a] * nvmax + d.p[c]];
            sd[0].add((double)d.phase * tr * (double)Cd[u]);
        }
        __syncthreads();
    }
    double sdd[1];
    block_sum_to0<1>(sd, scratch, sdd);
    if (threadIdx.x == 0) {
        eloc[w] += sdd[0] / S;
        if (logpsi) logpsi[w] += log(fabs(S));
        if (sign) sign[w] = wk.sgn[2 * w] * wk.sgn[2 * w + 1] * (S < 0.0 ? -1.0 : 1.0);
    }
    if (!grad) return;
    // electron gradients: d_i S / S = sum_u Cd_u phase_u sum_b W_i[p_b] det(M with column b <- A0^-1[H, i])
    for (int i = 0; i < N; ++i) {
        const int spin = i >= nu;
        const int n = spin ? s.n_dn : nu, nv = s.n_vir[spin], k = spin ? i - nu : i;
        const T* AT = (const T*)wk.Ainv[spin] + (size_t)w * n * n;
        const T* Gk = (const T*)wk.G[spin] + ((size_t)w * n + k) * 4 * n;
        const T* Gvk = (const T*)wk.Gv[spin] + ((size_t)w * n + k) * 4 * nv;
        const T* Tt = (const T*)wk.Tt[spin] + (size_t)w * n * nv;
        __syncthreads();
        for (int q = threadIdx.x; q < 3 * nv; q += blockDim.x) {
            const int c = q / nv, p = q - c * nv;
            double acc = (double)Gvk[c * nv + p];
            for (int j = 0; j < n; ++j) acc -= (double)Gk[c * n + j] * (double)Tt[(size_t)j * nv + p];
            Wg[c * nvmax + p] = acc;
        }
        __syncthreads();
        const T* Cd = (const T*)wk.Cd[spin] + (size_t)w * s.n_str[spin];
        Acc<T> g[3];
        for (int u = threadIdx.x; u < s.n_str[spin]; u += blockDim.x) {
            const StrDesc d = decode(s.str[spin][u]);
            if (d.e == 0) continue;
            T m[4][4], uh[4], gb[4];
            gather_minor<T>(d, Tt, nv, m);
            for (int a = 0; a < 4; ++a) uh[a] = a < d.e ? AT[(size_t)k * n + d.h[a]] : T(0);
            col_replaced_dets<T>(d.e, m, uh, gb);
            const T f = T(d.phase) * Cd[u];
            for (int b = 0; b < d.e; ++b)
                for (int c = 0; c < 3; ++c) g[c].add(f * T(Wg[c * nvmax + d.p[b]]) * gb[b]);
        }
        double gd[3];
        block_sum_to0<3>(g, scratch, gd);
        if (threadIdx.x == 0)
            for (int c = 0; c < 3; ++c) grad[((size_t)w * N + i) * 3 + c] += gd[c] / S;
    }
}


// ---------------------------------------------------------------------
// Particle-by-particle sweep of a multi-determinant wavefunction.
//
// On top of the reference-determinant move of k_sweep, a move of electron
// e (spin s) updates the table by a rank-1 term,
//   T' = T + c w^T / rho0,  c = A0^-1[:, e],  w = phi'_v - T^T phi'_occ,
// (no old orbital row is needed), evaluates every string ratio of spin s
// from T'[H,P], and S' = sum_u Cd_u R'_u with Cd_u = sum over the string's
// determinants of c_k R_other (fixed while spin s moves).  The wavefunction
// ratio is rho0 S'/S e^{dJ}.  Drifts add d_e S / S, the derivative of every
// string determinant along the rank-1 change of row e.
// ---------------------------------------------------------------------
template <typename T>
__host__ __device__ inline size_t msd_sweep_smem(int N, int nb, int nu, int nd, int nv0, int nv1) {
    const int nmax = nu > nd ? nu : nd, nvmax = nv0 > nv1 ? nv0 : nv1;
    size_t o = sizeof(double) * (3 * (size_t)N + kMaxWarps * 12 + 16);
    o += sizeof(T) * (5 * (size_t)nb + 5 * (size_t)nmax + 5 * (size_t)nvmax + nmax + nvmax + 3 * (size_t)nvmax);
    o += sizeof(T) * ((size_t)nu * nu + (size_t)nd * nd + (size_t)nu * nv0 + (size_t)nd * nv1);
    return o;
}

template <typename T>
__device__ __forceinline__ void refresh_cd(const DevSys& s, const DevWalkers& wk, int w, int spin) {
    const T* Ro = (const T*)wk.Rs[1 - spin] + (size_t)w * s.n_str[1 - spin];
    T* Cd = (T*)wk.Cd[spin] + (size_t)w * s.n_str[spin];
    for (int u = threadIdx.x; u < s.n_str[spin]; u += blockDim.x) {
        double acc = 0.0;
        for (int q = s.csr_off[spin][u]; q < s.csr_off[spin][u + 1]; ++q)
            acc += s.csr_c[spin][q] * (double)Ro[s.csr_other[spin][q]];
        Cd[u] = (T)acc;
    }
}

constexpr double kRefreshRho0F = 1e-2;   // mixed form
constexpr double kRefreshRho0D = 1e-4;   // FP64 form

template <typename T>
__global__ void k_sweep_msd(DevSys s, DevWalkers wk, int W, SweepParams p) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int w = blockIdx.x;
    if (w >= W) return;
    const int N = s.N, nu = s.n_up, nd = s.n_dn, nb = s.n_basis, nn = s.n_nuc;
    const int nmax = nu > nd ? nu : nd;
    const int nv0 = s.n_vir[0], nv1 = s.n_vir[1], nvmax = nv0 > nv1 ? nv0 : nv1;
    double* sR = (double*)smem;
    double* red = sR + 3 * N;
    double* scal = red + kMaxWarps * 12;
    T* bas = (T*)(scal + 16);
    T* phi = bas + 5 * nb;
    T* phv = phi + 5 * nmax;
    T* cold = phv + 5 * nvmax;
    T* wv = cold + nmax;
    T* Wc = wv + nvmax;          // [3][nvmax]
    T* sA = Wc + 3 * nvmax;
    T* sT = sA + nu * nu + nd * nd;
    T* Ainv[2] = {sA, sA + nu * nu};
    T* Tt[2] = {sT, sT + nu * nv0};
    {
        const T* g0 = (const T*)wk.Ainv[0] + (size_t)w * nu * nu;
        const T* g1 = (const T*)wk.Ainv[1] + (size_t)w * nd * nd;
        for (int q = threadIdx.x; q < nu * nu; q += blockDim.x) Ainv[0][q] = g0[q];
        for (int q = threadIdx.x; q < nd * nd; q += blockDim.x) Ainv[1][q] = g1[q];
        const T* t0 = (const T*)wk.Tt[0] + (size_t)w * nu * nv0;
        const T* t1 = (const T*)wk.Tt[1] + (size_t)w * nd * nv1;
        for (int q = threadIdx.x; q < nu * nv0; q += blockDim.x) Tt[0][q] = t0[q];
        for (int q = threadIdx.x; q < nd * nv1; q += blockDim.x) Tt[1][q] = t1[q];
    }
    for (int q = threadIdx.x; q < 3 * N; q += blockDim.x) sR[q] = wk.R[(size_t)w * 3 * N + q];
    double ld0 = 0.0, ld1 = 0.0, sg0 = 1.0, sg1 = 1.0;
    if (threadIdx.x == 0) {
        ld0 = wk.logdet[2 * w];
        ld1 = wk.logdet[2 * w + 1];
        sg0 = wk.sgn[2 * w];
        sg1 = wk.sgn[2 * w + 1];
        scal[8] = wk.Ssum[w];
    }
    unsigned long long acc = 0;
    __syncthreads();
    const double tau = p.tau;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    T* redT = (T*)red;

    for (int e = 0; e < N; ++e) {
        const int spin = e >= nu;
        const int n = spin ? nd : nu, nv = spin ? nv1 : nv0, ns = s.n_str[spin];
        const int k = spin ? e - nu : e;
        T* A = Ainv[spin];
        T* Ts = Tt[spin];
        const T* Ae = A + (size_t)k * n;
        T* Gk = (T*)wk.G[spin] + ((size_t)w * n + k) * 4 * n;
        T* Gvk = (T*)wk.Gv[spin] + ((size_t)w * n + k) * 4 * nv;
        T* Avk = (T*)wk.Av[spin] + ((size_t)w * n + k) * nv;
        T* Rcur = (T*)wk.Rs[spin] + (size_t)w * ns;
        T* Rnew = (T*)wk.Rn[spin] + (size_t)w * ns;
        const T* Cd = (const T*)wk.Cd[spin] + (size_t)w * ns;
        const int4* str = s.str[spin];
        const double re0 = sR[3 * e], re1 = sR[3 * e + 1], re2 = sR[3 * e + 2];

        // -- drift at the current position ---------------------------------
        for (int q = threadIdx.x; q < 3 * nv; q += blockDim.x) {
            const int c = q / nv, pp = q - c * nv;
            T a = Gvk[c * nv + pp];
            for (int j = 0; j < n; ++j) a -= Gk[c * n + j] * Ts[(size_t)j * nv + pp];
            Wc[c * nvmax + pp] = a;
        }
        Acc<T> va[9];
        T u_old = T(0);
        for (int j = threadIdx.x; j < n; j += blockDim.x) {
            const T a = Ae[j];
            va[0].add(Gk[j] * a);
            va[1].add(Gk[n + j] * a);
            va[2].add(Gk[2 * n + j] * a);
        }
        for (int q = threadIdx.x; q < N + nn; q += blockDim.x) {
            T x, y, z, a, b;
            if (q < N) {
                if (q == e) continue;
                x = T(re0 - sR[3 * q]); y = T(re1 - sR[3 * q + 1]); z = T(re2 - sR[3 * q + 2]);
                a = T(((q < nu) == (e < nu)) ? s.a_par : s.a_anti);
                b = T(s.b_ee);
            } else {
                const int c = q - N;
                x = T(re0 - s.Rn[3 * c]); y = T(re1 - s.Rn[3 * c + 1]); z = T(re2 - s.Rn[3 * c + 2]);
                a = T(s.a_en[c]);
                b = T(s.b_en);
            }
            const T ir = rsqrt_t(x * x + y * y + z * z);
            const T r = (x * x + y * y + z * z) * ir;
            const T qd = T(1) / (T(1) + b * r);
            u_old += a * r * qd;
            const T g = a * qd * qd * ir;
            va[3].add(g * x);
            va[4].add(g * y);
            va[5].add(g * z);
        }
        __syncthreads();
        for (int u = threadIdx.x; u < ns; u += blockDim.x) {
            const StrDesc d = decode(str[u]);
            if (d.e == 0) continue;
            T m[4][4], uh[4], gb[4];
            gather_minor<T>(d, Ts, nv, m);
#pragma unroll
            for (int a = 0; a < 4; ++a) uh[a] = a < d.e ? Ae[d.h[a]] : T(0);
            col_replaced_dets<T>(d.e, m, uh, gb);
            const T f = T(d.phase) * Cd[u];
            for (int b = 0; b < d.e; ++b) {
                const T fb = f * gb[b];
                va[6].add(fb * Wc[d.p[b]]);
                va[7].add(fb * Wc[nvmax + d.p[b]]);
                va[8].add(fb * Wc[2 * nvmax + d.p[b]]);
            }
        }
        double vd[9];
        block_sum_to0<9>(va, red, vd);
        if (threadIdx.x == 0) {
            const double iS = 1.0 / scal[8];
            const T g[3] = {T(vd[0] + vd[3] + vd[6] * iS), T(vd[1] + vd[4] + vd[7] * iS), T(vd[2] + vd[5] + vd[8] * iS)};
            const double r[3] = {re0, re1, re2};
            propose_move<T>(g, tau, r, p.key, p.sweep, (uint32_t)e, (uint32_t)w, scal);
        }
        __syncthreads();
        const double rn[3] = {scal[0], scal[1], scal[2]};

        // -- basis, occupied and virtual orbitals at r' -------------------
        for (int sh = threadIdx.x; sh < s.n_shell; sh += blockDim.x) shell_vgl<T>(s, sh, rn, bas, nb);
        __syncthreads();
        {
            const T* C = sys_C<T>(s, spin);
            const T* Cv = sys_Cv<T>(s, spin);
            for (int o = threadIdx.x; o < 5 * (n + nv); o += blockDim.x) {
                const int c = o / (n + nv), j = o - c * (n + nv);
                const T* b = bas + c * nb;
                T a0 = T(0), a1 = T(0);
                if (j < n) {
                    int l = 0;
                    for (; l + 2 <= nb; l += 2) {
                        a0 += C[(size_t)l * n + j] * b[l];
                        a1 += C[(size_t)(l + 1) * n + j] * b[l + 1];
                    }
                    for (; l < nb; ++l) a0 += C[(size_t)l * n + j] * b[l];
                    phi[c * nmax + j] = a0 + a1;
                } else {
                    const int pp = j - n;
                    int l = 0;
                    for (; l + 2 <= nb; l += 2) {
                        a0 += Cv[(size_t)l * nv + pp] * b[l];
                        a1 += Cv[(size_t)(l + 1) * nv + pp] * b[l + 1];
                    }
                    for (; l < nb; ++l) a0 += Cv[(size_t)l * nv + pp] * b[l];
                    phv[c * nvmax + pp] = a0 + a1;
                }
            }
        }
        __syncthreads();

        // -- reference ratio, its gradient, Jastrow change -----------------
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
                x = T(rn[0] - sR[3 * q]); y = T(rn[1] - sR[3 * q + 1]); z = T(rn[2] - sR[3 * q + 2]);
                a = T(((q < nu) == (e < nu)) ? s.a_par : s.a_anti);
                b = T(s.b_ee);
            } else {
                const int c = q - N;
                x = T(rn[0] - s.Rn[3 * c]); y = T(rn[1] - s.Rn[3 * c + 1]); z = T(rn[2] - s.Rn[3 * c + 2]);
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
        block_sum8<T>(vb2, redT);
        const T rho0 = vb2[0];
        const T rinv0 = T(1) / rho0;

        // -- new table column weights, string ratios and gradients ----------
        for (int q = threadIdx.x; q < 4 * nv; q += blockDim.x) {
            const int c = q / nv, pp = q - c * nv;
            T a = phv[c * nvmax + pp];
            for (int h = 0; h < n; ++h) a -= Ts[(size_t)h * nv + pp] * phi[c * nmax + h];
            if (c == 0)
                wv[pp] = a;
            else
                Wc[(c - 1) * nvmax + pp] = a;   // grad phi'_v - T^T grad phi'_occ (before the w term)
        }
        __syncthreads();
        for (int q = threadIdx.x; q < 3 * nv; q += blockDim.x) {
            const int c = q / nv, pp = q - c * nv;
            Wc[c * nvmax + pp] -= wv[pp] * vb2[1 + c] * rinv0;
        }
        __syncthreads();
        Acc<T> vs[4];
        for (int u = threadIdx.x; u < ns; u += blockDim.x) {
            const StrDesc d = decode(str[u]);
            T m[4][4], uh[4], gb[4];
            gather_minor<T>(d, Ts, nv, m);
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                const T ca = a < d.e ? Ae[d.h[a]] * rinv0 : T(0);
                uh[a] = ca;
#pragma unroll
                for (int b = 0; b < 4; ++b) m[a][b] += (a < d.e && b < d.e) ? ca * wv[d.p[b]] : T(0);
            }
            const T Ru = T(d.phase) * det_small<T>(d.e, m);
            Rnew[u] = Ru;
            vs[0].add(Cd[u] * Ru);
            if (d.e == 0) continue;
            col_replaced_dets<T>(d.e, m, uh, gb);
            const T f = T(d.phase) * Cd[u];
            for (int b = 0; b < d.e; ++b) {
                const T fb = f * gb[b];
                vs[1].add(fb * Wc[d.p[b]]);
                vs[2].add(fb * Wc[nvmax + d.p[b]]);
                vs[3].add(fb * Wc[2 * nvmax + d.p[b]]);
            }
        }
        double vsd[4];
        block_sum_to0<4>(vs, red + kMaxWarps * 8, vsd);
        if (threadIdx.x == 0) {
            const double S = scal[8], Sn = vsd[0];
            const double ratio = (double)rho0 * Sn / S;
            const double iSn = 1.0 / Sn;
            const T g[3] = {T((double)vb2[1] / (double)rho0 + (double)vb2[5] + vsd[1] * iSn),
                            T((double)vb2[2] / (double)rho0 + (double)vb2[6] + vsd[2] * iSn),
                            T((double)vb2[3] / (double)rho0 + (double)vb2[7] + vsd[3] * iSn)};
            const double ro3[3] = {re0, re1, re2};
            const int accept = accept_move_g<T>(T(ratio), g, vb2[4], tau, ro3, rn, scal + 3, p.key, p.sweep,
                                                (uint32_t)e, (uint32_t)w);
            scal[6] = (double)rho0;
            scal[7] = accept ? 1.0 : 0.0;
            scal[9] = Sn;
        }
        __syncthreads();
        if (scal[7] != 0.0) {
            for (int j = threadIdx.x; j < n; j += blockDim.x) cold[j] = A[(size_t)k * n + j];
            __syncthreads();
            for (int q = wid; q < n; q += nw) {
                T* Aq = A + (size_t)q * n;
                T t = T(0);
                for (int j = lane; j < n; j += 32) t += phi[j] * Aq[j];
                t = warp_sum(t);
                if (q == k) t -= T(1);
                const T f = t * rinv0;
                for (int j = lane; j < n; j += 32) Aq[j] -= f * cold[j];
            }
            for (int q = threadIdx.x; q < n * nv; q += blockDim.x) {
                const int h = q / nv, pp = q - h * nv;
                Ts[q] += cold[h] * wv[pp] * rinv0;
            }
            for (int o = threadIdx.x; o < 4 * n; o += blockDim.x) {
                const int c = o / n, j = o - c * n;
                Gk[o] = phi[(c + 1) * nmax + j];
            }
            for (int o = threadIdx.x; o < 5 * nv; o += blockDim.x) {
                const int c = o / nv, pp = o - c * nv;
                if (c == 0)
                    Avk[pp] = phv[pp];
                else
                    Gvk[(c - 1) * nv + pp] = phv[c * nvmax + pp];
            }
            for (int u = threadIdx.x; u < ns; u += blockDim.x) Rcur[u] = Rnew[u];
            if (threadIdx.x == 0) {
                const double r0 = scal[6];
                if (spin) {
                    ld1 += log(fabs(r0));
                    if (r0 < 0.0) sg1 = -sg1;
                } else {
                    ld0 += log(fabs(r0));
                    if (r0 < 0.0) sg0 = -sg0;
                }
                // The expansion accepts moves on its own ratio; the rank-1
                // updates of A0^-1 and T divide by the reference ratio, which
                // may be near zero there (the reference near its node while
                // the expansion is not).  Such a walker is rebuilt from scratch
                // in FP64 after the sweep.
                if (fabs(r0) < (sizeof(T) == 4 ? kRefreshRho0F : kRefreshRho0D) && wk.refresh) wk.refresh[w] = 1;
                scal[8] = scal[9];
                sR[3 * e] = rn[0];
                sR[3 * e + 1] = rn[1];
                sR[3 * e + 2] = rn[2];
                ++acc;
            }
            __syncthreads();
        }
        if (e == nu - 1 && nd > 0) {
            // the up block is done: the down strings' partial sums see the new R_up
            refresh_cd<T>(s, wk, w, 1);
            __syncthreads();
        }
    }
    refresh_cd<T>(s, wk, w, 0);
    __syncthreads();
    for (int q = threadIdx.x; q < 3 * N; q += blockDim.x) wk.R[(size_t)w * 3 * N + q] = sR[q];
    {
        T* g0 = (T*)wk.Ainv[0] + (size_t)w * nu * nu;
        T* g1 = (T*)wk.Ainv[1] + (size_t)w * nd * nd;
        for (int q = threadIdx.x; q < nu * nu; q += blockDim.x) g0[q] = Ainv[0][q];
        for (int q = threadIdx.x; q < nd * nd; q += blockDim.x) g1[q] = Ainv[1][q];
        T* t0 = (T*)wk.Tt[0] + (size_t)w * nu * nv0;
        T* t1 = (T*)wk.Tt[1] + (size_t)w * nd * nv1;
        for (int q = threadIdx.x; q < nu * nv0; q += blockDim.x) t0[q] = Tt[0][q];
        for (int q = threadIdx.x; q < nd * nv1; q += blockDim.x) t1[q] = Tt[1][q];
    }
    if (threadIdx.x == 0) {
        wk.logdet[2 * w] = ld0;
        wk.logdet[2 * w + 1] = ld1;
        wk.sgn[2 * w] = sg0;
        wk.sgn[2 * w + 1] = sg1;
        wk.Ssum[w] = scal[8];
        if (acc) atomicAdd(wk.n_acc, acc);
    }
}

template <typename T>
size_t msd_sweep_smem_bytes(const DevSys& s) {
    return msd_sweep_smem<T>(s.N, s.n_basis, s.n_up, s.n_dn, s.n_vir[0], s.n_vir[1]);
}

template <typename T>
cudaError_t launch_sweep_msd(const DevSys& s, const DevWalkers& wk, int W, const SweepParams& p, cudaStream_t st) {
    if (W == 0) return cudaSuccess;
    const size_t smem = msd_sweep_smem_bytes<T>(s);
    cudaError_t e = cudaFuncSetAttribute(k_sweep_msd<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_sweep_msd<T><<<W, 256, smem, st>>>(s, wk, W, p);
    return cudaGetLastError();
}

template size_t msd_sweep_smem_bytes<double>(const DevSys&);
template size_t msd_sweep_smem_bytes<float>(const DevSys&);
template cudaError_t launch_sweep_msd<double>(const DevSys&, const DevWalkers&, int, const SweepParams&, cudaStream_t);
template cudaError_t launch_sweep_msd<float>(const DevSys&, const DevWalkers&, int, const SweepParams&, cudaStream_t);

template <typename T>
cudaError_t launch_msd_table(const DevSys& s, const DevWalkers& wk, int W, cudaStream_t st, const int* only) {
    if (W == 0) return cudaSuccess;
    k_msd_table<T><<<W, 256, 0, st>>>(s, wk, W, only);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_msd_eloc(const DevSys& s, const DevWalkers& wk, int W, double* eloc, double* logpsi,
                            double* sign, double* grad, cudaStream_t st) {
    if (W == 0) return cudaSuccess;
    const int nmax = s.n_up > s.n_dn ? s.n_up : s.n_dn;
    const int nvmax = s.n_vir[0] > s.n_vir[1] ? s.n_vir[0] : s.n_vir[1];
    const size_t smem = sizeof(double) * (6 * (size_t)s.N + (2 * (size_t)nmax + 3) * (nvmax > 0 ? nvmax : 1));
    cudaError_t e = cudaFuncSetAttribute(k_msd_eloc<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_msd_eloc<T><<<W, 256, smem, st>>>(s, wk, W, eloc, logpsi, sign, grad);
    return cudaGetLastError();
}

template cudaError_t launch_msd_table<double>(const DevSys&, const DevWalkers&, int, cudaStream_t, const int*);
template cudaError_t launch_msd_table<float>(const DevSys&, const DevWalkers&, int, cudaStream_t, const int*);
template cudaError_t launch_msd_eloc<double>(const DevSys&, const DevWalkers&, int, double*, double*, double*,
                                             double*, cudaStream_t);
template cudaError_t launch_msd_eloc<float>(const DevSys&, const DevWalkers&, int, double*, double*, double*,
                                            double*, cudaStream_t);

}  // namespace qmc
