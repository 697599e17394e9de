// Ionic derivatives of E_L and ln|psi| for every walker by an adjoint
// (reverse-mode) pass.
//
// Sec. "Single Determinant QMC Forces" writes the derivative of a
// determinant one-body operator as tr(A^-1 dB/dR_a - X dA/dR_a) with
// X = A^-1 B A^-1 (Eq. 4) and d ln D = tr(A^-1 dA) (Eq. 3), evaluated there
// once per nuclear coordinate (cost O(N^3 3 N_atom)).  Here the kinetic
// determinant term is written as tr(B A^-1) with
//   B_ij = -1/2 lap phi_j(r_i) - grad_i J . grad phi_j(r_i),
// and since every dA, dB is a contraction of basis-function derivatives with
// the coefficient matrix C, the traces are pulled back to basis space once:
//   M = C^T A^-1         (n_basis x n),  weights of dPhi in d ln D and dB,
//   Y = M (B A^-1)       (n_basis x n),  weights of dPhi in -tr(X dA).
// Then for each electron i and basis function l on nucleus a
//   d ln D / dR_a += -M_li d Phi_l(r_i)
//   dT_det / dR_a += -M_li (-1/2 d lap Phi_l - grad_i J . d grad Phi_l)
//                    + Y_li d Phi_l(r_i)
// (the basis function moves with its nucleus: d/dR_a = -d/dr).  The cost
// is O(n^2 n_basis + n^3 + N n_basis) per walker, independent of N_atom.
// Basis derivatives to third order are recomputed per walker rather than
// stored.  The e-n Jastrow, V_en and V_nn terms are added directly.
#include "batch.cuh"
#include "qmc_internal.cuh"

namespace qmc {

constexpr int kForceTile = 32;  // basis functions per tile of M and Y

// First derivatives d_q Phi, derivatives of the Laplacian d_q lap Phi and
// the Hessian applied to a vector, (Hess Phi . g)_q, of one function of a
// shell at offset x (f0..f3: the radial sums at t = |x|^2).  With
// Phi = P S, S_k = d_k S = 2 x_k f1, S_kq = 4 x_k x_q f2 + 2 delta_kq f1:
//   d_q Phi        = P S_q + P_q S,
//   d_q lap Phi    = P_q lap S + P d_q lap S + 2 sum_k (P_kq S_k + P_k S_kq) + S_q lap P,
//   (Hess Phi g)_q = P sum_k S_kq g_k + S_q (grad P . g) + P_q (grad S . g) + S (Hess P g)_q,
// with sum_k S_kq g_k = 4 x_q f2 (x . g) + 2 f1 g_q: the Hessian is never
// formed, only its product with g (the adjoint needs nothing else).
template <typename F>
struct Deriv3 {
    F d1[3];   // d/dq Phi
    F hg[3];   // (Hess Phi . g)_q
    F dl[3];   // d/dq lap Phi
};

__device__ __forceinline__ int hidx(int a, int b) {
    // symmetric index into (xx, xy, xz, yy, yz, zz)
    const int lo = a < b ? a : b, hi = a < b ? b : a;
    return lo == 0 ? hi : (lo == 1 ? 2 + hi : 5);
}

template <typename F>
__device__ __forceinline__ void shell_d3(int l, int pure, const F x[3], const F g[3], int fi, F f0, F f1, F f2,
                                         F f3, Deriv3<F>& out) {
    const F t = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
    const AngPoly<F> a = angular<F>(l, pure, fi, x[0], x[1], x[2]);
    const F Pk[3] = {a.Px, a.Py, a.Pz};
    const F HP[6] = {a.Hxx, a.Hxy, a.Hxz, a.Hyy, a.Hyz, a.Hzz};
    const F LP = a.Hxx + a.Hyy + a.Hzz;
    F Sk[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) Sk[k] = F(2) * x[k] * f1;
    const F LS = F(6) * f1 + F(4) * t * f2;
    const F Px = Pk[0] * x[0] + Pk[1] * x[1] + Pk[2] * x[2];
    const F Pg = Pk[0] * g[0] + Pk[1] * g[1] + Pk[2] * g[2];
    const F xg = x[0] * g[0] + x[1] * g[1] + x[2] * g[2];
    const F c3 = F(20) * f2 + F(8) * t * f3;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const F HSk = HP[hidx(0, q)] * Sk[0] + HP[hidx(1, q)] * Sk[1] + HP[hidx(2, q)] * Sk[2];
        const F Hg = HP[hidx(0, q)] * g[0] + HP[hidx(1, q)] * g[1] + HP[hidx(2, q)] * g[2];
        out.d1[q] = a.P * Sk[q] + Pk[q] * f0;
        // sum_k (P_kq S_k + P_k S_kq) = (Hess P S)_q + 4 x_q f2 (grad P . x) + 2 f1 P_q
        const F acc = HSk + F(4) * x[q] * f2 * Px + F(2) * f1 * Pk[q];
        out.dl[q] = Pk[q] * LS + a.P * x[q] * c3 + F(2) * acc + Sk[q] * LP;
        out.hg[q] = a.P * (F(4) * x[q] * f2 * xg + F(2) * f1 * g[q]) + Sk[q] * Pg + Pk[q] * (F(2) * f1 * xg) +
                    f0 * Hg;
    }
}

// Adjoint terms of the functions of one shell at one electron: with M, Y
// the basis-space weights of the function rows (m = Mrow[fi * ld], y =
// Yrow[fi * ld]) and gj = grad_i J,
//   vt[q]     += -m (-1/2 d_q lap Phi - gj . d_q grad Phi) + y d_q Phi,
//   vt[3 + q] +=  m d_q Phi
// (derivatives with respect to the electron coordinate; the callers turn
// them into nuclear ones).  L = 0 or 1 fixes the angular momentum at compile
// time, so the constant angular factors of s and p shells fold away (on
// GB300 every FP64 instruction counts); L = -1 takes l, pure, nf at run time.
template <typename T, int L>
__device__ __forceinline__ void shell_terms(int l, int pure, int nf, const T x[3], T f0, T f1, T f2, T f3,
                                            const T gj[3], const T* Mrow, const T* Yrow, int ld, T (&vt)[6]) {
    auto body = [&](int fi) {
        Deriv3<T> D;
        shell_d3<T>(L >= 0 ? L : l, pure, x, gj, fi, f0, f1, f2, f3, D);
        const T m = Mrow[(size_t)fi * ld], y = Yrow[(size_t)fi * ld];
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            vt[q] += -m * (T(-0.5) * D.dl[q] - D.hg[q]) + y * D.d1[q];
            vt[3 + q] += m * D.d1[q];
        }
    };
    if constexpr (L >= 0) {
#pragma unroll
        for (int fi = 0; fi < (L == 0 ? 1 : 3); ++fi) body(fi);
    } else {
        for (int fi = 0; fi < nf; ++fi) body(fi);
    }
}

template <typename T>
__device__ __forceinline__ void shell_terms_any(int l, int pure, int nf, const T x[3], T f0, T f1, T f2, T f3,
                                                const T gj[3], const T* Mrow, const T* Yrow, int ld, T (&vt)[6]) {
    if (l == 0)
        shell_terms<T, 0>(l, pure, nf, x, f0, f1, f2, f3, gj, Mrow, Yrow, ld, vt);
    else if (l == 1)
        shell_terms<T, 1>(l, pure, nf, x, f0, f1, f2, f3, gj, Mrow, Yrow, ld, vt);
    else
        shell_terms<T, -1>(l, pure, nf, x, f0, f1, f2, f3, gj, Mrow, Yrow, ld, vt);
}

// Shared-memory head of every force kernel: positions (FP64), the per-atom
// sums acc[nn][6] (FP64: dT (3), dlnpsi (3)), grad_i J and grad_i ln|psi|
// in the form's type T, and the positions split as hi + lo floats, from
// which the mixed form takes its FP32 offsets without an FP64 instruction.
template <typename T>
__host__ __device__ inline size_t force_head_bytes(int N, int nn) {
    return sizeof(double) * (3 * (size_t)N + 6 * (size_t)nn) + sizeof(T) * 6 * (size_t)N + sizeof(float) * 6 * (size_t)N;
}

template <typename T>
struct ForceHead {
    double* sR;
    double* acc;
    T* gJ;
    T* gt;
    float* sRh;
    float* sRl;
    __device__ ForceHead(double* sm, int N, int nn) {
        sR = sm;
        acc = sR + 3 * N;
        gJ = (T*)(acc + 6 * nn);
        gt = gJ + 3 * N;
        sRh = (float*)(gt + 3 * N);
        sRl = sRh + 3 * N;
    }
    __device__ T* end(int N) const { return (T*)(void*)(sRl + 3 * N); }
};

template <typename T>
__device__ __forceinline__ void force_load_positions(const ForceHead<T>& h, const double* R, int N) {
    for (int q = threadIdx.x; q < 3 * N; q += blockDim.x) {
        const double r = R[q];
        h.sR[q] = r;
        if constexpr (sizeof(T) == 4) {
            const float hi = (float)r;
            h.sRh[q] = hi;
            h.sRl[q] = (float)(r - (double)hi);
        }
    }
}

// Offsets r_i - r_j and r_i - R_a, component c, in the form's precision.
template <typename T>
__device__ __forceinline__ T off_ee(const ForceHead<T>& h, int i, int j, int c) {
    if constexpr (sizeof(T) == 4)
        return diff_f2(h.sRh[3 * i + c], h.sRl[3 * i + c], h.sRh[3 * j + c], h.sRl[3 * j + c]);
    else
        return h.sR[3 * i + c] - h.sR[3 * j + c];
}

template <typename T>
__device__ __forceinline__ T off_en(const ForceHead<T>& h, const DevSys& s, int i, int a, int c) {
    if constexpr (sizeof(T) == 4)
        return diff_f2(h.sRh[3 * i + c], h.sRl[3 * i + c], s.Rn_hi[3 * a + c], s.Rn_lo[3 * a + c]);
    else
        return h.sR[3 * i + c] - s.Rn[3 * a + c];
}

// grad_i J and grad_i ln|psi| of every electron (a warp per electron, lanes
// over its orbitals and its partners), then the e-n Jastrow, V_en and V_nn
// parts of the per-atom sums (a warp per nucleus, lanes over electrons).
// Terms and per-electron sums in T, per-atom sums in FP64.  Ends synchronised.
template <typename T>
__device__ __forceinline__ void force_gradients_en(const DevSys& s, const DevWalkers& wk, int w, const double* dvnn,
                                                   const ForceHead<T>& h) {
    const int N = s.N, nu = s.n_up, nn = s.n_nuc;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int i = wid; i < N; i += nw) {
        const int spin = i >= nu;
        const int n = spin ? s.n_dn : nu;
        const int k = spin ? i - nu : i;
        const T* Ai = (const T*)wk.Ainv[spin] + ((size_t)w * n + k) * n;
        const T* Gi = (const T*)wk.G[spin] + ((size_t)w * n + k) * 4 * n;
        T v[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};   // grad ln|D| (3), grad J (3)
        for (int j = lane; j < n; j += 32) {
            const T a = Ai[j];
            v[0] += Gi[j] * a;
            v[1] += Gi[n + j] * a;
            v[2] += Gi[2 * n + j] * a;
        }
        for (int j = lane; j < N + nn; j += 32) {
            T x[3], a, b;
            if (j < N) {
                if (j == i) continue;
#pragma unroll
                for (int c = 0; c < 3; ++c) x[c] = off_ee(h, i, j, c);
                a = T(((i < nu) == (j < nu)) ? s.a_par : s.a_anti);
                b = T(s.b_ee);
            } else {
                const int c0 = j - N;
#pragma unroll
                for (int c = 0; c < 3; ++c) x[c] = off_en(h, s, i, c0, c);
                a = T(s.a_en[c0]);
                b = T(s.b_en);
            }
            const T r2 = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
            const T ir = rsqrt_t(r2);
            const T qd = T(1) / (T(1) + b * r2 * ir);
            const T gr = a * qd * qd * ir;  // u'(r) / r
#pragma unroll
            for (int c = 0; c < 3; ++c) v[3 + c] += gr * x[c];
        }
#pragma unroll
        for (int q = 0; q < 6; ++q) v[q] = warp_sum(v[q]);
        if (lane == 0)
            for (int c = 0; c < 3; ++c) {
                h.gJ[3 * i + c] = v[3 + c];
                h.gt[3 * i + c] = v[3 + c] + v[c];
            }
    }
    __syncthreads();

    for (int a = wid; a < nn; a += nw) {
        const T Za = T(s.Z[a]), aen = T(s.a_en[a]), ben = T(s.b_en);
        T dT[3] = {T(0), T(0), T(0)}, dJ[3] = {T(0), T(0), T(0)};
        for (int i = lane; i < N; i += 32) {
            T x[3], g[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                x[c] = off_en(h, s, i, a, c);
                g[c] = h.gt[3 * i + c];
            }
            const T r2 = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
            const T ir = rsqrt_t(r2), r = r2 * ir;
            T u, du, d2u, d3u;
            pade3<T>(aen, ben, r, u, du, d2u, d3u);
            const T cl = T(0.5) * (d3u + T(2) * d2u * ir - T(2) * du * ir * ir) * ir;
            const T hx = (d2u - du * ir) * ir * ir;
            const T gdot = g[0] * x[0] + g[1] * x[1] + g[2] * x[2];
            T vr3 = Za * ir * ir * ir;
            if (s.npp)   // local pseudopotential terms: d v(r)/dR_a = -v'(r) x / r, folded into the -Z x / r^3 slot
                for (int t = s.pp_off[a]; t < s.pp_off[a + 1]; ++t) {
                    const int2 ln = s.pp_ln[t];
                    if (ln.x == -1) vr3 += pp_term_dr<T>(s, t, ln.y, r) * ir;
                }
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                // sum_c H_cq g_c with H = hx x x^T + (du/r) I
                const T Hg = hx * x[q] * gdot + du * ir * g[q];
                dT[q] += cl * x[q] + Hg - vr3 * x[q];
                dJ[q] -= du * x[q] * ir;
            }
        }
        double v[6];
        for (int q = 0; q < 3; ++q) {
            v[q] = warp_sum(double(dT[q]));
            v[3 + q] = warp_sum(double(dJ[q]));
        }
        if (lane == 0)
            for (int q = 0; q < 3; ++q) {
                h.acc[6 * a + q] = v[q] + dvnn[3 * a + q];
                h.acc[6 * a + 3 + q] = v[3 + q];
            }
    }
    __syncthreads();
}

// The transposed inverse and P^T = (B A^-1)^T of a spin are read n times
// each by the tile products of force_walker; when both fit beside the tiles
// (at most 100 KB in all, two CTAs per SM) they are staged in shared memory
// with row stride n + 1 (conflict-free column walks).
template <typename T>
__host__ __device__ inline bool force_stage_fits(int N, int nn, int nmax) {
    const size_t base = force_head_bytes<T>(N, nn) + sizeof(T) * 2 * (size_t)kForceTile * nmax;
    const size_t extra = sizeof(T) * 2 * (size_t)nmax * (nmax + 1);
    return base + extra <= 100 * 1024;
}

template <typename T>
__host__ __device__ inline size_t force_smem(int N, int nn, int nmax) {
    const size_t base = force_head_bytes<T>(N, nn) + sizeof(T) * 2 * (size_t)kForceTile * nmax;
    return base + (force_stage_fits<T>(N, nn, nmax) ? sizeof(T) * 2 * (size_t)nmax * (nmax + 1) : 0);
}

// Per-electron accumulators of the space-warp form (kE): 3N doubles placed
// after the force kernel's own shared memory.
template <typename T>
__host__ __device__ inline size_t force_smem_e(int N, int nn, int nmax, bool kE) {
    const size_t b = (force_smem<T>(N, nn, nmax) + 15) & ~(size_t)15;
    return kE ? b + sizeof(double) * 3 * (size_t)N : force_smem<T>(N, nn, nmax);
}

// Adjoint ionic derivatives of walker w (body of k_force).  sm: the
// dynamic shared memory of launch_force (force_smem_e).  kE: also the
// determinant part of dE_L/dr_i (the same basis-space terms, every basis
// function moving with the electron, d/dr_i = -d/dR) into gEdet [W][N][3]
// and grad_i ln|psi| into gtot [W][N][3], for the space warp.
template <typename T, bool kE = false>
__device__ __forceinline__ void force_walker(const DevSys& s, const DevWalkers& wk, int w, const double* dvnn, double* Bscr,
                                             double* Pscr, double* dEL, double* dlog, double* sm,
                                             double* gEdet = nullptr, double* gtot = nullptr) {
    const int N = s.N, nu = s.n_up, nn = s.n_nuc;
    const int nmax = nu > s.n_dn ? nu : s.n_dn;
    const ForceHead<T> h(sm, N, nn);
    double* acc = h.acc;
    T* Mt = h.end(N);                  // [kForceTile][nmax]
    T* Yt = Mt + kForceTile * nmax;
    T* B = (T*)(Bscr + (size_t)w * nmax * nmax);
    T* PTg = (T*)(Pscr + (size_t)w * nmax * nmax);
    const bool stg = force_stage_fits<T>(N, nn, nmax);
    T* sAT = Yt + kForceTile * nmax;
    T* sPT = sAT + nmax * (nmax + 1);
    double* gEs = (double*)((unsigned char*)sm + ((force_smem<T>(N, nn, nmax) + 15) & ~(size_t)15));

    force_load_positions(h, wk.R + (size_t)w * 3 * N, N);
    if constexpr (kE)
        for (int q = threadIdx.x; q < 3 * N; q += blockDim.x) gEs[q] = 0.0;
    __syncthreads();
    force_gradients_en<T>(s, wk, w, dvnn, h);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;

    for (int spin = 0; spin < 2; ++spin) {
        const int n = spin ? s.n_dn : nu;
        if (n == 0) continue;
        const int i0 = spin ? nu : 0;
        const T* ATg = (const T*)wk.Ainv[spin] + (size_t)w * n * n;
        const T* Gs = (const T*)wk.G[spin] + (size_t)w * 4 * n * n;
        const T* C = sys_C<T>(s, spin);
        const int ld = stg ? n + 1 : n;   // row stride of AT and PT as read below
        const T* AT = stg ? sAT : ATg;
        T* PT = stg ? sPT : PTg;
        if (stg)
            for (int q2 = threadIdx.x; q2 < n * n; q2 += blockDim.x) sAT[(q2 / n) * ld + q2 % n] = ATg[q2];
        // B_pq = -1/2 lap phi_q(r_p) - grad_p J . grad phi_q(r_p)
        for (int q2 = threadIdx.x; q2 < n * n; q2 += blockDim.x) {
            const int pp = q2 / n, qq = q2 - pp * n;
            const T* Gp = Gs + (size_t)pp * 4 * n;
            const T* gj = h.gJ + 3 * (i0 + pp);
            B[q2] = T(-0.5) * Gp[3 * n + qq] - gj[0] * Gp[qq] - gj[1] * Gp[n + qq] - gj[2] * Gp[2 * n + qq];
            // non-local pseudopotential rows: E_L gains tr(B_NL A^-1), so the
            // same -tr(X dA) pull-back covers them
            if (wk.nlB[spin]) B[q2] += ((const T*)wk.nlB[spin])[(size_t)w * n * n + q2];
        }
        __syncthreads();
        // PT[i][p] = (B A^-1)_{p i} = sum_q B_pq AT[i][q].  With AT staged,
        // lanes take consecutive i (row p of B is one broadcast address per
        // step, the AT rows sit at stride n + 1); otherwise consecutive p (the
        // global AT row is the broadcast one)
        for (int q2 = threadIdx.x; q2 < n * n; q2 += blockDim.x) {
            const int r = q2 / n, c = q2 - r * n;
            const int i = stg ? c : r, pp = stg ? r : c;
            const T* ATi = AT + (size_t)i * ld;
            const T* Bp = B + (size_t)pp * n;
            T v = T(0);
            for (int q = 0; q < n; ++q) v += Bp[q] * ATi[q];
            PT[i * ld + pp] = v;
        }
        __syncthreads();
        int sh0 = 0;
        while (sh0 < s.n_shell) {
            const int fl0 = s.shell_fn[sh0];
            int sh1 = sh0 + 1;
            while (sh1 < s.n_shell && s.shell_fn[sh1 + 1] - fl0 <= kForceTile) ++sh1;
            const int nfl = s.shell_fn[sh1] - fl0;
            // M[l][i] = sum_j C[l][j] AT[i][j]
            for (int q2 = threadIdx.x; q2 < nfl * n; q2 += blockDim.x) {
                const int l = q2 / n, i = q2 - l * n;
                const T* Cl = C + (size_t)(fl0 + l) * n;
                const T* ATi = AT + (size_t)i * ld;
                T v = T(0);
                for (int j = 0; j < n; ++j) v += Cl[j] * ATi[j];
                Mt[l * nmax + i] = v;
            }
            __syncthreads();
            // Y[l][i] = sum_p M[l][p] PT[i][p]
            for (int q2 = threadIdx.x; q2 < nfl * n; q2 += blockDim.x) {
                const int l = q2 / n, i = q2 - l * n;
                const T* Ml = Mt + l * nmax;
                const T* Pi = PT + (size_t)i * ld;
                T v = T(0);
                for (int p = 0; p < n; ++p) v += Ml[p] * Pi[p];
                Yt[l * nmax + i] = v;
            }
            __syncthreads();
            // warp per shell, lanes over electrons of this spin
            for (int sh = sh0 + wid; sh < sh1; sh += nw) {
                const int4 d = s.shell[sh];
                const int l = d.y & 0xff, pure = d.y >> 8;
                const int nf = shell_nfn(l, pure);
                const int lb = s.shell_fn[sh] - fl0;
                T v[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
                for (int i = lane; i < n; i += 32) {
                    const T x[3] = {off_en(h, s, i0 + i, d.x, 0), off_en(h, s, i0 + i, d.x, 1),
                                    off_en(h, s, i0 + i, d.x, 2)};
                    T f0, f1, f2, f3;
                    radial<T, true>(sys_alpha<T>(s), sys_cn<T>(s), d.z, d.w, x[0] * x[0] + x[1] * x[1] + x[2] * x[2],
                                    f0, f1, f2, f3);
                    if (f0 == T(0) && f1 == T(0) && f2 == T(0) && f3 == T(0)) continue;  // screened
                    const T gj[3] = {h.gJ[3 * (i0 + i)], h.gJ[3 * (i0 + i) + 1], h.gJ[3 * (i0 + i) + 2]};
                    // the basis function moves with its nucleus, d/dR = -d/dr:
                    // dT = sum M (wL dlap + w.dgrad) - Y dPhi with each d -> -d/dr
                    T vt[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
                    shell_terms_any<T>(l, pure, nf, x, f0, f1, f2, f3, gj, Mt + lb * nmax + i, Yt + lb * nmax + i,
                                       nmax, vt);
#pragma unroll
                    for (int q = 0; q < 6; ++q) v[q] += vt[q];
                    if constexpr (kE)
#pragma unroll
                        for (int q = 0; q < 3; ++q) atomicAdd(&gEs[3 * (i0 + i) + q], -double(vt[q]));
                }
                // one shell's sum over this spin's electrons; shells add in FP64
                for (int q = 0; q < 6; ++q) v[q] = warp_sum(v[q]);
                if (lane == 0)
                    for (int q = 0; q < 6; ++q) atomicAdd(&acc[6 * d.x + q], q < 3 ? double(v[q]) : -double(v[q]));
            }
            __syncthreads();
            sh0 = sh1;
        }
    }
    __syncthreads();
    for (int q = threadIdx.x; q < 3 * nn; q += blockDim.x) {
        const int a = q / 3, c = q - 3 * a;
        dEL[(size_t)w * 3 * nn + q] = acc[6 * a + c] + (wk.nlF ? wk.nlF[(size_t)w * 3 * nn + q] : 0.0);
        dlog[(size_t)w * 3 * nn + q] = acc[6 * a + 3 + c];
    }
    if constexpr (kE)
        for (int q = threadIdx.x; q < 3 * N; q += blockDim.x) {
            gEdet[(size_t)w * 3 * N + q] = gEs[q];
            gtot[(size_t)w * 3 * N + q] = double(h.gt[q]);
        }
}

// Three CTAs per SM in the FP32 form (80 registers, no spills); the FP64
// form keeps two (at three it spills).
template <typename T, bool kE>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 3 : 2) k_force(DevSys s, DevWalkers wk, int W, const double* dvnn,
                                                  double* Bscr, double* Pscr, double* dEL, double* dlog,
                                                  double* gEdet, double* gtot) {
    extern __shared__ double sm[];
    const int w = blockIdx.x;
    if (w >= W) return;
    force_walker<T, kE>(s, wk, w, dvnn, Bscr, Pscr, dEL, dlog, sm, gEdet, gtot);
}

// ---------------------------------------------------------------------
// Large determinants: the same adjoint with its dense products done as
// batched GEMMs (k_force_prep -> GEMMs -> k_force_contract).  Per walker and
// spin, with X^T = AT (the stored transposed inverse) and B as above:
//   PT = AT B^T,  Q = PT AT        (n x n, batched over walkers)
//   M  = C AT^T,  Y = C Q^T        (n_basis x n, C shared by all walkers)
// M and Y are exactly the tiles k_force builds on chip; for n above ~64
// they no longer fit, and as GEMMs they run near the ALU roofline.
// ---------------------------------------------------------------------

// Per walker: grad J (stored), B for both spins (stored, type T), and the
// e-n Jastrow / V_en / V_nn part of the per-atom sums (stored).
template <typename T, bool kE>
__global__ void k_force_prep(DevSys s, DevWalkers wk, int w0, int W, const double* dvnn, T* Bw, double* gJw,
                             double* accw, double* gtot) {
    extern __shared__ double sm[];
    const int wl = blockIdx.x, w = w0 + wl;
    if (wl >= W) return;
    const int N = s.N, nu = s.n_up, nn = s.n_nuc;
    const int nmax = nu > s.n_dn ? nu : s.n_dn;
    const ForceHead<T> h(sm, N, nn);
    force_load_positions(h, wk.R + (size_t)w * 3 * N, N);
    __syncthreads();
    force_gradients_en<T>(s, wk, w, dvnn, h);
    for (int q = threadIdx.x; q < 3 * N; q += blockDim.x) gJw[(size_t)wl * 3 * N + q] = double(h.gJ[q]);
    for (int q = threadIdx.x; q < 6 * nn; q += blockDim.x) accw[(size_t)wl * 6 * nn + q] = h.acc[q];
    if constexpr (kE)
        for (int q = threadIdx.x; q < 3 * N; q += blockDim.x) gtot[(size_t)w * 3 * N + q] = double(h.gt[q]);
    for (int spin = 0; spin < 2; ++spin) {
        const int n = spin ? s.n_dn : nu, i0 = spin ? nu : 0;
        const T* Gs = (const T*)wk.G[spin] + (size_t)w * 4 * n * n;
        T* B = Bw + ((size_t)(spin * W + wl)) * nmax * nmax;
        const T* nlB = (const T*)wk.nlB[spin];
        for (int q2 = threadIdx.x; q2 < n * n; q2 += blockDim.x) {
            const int pp = q2 / n, qq = q2 - pp * n;
            const T* Gp = Gs + (size_t)pp * 4 * n;
            const T* gj = h.gJ + 3 * (i0 + pp);
            B[q2] = T(-0.5) * Gp[3 * n + qq] - gj[0] * Gp[qq] - gj[1] * Gp[n + qq] - gj[2] * Gp[2 * n + qq];
            if (nlB) B[q2] += nlB[(size_t)w * n * n + q2];   // non-local pseudopotential rows
        }
    }
}

// Third-order basis contraction with M, Y read from the GEMM outputs
// Mw/Yw [spin][walker][n_basis][n] (type T).
template <typename T, bool kE>
__global__ void __launch_bounds__(256) k_force_contract(DevSys s, DevWalkers wk, int w0, int W, const T* Mw,
                                                        const T* Yw, const double* gJw, const double* accw,
                                                        double* dEL, double* dlog, double* gEdet) {
    extern __shared__ double sm[];
    const int wl = blockIdx.x, w = w0 + wl;
    if (wl >= W) return;
    const int N = s.N, nu = s.n_up, nn = s.n_nuc, nb = s.n_basis;
    const ForceHead<T> h(sm, N, nn);
    double* acc = h.acc;
    double* gEs = (double*)((unsigned char*)sm + ((force_head_bytes<T>(N, nn) + 15) & ~(size_t)15));
    force_load_positions(h, wk.R + (size_t)w * 3 * N, N);
    if constexpr (kE)
        for (int q = threadIdx.x; q < 3 * N; q += blockDim.x) gEs[q] = 0.0;
    for (int q = threadIdx.x; q < 3 * N; q += blockDim.x) h.gJ[q] = T(gJw[(size_t)wl * 3 * N + q]);
    for (int q = threadIdx.x; q < 6 * nn; q += blockDim.x) acc[q] = accw[(size_t)wl * 6 * nn + q];
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int spin = 0; spin < 2; ++spin) {
        const int n = spin ? s.n_dn : nu;
        if (n == 0) continue;
        const int i0 = spin ? nu : 0;
        const T* M = Mw + ((size_t)(spin * W + wl)) * nb * n;
        const T* Y = Yw + ((size_t)(spin * W + wl)) * nb * n;
        // warp per run of shells on one centre, lanes over electrons: the
        // electron-centre offset is formed once per run, term sums in T, one
        // FP64 atomic per run and component
        for (int run = wid; run < s.n_run; run += nw) {
            const int sh0 = s.run_sh[run], sh1 = s.run_sh[run + 1];
            const int ctr = s.shell[sh0].x;
            T v[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
            for (int i = lane; i < n; i += 32) {
                const T x[3] = {off_en(h, s, i0 + i, ctr, 0), off_en(h, s, i0 + i, ctr, 1),
                                off_en(h, s, i0 + i, ctr, 2)};
                const T t = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
                const T gj[3] = {h.gJ[3 * (i0 + i)], h.gJ[3 * (i0 + i) + 1], h.gJ[3 * (i0 + i) + 2]};
                T ve[3] = {T(0), T(0), T(0)};
                for (int sh = sh0; sh < sh1; ++sh) {
                    const int4 d = s.shell[sh];
                    const int l = d.y & 0xff, pure = d.y >> 8;
                    const int nf = shell_nfn(l, pure);
                    const int fl = s.shell_fn[sh];
                    T f0, f1, f2, f3;
                    radial<T, true>(sys_alpha<T>(s), sys_cn<T>(s), d.z, d.w, t, f0, f1, f2, f3);
                    if (f0 == T(0) && f1 == T(0) && f2 == T(0) && f3 == T(0)) continue;  // screened
                    T vt[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
                    shell_terms_any<T>(l, pure, nf, x, f0, f1, f2, f3, gj, M + (size_t)fl * n + i,
                                       Y + (size_t)fl * n + i, n, vt);
#pragma unroll
                    for (int q = 0; q < 6; ++q) v[q] += vt[q];
                    if constexpr (kE)
#pragma unroll
                        for (int q = 0; q < 3; ++q) ve[q] += vt[q];
                }
                if constexpr (kE)
#pragma unroll
                    for (int q = 0; q < 3; ++q) atomicAdd(&gEs[3 * (i0 + i) + q], -double(ve[q]));
            }
            for (int q = 0; q < 6; ++q) v[q] = warp_sum(v[q]);
            if (lane == 0)
                for (int q = 0; q < 6; ++q) atomicAdd(&acc[6 * ctr + q], q < 3 ? double(v[q]) : -double(v[q]));
        }
    }
    __syncthreads();
    for (int q = threadIdx.x; q < 3 * nn; q += blockDim.x) {
        const int a = q / 3, c = q - 3 * a;
        dEL[(size_t)w * 3 * nn + q] = acc[6 * a + c] + (wk.nlF ? wk.nlF[(size_t)w * 3 * nn + q] : 0.0);
        dlog[(size_t)w * 3 * nn + q] = acc[6 * a + 3 + c];
    }
    if constexpr (kE)
        for (int q = threadIdx.x; q < 3 * N; q += blockDim.x) gEdet[(size_t)w * 3 * N + q] = gEs[q];
}

// gtot (may be null): grad_i ln|psi| [W][N][3] of the space-warp form.
template <typename T>
cudaError_t launch_force_prep(const DevSys& s, const DevWalkers& wk, int w0, int W, const double* dvnn, void* Bw,
                              double* gJw, double* accw, double* gtot, cudaStream_t st) {
    if (W == 0) return cudaSuccess;
    const size_t smem = force_head_bytes<T>(s.N, s.n_nuc);
    if (gtot) {
        if (smem > 48 * 1024) {
            cudaError_t e =
                cudaFuncSetAttribute(k_force_prep<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
        }
        k_force_prep<T, true><<<W, 256, smem, st>>>(s, wk, w0, W, dvnn, (T*)Bw, gJw, accw, gtot);
        return cudaGetLastError();
    }
    if (smem > 48 * 1024) {
        cudaError_t e =
            cudaFuncSetAttribute(k_force_prep<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    k_force_prep<T, false><<<W, 256, smem, st>>>(s, wk, w0, W, dvnn, (T*)Bw, gJw, accw, nullptr);
    return cudaGetLastError();
}

// gEdet (may be null): determinant part of dE_L/dr_i [W][N][3] (walker
// index w0 + local) of the space-warp form.
template <typename T>
cudaError_t launch_force_contract(const DevSys& s, const DevWalkers& wk, int w0, int W, const void* Mw, const void* Yw,
                                  const double* gJw, const double* accw, double* dEL, double* dlog, double* gEdet,
                                  cudaStream_t st) {
    if (W == 0) return cudaSuccess;
    if (gEdet) {
        const size_t smem = ((force_head_bytes<T>(s.N, s.n_nuc) + 15) & ~(size_t)15) + sizeof(double) * 3 * (size_t)s.N;
        if (smem > 48 * 1024) {
            cudaError_t e = cudaFuncSetAttribute(k_force_contract<T, true>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
        }
        k_force_contract<T, true><<<W, 256, smem, st>>>(s, wk, w0, W, (const T*)Mw, (const T*)Yw, gJw, accw, dEL,
                                                         dlog, gEdet);
        return cudaGetLastError();
    }
    const size_t smem = force_head_bytes<T>(s.N, s.n_nuc);
    if (smem > 48 * 1024) {
        cudaError_t e =
            cudaFuncSetAttribute(k_force_contract<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    k_force_contract<T, false><<<W, 256, smem, st>>>(s, wk, w0, W, (const T*)Mw, (const T*)Yw, gJw, accw, dEL, dlog,
                                                      nullptr);
    return cudaGetLastError();
}

template cudaError_t launch_force_prep<double>(const DevSys&, const DevWalkers&, int, int, const double*, void*,
                                               double*, double*, double*, cudaStream_t);
template cudaError_t launch_force_prep<float>(const DevSys&, const DevWalkers&, int, int, const double*, void*,
                                              double*, double*, double*, cudaStream_t);
template cudaError_t launch_force_contract<double>(const DevSys&, const DevWalkers&, int, int, const void*,
                                                   const void*, const double*, const double*, double*, double*,
                                                   double*, cudaStream_t);
template cudaError_t launch_force_contract<float>(const DevSys&, const DevWalkers&, int, int, const void*, const void*,
                                                  const double*, const double*, double*, double*, double*,
                                                  cudaStream_t);

// gEdet, gtot (both null, or both [W][N][3]): the space-warp form's
// per-electron outputs (see force_walker).
template <typename T>
cudaError_t launch_force(const DevSys& s, const DevWalkers& wk, int W, const double* dvnn, double* Bscr,
                         double* Pscr, double* dEL, double* dlog, double* gEdet, double* gtot, cudaStream_t st) {
    if (W == 0) return cudaSuccess;
    const int nmax = s.n_up > s.n_dn ? s.n_up : s.n_dn;
    if (gEdet) {
        const size_t smem = force_smem_e<T>(s.N, s.n_nuc, nmax, true);
        cudaError_t e = cudaFuncSetAttribute(k_force<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_force<T, true><<<W, 256, smem, st>>>(s, wk, W, dvnn, Bscr, Pscr, dEL, dlog, gEdet, gtot);
        return cudaGetLastError();
    }
    const size_t smem = force_smem<T>(s.N, s.n_nuc, nmax);
    cudaError_t e = cudaFuncSetAttribute(k_force<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_force<T, false><<<W, 256, smem, st>>>(s, wk, W, dvnn, Bscr, Pscr, dEL, dlog, nullptr, nullptr);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------
// Space warp (Filippi and Umrigar 2000; the paper adapts it to its batched
// force path, Sec. "Single Determinant QMC Forces").  When nucleus a moves
// by dR every electron i moves with it by omega_a(r_i) dR, with
//   omega_a(r) = F(|r - R_a|) / sum_b F(|r - R_b|),  F(d) = d^-4,
// which removes the divergent fluctuations of dE_L/dR_a from electrons near
// nucleus a.  Along coordinate c the warped derivatives are
//   dE_L^w/dR_ac      = dE_L/dR_ac + sum_i omega_a(r_i) dE_L/dr_ic,
//   d ln|psi|^w/dR_ac = d ln|psi|/dR_ac + sum_i omega_a(r_i) d ln|psi|/dr_ic
//                       + 1/2 sum_i d omega_a(r_i)/dr_ic     (Jacobian),
// and they replace the unwarped ones in the force estimator.  The force
// kernels (kE) leave the determinant part of dE_L/dr_i and grad_i ln|psi|;
// this kernel adds the Jastrow and potential parts of dE_L/dr_i,
//   -1/2 d/dr_i sum_j lap_j J - sum_j grad_j ln|psi| . d(grad_j J)/dr_i + dV/dr_i,
// and the warp.  One CTA per walker: a warp per electron over its partners
// (pair terms in T, per-electron sums in T, totals in FP64), then a warp
// per nucleus over the electrons.
// ---------------------------------------------------------------------
template <typename T>
__host__ __device__ inline size_t space_warp_smem(int N, int nn) {
    const size_t b = (force_head_bytes<T>(N, nn) + 15) & ~(size_t)15;
    return b + sizeof(double) * 3 * (size_t)N + sizeof(T) * (size_t)N;
}

// Space warp of walker w (body of k_space_warp and k_space_warp_batch).
// sm: space_warp_smem bytes of dynamic shared memory.
template <typename T>
__device__ __forceinline__ void space_warp_walker(const DevSys& s, const DevWalkers& wk, int w, const double* gEdet,
                                                  const double* gtot, double* dEL, double* dlog, double* sm) {
    const int N = s.N, nu = s.n_up, nn = s.n_nuc;
    const ForceHead<T> h(sm, N, nn);
    double* gEs = (double*)((unsigned char*)sm + ((force_head_bytes<T>(N, nn) + 15) & ~(size_t)15));
    T* Sk = (T*)(gEs + 3 * N);   // [N]    sum_b F(|r_k - R_b|)
    T* gS = h.gJ;                // [N][3] its gradient
    force_load_positions(h, wk.R + (size_t)w * 3 * N, N);
    for (int q = threadIdx.x; q < 3 * N; q += blockDim.x) {
        h.gt[q] = T(gtot[(size_t)w * 3 * N + q]);
        gEs[q] = gEdet[(size_t)w * 3 * N + q];
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;

    // Jastrow and potential terms of dE_L/dr_k.  For a pair term u(r),
    // x = r_k - r_j: d(grad u)/dx = hx x x^T + (u'/r) I with
    // hx = (u'' - u'/r)/r^2, d(u'' + 2u'/r)/dx = d3 x with
    // d3 = (u''' + 2u''/r - 2u'/r^2)/r.  An e-e pair changes both electrons'
    // Laplacian terms and both gradients (the partner's with opposite sign).
    for (int k = wid; k < N; k += nw) {
        T v[3] = {T(0), T(0), T(0)};
        const T gk[3] = {h.gt[3 * k], h.gt[3 * k + 1], h.gt[3 * k + 2]};
        for (int j = lane; j < N + nn; j += 32) {
            if (j == k) continue;
            const bool nuc = j >= N;
            T x[3], g[3], a, b, qv, lapf;
            if (!nuc) {
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    x[c] = off_ee(h, k, j, c);
                    g[c] = gk[c] - h.gt[3 * j + c];
                }
                a = T(((k < nu) == (j < nu)) ? s.a_par : s.a_anti);
                b = T(s.b_ee);
                qv = T(1);       // V_ee = 1/r
                lapf = T(1);
            } else {
                const int c0 = j - N;
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    x[c] = off_en(h, s, k, c0, c);
                    g[c] = gk[c];
                }
                a = T(s.a_en[c0]);
                b = T(s.b_en);
                qv = T(-s.Z[c0]);   // V_en = -Z/r
                lapf = T(0.5);
            }
            const T r2 = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
            const T ir = rsqrt_t(r2), r = r2 * ir;
            T u, du, d2u, d3u;
            pade3<T>(a, b, r, u, du, d2u, d3u);
            const T hx = (d2u - du * ir) * ir * ir;
            const T d3 = (d3u + T(2) * d2u * ir - T(2) * du * ir * ir) * ir;
            const T gdot = g[0] * x[0] + g[1] * x[1] + g[2] * x[2];
            const T vr3 = qv * ir * ir * ir;
#pragma unroll
            for (int c = 0; c < 3; ++c) v[c] += -(lapf * d3 + hx * gdot + vr3) * x[c] - du * ir * g[c];
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) v[c] = warp_sum(v[c]);
        if (lane == 0)
            for (int c = 0; c < 3; ++c) gEs[3 * k + c] += double(v[c]);
    }
    // warp normalisation per electron: S = sum_b F_b, grad S = sum_b -4 x_b F_b / d_b^2
    for (int k = threadIdx.x; k < N; k += blockDim.x) {
        T S = T(0), g[3] = {T(0), T(0), T(0)};
        for (int b = 0; b < nn; ++b) {
            T x[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) x[c] = off_en(h, s, k, b, c);
            const T d2 = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
            const T id2 = T(1) / d2;
            const T F = id2 * id2;
            S += F;
#pragma unroll
            for (int c = 0; c < 3; ++c) g[c] += T(-4) * x[c] * F * id2;
        }
        Sk[k] = S;
#pragma unroll
        for (int c = 0; c < 3; ++c) gS[3 * k + c] = g[c];
    }
    __syncthreads();
    // warp of every electron onto nucleus a: grad omega_a = (grad F_a - omega_a grad S) / S
    for (int a = wid; a < nn; a += nw) {
        double dE[3] = {0.0, 0.0, 0.0}, dL[3] = {0.0, 0.0, 0.0};
        for (int k = lane; k < N; k += 32) {
            T x[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) x[c] = off_en(h, s, k, a, c);
            const T d2 = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
            const T id2 = T(1) / d2;
            const T F = id2 * id2;
            const T iS = T(1) / Sk[k];
            const T om = F * iS;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const T gom = (T(-4) * x[c] * F * id2 - om * gS[3 * k + c]) * iS;
                dE[c] += double(om) * gEs[3 * k + c];
                dL[c] += double(om * h.gt[3 * k + c] + T(0.5) * gom);
            }
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            dE[c] = warp_sum(dE[c]);
            dL[c] = warp_sum(dL[c]);
        }
        if (lane == 0)
            for (int c = 0; c < 3; ++c) {
                dEL[(size_t)w * 3 * nn + 3 * a + c] += dE[c];
                dlog[(size_t)w * 3 * nn + 3 * a + c] += dL[c];
            }
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_space_warp(DevSys s, DevWalkers wk, int W, const double* gEdet,
                                                    const double* gtot, double* dEL, double* dlog) {
    extern __shared__ double sm[];
    const int w = blockIdx.x;
    if (w >= W) return;
    space_warp_walker<T>(s, wk, w, gEdet, gtot, dEL, dlog, sm);
}

template <typename T>
cudaError_t launch_space_warp(const DevSys& s, const DevWalkers& wk, int W, const double* gEdet, const double* gtot,
                              double* dEL, double* dlog, cudaStream_t st) {
    if (W == 0) return cudaSuccess;
    const size_t smem = space_warp_smem<T>(s.N, s.n_nuc);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_space_warp<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    k_space_warp<T><<<W, 256, smem, st>>>(s, wk, W, gEdet, gtot, dEL, dlog);
    return cudaGetLastError();
}

template cudaError_t launch_space_warp<double>(const DevSys&, const DevWalkers&, int, const double*, const double*,
                                               double*, double*, cudaStream_t);
template cudaError_t launch_space_warp<float>(const DevSys&, const DevWalkers&, int, const double*, const double*,
                                              double*, double*, cudaStream_t);

// Batched form: persistent CTAs over the walkers of every system.
// kWarp: some member of the batch has the space warp on (its walkers also
// get the per-electron outputs); batches without it run the plain body.
template <typename T, bool kWarp>
__global__ void __launch_bounds__(256, 2) k_force_batch(const BatchSys* __restrict__ sys, BatchPlan* plan,
                                                        int parity, int ctr) {
    extern __shared__ double sm[];
    __shared__ BatchSys bs;
    __shared__ int s_sys, s_idx;
    for (;;) {
        if (threadIdx.x == 0) batch_next(plan, kUnitWalker, ctr, &s_sys, &s_idx);
        __syncthreads();
        const int q = s_sys;
        if (q < 0) break;
        batch_load(&bs, sys + q);
        __syncthreads();
        bool warped = false;
        if constexpr (kWarp) {
            if (bs.space_warp) {
                force_walker<T, true>(bs.s, bs.wk[parity], s_idx, bs.dvnn, bs.Bscr, bs.Pscr, bs.dEL, bs.dlog, sm,
                                      bs.gEdet, bs.gtot);
                warped = true;
            }
        }
        if (!warped) force_walker<T>(bs.s, bs.wk[parity], s_idx, bs.dvnn, bs.Bscr, bs.Pscr, bs.dEL, bs.dlog, sm);
        __syncthreads();
    }
}

size_t force_batch_smem_bytes(const DevSys& s, int elem, int space_warp) {
    const int nmax = s.n_up > s.n_dn ? s.n_up : s.n_dn;
    return elem == 4 ? force_smem_e<float>(s.N, s.n_nuc, nmax, space_warp != 0)
                     : force_smem_e<double>(s.N, s.n_nuc, nmax, space_warp != 0);
}

// Batched space warp: persistent CTAs over the walkers of every system; the
// walkers of systems without the warp are skipped.
template <typename T>
__global__ void __launch_bounds__(256) k_space_warp_batch(const BatchSys* __restrict__ sys, BatchPlan* plan,
                                                          int parity, int ctr) {
    extern __shared__ double sm[];
    __shared__ BatchSys bs;
    __shared__ int s_sys, s_idx;
    for (;;) {
        if (threadIdx.x == 0) batch_next(plan, kUnitWalker, ctr, &s_sys, &s_idx);
        __syncthreads();
        const int q = s_sys;
        if (q < 0) break;
        batch_load(&bs, sys + q);
        __syncthreads();
        if (bs.space_warp)
            space_warp_walker<T>(bs.s, bs.wk[parity], s_idx, bs.gEdet, bs.gtot, bs.dEL, bs.dlog, sm);
        __syncthreads();
    }
}

size_t space_warp_batch_smem_bytes(const DevSys& s, int elem) {
    return elem == 4 ? space_warp_smem<float>(s.N, s.n_nuc) : space_warp_smem<double>(s.N, s.n_nuc);
}

template <typename T>
int space_warp_batch_prepare(size_t smem) {
    int nb = 0;
    if (cudaFuncSetAttribute(k_space_warp_batch<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_space_warp_batch<T>, 256, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return nb;
}

template <typename T>
cudaError_t launch_space_warp_batch(const BatchSys* sys, BatchPlan* plan, int parity, int ctr, int grid, size_t smem,
                                    cudaStream_t st) {
    k_space_warp_batch<T><<<grid, 256, smem, st>>>(sys, plan, parity, ctr);
    return cudaGetLastError();
}

template int space_warp_batch_prepare<double>(size_t);
template int space_warp_batch_prepare<float>(size_t);
template cudaError_t launch_space_warp_batch<double>(const BatchSys*, BatchPlan*, int, int, int, size_t,
                                                     cudaStream_t);
template cudaError_t launch_space_warp_batch<float>(const BatchSys*, BatchPlan*, int, int, int, size_t, cudaStream_t);

template <typename T>
int force_batch_prepare(size_t smem, int any_warp) {
    int nb = 0;
    const void* f = any_warp ? (const void*)k_force_batch<T, true> : (const void*)k_force_batch<T, false>;
    if (cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, f, 256, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return nb;
}

template <typename T>
cudaError_t launch_force_batch(const BatchSys* sys, BatchPlan* plan, int parity, int ctr, int grid, size_t smem,
                               int any_warp, cudaStream_t st) {
    if (any_warp)
        k_force_batch<T, true><<<grid, 256, smem, st>>>(sys, plan, parity, ctr);
    else
        k_force_batch<T, false><<<grid, 256, smem, st>>>(sys, plan, parity, ctr);
    return cudaGetLastError();
}

template int force_batch_prepare<double>(size_t, int);
template int force_batch_prepare<float>(size_t, int);
template cudaError_t launch_force_batch<double>(const BatchSys*, BatchPlan*, int, int, int, size_t, int,
                                                cudaStream_t);
template cudaError_t launch_force_batch<float>(const BatchSys*, BatchPlan*, int, int, int, size_t, int, cudaStream_t);

template cudaError_t launch_force<double>(const DevSys&, const DevWalkers&, int, const double*, double*, double*,
                                          double*, double*, double*, double*, cudaStream_t);
template cudaError_t launch_force<float>(const DevSys&, const DevWalkers&, int, const double*, double*, double*,
                                         double*, double*, double*, double*, cudaStream_t);

}  // namespace qmc
