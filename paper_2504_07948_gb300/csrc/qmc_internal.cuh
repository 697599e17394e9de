// Internal declarations shared by the CUDA translation units of libqmc.
//
// Layout conventions (walker-major, all walkers of one array contiguous):
//   R      [cap][N][3]          double   electron positions, up-spin block first
//   AinvT  [cap][n_s][n_s]      T        transposed inverse Slater matrix of
//                                        spin s: AinvT[e][j] = (A^-1)[j][e], so
//                                        the column of A^-1 that an electron's
//                                        ratio needs is one contiguous row
//   G      [cap][n_s][4][n_s]   T        cached orbital gradient (3 rows) and
//                                        Laplacian (1 row) at each electron
//   Ascr   [cap][n_s][n_s]      double   recompute scratch (A itself)
//   logdet, sgn [cap][2]        double
//   eloc, weight [cap]          double
// A_ij = phi_j(r_i) (row = electron, column = orbital), as in Sec. "Single
// Determinant QMC Forces" of the paper.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace qmc {

constexpr int kMaxWarps = 32;

// Error flags raised by kernels (bitmask in device memory).
enum : unsigned { kErrSingular = 1u, kErrNonFinite = 2u, kErrPopulation = 4u, kErrTimeout = 8u };

struct DevSys {
    int n_nuc, n_up, n_dn, N;
    int n_shell, n_basis, n_prim;
    const double* Z;      // [n_nuc]
    const double* Rn;     // [n_nuc][3]
    const float* Rn_hi;   // [n_nuc][3] float(Rn) and float(Rn - float(Rn)): with the same split
    const float* Rn_lo;   // of an electron position, FP32 offsets keep FP32 relative accuracy
    const double* a_en;   // [n_nuc]
    double a_anti, a_par, b_ee, b_en;
    double vnn;           // nuclear repulsion
    const int4* shell;    // (center, l | pure << 8, first_prim, nprim)
    const int* shell_fn;  // first basis function of each shell
    int n_run;            // maximal runs of consecutive shells on one centre
    const int* run_sh;    // [n_run + 1] first shell of each run
    const double* shell_amin;   // [n_shell] smallest exponent of each shell (+inf if none):
    const float* shell_amin_f;  // the shell is screened where shell_amin * r^2 > kScreenExponent
    const double* alpha;  // [n_prim]
    const double* cn;     // [n_prim] normalised contraction coefficients
    const float* alpha_f;
    const float* cn_f;
    const double* C[2];   // [n_basis][n_s] occupied orbital coefficients per spin
    const float* C_f[2];
    // Multi-determinant expansion (table method); msd == 0: one determinant.
    // Spin strings are stored relative to the reference determinant: e
    // holes (positions 0..n_s-1 in the reference orbital list, ascending)
    // and e particles (positions 0..n_vir-1 in the active virtual list,
    // ascending), with the sign of the permutation that sorts the reference
    // list after the in-place replacement hole_a -> particle_a.
    int msd;
    int n_vir[2];             // active virtual orbitals per spin
    const double* Cv[2];      // [n_basis][n_vir] virtual orbital coefficients
    const float* Cv_f[2];
    int n_str[2];             // unique strings per spin (string 0 = reference)
    const int4* str[2];       // x = e | (phase < 0) << 8, y = holes, z = particles (4 x 8 bit)
    const int* csr_off[2];    // [n_str + 1]: the determinants that contain each string
    const int* csr_other[2];  // string of the other spin in each of those determinants
    const double* csr_c[2];   // and its CI coefficient
    // three-body (electron-electron-nucleus) Jastrow, n3 == 0: none.
    // J3 = sum_a sum_{i<j} sum_k c3[a][k] (s_ia^m s_ja^n + s_ia^n s_ja^m) s_ij^o,
    // s(r) = r / (1 + b3 r), (m, n, o) = e3[3k .. 3k+2]
    int n3;
    const int* e3;       // [n3][3]
    const double* c3;    // [n_nuc][n3]
    double b3;
    // semi-local pseudopotential, npp == 0: none.  Radial terms sorted by
    // nucleus (pp_off[a] .. pp_off[a + 1] - 1 are nucleus a's), each
    // beta r^(n-2) exp(-alpha r^2) in channel l (-1: local, added to -Z/r
    // for every electron; l = 0..3: projector on angular momentum l about
    // the nucleus for electrons within pp_rcut[a]).  The non-local matrix
    // elements use the quadrature rule (pp_quad, pp_qw), rotated per
    // (walker slot, nucleus) when pp_rotate != 0.
    int npp;
    const int* pp_off;       // [n_nuc + 1]
    const int2* pp_ln;       // [npp] (l, n)
    const double2* pp_ab;    // [npp] (alpha, beta)
    const float2* pp_ab_f;
    const double* pp_rcut;   // [n_nuc]
    int n_ecp;               // nuclei with a non-local channel
    const int* ecp_nuc;      // [n_ecp]
    const double* CT[2];     // [n_s][n_basis] occupied coefficients, orbital-major (coalesced over the basis)
    const float* CT_f[2];
    const float* a_en_f;     // [n_nuc]
    const int* shell_by_type;  // [n_shell] shells sorted by (l, pure), stable
    int pp_nq, pp_rotate;
    const double* pp_quad;   // [pp_nq][3] unit vectors
    const double* pp_qw;     // [pp_nq] weights (sum 1)
};

constexpr int kMaxExcitation = 4;
constexpr int kMaxVirtual = 64;

// Per-walker state.  Pointers are to element 0 of walker 0.
struct DevWalkers {
    int cap;
    double* R;
    void* Ainv[2];
    void* G[2];
    double* Ascr[2];
    double* logdet;
    double* sgn;
    double* eloc;
    double* weight;
    unsigned long long* n_acc;   // one counter of accepted moves (statistics)
    unsigned* err;               // device error flags of the handle
    int* refresh;                // [cap] walkers whose state must be rebuilt in FP64 (see k_sweep_msd)
    // multi-determinant state (msd only)
    void* Av[2];     // [cap][n_s][n_vir]      virtual orbital values at each electron
    void* Gv[2];     // [cap][n_s][4][n_vir]   their gradients and Laplacians
    void* Tt[2];     // [cap][n_s][n_vir]      table T = A0^-1 A_v (row = hole, column = particle)
    void* Rs[2];     // [cap][n_str]           string ratios D_u / D_0 (sign included)
    void* Rn[2];     // [cap][n_str]           ratios at a proposed move
    void* Cd[2];     // [cap][n_str]           sum over the string's dets of c_k R_other
    double* Ssum;    // [cap]                  S = sum_k c_k R_up R_dn
    // non-local pseudopotential terms of the ionic derivatives (set for the
    // force pass only, else null): rows of the non-local matrix B_NL per spin
    // [cap][n_s][n_s] (type T; B_NL[k][j] = sum over electron k's quadrature
    // points of c_p phi_j(r'_p)), and the direct derivative terms [cap][3 n_nuc]
    const void* nlB[2];
    const double* nlF;
};

// ---------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11).
// ---------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k.x += 0x9E3779B9u;
            k.y += 0xBB67AE85u;
        }
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    }
    return c;
}

// Uniform on (0,1) from one 32-bit word: (x + 1/2) 2^-32.
__device__ __forceinline__ double u01(uint32_t x) { return ((double)x + 0.5) * 2.3283064365386963e-10; }

// Stream layout: counter = (sweep, electron, walker slot, purpose);
// purpose 0 = three Box-Muller normals, 1 = acceptance uniform, 2 =
// branching uniform (electron field 0xFFFFFFFF).
__device__ __forceinline__ void draw_normals(uint2 key, uint32_t sweep, uint32_t e, uint32_t slot,
                                             double chi[3]) {
    const uint4 x = philox4x32_10(make_uint4(sweep, e, slot, 0u), key);
    const double r1 = sqrt(-2.0 * log(u01(x.x))), r2 = sqrt(-2.0 * log(u01(x.z)));
    double s1, c1, s2, c2;
    sincospi(2.0 * u01(x.y), &s1, &c1);
    sincospi(2.0 * u01(x.w), &s2, &c2);
    chi[0] = r1 * c1;
    chi[1] = r1 * s1;
    chi[2] = r2 * c2;
}

__device__ __forceinline__ double draw_uniform(uint2 key, uint32_t sweep, uint32_t e, uint32_t slot,
                                               uint32_t purpose) {
    return u01(philox4x32_10(make_uint4(sweep, e, slot, purpose), key).x);
}

// ---------------------------------------------------------------------
// Per-move helpers shared by the sweeps.
// ---------------------------------------------------------------------
// Umrigar-Nightingale-Runge drift cap (a = 1) in the cancellation-free
// form v * 2 / (1 + sqrt(1 + 2 v^2 tau)).
__device__ __forceinline__ void capped_drift(const double g[3], double tau, double vb[3]) {
    const double v2 = g[0] * g[0] + g[1] * g[1] + g[2] * g[2];
    const double f = 2.0 / (1.0 + sqrt(1.0 + 2.0 * v2 * tau));
    vb[0] = f * g[0];
    vb[1] = f * g[1];
    vb[2] = f * g[2];
}

__device__ __forceinline__ double rsqrt_t(double v) { return rsqrt(v); }
__device__ __forceinline__ float rsqrt_t(float v) { return rsqrtf(v); }

// Proposal normals in the precision of the form: FP64 (the stream both the
// FP64 form and the oracle use) or FP32 Box-Muller from the same words.
template <typename T>
__device__ __forceinline__ void draw_normals_t(uint2 key, uint32_t sweep, uint32_t e, uint32_t slot, double chi[3]);
template <>
__device__ __forceinline__ void draw_normals_t<double>(uint2 key, uint32_t sweep, uint32_t e, uint32_t slot,
                                                       double chi[3]) {
    draw_normals(key, sweep, e, slot, chi);
}
template <>
__device__ __forceinline__ void draw_normals_t<float>(uint2 key, uint32_t sweep, uint32_t e, uint32_t slot,
                                                      double chi[3]) {
    const uint4 x = philox4x32_10(make_uint4(sweep, e, slot, 0u), key);
    const float k = 2.3283064365386963e-10f;
    const float r1 = sqrtf(-2.0f * logf(((float)x.x + 0.5f) * k)), r2 = sqrtf(-2.0f * logf(((float)x.z + 0.5f) * k));
    float s1, c1, s2, c2;
    sincospif(2.0f * ((float)x.y + 0.5f) * k, &s1, &c1);
    sincospif(2.0f * ((float)x.w + 0.5f) * k, &s2, &c2);
    chi[0] = r1 * c1;
    chi[1] = r1 * s1;
    chi[2] = r2 * c2;
}

// ---------------------------------------------------------------------
// Thread-0 steps of one move (the serial part of every sweep).
//
// propose_move: UNR-capped drift of the gradient g, normals of the (sweep,
// electron, slot) stream, r' = r + tau vb + sqrt(tau) chi; writes r' to
// scal[0..2] and vb to scal[3..5].
// accept_move: ratio rho, gradient at r' (determinant part gd / rho plus
// Jastrow part gj), Jastrow change dJ; Green's-function ratio of the drifted
// moves and the Metropolis decision (fixed node: rho > 0).
// The FP64 form does all of it in double.  The mixed form keeps positions in
// double but evaluates drifts, Green's function and acceptance probability
// in float: on GB300 a double instruction costs the FP64 pipe 64 times a
// float one, and this serial section otherwise holds every other thread of
// the CTA at the next barrier.
// ---------------------------------------------------------------------
__device__ __forceinline__ void draw_normals_f(uint2 key, uint32_t sweep, uint32_t e, uint32_t slot, float chi[3]) {
    const uint4 x = philox4x32_10(make_uint4(sweep, e, slot, 0u), key);
    const float k = 2.3283064365386963e-10f;
    const float r1 = sqrtf(-2.0f * logf(((float)x.x + 0.5f) * k)), r2 = sqrtf(-2.0f * logf(((float)x.z + 0.5f) * k));
    float s1, c1, s2, c2;
    sincospif(2.0f * ((float)x.y + 0.5f) * k, &s1, &c1);
    sincospif(2.0f * ((float)x.w + 0.5f) * k, &s2, &c2);
    chi[0] = r1 * c1;
    chi[1] = r1 * s1;
    chi[2] = r2 * c2;
}

template <typename T>
__device__ __forceinline__ void propose_move(const T g[3], double tau, const double r[3], uint2 key, uint32_t sweep,
                                             uint32_t e, uint32_t slot, double* scal) {
    if constexpr (sizeof(T) == 8) {
        const double gd[3] = {g[0], g[1], g[2]};
        double vb[3], chi[3];
        capped_drift(gd, tau, vb);
        draw_normals(key, sweep, e, slot, chi);
        const double sqt = sqrt(tau);
        for (int c = 0; c < 3; ++c) {
            scal[c] = r[c] + tau * vb[c] + sqt * chi[c];
            scal[3 + c] = vb[c];
        }
    } else {
        const float tf = (float)tau;
        const float v2 = g[0] * g[0] + g[1] * g[1] + g[2] * g[2];
        const float f = 2.0f / (1.0f + sqrtf(1.0f + 2.0f * v2 * tf));
        float chi[3];
        draw_normals_f(key, sweep, e, slot, chi);
        const float sq = sqrtf(tf);
        for (int c = 0; c < 3; ++c) {
            const float vb = f * g[c];
            scal[c] = r[c] + (double)(tf * vb + sq * chi[c]);
            scal[3 + c] = (double)vb;
        }
    }
}

// FP64 proposal computed by lanes 0 and 1 of warp 0 together: each lane
// forms one Box-Muller pair from the same Philox words as draw_normals (lane
// 0: words 0, 1; lane 1: words 2, 3), so the logarithm, square root and
// sine/cosine of the two pairs issue once instead of twice (each FP64
// instruction costs its warp the same with one or two lanes active).  The
// result equals propose_move<double>; lane 0 writes it.  g is read by lane 0
// only.
__device__ __forceinline__ void propose_move_fp64_pair(const double g[3], double tau, const double r[3], uint2 key,
                                                       uint32_t sweep, uint32_t e, uint32_t slot, double* scal) {
    const int lane = threadIdx.x & 31;
    const uint4 x = philox4x32_10(make_uint4(sweep, e, slot, 0u), key);
    const double rr = sqrt(-2.0 * log(u01(lane ? x.z : x.x)));
    double sn, cs;
    sincospi(2.0 * u01(lane ? x.w : x.y), &sn, &cs);
    const double chi2 = __shfl_sync(0x3u, rr * cs, 1);
    if (lane == 0) {
        double vb[3];
        capped_drift(g, tau, vb);
        const double chi[3] = {rr * cs, rr * sn, chi2};
        const double sqt = sqrt(tau);
        for (int c = 0; c < 3; ++c) {
            scal[c] = r[c] + tau * vb[c] + sqt * chi[c];
            scal[3 + c] = vb[c];
        }
    }
}

// Metropolis test of a move with wavefunction ratio `ratio`, full gradient
// of ln|psi| at r' g, Jastrow change dJ (see propose_move for precisions).
template <typename T>
__device__ __forceinline__ int accept_move_g(T ratio, const T g[3], T dJ, double tau, const double ro[3],
                                             const double rn[3], const double* vb_old, uint2 key, uint32_t sweep,
                                             uint32_t e, uint32_t slot) {
    if constexpr (sizeof(T) == 8) {
        if (!(ratio > 0.0 && isfinite(ratio))) return 0;
        double vbn[3];
        capped_drift(g, tau, vbn);
        double fwd = 0.0, bwd = 0.0;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const double f = rn[c] - ro[c] - tau * vb_old[c];
            const double bk = ro[c] - rn[c] - tau * vbn[c];
            fwd += f * f;
            bwd += bk * bk;
        }
        const double lnp = 2.0 * log(ratio) + 2.0 * dJ - (bwd - fwd) / (2.0 * tau);
        const double u = draw_uniform(key, sweep, e, slot, 1u);
        return (lnp >= 0.0) || (u < exp(lnp));
    } else {
        if (!(ratio > 0.0f && isfinite(ratio))) return 0;
        const float tf = (float)tau;
        const float v2 = g[0] * g[0] + g[1] * g[1] + g[2] * g[2];
        const float f = 2.0f / (1.0f + sqrtf(1.0f + 2.0f * v2 * tf));
        float fwd = 0.0f, bwd = 0.0f;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float d = (float)(rn[c] - ro[c]);
            const float fw = d - tf * (float)vb_old[c];
            const float bk = -d - tf * f * g[c];
            fwd += fw * fw;
            bwd += bk * bk;
        }
        const float lnp = 2.0f * logf(ratio) + 2.0f * dJ - (bwd - fwd) / (2.0f * tf);
        const uint4 x = philox4x32_10(make_uint4(sweep, e, slot, 1u), key);
        const float u = ((float)x.x + 0.5f) * 2.3283064365386963e-10f;
        return (lnp >= 0.0f) || (u < expf(lnp));
    }
}

// One determinant: ratio rho, determinant gradient gd / rho plus Jastrow
// gradient gj.
template <typename T>
__device__ __forceinline__ int accept_move(T rho, const T gd[3], const T gj[3], T dJ, double tau, const double ro[3],
                                           const double rn[3], const double* vb_old, uint2 key, uint32_t sweep,
                                           uint32_t e, uint32_t slot) {
    const T ir = T(1) / rho;
    T g[3];
    if constexpr (sizeof(T) == 8) {
        for (int c = 0; c < 3; ++c) g[c] = gd[c] / rho + gj[c];
    } else {
        for (int c = 0; c < 3; ++c) g[c] = gd[c] * ir + gj[c];
    }
    return accept_move_g<T>(rho, g, dJ, tau, ro, rn, vb_old, key, sweep, e, slot);
}

// Mixed-form move of the Sherman-Morrison sweep: the same arithmetic as
// propose_move<float> / accept_move<float>, with the results every thread
// needs left as floats in fs: r' as hi/lo floats [0..5], the step r' - r
// [6..8] and the drift at r [9..11].  The acceptance test reads the step and
// drift back instead of forming r' - r in FP64 (the step is the float that
// was added to r, so both agree).
__device__ __forceinline__ void propose_move_mixed(const float g[3], double tau, const double r[3], uint2 key,
                                                   uint32_t sweep, uint32_t e, uint32_t slot, double* scal,
                                                   float* fs) {
    const float tf = (float)tau;
    const float v2 = g[0] * g[0] + g[1] * g[1] + g[2] * g[2];
    const float f = 2.0f / (1.0f + sqrtf(1.0f + 2.0f * v2 * tf));
    float chi[3];
    draw_normals_f(key, sweep, e, slot, chi);
    const float sq = sqrtf(tf);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float vb = f * g[c];
        const float d = tf * vb + sq * chi[c];
        const double rn = r[c] + (double)d;
        const float hi = (float)rn;
        scal[c] = rn;
        fs[c] = hi;
        fs[3 + c] = (float)(rn - (double)hi);
        fs[6 + c] = d;
        fs[9 + c] = vb;
    }
}

__device__ __forceinline__ int accept_move_mixed(float rho, const float gd[3], const float gj[3], float dJ,
                                                 double tau, const float* fs, uint2 key, uint32_t sweep, uint32_t e,
                                                 uint32_t slot) {
    if (!(rho > 0.0f && isfinite(rho))) return 0;
    const float ir = 1.0f / rho;
    float g[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) g[c] = gd[c] * ir + gj[c];
    const float tf = (float)tau;
    const float v2 = g[0] * g[0] + g[1] * g[1] + g[2] * g[2];
    const float f = 2.0f / (1.0f + sqrtf(1.0f + 2.0f * v2 * tf));
    float fwd = 0.0f, bwd = 0.0f;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float d = fs[6 + c];
        const float fw = d - tf * fs[9 + c];
        const float bk = -d - tf * f * g[c];
        fwd += fw * fw;
        bwd += bk * bk;
    }
    const float lnp = 2.0f * logf(rho) + 2.0f * dJ - (bwd - fwd) / (2.0f * tf);
    const uint4 x = philox4x32_10(make_uint4(sweep, e, slot, 1u), key);
    const float u = ((float)x.x + 0.5f) * 2.3283064365386963e-10f;
    return (lnp >= 0.0f) || (u < expf(lnp));
}

// ---------------------------------------------------------------------
// Three-body (electron-electron-nucleus) Jastrow.  Scaled distance s(r) =
// r / (1 + b r) with s' = 1 / (1 + b r)^2, s'' = -2 b / (1 + b r)^3; a
// radial function F(s(r)) has grad F = F'(s) s' u (u the unit vector) and
// lap F = F''(s) s'^2 + F'(s) (s'' + 2 s' / r).
// ---------------------------------------------------------------------
struct SDist {
    double s, s1, l;   // s, s', s'' + 2 s' / r
    double u[3];       // unit vector
};
__device__ __forceinline__ SDist sdist(double b, double x, double y, double z) {
    SDist d;
    const double r2 = x * x + y * y + z * z;
    const double ir = rsqrt(r2), r = r2 * ir;
    const double q = 1.0 / (1.0 + b * r);
    d.s = r * q;
    d.s1 = q * q;
    d.l = -2.0 * b * q * q * q + 2.0 * d.s1 * ir;
    d.u[0] = x * ir;
    d.u[1] = y * ir;
    d.u[2] = z * ir;
    return d;
}
__device__ __forceinline__ double ipow_d(double x, int k) {
    double p = 1.0;
    for (int q = 0; q < k; ++q) p *= x;
    return p;
}
// One term (m, n, o) of nucleus a for electron i and partner j seen from
// electron i: value P Q, gradient in r_i and Laplacian in r_i (coefficient 1).
__device__ __forceinline__ void j3_term(int m, int n, int o, const SDist& xi, const SDist& xj, const SDist& y,
                                        double& val, double g[3], double& lap) {
    const double P = ipow_d(xi.s, m) * ipow_d(xj.s, n) + ipow_d(xi.s, n) * ipow_d(xj.s, m);
    const double Pi = (m ? m * ipow_d(xi.s, m - 1) : 0.0) * ipow_d(xj.s, n) +
                      (n ? n * ipow_d(xi.s, n - 1) : 0.0) * ipow_d(xj.s, m);
    const double Pii = (m > 1 ? m * (m - 1) * ipow_d(xi.s, m - 2) : 0.0) * ipow_d(xj.s, n) +
                       (n > 1 ? n * (n - 1) * ipow_d(xi.s, n - 2) : 0.0) * ipow_d(xj.s, m);
    const double Q = ipow_d(y.s, o);
    const double Q1 = o ? o * ipow_d(y.s, o - 1) : 0.0;
    const double Q2 = o > 1 ? o * (o - 1) * ipow_d(y.s, o - 2) : 0.0;
    val = P * Q;
    double dot = 0.0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        g[c] = Pi * Q * xi.s1 * xi.u[c] + P * Q1 * y.s1 * y.u[c];
        dot += xi.u[c] * y.u[c];
    }
    lap = Pii * Q * xi.s1 * xi.s1 + Pi * Q * xi.l + P * Q2 * y.s1 * y.s1 + P * Q1 * y.l + 2.0 * Pi * Q1 * xi.s1 * y.s1 * dot;
}
// ---------------------------------------------------------------------
// Pseudopotential radial terms beta r^(n-2) exp(-alpha r^2).
// ---------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T pp_term(const DevSys& s, int t, int n, T r) {
    T a, b;
    if constexpr (sizeof(T) == 8) {
        a = s.pp_ab[t].x;
        b = s.pp_ab[t].y;
    } else {
        a = s.pp_ab_f[t].x;
        b = s.pp_ab_f[t].y;
    }
    T rk = T(1);
    if (n >= 2) {
        for (int q = 2; q < n; ++q) rk *= r;
    } else {
        for (int q = n; q < 2; ++q) rk *= r;
        rk = T(1) / rk;
    }
    T e;
    if constexpr (sizeof(T) == 8) e = exp(-a * r * r);
    else e = expf(-a * r * r);
    return b * rk * e;
}
// d/dr of a radial term: beta exp(-alpha r^2) r^(n-2) ((n-2)/r - 2 alpha r).
template <typename T>
__device__ __forceinline__ T pp_term_dr(const DevSys& s, int t, int n, T r) {
    T a;
    if constexpr (sizeof(T) == 8) a = s.pp_ab[t].x;
    else a = s.pp_ab_f[t].x;
    return pp_term<T>(s, t, n, r) * (T(n - 2) / r - T(2) * a * r);
}
// Local terms (l = -1) of nucleus a at distance r.
template <typename T>
__device__ __forceinline__ T pp_local(const DevSys& s, int a, T r) {
    T v = T(0);
    for (int t = s.pp_off[a]; t < s.pp_off[a + 1]; ++t) {
        const int2 ln = s.pp_ln[t];
        if (ln.x == -1) v += pp_term<T>(s, t, ln.y, r);
    }
    return v;
}
// ---------------------------------------------------------------------
// Pade pair function u(r) = a r / (1 + b r) and radial derivatives.
// ---------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void pade(T a, T b, T r, T& u, T& du, T& d2u) {
    const T q = T(1) / (T(1) + b * r);
    u = a * r * q;
    du = a * q * q;
    d2u = T(-2) * a * b * q * q * q;
}

template <typename T>
__device__ __forceinline__ void pade3(T a, T b, T r, T& u, T& du, T& d2u, T& d3u) {
    const T q = T(1) / (T(1) + b * r);
    u = a * r * q;
    du = a * q * q;
    d2u = T(-2) * a * b * q * q * q;
    d3u = T(6) * a * b * b * q * q * q * q;
}

// ---------------------------------------------------------------------
// Contracted shell = P(x,y,z) * S(t), t = r^2, S(t) = sum_p c_p e^{-a_p t}.
// With f^(m) = d^m S / dt^m:  grad S = 2 x f',  lap S = 6 f' + 4 t f'',
// d_k d_q S = 4 x_k x_q f'' + 2 delta_kq f',
// d_q lap S = x_q (20 f'' + 8 t f''').
// Angular polynomials P have degree <= 2, so their Hessians are constant.
// ---------------------------------------------------------------------
template <typename T>
struct AngPoly {
    T P, Px, Py, Pz;      // value and gradient
    T Hxx, Hxy, Hxz, Hyy, Hyz, Hzz;  // constant Hessian
};

// Angular function fi of a shell (l, pure) at (x, y, z).
template <typename T>
__device__ __forceinline__ AngPoly<T> angular(int l, int pure, int fi, T x, T y, T z) {
    const T s3 = T(1.7320508075688772);
    AngPoly<T> a;
    a.Hxx = a.Hxy = a.Hxz = a.Hyy = a.Hyz = a.Hzz = T(0);
    if (l == 0) {
        a.P = T(1); a.Px = a.Py = a.Pz = T(0);
    } else if (l == 1) {
        a.P = fi == 0 ? x : (fi == 1 ? y : z);
        a.Px = fi == 0 ? T(1) : T(0);
        a.Py = fi == 1 ? T(1) : T(0);
        a.Pz = fi == 2 ? T(1) : T(0);
    } else if (pure) {
        switch (fi) {
            case 0:  // sqrt3 xy
                a.P = s3 * x * y; a.Px = s3 * y; a.Py = s3 * x; a.Pz = T(0); a.Hxy = s3; break;
            case 1:  // sqrt3 yz
                a.P = s3 * y * z; a.Px = T(0); a.Py = s3 * z; a.Pz = s3 * y; a.Hyz = s3; break;
            case 2:  // z^2 - (x^2 + y^2)/2
                a.P = z * z - T(0.5) * (x * x + y * y); a.Px = -x; a.Py = -y; a.Pz = T(2) * z;
                a.Hxx = T(-1); a.Hyy = T(-1); a.Hzz = T(2); break;
            case 3:  // sqrt3 xz
                a.P = s3 * x * z; a.Px = s3 * z; a.Py = T(0); a.Pz = s3 * x; a.Hxz = s3; break;
            default:  // sqrt3/2 (x^2 - y^2)
                a.P = T(0.5) * s3 * (x * x - y * y); a.Px = s3 * x; a.Py = -s3 * y; a.Pz = T(0);
                a.Hxx = s3; a.Hyy = -s3; break;
        }
    } else {
        switch (fi) {  // xx, xy, xz, yy, yz, zz relative to the (2,0,0) normalisation
            case 0: a.P = x * x; a.Px = T(2) * x; a.Py = a.Pz = T(0); a.Hxx = T(2); break;
            case 1: a.P = s3 * x * y; a.Px = s3 * y; a.Py = s3 * x; a.Pz = T(0); a.Hxy = s3; break;
            case 2: a.P = s3 * x * z; a.Px = s3 * z; a.Py = T(0); a.Pz = s3 * x; a.Hxz = s3; break;
            case 3: a.P = y * y; a.Py = T(2) * y; a.Px = a.Pz = T(0); a.Hyy = T(2); break;
            case 4: a.P = s3 * y * z; a.Px = T(0); a.Py = s3 * z; a.Pz = s3 * y; a.Hyz = s3; break;
            default: a.P = z * z; a.Pz = T(2) * z; a.Px = a.Py = T(0); a.Hzz = T(2); break;
        }
    }
    return a;
}

__host__ __device__ __forceinline__ int shell_nfn(int l, int pure) {
    return l == 0 ? 1 : (l == 1 ? 3 : (pure ? 5 : 6));
}

template <typename T>
__device__ __forceinline__ T dexp(T v);
template <>
__device__ __forceinline__ double dexp<double>(double v) { return exp(v); }
template <>
__device__ __forceinline__ float dexp<float>(float v) { return expf(v); }

// Primitives with a r^2 above this are skipped: their value and every
// derivative used here (at most a^3 r^3 times the value) stay below
// 1e-26 * a^(3/2), far under the FP64 tolerance of the path.
constexpr double kScreenExponent = 60.0;

// Radial sums f, f', f'' (and f''' when want3) at t.
template <typename T, bool want3>
__device__ __forceinline__ void radial(const T* alpha, const T* cn, int p0, int np, T t, T& f0, T& f1,
                                       T& f2, T& f3) {
    f0 = f1 = f2 = f3 = T(0);
    for (int p = p0; p < p0 + np; ++p) {
        const T a = alpha[p];
        if (a * t > T(kScreenExponent)) continue;
        const T e = cn[p] * dexp<T>(-a * t);
        f0 += e;
        f1 -= a * e;
        f2 += a * a * e;
        if (want3) f3 -= a * a * a * e;
    }
}

template <typename T>
__device__ __forceinline__ const T* sys_alpha(const DevSys& s);
template <>
__device__ __forceinline__ const double* sys_alpha<double>(const DevSys& s) { return s.alpha; }
template <>
__device__ __forceinline__ const float* sys_alpha<float>(const DevSys& s) { return s.alpha_f; }
template <typename T>
__device__ __forceinline__ const T* sys_cn(const DevSys& s);
template <>
__device__ __forceinline__ const double* sys_cn<double>(const DevSys& s) { return s.cn; }
template <>
__device__ __forceinline__ const float* sys_cn<float>(const DevSys& s) { return s.cn_f; }
template <typename T>
__device__ __forceinline__ const T* sys_C(const DevSys& s, int spin);
template <>
__device__ __forceinline__ const double* sys_C<double>(const DevSys& s, int spin) { return s.C[spin]; }
template <>
__device__ __forceinline__ const float* sys_C<float>(const DevSys& s, int spin) { return s.C_f[spin]; }

template <typename T>
__device__ __forceinline__ const T* sys_Cv(const DevSys& s, int spin);
template <>
__device__ __forceinline__ const double* sys_Cv<double>(const DevSys& s, int spin) { return s.Cv[spin]; }
template <>
__device__ __forceinline__ const float* sys_Cv<float>(const DevSys& s, int spin) { return s.Cv_f[spin]; }

template <typename T>
__device__ __forceinline__ const T* sys_amin(const DevSys& s);
template <>
__device__ __forceinline__ const double* sys_amin<double>(const DevSys& s) { return s.shell_amin; }
template <>
__device__ __forceinline__ const float* sys_amin<float>(const DevSys& s) { return s.shell_amin_f; }

// Value, gradient and Laplacian of every function of shell sh at electron
// position r; writes out[c * ld + fn] for c = 0 (value), 1..3 (gradient),
// 4 (Laplacian).
template <typename T>
__device__ __forceinline__ void shell_vgl_at(const DevSys& s, int sh, int4 d, T x, T y, T z, T* out, int ld,
                                             int fn0 = -1);

template <typename T>
__device__ __forceinline__ void shell_vgl(const DevSys& s, int sh, const double r[3], T* out, int ld) {
    const int4 d = s.shell[sh];
    shell_vgl_at<T>(s, sh, d, T(r[0] - s.Rn[3 * d.x]), T(r[1] - s.Rn[3 * d.x + 1]), T(r[2] - s.Rn[3 * d.x + 2]), out,
                    ld);
}

// FP32 difference of two positions split as hi + lo floats: the hi parts
// subtract exactly when close (Sterbenz) and the lo parts restore the bits a
// single float drops, so the offset keeps FP32 relative accuracy without an
// FP64 instruction.
__device__ __forceinline__ float diff_f2(float ah, float al, float bh, float bl) { return (ah - bh) + (al - bl); }

// The mixed form's shells at an electron given as hi/lo floats.
__device__ __forceinline__ void shell_vgl_f2(const DevSys& s, int sh, const float rh[3], const float rl[3], float* out,
                                             int ld) {
    const int4 d = s.shell[sh];
    const int c = 3 * d.x;
    shell_vgl_at<float>(s, sh, d, diff_f2(rh[0], rl[0], s.Rn_hi[c], s.Rn_lo[c]),
                        diff_f2(rh[1], rl[1], s.Rn_hi[c + 1], s.Rn_lo[c + 1]),
                        diff_f2(rh[2], rl[2], s.Rn_hi[c + 2], s.Rn_lo[c + 2]), out, ld);
}

// fn0: first output column (default: the shell's first basis function).
template <typename T>
__device__ __forceinline__ void shell_vgl_at(const DevSys& s, int sh, int4 d, T x, T y, T z, T* out, int ld,
                                             int fn0) {
    const int l = d.y & 0xff, pure = d.y >> 8;
    const T t = x * x + y * y + z * z;
    T f0, f1, f2, f3;
    radial<T, false>(sys_alpha<T>(s), sys_cn<T>(s), d.z, d.w, t, f0, f1, f2, f3);
    if (fn0 < 0) fn0 = s.shell_fn[sh];
    const int nf = shell_nfn(l, pure);
    if (f0 == T(0) && f1 == T(0) && f2 == T(0)) {
        for (int fi = 0; fi < nf; ++fi)
#pragma unroll
            for (int c = 0; c < 5; ++c) out[c * ld + fn0 + fi] = T(0);
        return;
    }
    const T Sx = T(2) * x * f1, Sy = T(2) * y * f1, Sz = T(2) * z * f1;
    const T LS = T(6) * f1 + T(4) * t * f2;
    for (int fi = 0; fi < nf; ++fi) {
        const AngPoly<T> a = angular<T>(l, pure, fi, x, y, z);
        const T LP = a.Hxx + a.Hyy + a.Hzz;
        out[0 * ld + fn0 + fi] = a.P * f0;
        out[1 * ld + fn0 + fi] = a.P * Sx + a.Px * f0;
        out[2 * ld + fn0 + fi] = a.P * Sy + a.Py * f0;
        out[3 * ld + fn0 + fi] = a.P * Sz + a.Pz * f0;
        out[4 * ld + fn0 + fi] = a.P * LS + T(2) * (a.Px * Sx + a.Py * Sy + a.Pz * Sz) + LP * f0;
    }
}

// Shared-memory bytes of basis_live's outputs for n_basis = nb: the packed
// rows bas_c [5][ld], rows [ld], the scan scratch and, with kCompact, the
// list of live shells [ld] (int2; a shell has at least one function, so
// n_shell <= nb), ld = basis_live_ld(nb).
__host__ __device__ inline int basis_live_ld(int nb) { return (nb + 3) & ~3; }
template <typename T, bool kCompact = true>
__host__ __device__ inline size_t basis_live_bytes(int nb) {
    const size_t ld = (size_t)basis_live_ld(nb);
    return (sizeof(T) * 5 * ld + sizeof(int) * (ld + kMaxWarps) + (kCompact ? sizeof(int2) * ld : 0) + 15) &
           ~(size_t)15;
}

// Offset of electron r from the centre of shell d: in double rounded to T
// (rd) or from hi/lo floats (rh, rl; FP32 offsets of the mixed form).
template <typename T>
__device__ __forceinline__ void shell_offset(const DevSys& s, int4 d, const double* rd, const float* rh,
                                             const float* rl, T& x, T& y, T& z) {
    const int c = 3 * d.x;
    if (rd == nullptr) {
        x = T(diff_f2(rh[0], rl[0], s.Rn_hi[c], s.Rn_lo[c]));
        y = T(diff_f2(rh[1], rl[1], s.Rn_hi[c + 1], s.Rn_lo[c + 1]));
        z = T(diff_f2(rh[2], rl[2], s.Rn_hi[c + 2], s.Rn_lo[c + 2]));
    } else {
        x = T(rd[0] - s.Rn[c]);
        y = T(rd[1] - s.Rn[c + 1]);
        z = T(rd[2] - s.Rn[c + 2]);
    }
}

// Live-shell basis of one move.  A shell whose most diffuse primitive is
// screened at the electron (shell_amin r^2 > kScreenExponent: the test
// radial() applies per primitive, with the same offsets and rounding, so all
// its primitives are skipped and its functions are exactly zero) is left
// out.  A block-wide scan gives every live shell the packed position of its
// first function; the functions of the live shells are written packed,
// bas_c[c * ldc + t] (c = value, d/dx, d/dy, d/dz, Laplacian), with rows[t]
// the basis function of packed row t, and the packed rows are padded with
// zero rows (rows[] = 0) to a multiple of 4 (ldc = basis_live_ld(n_basis)).
// kCompact: the scan also lists the live shells and they are evaluated one
// per thread on consecutive threads, so a warp runs the basis code only for
// live shells (one more barrier and n_basis int2 of shared memory); else
// each thread evaluates its own shell during the scan.  The electron is
// given in double (rd) or, with rd null, as hi/lo floats (rh, rl); see
// shell_offset.  scan: the scratch after rows (basis_live_bytes).  lst_buf:
// n_shell int2 of shared memory for the shell list, idle during the call
// (null: the list follows the scan scratch, as basis_live_bytes<T, true>
// lays it out).  Returns the padded row count in every thread; ends
// synchronised.
template <typename T, bool kCompact = true>
__device__ __forceinline__ int basis_live(const DevSys& s, const double* rd, const float* rh, const float* rl,
                                          T* bas_c, int ldc, int* rows, int* scan, int2* lst_buf = nullptr) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    int2* lst = lst_buf ? lst_buf
                        : reinterpret_cast<int2*>(((uintptr_t)(scan + kMaxWarps) + 7) & ~(uintptr_t)7);
    const T* amin = sys_amin<T>(s);
    int base = 0, nlive = 0;   // packed functions and live shells of the rounds so far
    for (int sh0 = 0; sh0 < s.n_shell; sh0 += blockDim.x) {
        const int sh = sh0 + threadIdx.x;
        int cnt = 0;
        int4 d = make_int4(0, 0, 0, 0);
        T x = T(0), y = T(0), z = T(0);
        if (sh < s.n_shell) {
            d = s.shell[sh];
            shell_offset<T>(s, d, rd, rh, rl, x, y, z);
            const T t = x * x + y * y + z * z;
            if (!(amin[sh] * t > T(kScreenExponent))) cnt = shell_nfn(d.y & 0xff, d.y >> 8);
        }
        // exclusive prefix over the block of (live functions | live shells << 16)
        const int key = cnt | ((cnt ? 1 : 0) << 16);
        int inc = key;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += v;
        }
        if (lane == 31) scan[wid] = inc;
        __syncthreads();
        int woff = 0, tot = 0;
        for (int q = 0; q < nw; ++q) {
            const int v = scan[q];
            woff += q < wid ? v : 0;
            tot += v;
        }
        const int ex = woff + inc - key;
        if (cnt) {
            const int pos = base + (ex & 0xffff);
            if constexpr (kCompact) {
                lst[nlive + (ex >> 16)] = make_int2(sh, pos);
            } else {
                shell_vgl_at<T>(s, sh, d, x, y, z, bas_c, ldc, pos);
                const int f0 = s.shell_fn[sh];
                for (int fi = 0; fi < cnt; ++fi) rows[pos + fi] = f0 + fi;
            }
        }
        base += tot & 0xffff;
        nlive += tot >> 16;
        if constexpr (!kCompact) {
            if (sh0 + (int)blockDim.x >= s.n_shell)
                for (int t = base + (int)threadIdx.x; t < ((base + 3) & ~3); t += blockDim.x) {
                    rows[t] = 0;
#pragma unroll
                    for (int c = 0; c < 5; ++c) bas_c[c * ldc + t] = T(0);
                }
        }
        __syncthreads();   // scan[] is reused by the next round; lst complete after the last
    }
    const int nrow = (base + 3) & ~3;
    if constexpr (kCompact) {
        for (int q = threadIdx.x; q < nlive; q += blockDim.x) {
            const int2 e = lst[q];
            const int4 d = s.shell[e.x];
            T x, y, z;
            shell_offset<T>(s, d, rd, rh, rl, x, y, z);
            shell_vgl_at<T>(s, e.x, d, x, y, z, bas_c, ldc, e.y);
            const int f0 = s.shell_fn[e.x], nf = shell_nfn(d.y & 0xff, d.y >> 8);
            for (int fi = 0; fi < nf; ++fi) rows[e.y + fi] = f0 + fi;
        }
        for (int t = base + (int)threadIdx.x; t < nrow; t += blockDim.x) {
            rows[t] = 0;
#pragma unroll
            for (int c = 0; c < 5; ++c) bas_c[c * ldc + t] = T(0);
        }
        __syncthreads();
    }
    return nrow;
}

// ---------------------------------------------------------------------
// Orbital contraction of one move (Eq. 2) over the packed live basis rows
// of basis_live:
//   phi[c * ldphi + j] = sum_{t < nrow} C[rows[t]][j] bas[c * ldb + t],
//   c = value, d/dx, d/dy, d/dz, Laplacian;  C is [n_basis][n] (orbital
// index contiguous).  Screened shells contribute exactly zero and are not
// visited.  nrow and ldb are multiples of 4, rows and bas 16-byte aligned.
// Small n (C stays in L1): one thread per (c, j), four partial sums.  Large
// n (C of the 32-water cluster is 0.5 MB and lives in L2): each coefficient
// is fetched once per move instead of five times; the mixed form splits the
// basis rows over thread slices as well (below), the FP64 form keeps one
// thread per orbital with sixteen rows of C in flight.  (Staging C through shared memory by bulk
// copies was measured slower: the chunk handshakes cost more than the
// latency they hide at the shared-memory budget the delayed update leaves.)
// ---------------------------------------------------------------------
template <int kV>
struct VecF;
template <>
struct VecF<1> {
    using type = float;
    __device__ static float at(const float& v, int) { return v; }
};
template <>
struct VecF<2> {
    using type = float2;
    __device__ static float at(const float2& v, int u) { return u == 0 ? v.x : v.y; }
};
template <>
struct VecF<4> {
    using type = float4;
    __device__ static float at(const float4& v, int u) { return u == 0 ? v.x : u == 1 ? v.y : u == 2 ? v.z : v.w; }
};

// Body of the sliced mixed-form contraction (see contract5).  Requires
// n % kV == 0 and C aligned to kV floats.
template <int kV>
__device__ __forceinline__ void contract5_sliced(const float* __restrict__ C, int n, int nrow, int ldb, const int* rows,
                                                 const float* bas, float* phi, int ldphi) {
    using V = typename VecF<kV>::type;
    const int ng = n / kV;
    int nks = (int)blockDim.x / ng;
    if (nks > 8) nks = 8;
    const int ks = (int)threadIdx.x / ng, jg = (int)threadIdx.x - ks * ng;
    const int nq = nrow >> 2, lq = ldb >> 2, qper = (nq + nks - 1) / nks;
    float a[5 * kV];
#pragma unroll
    for (int u = 0; u < 5 * kV; ++u) a[u] = 0.f;
    if (ks < nks) {
        const int q0 = ks * qper, q1 = min(nq, q0 + qper);
        const V* Cv = reinterpret_cast<const V*>(C) + jg;
        const float4* B4 = reinterpret_cast<const float4*>(bas);
        const int4* R4 = reinterpret_cast<const int4*>(rows);
#pragma unroll 2
        for (int q = q0; q < q1; ++q) {
            const int4 r = R4[q];
            const V c0 = Cv[(size_t)r.x * ng], c1 = Cv[(size_t)r.y * ng], c2 = Cv[(size_t)r.z * ng],
                    c3 = Cv[(size_t)r.w * ng];
#pragma unroll
            for (int c = 0; c < 5; ++c) {
                const float4 b = B4[c * lq + q];
#pragma unroll
                for (int u = 0; u < kV; ++u) {
                    float& acc = a[kV * c + u];
                    acc += VecF<kV>::at(c0, u) * b.x;
                    acc += VecF<kV>::at(c1, u) * b.y;
                    acc += VecF<kV>::at(c2, u) * b.z;
                    acc += VecF<kV>::at(c3, u) * b.w;
                }
            }
        }
    }
    for (int r = 0; r < nks; ++r) {
        if (ks == r)
#pragma unroll
            for (int c = 0; c < 5; ++c) {
                float* dst = phi + c * ldphi + kV * jg;
#pragma unroll
                for (int u = 0; u < kV; ++u) dst[u] = (r == 0 ? 0.f : dst[u]) + a[kV * c + u];
            }
        __syncthreads();
    }
}

// Mixed form, n <= 64: the rows are split over the 8 low lanes of a warp
// instead (4 groups of kV orbitals x 8 row slices per warp), so the slices
// reduce by three butterfly shuffles with no barrier; each lane reads kV
// coefficients and five 16-byte basis vectors per four rows (L1-resident C).
// Requires n % kV == 0 and C aligned to kV floats.
template <int kV>
__device__ __forceinline__ void contract5_lanes(const float* __restrict__ C, int n, int nrow, int ldb, const int* rows,
                                                const float* bas, float* phi, int ldphi) {
    using V = typename VecF<kV>::type;
    constexpr int kS = 8, kGpw = 32 / kS;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int ks = lane & (kS - 1), gl = lane >> 3;
    const int ng = n / kV, nq = nrow >> 2, lq = ldb >> 2, qper = (nq + kS - 1) / kS;
    const int q0 = ks * qper, q1 = min(nq, q0 + qper);
    const float4* B4 = reinterpret_cast<const float4*>(bas);
    const int4* R4 = reinterpret_cast<const int4*>(rows);
    for (int g0 = wid * kGpw; g0 < ng; g0 += nw * kGpw) {   // warp-uniform
        const int g = g0 + gl;
        float a[5 * kV];
#pragma unroll
        for (int u = 0; u < 5 * kV; ++u) a[u] = 0.f;
        if (g < ng) {
            const V* Cv = reinterpret_cast<const V*>(C) + g;
#pragma unroll 2
            for (int q = q0; q < q1; ++q) {
                const int4 r = R4[q];
                const V c0 = Cv[(size_t)r.x * ng], c1 = Cv[(size_t)r.y * ng], c2 = Cv[(size_t)r.z * ng],
                        c3 = Cv[(size_t)r.w * ng];
#pragma unroll
                for (int c = 0; c < 5; ++c) {
                    const float4 b = B4[c * lq + q];
#pragma unroll
                    for (int u = 0; u < kV; ++u) {
                        float& acc = a[kV * c + u];
                        acc += VecF<kV>::at(c0, u) * b.x;
                        acc += VecF<kV>::at(c1, u) * b.y;
                        acc += VecF<kV>::at(c2, u) * b.z;
                        acc += VecF<kV>::at(c3, u) * b.w;
                    }
                }
            }
        }
#pragma unroll
        for (int u = 0; u < 5 * kV; ++u) {
            a[u] += __shfl_xor_sync(0xffffffffu, a[u], 1);
            a[u] += __shfl_xor_sync(0xffffffffu, a[u], 2);
            a[u] += __shfl_xor_sync(0xffffffffu, a[u], 4);
        }
        if (ks == 0 && g < ng)
#pragma unroll
            for (int c = 0; c < 5; ++c)
#pragma unroll
                for (int u = 0; u < kV; ++u) phi[c * ldphi + kV * g + u] = a[kV * c + u];
    }
}

// kSliced = false compiles the sliced path out (kernels that never see
// n > 64 keep their registers for the rest).
template <typename T, bool kSliced = true>
__device__ __forceinline__ void contract5(const T* __restrict__ C, int n, int nrow, int ldb, const int* rows,
                                          const T* bas, T* phi, int ldphi) {
    if constexpr (sizeof(T) == 4) {
        if (n <= 64) {
            const uintptr_t ca = (uintptr_t)C;
            if ((n & 1) == 0 && (ca & 7) == 0) {
                contract5_lanes<2>(C, n, nrow, ldb, rows, bas, phi, ldphi);
                return;
            }
            contract5_lanes<1>(C, n, nrow, ldb, rows, bas, phi, ldphi);
            return;
        }
    }
    if constexpr (sizeof(T) == 4 && kSliced) {
        // Mixed form, n > 64: threads are (group of kV orbitals, slice of basis
        // rows); each accumulates kV orbitals x 5 components over its slice,
        // with four kV-wide coefficient loads and five 16-byte basis loads per
        // four rows (20 kV FMAs per 4 + 5 memory instructions instead of 5 per
        // 6), and the slices then add up into phi in slice order
        // (deterministic).  kV = 4 when n % 4 == 0 (measured fastest on the
        // 32-water cluster), else 2.
        if (n > 64 && (n & 1) == 0 && (((uintptr_t)C) & 7) == 0) {
            if ((n & 3) == 0 && (((uintptr_t)C) & 15) == 0 && (n >> 2) <= (int)blockDim.x) {
                contract5_sliced<4>(C, n, nrow, ldb, rows, bas, phi, ldphi);
                return;
            }
            if ((n >> 1) <= (int)blockDim.x) {
                contract5_sliced<2>(C, n, nrow, ldb, rows, bas, phi, ldphi);
                return;
            }
        }
    }
    if (2 * n >= (int)blockDim.x) {
        if constexpr (sizeof(T) == 4) {
            // basis values four at a time (16-byte shared loads: 5 loads per
            // 4 coefficients instead of 20).
            if (n <= 128) {
                for (int j = threadIdx.x; j < n; j += blockDim.x) {
                    float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f, a4 = 0.f;
#pragma unroll 4
                    for (int l = 0; l < nrow; l += 4) {
                        const int4 r = *reinterpret_cast<const int4*>(rows + l);
                        const float c0 = C[(size_t)r.x * n + j], c1 = C[(size_t)r.y * n + j];
                        const float c2 = C[(size_t)r.z * n + j], c3 = C[(size_t)r.w * n + j];
                        const float4 b0 = *reinterpret_cast<const float4*>(bas + l);
                        const float4 b1 = *reinterpret_cast<const float4*>(bas + ldb + l);
                        const float4 b2 = *reinterpret_cast<const float4*>(bas + 2 * ldb + l);
                        const float4 b3 = *reinterpret_cast<const float4*>(bas + 3 * ldb + l);
                        const float4 b4 = *reinterpret_cast<const float4*>(bas + 4 * ldb + l);
                        a0 += c0 * b0.x + c1 * b0.y + c2 * b0.z + c3 * b0.w;
                        a1 += c0 * b1.x + c1 * b1.y + c2 * b1.z + c3 * b1.w;
                        a2 += c0 * b2.x + c1 * b2.y + c2 * b2.z + c3 * b2.w;
                        a3 += c0 * b3.x + c1 * b3.y + c2 * b3.z + c3 * b3.w;
                        a4 += c0 * b4.x + c1 * b4.y + c2 * b4.z + c3 * b4.w;
                    }
                    phi[j] = a0;
                    phi[ldphi + j] = a1;
                    phi[2 * ldphi + j] = a2;
                    phi[3 * ldphi + j] = a3;
                    phi[4 * ldphi + j] = a4;
                }
                return;
            }
        }
        for (int j = threadIdx.x; j < n; j += blockDim.x) {
            T a0 = T(0), a1 = T(0), a2 = T(0), a3 = T(0), a4 = T(0);
#pragma unroll 16
            for (int l = 0; l < nrow; ++l) {
                const T c = C[(size_t)rows[l] * n + j];
                a0 += c * bas[l];
                a1 += c * bas[ldb + l];
                a2 += c * bas[2 * ldb + l];
                a3 += c * bas[3 * ldb + l];
                a4 += c * bas[4 * ldb + l];
            }
            phi[j] = a0;
            phi[ldphi + j] = a1;
            phi[2 * ldphi + j] = a2;
            phi[3 * ldphi + j] = a3;
            phi[4 * ldphi + j] = a4;
        }
        return;
    }
    for (int o = threadIdx.x; o < 5 * n; o += blockDim.x) {
        const int c = o / n, j = o - c * n;
        const T* b = bas + c * ldb;
        T a0 = T(0), a1 = T(0), a2 = T(0), a3 = T(0);
        for (int l = 0; l < nrow; l += 4) {
            const int4 r = *reinterpret_cast<const int4*>(rows + l);
            a0 += C[(size_t)r.x * n + j] * b[l];
            a1 += C[(size_t)r.y * n + j] * b[l + 1];
            a2 += C[(size_t)r.z * n + j] * b[l + 2];
            a3 += C[(size_t)r.w * n + j] * b[l + 3];
        }
        phi[c * ldphi + j] = (a0 + a1) + (a2 + a3);
    }
}

// ---------------------------------------------------------------------
// Block reductions (sums of K doubles); every thread gets the result.
// scratch: >= kMaxWarps * K doubles of shared memory.
// ---------------------------------------------------------------------
template <int K>
__device__ __forceinline__ void block_sum(double (&v)[K], double* scratch) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k)
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < K; ++k) scratch[wid * K + k] = v[k];
    __syncthreads();
#pragma unroll
    for (int k = 0; k < K; ++k) {
        double a = 0.0;
        for (int q = 0; q < nw; ++q) a += scratch[q * K + k];
        v[k] = a;
    }
}

// Per-thread running sums.  In double a plain sum; in float a compensated
// pair (Knuth's two-sum): the rounding error of every addition is kept in
// the low word, so long sums of float terms reach about twice the float
// precision on the FP32 pipe instead of FP64 instructions (GB300 issues
// FP64 at 1/64 of the FP32 rate).
template <typename T>
struct Acc;
template <>
struct Acc<double> {
    double h = 0.0;
    __device__ __forceinline__ void add(double x) { h += x; }
};
template <>
struct Acc<float> {
    float h = 0.f, l = 0.f;
    __device__ __forceinline__ void add(float x) {
        const float s = h + x;
        const float bp = s - h;
        l += (h - (s - bp)) + (x - bp);
        h = s;
    }
    __device__ __forceinline__ void add_pair(float xh, float xl) {
        add(xh);
        l += xl;
    }
};

// Block total of K accumulators, delivered in double to thread 0 only
// (out[] is undefined elsewhere).  The float form adds the pairs with two-sum
// at every level of the tree and converts to double once, in thread 0.
// scratch: >= 2 * kMaxWarps * K doubles.
template <int K>
__device__ __forceinline__ void block_sum_to0(Acc<double> (&v)[K], double* scratch, double (&out)[K]) {
    double t[K];
#pragma unroll
    for (int k = 0; k < K; ++k) t[k] = v[k].h;
    block_sum<K>(t, scratch);
#pragma unroll
    for (int k = 0; k < K; ++k) out[k] = t[k];
}
template <int K>
__device__ __forceinline__ void block_sum_to0(Acc<float> (&v)[K], double* scratch, double (&out)[K]) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    float* sc = (float*)scratch;
#pragma unroll
    for (int k = 0; k < K; ++k)
        for (int o = 16; o > 0; o >>= 1) {
            const float oh = __shfl_xor_sync(0xffffffffu, v[k].h, o);
            const float ol = __shfl_xor_sync(0xffffffffu, v[k].l, o);
            v[k].add_pair(oh, ol);
        }
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < K; ++k) {
            sc[2 * (wid * K + k)] = v[k].h;
            sc[2 * (wid * K + k) + 1] = v[k].l;
        }
    __syncthreads();
    if (threadIdx.x == 0)
#pragma unroll
        for (int k = 0; k < K; ++k) {
            Acc<float> a;
            for (int q = 0; q < nw; ++q) a.add_pair(sc[2 * (q * K + k)], sc[2 * (q * K + k) + 1]);
            out[k] = (double)a.h + (double)a.l;
        }
}

// Sum of 8 values over the block with a transposing butterfly: each lane
// ends a warp holding the warp total of one of the 8 values (9 adds per lane
// instead of 40), then the warp totals are added through shared memory.
// Every thread gets the 8 block totals.  scratch: >= kMaxWarps * 8 doubles.
template <typename A>
__device__ __forceinline__ void block_sum8(A (&v)[8], A* scratch) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    {
        const bool h = (lane >> 4) & 1;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const A send = h ? v[i] : v[i + 4];
            const A keep = h ? v[i + 4] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
        }
    }
    {
        const bool h = (lane >> 3) & 1;
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const A send = h ? v[i] : v[i + 2];
            const A keep = h ? v[i + 2] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
        }
    }
    {
        const bool h = (lane >> 2) & 1;
        const A send = h ? v[0] : v[1];
        const A keep = h ? v[1] : v[0];
        v[0] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
    }
    v[0] += __shfl_xor_sync(0xffffffffu, v[0], 2);
    v[0] += __shfl_xor_sync(0xffffffffu, v[0], 1);
    // lane bits (4, 3, 2) = (h1, h2, h3) select value index h3 + 2 h2 + 4 h1
    __syncthreads();
    if ((lane & 3) == 0) {
        const int k = ((lane >> 2) & 1) | (((lane >> 3) & 1) << 1) | (((lane >> 4) & 1) << 2);
        scratch[wid * 8 + k] = v[0];
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        A a = A(0);
        for (int q = 0; q < nw; ++q) a += scratch[q * 8 + k];
        v[k] = a;
    }
}


// block_sum8 for callers that need the totals in thread 0 only (the serial
// move logic of the sweeps): warp 0's lanes 0..7 each add one value over the
// warps and thread 0 gathers the 8 totals by shuffles, instead of every
// thread adding all 8 x (warps) partial sums.  The totals in thread 0 are
// bit-identical to block_sum8's; v of every other thread is left undefined.
template <typename A>
__device__ __forceinline__ void block_sum8_to0(A (&v)[8], A* scratch) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    {
        const bool h = (lane >> 4) & 1;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const A send = h ? v[i] : v[i + 4];
            const A keep = h ? v[i + 4] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
        }
    }
    {
        const bool h = (lane >> 3) & 1;
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const A send = h ? v[i] : v[i + 2];
            const A keep = h ? v[i + 2] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
        }
    }
    {
        const bool h = (lane >> 2) & 1;
        const A send = h ? v[0] : v[1];
        const A keep = h ? v[1] : v[0];
        v[0] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
    }
    v[0] += __shfl_xor_sync(0xffffffffu, v[0], 2);
    v[0] += __shfl_xor_sync(0xffffffffu, v[0], 1);
    __syncthreads();
    if ((lane & 3) == 0) {
        const int k = ((lane >> 2) & 1) | (((lane >> 3) & 1) << 1) | (((lane >> 4) & 1) << 2);
        scratch[wid * 8 + k] = v[0];
    }
    __syncthreads();
    if (wid == 0) {
        A a = A(0);
        if (lane < 8)
            for (int q = 0; q < nw; ++q) a += scratch[q * 8 + lane];
#pragma unroll
        for (int k = 0; k < 8; ++k) v[k] = __shfl_sync(0xffffffffu, a, k);
    }
}

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ float warp_sum(float v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}


// ---------------------------------------------------------------------
// Launchers (defined in the kernel translation units).
// ---------------------------------------------------------------------
struct SweepParams {
    double tau;
    uint2 key;
    uint32_t sweep;
    int ainv_smem;   // keep A^-1 in shared memory for the sweep
    int g_smem;      // keep the gradient/Laplacian cache in shared memory
};

template <typename T>
cudaError_t launch_orbitals_all(const DevSys& s, const DevWalkers& wk, int W, cudaStream_t st,
                                const int* only = nullptr);
// only (optional, [W]): rebuild just the walkers whose flag is nonzero.
cudaError_t launch_invert(const DevSys& s, const DevWalkers& wk, int W, int store_fp32, unsigned* err,
                          cudaStream_t st, const int* only = nullptr);
// Jastrow parameter derivatives (k_wavefunction.cu): for P = 4 + n_nuc +
// n_nuc n3 parameters (a_anti, a_par, b_ee, b_en, a_en[], c3[][]),
// Non-local pseudopotential energy (locality approximation) of walkers
// [w0, W), added to eloc[w]; rotations of the quadrature rule from Philox key
// `key` at counter (sweep, nucleus, slot, 3).  U0 / U1: u_k = C_s A^-1 e_k of
// every electron of those walkers per spin, [w - w0][k][ldu] with ldu =
// n_basis rounded up to 4 (the tensor-core product), or nullptr to form
// them in the kernel.
template <typename T>
cudaError_t launch_nlpp(const DevSys& s, const DevWalkers& wk, int w0, int W, double* eloc, uint2 key, uint32_t sweep,
                        const void* U0, const void* U1, cudaStream_t st);
// The non-local terms of the ionic derivatives: B_NL rows into nlB[spin]
// (zeroed first by the caller; rows of electrons out of range stay zero) and
// the direct terms into nlF [W][3 n_nuc].
template <typename T>
cudaError_t launch_nlpp_force(const DevSys& s, const DevWalkers& wk, int w0, int W, void* nlB0, void* nlB1,
                              double* nlF, uint2 key, uint32_t sweep, const void* U0, const void* U1,
                              cudaStream_t st);
// The non-local energy's Jastrow parameter derivatives added to deloc[W][P]
// (same parameter order and rotations as launch_jastrow_derivs and
// launch_nlpp): sum_p W_p rho_p (dJ/dp(R'_p) - dJ/dp(R)).
template <typename T>
cudaError_t launch_nlpp_param(const DevSys& s, const DevWalkers& wk, int w0, int W, double* deloc, uint2 key,
                              uint32_t sweep, const void* U0, const void* U1, cudaStream_t st);
// dlog[W][P] = d ln|psi| / dp and deloc[W][P] = dE_L / dp from the positions
// and the total gradient grad_i ln|psi| [W][N][3].
cudaError_t launch_jastrow_derivs(const DevSys& s, const double* R, const double* G, int W, double* dlog,
                                  double* deloc, cudaStream_t st);
template <typename T>
cudaError_t launch_eloc(const DevSys& s, const DevWalkers& wk, int W, double* eloc_out, double* logpsi,
                        double* grad, double* lap, unsigned* err, cudaStream_t st);
template <typename T>
cudaError_t launch_sweep(const DevSys& s, const DevWalkers& wk, int W, const SweepParams& p,
                         const int* n_live, cudaStream_t st);
template <typename T>
size_t sweep_smem_bytes(const DevSys& s, int ainv_smem, int g_smem);
constexpr int kMaxDelayRank = 32;
template <typename T>
size_t delayed_smem_bytes(const DevSys& s, int kmax);
template <typename T>
cudaError_t launch_sweep_delayed(const DevSys& s, const DevWalkers& wk, int W, const SweepParams& p, int kmax,
                                 cudaStream_t st);
// Ionic derivatives (k_force.cu).  gEdet, gtot: null, or the space-warp
// form's per-electron outputs [W][N][3] (determinant part of dE_L/dr_i and
// grad_i ln|psi|), consumed by launch_space_warp.
template <typename T>
cudaError_t launch_force(const DevSys& s, const DevWalkers& wk, int W, const double* dvnn, double* Bscr,
                         double* Pscr, double* dEL, double* dlog, double* gEdet, double* gtot, cudaStream_t st);
template <typename T>
cudaError_t launch_force_prep(const DevSys& s, const DevWalkers& wk, int w0, int W, const double* dvnn, void* Bw,
                              double* gJw, double* accw, double* gtot, cudaStream_t st);
template <typename T>
cudaError_t launch_force_contract(const DevSys& s, const DevWalkers& wk, int w0, int W, const void* Mw, const void* Yw,
                                  const double* gJw, const double* accw, double* dEL, double* dlog, double* gEdet,
                                  cudaStream_t st);
// Space warp (k_force.cu): completes dE_L/dr_i with the Jastrow and
// potential terms and adds the warp of every electron to the per-walker
// ionic derivatives dEL, dlog [W][n_nuc][3] in place.
template <typename T>
cudaError_t launch_space_warp(const DevSys& s, const DevWalkers& wk, int W, const double* gEdet, const double* gtot,
                              double* dEL, double* dlog, cudaStream_t st);
cudaError_t launch_weighted_sum(const double* x /*[W][K]*/, const double* g /*[W] or null*/, int W, int K,
                                double* out /*[K]*/, int accumulate, cudaStream_t st);

// Multi-determinant kernels (k_msd.cu).
template <typename T>
cudaError_t launch_msd_table(const DevSys& s, const DevWalkers& wk, int W, cudaStream_t st, const int* only = nullptr);
template <typename T>
size_t msd_sweep_smem_bytes(const DevSys& s);
template <typename T>
cudaError_t launch_sweep_msd(const DevSys& s, const DevWalkers& wk, int W, const SweepParams& p, cudaStream_t st);
size_t force_msd_scratch_words(const DevSys& s);
// Batched FP32 GEMM on the tensor cores (3xTF32 split), D_b = A_b B_b^T
// (B_b^T replaced by B_b when b_trans); N <= 256 (k_tc_gemm.cu).
size_t tc_gemm_smem_bytes(int N);
cudaError_t launch_tc_gemm(int batch, int M, int N, int K, const float* A, long long sA, int lda, const float* B,
                           long long sB, int ldb, int b_trans, float* D, long long sD, int ldd, unsigned* err,
                           cudaStream_t st);
// D_b = alpha A_b B_b^T + beta D_b (B_b^T replaced by B_b when b_trans) on the
// pipelined TMA kernel alone; cudaErrorNotSupported when TMA cannot describe
// the operands (16-byte aligned bases, row and batch strides required).
// D = A B^T for operands given as TF32 hi / lo pairs ([M][K] and [N][K],
// row strides lda, ldb, 16-byte aligned): the tensor maps are encoded once
// by tc_split_plan (false when TMA cannot describe the operands) and the
// launch reuses them; tc_split_prepare sets the kernel's shared-memory limit
// (call it outside any stream capture).
struct alignas(64) TcSplitPlan {
    unsigned char map[4][128];   // CUtensorMap of A_hi, A_lo, B_hi, B_lo
    int M, N, K;
};
bool tc_split_plan(TcSplitPlan* p, int M, int N, int K, const float* Ah, const float* Al, int lda, const float* Bh,
                   const float* Bl, int ldb);
cudaError_t tc_split_prepare(int N);
cudaError_t launch_tc_gemm_split(const TcSplitPlan& p, float* D, int ldd, unsigned* err, cudaStream_t st);
cudaError_t launch_tc_gemm_ab(int batch, int M, int N, int K, float alpha, const float* A, long long sA, int lda,
                              const float* B, long long sB, int ldb, int b_trans, float beta, float* D, long long sD,
                              int ldd, unsigned* err, cudaStream_t st);

template <typename T>
cudaError_t launch_force_msd(const DevSys& s, const DevWalkers& wk, int W, const double* dvnn, double* scr,
                             double* dEL, double* dlog, double* gEdet, double* gtot, cudaStream_t st);
template <typename T>
cudaError_t launch_msd_eloc(const DevSys& s, const DevWalkers& wk, int W, double* eloc, double* logpsi,
                            double* sign, double* grad, cudaStream_t st);

// Branching (Eq. 1 projection with population control).
struct BranchParams {
    double tau, e_trial, e_cut;
    uint2 key;
    uint32_t sweep;
    int cap;
    int fixed_pop;   // > 0: resample exactly this many walkers (systematic comb)
};
cudaError_t launch_branch(const DevSys& s, const DevWalkers& src, const DevWalkers& dst, int W,
                          const double* eloc_new, const BranchParams& p, int* copies, int* offsets,
                          double* wts, double* stats /*[5]: sum w, sum w E, W_new, overflow, sum w clip(E)*/,
                          int elem_bytes, cudaStream_t st);

}  // namespace qmc
