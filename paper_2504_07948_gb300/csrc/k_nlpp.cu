// Non-local pseudopotential energy in the locality approximation (the
// valence Hamiltonian with effective core potentials, Sec. "Quantum Monte
// Carlo" and Sec. "The SPICE2(+)-ccECP dataset").  For every electron i
// within the cutoff radius of a pseudopotential nucleus a,
//   V_i,a = sum_l v_l(r_ia) (2l + 1) sum_q w_q P_l(r_hat_ia . d_q)
//           psi(R with r_i -> R_a + r_ia d_q) / psi(R),
// d_q the quadrature directions rotated per (walker slot, nucleus).
//
// The determinant ratio of moving electron i (row k of spin block s) to r'
// is phi(r')^T A^-1 e_k = chi(r')^T u_k with u_k = C_s (A^-1 e_k): the
// occupied coefficients [N_b x n] times the k-th column of the inverse (one
// contiguous row of the stored transposed inverse).  So an electron costs
// one N_b x n product and each quadrature point only its basis values and
// an N_b dot product, instead of an N_b x n contraction per point.  The
// Jastrow ratio is exp of the change of every term that involves electron i,
// summed term by term (differences of pair functions, not of totals).
//
// One CTA per walker:
//   1. the quadrature rotation of every pseudopotential nucleus (Shoemake's
//      quaternion from Philox counter (sweep, nucleus, slot, 3));
//   2. the ascending list of electrons within some cutoff (warp ballots);
//   3. per chunk of up to kChunk listed electrons of one spin: their inverse
//      columns and u_k in shared memory, and their (electron, nucleus) pairs;
//   4. per pass of at most kPtCap points: pair data (direction, distance,
//      channel potentials) once per pair and point data (position, weight)
//      once per point, by one thread each, into shared memory;
//   5. one warp per quadrature point: lanes over shells for chi(r') . u_k,
//      then over electrons and nuclei for the Jastrow change;
//   6. the walker total, summed in a fixed order, added to E_L.
// The mixed form runs the basis, dot products and pair terms in FP32
// (offsets from hi/lo split positions) and keeps FP64 to the per-pair and
// per-point set-up (one thread each, not one warp) and the walker total:
// GB300 issues FP64 at about 1/64 of the FP32 rate, so FP64 work repeated
// across the lanes of every point would dominate.  The FP64 form takes the
// Jastrow terms of each chunk electron at its old position once and only
// the new terms per point.
#include "qmc_internal.cuh"

namespace qmc {

namespace {

constexpr int kNlThreads = 256;
constexpr int kNlWarps = kNlThreads / 32;
constexpr int kChunk = 8;

// Points of one pass: at most kPtCap quadrature points (pairs x rule).
constexpr int kPtCap = 192;

struct NlLayout {
    size_t sR, sRf, rot, el, Ak, U, pairs, pg, pt, ptf, jold, beta, Fd, dvw, total;
};

// Passes of the kernel: the energy, the ionic-derivative terms, the Jastrow
// parameter derivatives.
enum NlMode { kNlEnergy = 0, kNlForce = 1, kNlParam = 2 };

template <typename T>
__host__ __device__ inline NlLayout nl_layout(int N, int nmax, int nb, int n_ecp, int n_shell, int n_nuc,
                                              int mode, int n_par) {
    const bool force = mode == kNlForce;
    NlLayout L;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o = (o + bytes + 15) & ~(size_t)15;
        return at;
    };
    L.sR = take(sizeof(double) * 3 * N);
    L.sRf = take(sizeof(float) * 3 * N);
    L.rot = take(sizeof(double) * 9 * (n_ecp > 0 ? n_ecp : 1));
    L.el = take(sizeof(int) * (N + 1));
    L.Ak = take(sizeof(T) * kChunk * ((nmax + 3) & ~3));
    L.U = take(sizeof(T) * kChunk * ((nb + 3) & ~3));
    L.pairs = take(sizeof(int2) * kChunk * (n_ecp > 0 ? n_ecp : 1));
    L.pg = take(sizeof(double) * 12 * kPtCap);   // per pair: x_hat[3], r, v_l[4], dv_l/dr[4]
    L.pt = take(sizeof(double) * 8 * kPtCap);    // per point: r d_q [3], weight, dW/dR_a [3]
    L.ptf = take(sizeof(float) * 3 * kPtCap);    // per point: r d_q in FP32
    L.jold = take(sizeof(double) * kChunk);      // FP64 form: J terms of each chunk electron
    // force pass: sum_p c_p chi(r'_p) per chunk electron, direct terms per nucleus
    L.beta = take(force ? sizeof(T) * kChunk * ((nb + 3) & ~3) : 0);
    L.Fd = take(force ? sizeof(double) * 3 * n_nuc : 0);
    // parameter pass: one row of parameter derivatives per warp
    L.dvw = take(mode == kNlParam ? sizeof(double) * kNlWarps * n_par : 0);
    L.total = o;
    return L;
}

// Shoemake's uniform random rotation ("Uniform random rotations", Graphics
// Gems III, 1992) from three uniforms: the unit quaternion
// (x, y, z, w) = (sqrt(1-u1) sin 2 pi u2, sqrt(1-u1) cos 2 pi u2,
// sqrt(u1) sin 2 pi u3, sqrt(u1) cos 2 pi u3) and its rotation matrix.
__device__ void pp_rotation(uint2 key, uint32_t sweep, uint32_t nucleus, uint32_t slot, double* rot) {
    const uint4 v = philox4x32_10(make_uint4(sweep, nucleus, slot, 3u), key);
    const double u1 = u01(v.x), u2 = u01(v.y), u3 = u01(v.z);
    const double a = sqrt(1.0 - u1), b = sqrt(u1);
    double s2, c2, s3, c3;
    sincospi(2.0 * u2, &s2, &c2);
    sincospi(2.0 * u3, &s3, &c3);
    const double x = a * s2, y = a * c2, z = b * s3, w = b * c3;
    rot[0] = 1.0 - 2.0 * (y * y + z * z);
    rot[1] = 2.0 * (x * y - z * w);
    rot[2] = 2.0 * (x * z + y * w);
    rot[3] = 2.0 * (x * y + z * w);
    rot[4] = 1.0 - 2.0 * (x * x + z * z);
    rot[5] = 2.0 * (y * z - x * w);
    rot[6] = 2.0 * (x * z - y * w);
    rot[7] = 2.0 * (y * z + x * w);
    rot[8] = 1.0 - 2.0 * (x * x + y * y);
}

__device__ __forceinline__ double legendre(int l, double x) {
    return l == 0 ? 1.0 : l == 1 ? x : l == 2 ? 0.5 * (3.0 * x * x - 1.0) : 0.5 * (5.0 * x * x * x - 3.0 * x);
}

__device__ __forceinline__ double legendre_dx(int l, double x) {
    return l == 0 ? 0.0 : l == 1 ? 1.0 : l == 2 ? 3.0 * x : 0.5 * (15.0 * x * x - 3.0);
}

// Value-only contracted shell at offset (x, y, z): sum_p c_p exp(-a_p t).
template <typename T>
__device__ __forceinline__ T radial0(const DevSys& s, int p0, int np, T t) {
    const T* al = sys_alpha<T>(s);
    const T* cn = sys_cn<T>(s);
    T f = T(0);
    for (int p = p0; p < p0 + np; ++p) {
        const T a = al[p];
        if (a * t > T(kScreenExponent)) continue;
        f += cn[p] * dexp<T>(-a * t);
    }
    return f;
}

// Quadrature points of one pair processed together in registers.
constexpr int kQ = 12;

// Sum over a shell's functions of P_f(x, y, z) u_f (values only; the angular
// forms and their order as in `angular`).
template <typename T>
__device__ __forceinline__ T shell_dot(int l, int pure, T x, T y, T z, const T (&uf)[6]) {
    const T s3 = T(1.7320508075688772);
    if (l == 0) return uf[0];
    if (l == 1) return x * uf[0] + y * uf[1] + z * uf[2];
    if (pure)
        return s3 * (x * y * uf[0] + y * z * uf[1] + x * z * uf[3]) + (z * z - T(0.5) * (x * x + y * y)) * uf[2] +
               T(0.5) * s3 * (x * x - y * y) * uf[4];
    return x * x * uf[0] + y * y * uf[3] + z * z * uf[5] + s3 * (x * y * uf[1] + x * z * uf[2] + y * z * uf[4]);
}

// Lane's share of chi(R_a + r d_q) . u at the batch's points q < nqb of one
// pair (nucleus a, distance r; dq[q] = r d_q): each lane takes shells in
// (l, pure) order (neighbouring lanes mostly of one type), loads a shell's
// data once and evaluates it at every point of the batch, so the loads are
// shared by the points and the points give independent work.  A shell is
// skipped when even the sphere's nearest point is screened.
template <typename T>
__device__ __forceinline__ void pair_basis_lane(const DevSys& s, int a, T r, const T (&dq)[kQ][3], int nqb,
                                                const T* __restrict__ u, T (&dr)[kQ], int lane) {
    for (int k = lane; k < s.n_shell; k += 32) {
        const int sh = s.shell_by_type[k];
        const int4 d = s.shell[sh];
        const int c = 3 * d.x;
        T cx, cy, cz;   // R_a - R_c
        if constexpr (sizeof(T) == 8) {
            cx = s.Rn[3 * a] - s.Rn[c];
            cy = s.Rn[3 * a + 1] - s.Rn[c + 1];
            cz = s.Rn[3 * a + 2] - s.Rn[c + 2];
        } else {
            cx = diff_f2(s.Rn_hi[3 * a], s.Rn_lo[3 * a], s.Rn_hi[c], s.Rn_lo[c]);
            cy = diff_f2(s.Rn_hi[3 * a + 1], s.Rn_lo[3 * a + 1], s.Rn_hi[c + 1], s.Rn_lo[c + 1]);
            cz = diff_f2(s.Rn_hi[3 * a + 2], s.Rn_lo[3 * a + 2], s.Rn_hi[c + 2], s.Rn_lo[c + 2]);
        }
        const T amin = sys_amin<T>(s)[sh];
        const T gap = sqrt(cx * cx + cy * cy + cz * cz) - r;
        if (gap > T(0) && amin * gap * gap > T(kScreenExponent)) continue;
        const int l = d.y & 0xff, pure = d.y >> 8, fn0 = s.shell_fn[sh];
        const int nf = shell_nfn(l, pure);
        T uf[6];
#pragma unroll
        for (int f = 0; f < 6; ++f) uf[f] = f < nf ? u[fn0 + f] : T(0);
#pragma unroll
        for (int q = 0; q < kQ; ++q) {
            if (q < nqb) {
                const T x = cx + dq[q][0], y = cy + dq[q][1], z = cz + dq[q][2];
                const T t = x * x + y * y + z * z;
                if (amin * t <= T(kScreenExponent)) dr[q] += radial0<T>(s, d.z, d.w, t) * shell_dot<T>(l, pure, x, y, z, uf);
            }
        }
    }
}

// Lane's share of the Jastrow change of electron i moved to R_a + r d_q for
// the batch's points (mixed form): pair distances in FP32, each term's change
// u(r') - u(r) = a (r' - r) / ((1 + b r')(1 + b r)) formed directly so that
// no two large totals cancel.
__device__ __forceinline__ void pair_jastrow_lane_f(const DevSys& s, const float* sRf, int i, int a,
                                                    const float (&dq)[kQ][3], int nqb, float (&dj)[kQ], int lane) {
    const int N = s.N, nu = s.n_up;
    const float bee = (float)s.b_ee, ben = (float)s.b_en;
    const float apar = (float)s.a_par, aanti = (float)s.a_anti;
    const float ex = sRf[3 * i], ey = sRf[3 * i + 1], ez = sRf[3 * i + 2];
    const float ax = s.Rn_hi[3 * a] + s.Rn_lo[3 * a], ay = s.Rn_hi[3 * a + 1] + s.Rn_lo[3 * a + 1],
                az = s.Rn_hi[3 * a + 2] + s.Rn_lo[3 * a + 2];
    for (int j = lane; j < N; j += 32) {
        if (j == i) continue;
        const float aa = ((i < nu) == (j < nu)) ? apar : aanti;
        const float xj = sRf[3 * j], yj = sRf[3 * j + 1], zj = sRf[3 * j + 2];
        const float ro = sqrtf((ex - xj) * (ex - xj) + (ey - yj) * (ey - yj) + (ez - zj) * (ez - zj));
        const float go = aa / (1.f + bee * ro);
        const float cx = ax - xj, cy = ay - yj, cz = az - zj;
#pragma unroll
        for (int q = 0; q < kQ; ++q) {
            if (q < nqb) {
                const float x = cx + dq[q][0], y = cy + dq[q][1], z = cz + dq[q][2];
                const float rn = sqrtf(x * x + y * y + z * z);
                dj[q] += __fdividef((rn - ro) * go, 1.f + bee * rn);
            }
        }
    }
    for (int b = lane; b < s.n_nuc; b += 32) {
        const int c = 3 * b;
        const float ro = sqrtf((ex - s.Rn_hi[c]) * (ex - s.Rn_hi[c]) + (ey - s.Rn_hi[c + 1]) * (ey - s.Rn_hi[c + 1]) +
                               (ez - s.Rn_hi[c + 2]) * (ez - s.Rn_hi[c + 2]));
        const float go = s.a_en_f[b] / (1.f + ben * ro);
        const float cx = diff_f2(s.Rn_hi[3 * a], s.Rn_lo[3 * a], s.Rn_hi[c], s.Rn_lo[c]);
        const float cy = diff_f2(s.Rn_hi[3 * a + 1], s.Rn_lo[3 * a + 1], s.Rn_hi[c + 1], s.Rn_lo[c + 1]);
        const float cz = diff_f2(s.Rn_hi[3 * a + 2], s.Rn_lo[3 * a + 2], s.Rn_hi[c + 2], s.Rn_lo[c + 2]);
#pragma unroll
        for (int q = 0; q < kQ; ++q) {
            if (q < nqb) {
                const float x = cx + dq[q][0], y = cy + dq[q][1], z = cz + dq[q][2];
                const float rn = sqrtf(x * x + y * y + z * z);
                dj[q] += __fdividef((rn - ro) * go, 1.f + ben * rn);
            }
        }
    }
}

// Lane's share of the pair and nucleus Jastrow terms of electron i at the
// batch's points R_a + r d_q (FP64 form: the new terms themselves; the old
// ones are subtracted once per electron).
__device__ __forceinline__ void pair_jastrow_lane_d(const DevSys& s, const double* sR, int i, int a,
                                                    const double (&dq)[kQ][3], int nqb, double (&dj)[kQ], int lane) {
    const int N = s.N, nu = s.n_up;
    const double* Ra = s.Rn + 3 * a;
    for (int j = lane; j < N; j += 32) {
        if (j == i) continue;
        const double aa = ((i < nu) == (j < nu)) ? s.a_par : s.a_anti;
        const double cx = Ra[0] - sR[3 * j], cy = Ra[1] - sR[3 * j + 1], cz = Ra[2] - sR[3 * j + 2];
#pragma unroll
        for (int q = 0; q < kQ; ++q) {
            if (q < nqb) {
                const double x = cx + dq[q][0], y = cy + dq[q][1], z = cz + dq[q][2];
                const double rn = sqrt(x * x + y * y + z * z);
                dj[q] += aa * rn / (1.0 + s.b_ee * rn);
            }
        }
    }
    for (int b = lane; b < s.n_nuc; b += 32) {
        const double cx = Ra[0] - s.Rn[3 * b], cy = Ra[1] - s.Rn[3 * b + 1], cz = Ra[2] - s.Rn[3 * b + 2];
#pragma unroll
        for (int q = 0; q < kQ; ++q) {
            if (q < nqb) {
                const double x = cx + dq[q][0], y = cy + dq[q][1], z = cz + dq[q][2];
                const double rn = sqrt(x * x + y * y + z * z);
                dj[q] += s.a_en[b] * rn / (1.0 + s.b_en * rn);
            }
        }
    }
}

// Lane's share of the three-body terms of electron e at position x with
// every partner j and nucleus a (pairs (a, j) over the lanes).
__device__ __forceinline__ double jastrow3_lane(const DevSys& s, const double* sR, int e, const double* x, int lane) {
    const int N = s.N, T3 = s.n_nuc * N;
    double J = 0.0;
    for (int q = lane; q < T3; q += 32) {
        const int a = q / N, j = q - a * N;
        if (j == e) continue;
        const double* Ra = s.Rn + 3 * a;
        const SDist xi = sdist(s.b3, x[0] - Ra[0], x[1] - Ra[1], x[2] - Ra[2]);
        const SDist xj = sdist(s.b3, sR[3 * j] - Ra[0], sR[3 * j + 1] - Ra[1], sR[3 * j + 2] - Ra[2]);
        const SDist y = sdist(s.b3, x[0] - sR[3 * j], x[1] - sR[3 * j + 1], x[2] - sR[3 * j + 2]);
        const double* c = s.c3 + (size_t)a * s.n3;
        for (int k = 0; k < s.n3; ++k) {
            if (c[k] == 0.0) continue;
            const int m = s.e3[3 * k], n = s.e3[3 * k + 1], o = s.e3[3 * k + 2];
            J += c[k] * (ipow_d(xi.s, m) * ipow_d(xj.s, n) + ipow_d(xi.s, n) * ipow_d(xj.s, m)) * ipow_d(y.s, o);
        }
    }
    return J;
}

// Lane's share of every Jastrow term that involves electron e, with e at
// position x (FP64 form): pair terms with the other electrons, nucleus
// terms and three-body terms.
__device__ __forceinline__ double jastrow_terms_lane(const DevSys& s, const double* sR, int e, const double* x,
                                                     int lane) {
    const int N = s.N, nu = s.n_up;
    double J = 0.0;
    for (int j = lane; j < N; j += 32) {
        if (j == e) continue;
        const double a = ((e < nu) == (j < nu)) ? s.a_par : s.a_anti;
        const double dx = x[0] - sR[3 * j], dy = x[1] - sR[3 * j + 1], dz = x[2] - sR[3 * j + 2];
        const double r = sqrt(dx * dx + dy * dy + dz * dz);
        J += a * r / (1.0 + s.b_ee * r);
    }
    for (int b = lane; b < s.n_nuc; b += 32) {
        const double dx = x[0] - s.Rn[3 * b], dy = x[1] - s.Rn[3 * b + 1], dz = x[2] - s.Rn[3 * b + 2];
        const double r = sqrt(dx * dx + dy * dy + dz * dz);
        J += s.a_en[b] * r / (1.0 + s.b_en * r);
    }
    if (s.n3 > 0) J += jastrow3_lane(s, sR, e, x, lane);
    return J;
}

// Force pass, lane's share for one pair's batch of points, given per point
// c_q = W_q exp(dJ_q) and the determinant ratio rho_q (warp totals of the
// energy pass), the pair's unit vector xh and distance r (dq[q] = r d_q):
//   beta[f] += sum_q c_q chi_f(r'_q)            (the pair's row of B_NL, in basis space)
//   Fd[b]   -= sum_q c_q sum_{f on b} grad chi_f(r'_q) u_f    (basis functions moving with b)
//   Fd[b]   += sum_q c_q rho_q (u'(|r_i - R_b|) e_old - u'(|r'_q - R_b|) e_new)   (e-n Jastrow)
//   mot     += sum_q c_q (g_q + rho_q gJ_q) (I - d_q x_hat^T)   (r'_q follows R_a)
// with g_q = grad_{r'} (chi . u) and gJ_q = grad_{r'} J at the moved electron.
template <typename T>
__device__ __forceinline__ void pair_force_lane(const DevSys& s, const double* sR, const float* sRf, int i, int a,
                                                T r, const T (&dq)[kQ][3], int nqb, const T (&cq)[kQ],
                                                const T (&rq)[kQ], const T (&xh)[3], const T* __restrict__ u,
                                                T* beta, double* Fd, T (&mot)[3], int lane) {
    const int N = s.N, nu = s.n_up;
    const T ir = T(1) / r;
    // basis: lanes over shells in (l, pure) order
    for (int k = lane; k < s.n_shell; k += 32) {
        const int sh = s.shell_by_type[k];
        const int4 d = s.shell[sh];
        const int c = 3 * d.x;
        T cx, cy, cz;   // R_a - R_c
        if constexpr (sizeof(T) == 8) {
            cx = s.Rn[3 * a] - s.Rn[c];
            cy = s.Rn[3 * a + 1] - s.Rn[c + 1];
            cz = s.Rn[3 * a + 2] - s.Rn[c + 2];
        } else {
            cx = diff_f2(s.Rn_hi[3 * a], s.Rn_lo[3 * a], s.Rn_hi[c], s.Rn_lo[c]);
            cy = diff_f2(s.Rn_hi[3 * a + 1], s.Rn_lo[3 * a + 1], s.Rn_hi[c + 1], s.Rn_lo[c + 1]);
            cz = diff_f2(s.Rn_hi[3 * a + 2], s.Rn_lo[3 * a + 2], s.Rn_hi[c + 2], s.Rn_lo[c + 2]);
        }
        const T amin = sys_amin<T>(s)[sh];
        const T gap = sqrt(cx * cx + cy * cy + cz * cz) - r;
        if (gap > T(0) && amin * gap * gap > T(kScreenExponent)) continue;
        const int l = d.y & 0xff, pure = d.y >> 8, fn0 = s.shell_fn[sh];
        const int nf = shell_nfn(l, pure);
        T uf[6], bs[6];
#pragma unroll
        for (int f = 0; f < 6; ++f) {
            uf[f] = f < nf ? u[fn0 + f] : T(0);
            bs[f] = T(0);
        }
        T fb[3] = {T(0), T(0), T(0)};
        const T* al = sys_alpha<T>(s);
        const T* cn = sys_cn<T>(s);
        for (int q = 0; q < nqb; ++q) {
            const T x = cx + dq[q][0], y = cy + dq[q][1], z = cz + dq[q][2];
            const T t = x * x + y * y + z * z;
            if (amin * t > T(kScreenExponent)) continue;
            T f0 = T(0), f1 = T(0);
            for (int pp = d.z; pp < d.z + d.w; ++pp) {
                const T aa = al[pp];
                if (aa * t > T(kScreenExponent)) continue;
                const T e = cn[pp] * dexp<T>(-aa * t);
                f0 += e;
                f1 -= aa * e;
            }
            T g[3] = {T(0), T(0), T(0)};
            for (int f = 0; f < nf; ++f) {
                const AngPoly<T> ap = angular<T>(l, pure, f, x, y, z);
                bs[f] += cq[q] * ap.P * f0;
                const T tf = T(2) * ap.P * f1;
                g[0] += (tf * x + ap.Px * f0) * uf[f];
                g[1] += (tf * y + ap.Py * f0) * uf[f];
                g[2] += (tf * z + ap.Pz * f0) * uf[f];
            }
            const T gd = (g[0] * dq[q][0] + g[1] * dq[q][1] + g[2] * dq[q][2]) * ir;
#pragma unroll
            for (int cc = 0; cc < 3; ++cc) {
                fb[cc] -= cq[q] * g[cc];
                mot[cc] += cq[q] * (g[cc] - gd * xh[cc]);
            }
        }
        for (int f = 0; f < nf; ++f) atomicAdd(&beta[fn0 + f], bs[f]);
#pragma unroll
        for (int cc = 0; cc < 3; ++cc) atomicAdd(&Fd[c + cc], (double)fb[cc]);
    }
    // Jastrow: electron pairs (gradient at r' only)
    const T ax = T(s.Rn[3 * a]), ay = T(s.Rn[3 * a + 1]), az = T(s.Rn[3 * a + 2]);
    const T ex = T(sR[3 * i]), ey = T(sR[3 * i + 1]), ez = T(sR[3 * i + 2]);
    for (int j = lane; j < N; j += 32) {
        if (j == i) continue;
        const T aa = T(((i < nu) == (j < nu)) ? s.a_par : s.a_anti), bb = T(s.b_ee);
        T jx, jy, jz;
        if constexpr (sizeof(T) == 8) {
            jx = sR[3 * j]; jy = sR[3 * j + 1]; jz = sR[3 * j + 2];
        } else {
            jx = sRf[3 * j]; jy = sRf[3 * j + 1]; jz = sRf[3 * j + 2];
        }
        const T cx = ax - jx, cy = ay - jy, cz = az - jz;
        for (int q = 0; q < nqb; ++q) {
            const T x = cx + dq[q][0], y = cy + dq[q][1], z = cz + dq[q][2];
            const T rn = sqrt(x * x + y * y + z * z);
            const T qd = T(1) / (T(1) + bb * rn);
            const T gr = aa * qd * qd / rn;   // u'(r) / r
            const T g[3] = {gr * x, gr * y, gr * z};
            const T gd = (g[0] * dq[q][0] + g[1] * dq[q][1] + g[2] * dq[q][2]) * ir;
            const T w = cq[q] * rq[q];
#pragma unroll
            for (int cc = 0; cc < 3; ++cc) mot[cc] += w * (g[cc] - gd * xh[cc]);
        }
    }
    // Jastrow: electron-nucleus terms (gradient at r' and the explicit nuclear derivative)
    for (int b = lane; b < s.n_nuc; b += 32) {
        const T aa = T(s.a_en[b]), bb = T(s.b_en);
        const T bx = T(s.Rn[3 * b]), by = T(s.Rn[3 * b + 1]), bz = T(s.Rn[3 * b + 2]);
        const T ox = ex - bx, oy = ey - by, oz = ez - bz;
        const T ro = sqrt(ox * ox + oy * oy + oz * oz);
        const T qo = T(1) / (T(1) + bb * ro);
        const T go = aa * qo * qo / ro;
        const T cx = ax - bx, cy = ay - by, cz = az - bz;
        T fe[3] = {T(0), T(0), T(0)};
        for (int q = 0; q < nqb; ++q) {
            const T x = cx + dq[q][0], y = cy + dq[q][1], z = cz + dq[q][2];
            const T rn = sqrt(x * x + y * y + z * z);
            const T qd = T(1) / (T(1) + bb * rn);
            const T gr = aa * qd * qd / rn;
            const T g[3] = {gr * x, gr * y, gr * z};
            const T gd = (g[0] * dq[q][0] + g[1] * dq[q][1] + g[2] * dq[q][2]) * ir;
            const T w = cq[q] * rq[q];
            fe[0] += w * (go * ox - g[0]);
            fe[1] += w * (go * oy - g[1]);
            fe[2] += w * (go * oz - g[2]);
#pragma unroll
            for (int cc = 0; cc < 3; ++cc) mot[cc] += w * (g[cc] - gd * xh[cc]);
        }
#pragma unroll
        for (int cc = 0; cc < 3; ++cc) atomicAdd(&Fd[3 * b + cc], (double)fe[cc]);
    }
}

// Parameter pass, lane's share for one pair's batch of points given per point
// f_q = W_q rho_q (the point's term of V_NL): adds f_q (B_p(r'_q) - B_p(r_i))
// for every Jastrow parameter p, B_p = dJ/dp restricted to the terms of
// electron i (parameter order a_anti, a_par, b_ee, b_en, a_en[n_nuc],
// c3[n_nuc][n3]).  The electron-pair parameters and b_en accumulate in the
// lane's acc; the nucleus-indexed ones in the warp's row dv, each nucleus
// owned by one lane, so the order of the sums is fixed.  Changes of the pair
// functions are formed directly, r/(1+br) as (r' - r) / ((1 + b r')(1 + b r)).
__device__ void param_lane(const DevSys& s, const double* sR, int i, int a, const double* pt, int p0,
                           const double (&f)[kQ], int nqb, double (&acc)[4], double* dv, int lane) {
    const int N = s.N, nu = s.n_up, nn = s.n_nuc;
    const double* ri = sR + 3 * i;
    const double* Ra = s.Rn + 3 * a;
    double rp[kQ][3];
#pragma unroll
    for (int q = 0; q < kQ; ++q)
#pragma unroll
        for (int c = 0; c < 3; ++c) rp[q][c] = q < nqb ? Ra[c] + pt[8 * (p0 + q) + c] : 0.0;
    for (int j = lane; j < N; j += 32) {
        if (j == i) continue;
        const bool like = (i < nu) == (j < nu);
        const double aa = like ? s.a_par : s.a_anti;
        const double* rj = sR + 3 * j;
        const double ro = sqrt((ri[0] - rj[0]) * (ri[0] - rj[0]) + (ri[1] - rj[1]) * (ri[1] - rj[1]) +
                               (ri[2] - rj[2]) * (ri[2] - rj[2]));
        const double qo = 1.0 / (1.0 + s.b_ee * ro);
#pragma unroll
        for (int q = 0; q < kQ; ++q)
            if (q < nqb) {
                const double x = rp[q][0] - rj[0], y = rp[q][1] - rj[1], z = rp[q][2] - rj[2];
                const double rn = sqrt(x * x + y * y + z * z), qn = 1.0 / (1.0 + s.b_ee * rn);
                const double dB = (rn - ro) * qn * qo;
                acc[like ? 1 : 0] += f[q] * dB;
                // d/db of a r / (1 + b r) is -a (r q)^2: its change is -a dB (r' q' + r q)
                acc[2] -= f[q] * aa * dB * (rn * qn + ro * qo);
            }
    }
    for (int b = lane; b < nn; b += 32) {
        const double* Rb = s.Rn + 3 * b;
        const double ro = sqrt((ri[0] - Rb[0]) * (ri[0] - Rb[0]) + (ri[1] - Rb[1]) * (ri[1] - Rb[1]) +
                               (ri[2] - Rb[2]) * (ri[2] - Rb[2]));
        const double qo = 1.0 / (1.0 + s.b_en * ro);
        double da = 0.0;
#pragma unroll
        for (int q = 0; q < kQ; ++q)
            if (q < nqb) {
                const double x = rp[q][0] - Rb[0], y = rp[q][1] - Rb[1], z = rp[q][2] - Rb[2];
                const double rn = sqrt(x * x + y * y + z * z), qn = 1.0 / (1.0 + s.b_en * rn);
                const double dB = (rn - ro) * qn * qo;
                da += f[q] * dB;
                acc[3] -= f[q] * s.a_en[b] * dB * (rn * qn + ro * qo);
            }
        dv[4 + b] += da;
        if (s.n3 == 0) continue;
        // three-body terms of nucleus b: pairs (i, j) with the moved electron
        double* d3 = dv + 4 + nn + (size_t)b * s.n3;
        const SDist xo = sdist(s.b3, ri[0] - Rb[0], ri[1] - Rb[1], ri[2] - Rb[2]);
        for (int j = 0; j < N; ++j) {
            if (j == i) continue;
            const double* rj = sR + 3 * j;
            const SDist xj = sdist(s.b3, rj[0] - Rb[0], rj[1] - Rb[1], rj[2] - Rb[2]);
            const SDist yo = sdist(s.b3, ri[0] - rj[0], ri[1] - rj[1], ri[2] - rj[2]);
            for (int q = 0; q < nqb; ++q) {
                const SDist xn = sdist(s.b3, rp[q][0] - Rb[0], rp[q][1] - Rb[1], rp[q][2] - Rb[2]);
                const SDist yn = sdist(s.b3, rp[q][0] - rj[0], rp[q][1] - rj[1], rp[q][2] - rj[2]);
                for (int k = 0; k < s.n3; ++k) {
                    const int m = s.e3[3 * k], n = s.e3[3 * k + 1], o = s.e3[3 * k + 2];
                    const double vn = (ipow_d(xn.s, m) * ipow_d(xj.s, n) + ipow_d(xn.s, n) * ipow_d(xj.s, m)) *
                                      ipow_d(yn.s, o);
                    const double vo = (ipow_d(xo.s, m) * ipow_d(xj.s, n) + ipow_d(xo.s, n) * ipow_d(xj.s, m)) *
                                      ipow_d(yo.s, o);
                    d3[k] += f[q] * (vn - vo);
                }
            }
        }
    }
}

// Walkers w0 + blockIdx.x < W.  Ug0 / Ug1: u_k of every electron of the
// launch's walkers per spin, [w - w0][k][ldu] (formed on the tensor cores
// beforehand), or nullptr: formed here.
template <typename T, int kMode>
__global__ void __launch_bounds__(kNlThreads) k_nlpp(DevSys s, DevWalkers wk, int w0, int W, double* eloc, uint2 key,
                                                      uint32_t sweep, const T* __restrict__ Ug0,
                                                      const T* __restrict__ Ug1, T* nlB0, T* nlB1, double* nlF) {
    constexpr bool kForce = kMode == kNlForce;
    // parameter pass: eloc is deloc [W][P], P = 4 + n_nuc (1 + n3)
    const int P = 4 + s.n_nuc * (1 + s.n3);
    extern __shared__ __align__(16) unsigned char smem[];
    const int w = w0 + (int)blockIdx.x;
    if (w >= W) return;
    const int N = s.N, nu = s.n_up, nmax = s.n_up > s.n_dn ? s.n_up : s.n_dn;
    const int nb = s.n_basis, ldu = (nb + 3) & ~3, nq = s.pp_nq;
    const NlLayout L = nl_layout<T>(N, nmax, nb, s.n_ecp, s.n_shell, s.n_nuc, kMode, P);
    double* sR = (double*)(smem + L.sR);
    float* sRf = (float*)(smem + L.sRf);
    double* rot = (double*)(smem + L.rot);
    int* el = (int*)(smem + L.el);
    T* Ak = (T*)(smem + L.Ak);
    T* U = (T*)(smem + L.U);
    int2* pairs = (int2*)(smem + L.pairs);
    double* pg = (double*)(smem + L.pg);
    double* pt = (double*)(smem + L.pt);
    float* ptf = (float*)(smem + L.ptf);
    double* jold = (double*)(smem + L.jold);
    T* beta = (T*)(smem + L.beta);
    double* Fd = (double*)(smem + L.Fd);
    double* dvw = (double*)(smem + L.dvw);
    if constexpr (kForce)
        for (int q = threadIdx.x; q < 3 * s.n_nuc; q += blockDim.x) Fd[q] = 0.0;
    if constexpr (kMode == kNlParam)
        for (int q = threadIdx.x; q < kNlWarps * P; q += blockDim.x) dvw[q] = 0.0;
    double pacc[4] = {0.0, 0.0, 0.0, 0.0};   // parameter pass: this lane's a_anti, a_par, b_ee, b_en parts
    const int nmax4 = (nmax + 3) & ~3;
    __shared__ int s_count, s_npair;
    __shared__ int s_wcnt[kNlWarps];
    __shared__ double s_part[kNlWarps];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;

    for (int q = tid; q < 3 * N; q += blockDim.x) {
        sR[q] = wk.R[(size_t)w * 3 * N + q];
        sRf[q] = (float)sR[q];
    }
    for (int k = tid; k < s.n_ecp; k += blockDim.x) {
        double* m = rot + 9 * k;
        if (s.pp_rotate) {
            pp_rotation(key, sweep, (uint32_t)s.ecp_nuc[k], (uint32_t)w, m);
        } else {
            for (int c = 0; c < 9; ++c) m[c] = (c % 4 == 0) ? 1.0 : 0.0;
        }
    }
    if (tid == 0) s_count = 0;
    __syncthreads();
    // electrons within some cutoff, ascending (warp-ordered ballots)
    for (int base = 0; base < N; base += blockDim.x) {
        const int i = base + tid;
        int in = 0;
        if (i < N)
            for (int k = 0; k < s.n_ecp && !in; ++k) {
                const int a = s.ecp_nuc[k];
                const double x = sR[3 * i] - s.Rn[3 * a], y = sR[3 * i + 1] - s.Rn[3 * a + 1],
                             z = sR[3 * i + 2] - s.Rn[3 * a + 2];
                in = sqrt(x * x + y * y + z * z) < s.pp_rcut[a];
            }
        const unsigned bal = __ballot_sync(0xffffffffu, in);
        if (lane == 0) s_wcnt[wid] = __popc(bal);
        __syncthreads();
        int off = s_count;
        for (int q = 0; q < wid; ++q) off += s_wcnt[q];
        if (in) el[off + __popc(bal & ((1u << lane) - 1u))] = i;
        __syncthreads();
        if (tid == 0) {
            int t = 0;
            for (int q = 0; q < kNlWarps; ++q) t += s_wcnt[q];
            s_count = s_count + t;
        }
        __syncthreads();
    }
    const int M = s_count;
    const int gsize = kPtCap / nq;   // pairs per pass (the setter keeps nq <= kPtCap)
    double part = 0.0;               // this warp's points (lane 0)

    for (int c0 = 0; c0 < M;) {
        // chunk: up to kChunk listed electrons of the spin of el[c0]
        const int spin = el[c0] >= nu;
        int c1 = c0;
        while (c1 < M && c1 - c0 < kChunk && (el[c1] >= nu) == spin) ++c1;
        const int nc = c1 - c0;
        const int n = spin ? s.n_dn : nu;
        const T* Ainv = (const T*)wk.Ainv[spin];
        const T* Ug = spin ? Ug1 : Ug0;
        const int n4 = (n + 3) & ~3;
        if (Ug) {
            // u_k precomputed: the chunk's rows into shared memory
            for (int q = tid; q < nc * ldu; q += blockDim.x) {
                const int ce = q / ldu, b = q - ce * ldu;
                const int k = el[c0 + ce] - (spin ? nu : 0);
                U[q] = Ug[((size_t)(w - w0) * n + k) * ldu + b];
            }
        } else {
            for (int q = tid; q < nc * n4; q += blockDim.x) {
                const int ce = q / n4, j = q - ce * n4;
                const int k = el[c0 + ce] - (spin ? nu : 0);
                Ak[ce * nmax4 + j] = j < n ? Ainv[((size_t)w * n + k) * n + j] : T(0);
            }
        }
        if constexpr (kForce)
            for (int q = tid; q < kChunk * ldu; q += blockDim.x) beta[q] = T(0);
        // (electron, nucleus) pairs of the chunk, ascending in both
        if (wid == 0) {
            int np = 0;
            for (int ce = 0; ce < nc; ++ce) {
                const int i = el[c0 + ce];
                for (int k0 = 0; k0 < s.n_ecp; k0 += 32) {
                    const int k = k0 + lane;
                    int in = 0;
                    if (k < s.n_ecp) {
                        const int a = s.ecp_nuc[k];
                        const double x = sR[3 * i] - s.Rn[3 * a], y = sR[3 * i + 1] - s.Rn[3 * a + 1],
                                     z = sR[3 * i + 2] - s.Rn[3 * a + 2];
                        in = sqrt(x * x + y * y + z * z) < s.pp_rcut[a];
                    }
                    const unsigned bal = __ballot_sync(0xffffffffu, in);
                    if (in) pairs[np + __popc(bal & ((1u << lane) - 1u))] = make_int2(ce, k);
                    np += __popc(bal);
                }
            }
            if (lane == 0) s_npair = np;
        }
        __syncthreads();
        // u_ce = C_spin A^-1 e_k over the basis (orbital-major coefficients:
        // consecutive threads read consecutive basis functions)
        if (!Ug) {
            const T* Cs;
            if constexpr (sizeof(T) == 8) Cs = s.CT[spin];
            else Cs = s.CT_f[spin];
            for (int b = tid; b < nb; b += blockDim.x) {
                T acc[kChunk];
#pragma unroll
                for (int ce = 0; ce < kChunk; ++ce) acc[ce] = T(0);
                for (int j = 0; j < n4; j += 4) {
                    // four coefficients, then each chunk electron's four
                    // inverse entries as one vector load (rows padded with zeros)
                    T cv[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) cv[q] = j + q < n ? Cs[(size_t)(j + q) * nb + b] : T(0);
#pragma unroll
                    for (int ce = 0; ce < kChunk; ++ce)
                        if (ce < nc) {
                            const T* a = Ak + ce * nmax4 + j;
                            if constexpr (sizeof(T) == 4) {
                                const float4 v = *reinterpret_cast<const float4*>(a);
                                acc[ce] += cv[0] * v.x + cv[1] * v.y + cv[2] * v.z + cv[3] * v.w;
                            } else {
                                const double2 v0 = *reinterpret_cast<const double2*>(a);
                                const double2 v1 = *reinterpret_cast<const double2*>(a + 2);
                                acc[ce] += cv[0] * v0.x + cv[1] * v0.y + cv[2] * v1.x + cv[3] * v1.y;
                            }
                        }
                }
#pragma unroll
                for (int ce = 0; ce < kChunk; ++ce)
                    if (ce < nc) U[ce * ldu + b] = acc[ce];
            }
        }
        if constexpr (sizeof(T) == 8) {
            // Jastrow terms of each chunk electron at its old position (one warp each)
            for (int ce = wid; ce < nc; ce += kNlWarps) {
                const int i = el[c0 + ce];
                double J = jastrow_terms_lane(s, sR, i, sR + 3 * i, lane);
                for (int o = 16; o > 0; o >>= 1) J += __shfl_xor_sync(0xffffffffu, J, o);
                if (lane == 0) jold[ce] = J;
            }
        }
        __syncthreads();
        const int npair = s_npair;
        for (int g0 = 0; g0 < npair; g0 += gsize) {
            const int ng = min(gsize, npair - g0), npts = ng * nq;
            // pair data: unit vector from the nucleus, distance, channel potentials
            for (int t = tid; t < ng; t += blockDim.x) {
                const int2 pk = pairs[g0 + t];
                const int i = el[c0 + pk.x], a = s.ecp_nuc[pk.y];
                double x[3], r2 = 0.0;
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    x[c] = sR[3 * i + c] - s.Rn[3 * a + c];
                    r2 += x[c] * x[c];
                }
                const double r = sqrt(r2);
                double* d = pg + 12 * t;
#pragma unroll
                for (int c = 0; c < 3; ++c) d[c] = x[c] / r;
                d[3] = r;
                double v[4] = {0.0, 0.0, 0.0, 0.0}, dv[4] = {0.0, 0.0, 0.0, 0.0};
                for (int k = s.pp_off[a]; k < s.pp_off[a + 1]; ++k) {
                    const int2 ln = s.pp_ln[k];
                    if (ln.x >= 0) {
                        v[ln.x] += pp_term<double>(s, k, ln.y, r);
                        if constexpr (kForce) dv[ln.x] += pp_term_dr<double>(s, k, ln.y, r);
                    }
                }
#pragma unroll
                for (int l = 0; l < 4; ++l) {
                    d[4 + l] = v[l];
                    d[8 + l] = dv[l];
                }
            }
            __syncthreads();
            // point data: offset r d_q from the nucleus and weight w_q sum_l (2l+1) v_l P_l(cos)
            for (int t = tid; t < npts; t += blockDim.x) {
                const int pr = t / nq, q = t - pr * nq;
                const int2 pk = pairs[g0 + pr];
                const double* m = rot + 9 * pk.y;
                const double* o = s.pp_quad + 3 * q;
                const double* d = pg + 12 * pr;
                double cth = 0.0, dqv[3];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const double dq = m[3 * c] * o[0] + m[3 * c + 1] * o[1] + m[3 * c + 2] * o[2];
                    dqv[c] = dq;
                    cth += dq * d[c];
                    pt[8 * t + c] = d[3] * dq;
                    ptf[3 * t + c] = (float)(d[3] * dq);
                }
                double wq = 0.0, dw[3] = {0.0, 0.0, 0.0};
#pragma unroll
                for (int l = 0; l < 4; ++l)
                    if (d[4 + l] != 0.0) {
                        const double f = 2.0 * l + 1.0;
                        wq += f * legendre(l, cth) * d[4 + l];
                        if constexpr (kForce) {
                            // d/dR_a of v_l(r) P_l(cos): dr/dR_a = -x_hat, dcos/dR_a = -(d - cos x_hat) / r
#pragma unroll
                            for (int c = 0; c < 3; ++c)
                                dw[c] += f * (d[8 + l] * legendre(l, cth) * (-d[c]) +
                                              d[4 + l] * legendre_dx(l, cth) * (-(dqv[c] - cth * d[c]) / d[3]));
                        }
                    }
                pt[8 * t + 3] = wq * s.pp_qw[q];
#pragma unroll
                for (int c = 0; c < 3; ++c) pt[8 * t + 4 + c] = dw[c] * s.pp_qw[q];
            }
            __syncthreads();
            // one warp per pair, its points in register batches of kQ
            for (int pr = wid; pr < ng; pr += kNlWarps) {
                const int2 pk = pairs[g0 + pr];
                const int ce = pk.x, i = el[c0 + ce], a = s.ecp_nuc[pk.y];
                const T r = (T)pg[12 * pr + 3];
                for (int q0 = 0; q0 < nq; q0 += kQ) {
                    const int nqb = min(kQ, nq - q0);
                    const int p0 = pr * nq + q0;
                    T dq[kQ][3], dr[kQ], dj[kQ];
#pragma unroll
                    for (int q = 0; q < kQ; ++q) {
                        dr[q] = dj[q] = T(0);
#pragma unroll
                        for (int c = 0; c < 3; ++c) {
                            if constexpr (sizeof(T) == 8) dq[q][c] = q < nqb ? pt[8 * (p0 + q) + c] : 0.0;
                            else dq[q][c] = q < nqb ? ptf[3 * (p0 + q) + c] : 0.f;
                        }
                    }
                    pair_basis_lane<T>(s, a, r, dq, nqb, U + ce * ldu, dr, lane);
                    if constexpr (sizeof(T) == 8) pair_jastrow_lane_d(s, sR, i, a, dq, nqb, dj, lane);
                    else pair_jastrow_lane_f(s, sRf, i, a, dq, nqb, dj, lane);
                    if (s.n3 > 0) {
                        // three-body change, point by point in FP64
                        const double re[3] = {sR[3 * i], sR[3 * i + 1], sR[3 * i + 2]};
                        const double J3o = jastrow3_lane(s, sR, i, re, lane);
                        for (int q = 0; q < nqb; ++q) {
                            const double rp[3] = {s.Rn[3 * a] + pt[8 * (p0 + q)], s.Rn[3 * a + 1] + pt[8 * (p0 + q) + 1],
                                                  s.Rn[3 * a + 2] + pt[8 * (p0 + q) + 2]};
                            const double d3 = jastrow3_lane(s, sR, i, rp, lane) - (sizeof(T) == 8 ? 0.0 : J3o);
#pragma unroll
                            for (int qq = 0; qq < kQ; ++qq)
                                if (qq == q) dj[qq] += (T)d3;
                        }
                    }
#pragma unroll
                    for (int q = 0; q < kQ; ++q)
                        for (int o = 16; o > 0; o >>= 1) {
                            dr[q] += __shfl_xor_sync(0xffffffffu, dr[q], o);
                            dj[q] += __shfl_xor_sync(0xffffffffu, dj[q], o);
                        }
                    if constexpr (kForce) {
                        T cq[kQ], ej[kQ];
#pragma unroll
                        for (int q = 0; q < kQ; ++q) {
                            if constexpr (sizeof(T) == 8) ej[q] = q < nqb ? exp(dj[q] - jold[ce]) : 0.0;
                            else ej[q] = q < nqb ? expf(dj[q]) : 0.f;
                            cq[q] = q < nqb ? (T)pt[8 * (p0 + q) + 3] * ej[q] : T(0);
                        }
                        const T xh[3] = {(T)pg[12 * pr], (T)pg[12 * pr + 1], (T)pg[12 * pr + 2]};
                        T mot[3] = {T(0), T(0), T(0)};
                        pair_force_lane<T>(s, sR, sRf, i, a, r, dq, nqb, cq, dr, xh, U + ce * ldu, beta + ce * ldu, Fd,
                                           mot, lane);
#pragma unroll
                        for (int c = 0; c < 3; ++c)
                            for (int o = 16; o > 0; o >>= 1) mot[c] += __shfl_xor_sync(0xffffffffu, mot[c], o);
                        if (lane == 0) {
                            double fa[3] = {(double)mot[0], (double)mot[1], (double)mot[2]};
                            for (int q = 0; q < nqb; ++q)
#pragma unroll
                                for (int c = 0; c < 3; ++c) fa[c] += pt[8 * (p0 + q) + 4 + c] * (double)(ej[q] * dr[q]);
#pragma unroll
                            for (int c = 0; c < 3; ++c) atomicAdd(&Fd[3 * a + c], fa[c]);
                        }
                    } else if constexpr (kMode == kNlParam) {
                        // every lane holds the warp totals dr, dj after the butterfly
                        double fq[kQ];
#pragma unroll
                        for (int q = 0; q < kQ; ++q) {
                            fq[q] = 0.0;
                            if (q < nqb) {
                                if constexpr (sizeof(T) == 8) fq[q] = pt[8 * (p0 + q) + 3] * dr[q] * exp(dj[q] - jold[ce]);
                                else fq[q] = pt[8 * (p0 + q) + 3] * (double)(dr[q] * expf(dj[q]));
                            }
                        }
                        param_lane(s, sR, i, a, pt, p0, fq, nqb, pacc, dvw + wid * P, lane);
                    } else if (lane == 0) {
#pragma unroll
                        for (int q = 0; q < kQ; ++q) {
                            if (q < nqb) {
                                if constexpr (sizeof(T) == 8) part += pt[8 * (p0 + q) + 3] * dr[q] * exp(dj[q] - jold[ce]);
                                else part += pt[8 * (p0 + q) + 3] * (double)(dr[q] * expf(dj[q]));
                            }
                        }
                    }
                }
            }
            __syncthreads();
        }
        if constexpr (kForce) {
            // rows of B_NL for the chunk's electrons: sum_l C[l][j] beta[l]
            const T* Cs = sys_C<T>(s, spin);
            T* out = spin ? nlB1 : nlB0;
            for (int q = tid; q < nc * n; q += blockDim.x) {
                const int ce = q / n, j = q - ce * n;
                const int k = el[c0 + ce] - (spin ? nu : 0);
                const T* bc = beta + ce * ldu;
                T v = T(0);
                for (int l = 0; l < nb; ++l) v += Cs[(size_t)l * n + j] * bc[l];
                out[((size_t)w * n + k) * n + j] = v;
            }
            __syncthreads();
        }
        c0 = c1;
    }
    if constexpr (kForce) {
        __syncthreads();
        for (int q = tid; q < 3 * s.n_nuc; q += blockDim.x) nlF[(size_t)w * 3 * s.n_nuc + q] = Fd[q];
        return;
    }
    if constexpr (kMode == kNlParam) {
#pragma unroll
        for (int c = 0; c < 4; ++c)
            for (int o = 16; o > 0; o >>= 1) pacc[c] += __shfl_xor_sync(0xffffffffu, pacc[c], o);
        if (lane == 0)
#pragma unroll
            for (int c = 0; c < 4; ++c) dvw[wid * P + c] += pacc[c];
        __syncthreads();
        for (int q = tid; q < P; q += blockDim.x) {
            double v = 0.0;
            for (int k = 0; k < kNlWarps; ++k) v += dvw[k * P + q];
            eloc[(size_t)w * P + q] += v;
        }
        return;
    }
    if (lane == 0) s_part[wid] = part;
    __syncthreads();
    if (tid == 0) {
        double v = 0.0;
        for (int q = 0; q < kNlWarps; ++q) v += s_part[q];
        eloc[w] += v;
        if (!isfinite(eloc[w]) && wk.err) atomicOr(wk.err, kErrNonFinite);
    }
}

}  // namespace

template <typename T>
cudaError_t launch_nlpp(const DevSys& s, const DevWalkers& wk, int w0, int W, double* eloc, uint2 key, uint32_t sweep,
                        const void* U0, const void* U1, cudaStream_t st) {
    if (W <= w0 || s.npp == 0 || s.n_ecp == 0) return cudaSuccess;
    if (s.pp_nq < 1 || s.pp_nq > kPtCap) return cudaErrorInvalidValue;
    const int nmax = s.n_up > s.n_dn ? s.n_up : s.n_dn;
    const size_t smem = nl_layout<T>(s.N, nmax, s.n_basis, s.n_ecp, s.n_shell, s.n_nuc, kNlEnergy, 0).total;
    if (smem > 227 * 1024) return cudaErrorNotSupported;   // the host reports QMC_ERR_UNSUPPORTED
    cudaError_t e =
        cudaFuncSetAttribute(k_nlpp<T, kNlEnergy>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_nlpp<T, kNlEnergy><<<W - w0, kNlThreads, smem, st>>>(s, wk, w0, W, eloc, key, sweep, (const T*)U0,
                                                          (const T*)U1, nullptr, nullptr, nullptr);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_nlpp_param(const DevSys& s, const DevWalkers& wk, int w0, int W, double* deloc, uint2 key,
                              uint32_t sweep, const void* U0, const void* U1, cudaStream_t st) {
    if (W <= w0 || s.npp == 0 || s.n_ecp == 0) return cudaSuccess;
    if (s.pp_nq < 1 || s.pp_nq > kPtCap) return cudaErrorInvalidValue;
    const int nmax = s.n_up > s.n_dn ? s.n_up : s.n_dn, P = 4 + s.n_nuc * (1 + s.n3);
    const size_t smem = nl_layout<T>(s.N, nmax, s.n_basis, s.n_ecp, s.n_shell, s.n_nuc, kNlParam, P).total;
    if (smem > 227 * 1024) return cudaErrorNotSupported;   // the host reports QMC_ERR_UNSUPPORTED
    cudaError_t e = cudaFuncSetAttribute(k_nlpp<T, kNlParam>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_nlpp<T, kNlParam><<<W - w0, kNlThreads, smem, st>>>(s, wk, w0, W, deloc, key, sweep, (const T*)U0, (const T*)U1,
                                                         nullptr, nullptr, nullptr);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_nlpp_force(const DevSys& s, const DevWalkers& wk, int w0, int W, void* nlB0, void* nlB1,
                              double* nlF, uint2 key, uint32_t sweep, const void* U0, const void* U1,
                              cudaStream_t st) {
    if (W <= w0 || s.npp == 0 || s.n_ecp == 0) return cudaSuccess;
    if (s.pp_nq < 1 || s.pp_nq > kPtCap) return cudaErrorInvalidValue;
    const int nmax = s.n_up > s.n_dn ? s.n_up : s.n_dn;
    const size_t smem = nl_layout<T>(s.N, nmax, s.n_basis, s.n_ecp, s.n_shell, s.n_nuc, kNlForce, 0).total;
    if (smem > 227 * 1024) return cudaErrorNotSupported;   // the host reports QMC_ERR_UNSUPPORTED
    cudaError_t e = cudaFuncSetAttribute(k_nlpp<T, kNlForce>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_nlpp<T, kNlForce><<<W - w0, kNlThreads, smem, st>>>(s, wk, w0, W, nullptr, key, sweep, (const T*)U0,
                                                         (const T*)U1, (T*)nlB0, (T*)nlB1, nlF);
    return cudaGetLastError();
}

template cudaError_t launch_nlpp<double>(const DevSys&, const DevWalkers&, int, int, double*, uint2, uint32_t,
                                         const void*, const void*, cudaStream_t);
template cudaError_t launch_nlpp<float>(const DevSys&, const DevWalkers&, int, int, double*, uint2, uint32_t,
                                        const void*, const void*, cudaStream_t);
template cudaError_t launch_nlpp_param<double>(const DevSys&, const DevWalkers&, int, int, double*, uint2, uint32_t,
                                               const void*, const void*, cudaStream_t);
template cudaError_t launch_nlpp_param<float>(const DevSys&, const DevWalkers&, int, int, double*, uint2, uint32_t,
                                              const void*, const void*, cudaStream_t);
template cudaError_t launch_nlpp_force<double>(const DevSys&, const DevWalkers&, int, int, void*, void*, double*,
                                               uint2, uint32_t, const void*, const void*, cudaStream_t);
template cudaError_t launch_nlpp_force<float>(const DevSys&, const DevWalkers&, int, int, void*, void*, double*,
                                              uint2, uint32_t, const void*, const void*, cudaStream_t);

}  // namespace qmc
