/*
 * CPU FP64 oracle for the walker-batched Slater-Jastrow DMC hot path.
 *
 * TEST INFRASTRUCTURE ONLY: only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  The CUDA library is
 * written independently and never calls into this file.
 *
 * Every quantity is computed from its plain definition in FP64, with no
 * incremental updates: determinants are refactorised by LU after every
 * proposed move, ionic derivatives are taken one nuclear coordinate at a
 * time (the forward form whose cost the paper states as O(N^3 * 3 N_atom),
 * Sec. "Single Determinant QMC Forces", Eqs. 3-4).
 *
 * Conventions (shared with the CUDA library only as documented interface,
 * never as code):
 *   - primitive x^i y^j z^k exp(-a r^2) with the Cartesian normalisation
 *     (2a/pi)^(3/4) (4a)^(l/2) / sqrt((2i-1)!!(2j-1)!!(2k-1)!!); a contracted
 *     shell is rescaled to unit norm with the closed-form overlap of
 *     normalised primitives (2 sqrt(a b)/(a+b))^(l+3/2).  Shells containing a
 *     zero exponent keep their raw weights (they are not normalisable);
 *   - pure d: (sqrt3 xy, sqrt3 yz, z^2-(x^2+y^2)/2, sqrt3 xz,
 *     sqrt3/2 (x^2-y^2)) times the (2,0,0) primitive normalisation;
 *   - Cartesian d order xx, xy, xz, yy, yz, zz; p order x, y, z;
 *   - Pade Jastrow u(r) = a r / (1 + b r); pairs of unlike spin use a_anti,
 *     like spins a_par; electron-nucleus pairs use a_en[a], b_en;
 *   - electrons 0..n_up-1 are spin up, the rest spin down.
 */
#include "qmc_oracle.h"

#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ------------------------------------------------------------------ */
/* threading: a plain parallel-for over walkers                        */
/* ------------------------------------------------------------------ */

typedef void (*walker_fn)(void* ctx, int w);

typedef struct {
    walker_fn fn;
    void* ctx;
    int n, stride, first;
} pf_arg;

static void* pf_thread(void* p) {
    pf_arg* a = (pf_arg*)p;
    for (int w = a->first; w < a->n; w += a->stride) a->fn(a->ctx, w);
    return NULL;
}

static void parallel_for(int n, int nthreads, walker_fn fn, void* ctx) {
    if (nthreads <= 1 || n <= 1) {
        for (int w = 0; w < n; ++w) fn(ctx, w);
        return;
    }
    if (nthreads > n) nthreads = n;
    pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * nthreads);
    pf_arg* args = (pf_arg*)malloc(sizeof(pf_arg) * nthreads);
    for (int t = 0; t < nthreads; ++t) {
        args[t].fn = fn; args[t].ctx = ctx; args[t].n = n; args[t].stride = nthreads; args[t].first = t;
        pthread_create(&th[t], NULL, pf_thread, &args[t]);
    }
    for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
    free(th);
    free(args);
}

/* ------------------------------------------------------------------ */
/* basis                                                               */
/* ------------------------------------------------------------------ */

static const int DSLOT[OD_N][3] = {
    {0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}, {2, 0, 0}, {1, 1, 0}, {1, 0, 1}, {0, 2, 0}, {0, 1, 1},
    {0, 0, 2}, {3, 0, 0}, {2, 1, 0}, {2, 0, 1}, {1, 2, 0}, {1, 1, 1}, {1, 0, 2}, {0, 3, 0}, {0, 2, 1},
    {0, 1, 2}, {0, 0, 3}};
static const int NSLOT_BY_ORDER[4] = {1, 4, 10, 20};

static int slot_of(int a, int b, int c) {
    for (int k = 0; k < OD_N; ++k)
        if (DSLOT[k][0] == a && DSLOT[k][1] == b && DSLOT[k][2] == c) return k;
    return -1;
}

static double dfact(int n) { /* n!!, with (-1)!! = 1 */
    double r = 1.0;
    for (int k = n; k > 1; k -= 2) r *= (double)k;
    return r;
}

static int shell_nfn(int l, int pure) {
    if (l == 0) return 1;
    if (l == 1) return 3;
    return pure ? 5 : 6;
}

/* One angular function of a shell as a sum of at most three monomials. */
typedef struct {
    int nterm;
    int ijk[3][3];
    double w[3];
} angfn;

static void shell_angular(int l, int pure, angfn* out) {
    if (l == 0) {
        out[0].nterm = 1; out[0].ijk[0][0] = 0; out[0].ijk[0][1] = 0; out[0].ijk[0][2] = 0; out[0].w[0] = 1.0;
        return;
    }
    if (l == 1) {
        for (int c = 0; c < 3; ++c) {
            out[c].nterm = 1;
            out[c].ijk[0][0] = (c == 0); out[c].ijk[0][1] = (c == 1); out[c].ijk[0][2] = (c == 2);
            out[c].w[0] = 1.0;
        }
        return;
    }
    if (!pure) {
        static const int cart[6][3] = {{2, 0, 0}, {1, 1, 0}, {1, 0, 1}, {0, 2, 0}, {0, 1, 1}, {0, 0, 2}};
        for (int c = 0; c < 6; ++c) {
            out[c].nterm = 1;
            for (int d = 0; d < 3; ++d) out[c].ijk[0][d] = cart[c][d];
            /* relative to the (2,0,0) normalisation */
            out[c].w[0] = sqrt(dfact(3) / (dfact(2 * cart[c][0] - 1) * dfact(2 * cart[c][1] - 1) *
                                           dfact(2 * cart[c][2] - 1)));
        }
        return;
    }
    const double s3 = sqrt(3.0);
    memset(out, 0, sizeof(angfn) * 5);
    /* m = -2 : sqrt3 xy */
    out[0].nterm = 1; out[0].ijk[0][0] = 1; out[0].ijk[0][1] = 1; out[0].w[0] = s3;
    /* m = -1 : sqrt3 yz */
    out[1].nterm = 1; out[1].ijk[0][1] = 1; out[1].ijk[0][2] = 1; out[1].w[0] = s3;
    /* m = 0 : z^2 - (x^2 + y^2)/2 */
    out[2].nterm = 3;
    out[2].ijk[0][2] = 2; out[2].w[0] = 1.0;
    out[2].ijk[1][0] = 2; out[2].w[1] = -0.5;
    out[2].ijk[2][1] = 2; out[2].w[2] = -0.5;
    /* m = +1 : sqrt3 xz */
    out[3].nterm = 1; out[3].ijk[0][0] = 1; out[3].ijk[0][2] = 1; out[3].w[0] = s3;
    /* m = +2 : sqrt3/2 (x^2 - y^2) */
    out[4].nterm = 2;
    out[4].ijk[0][0] = 2; out[4].w[0] = 0.5 * s3;
    out[4].ijk[1][1] = 2; out[4].w[1] = -0.5 * s3;
}

typedef struct {
    int n_basis;
    int* first_prim;  /* [n_shell] */
    int* first_fn;    /* [n_shell] */
    int* fn_center;   /* [n_basis] */
    double* cnorm;    /* [n_prim] normalised contraction coefficients */
} basis_prep;

static double prim_norm(double a, int l) {
    return pow(2.0 * a / M_PI, 0.75) * pow(4.0 * a, 0.5 * l) / sqrt(dfact(2 * l - 1));
}

static void prep_basis(const oracle_system* s, basis_prep* p) {
    int np = 0, nb = 0;
    p->first_prim = (int*)malloc(sizeof(int) * (s->n_shell + 1));
    p->first_fn = (int*)malloc(sizeof(int) * (s->n_shell + 1));
    for (int sh = 0; sh < s->n_shell; ++sh) {
        p->first_prim[sh] = np;
        p->first_fn[sh] = nb;
        np += s->sh_nprim[sh];
        nb += shell_nfn(s->sh_l[sh], s->sh_pure[sh]);
    }
    p->first_prim[s->n_shell] = np;
    p->first_fn[s->n_shell] = nb;
    p->n_basis = nb;
    p->fn_center = (int*)malloc(sizeof(int) * (nb > 0 ? nb : 1));
    p->cnorm = (double*)malloc(sizeof(double) * (np > 0 ? np : 1));
    for (int sh = 0; sh < s->n_shell; ++sh) {
        for (int f = p->first_fn[sh]; f < p->first_fn[sh + 1]; ++f) p->fn_center[f] = s->sh_center[sh];
        const int l = s->sh_l[sh];
        const int p0 = p->first_prim[sh], p1 = p->first_prim[sh + 1];
        int has_zero = 0;
        for (int q = p0; q < p1; ++q)
            if (s->alpha[q] == 0.0) has_zero = 1;
        if (has_zero) {
            for (int q = p0; q < p1; ++q) p->cnorm[q] = s->coef[q];
            continue;
        }
        double S = 0.0;
        for (int q = p0; q < p1; ++q)
            for (int r = p0; r < p1; ++r) {
                const double a = s->alpha[q], b = s->alpha[r];
                S += s->coef[q] * s->coef[r] * pow(2.0 * sqrt(a * b) / (a + b), l + 1.5);
            }
        for (int q = p0; q < p1; ++q) p->cnorm[q] = s->coef[q] * prim_norm(s->alpha[q], l) / sqrt(S);
    }
}

static void free_basis(basis_prep* p) {
    free(p->first_prim);
    free(p->first_fn);
    free(p->fn_center);
    free(p->cnorm);
}

/* m-th derivatives (m = 0..maxm) of t^i exp(-a t^2) for i = 0..imax at t. */
static void gauss1d(double a, double t, int imax, int maxm, double E[3][4]) {
    const double g = exp(-a * t * t);
    for (int i = 0; i <= imax; ++i) {
        double poly[8] = {0};
        poly[i] = 1.0;
        for (int m = 0; m <= maxm; ++m) {
            double v = 0.0, tp = 1.0;
            for (int k = 0; k < 8; ++k) {
                v += poly[k] * tp;
                tp *= t;
            }
            E[i][m] = v * g;
            double np[8] = {0};
            for (int k = 1; k < 8; ++k) np[k - 1] += k * poly[k];
            for (int k = 0; k < 7; ++k) np[k + 1] -= 2.0 * a * poly[k];
            memcpy(poly, np, sizeof(poly));
        }
    }
}

/* out[f * OD_N + slot], slots with total order <= maxorder. */
static void basis_eval(const oracle_system* s, const basis_prep* p, const double r[3], int maxorder,
                       double* out) {
    const int nslot = NSLOT_BY_ORDER[maxorder];
    memset(out, 0, sizeof(double) * (size_t)p->n_basis * OD_N);
    for (int sh = 0; sh < s->n_shell; ++sh) {
        const int l = s->sh_l[sh];
        const int c = s->sh_center[sh];
        const double x[3] = {r[0] - s->R[3 * c], r[1] - s->R[3 * c + 1], r[2] - s->R[3 * c + 2]};
        angfn ang[6];
        shell_angular(l, s->sh_pure[sh], ang);
        const int nf = shell_nfn(l, s->sh_pure[sh]);
        for (int q = p->first_prim[sh]; q < p->first_prim[sh + 1]; ++q) {
            double E[3][3][4];
            for (int d = 0; d < 3; ++d) gauss1d(s->alpha[q], x[d], l, maxorder, E[d]);
            const double cq = p->cnorm[q];
            for (int f = 0; f < nf; ++f) {
                double* o = out + (size_t)(p->first_fn[sh] + f) * OD_N;
                for (int t = 0; t < ang[f].nterm; ++t) {
                    const int* m = ang[f].ijk[t];
                    const double wt = cq * ang[f].w[t];
                    for (int k = 0; k < nslot; ++k)
                        o[k] += wt * E[0][m[0]][DSLOT[k][0]] * E[1][m[1]][DSLOT[k][1]] * E[2][m[2]][DSLOT[k][2]];
                }
            }
        }
    }
}

int oracle_n_basis(const oracle_system* s) {
    int nb = 0;
    for (int sh = 0; sh < s->n_shell; ++sh) nb += shell_nfn(s->sh_l[sh], s->sh_pure[sh]);
    return nb;
}

int oracle_basis(const oracle_system* s, const double r[3], double* out) {
    basis_prep p;
    prep_basis(s, &p);
    basis_eval(s, &p, r, 3, out);
    free_basis(&p);
    return 0;
}

/* ------------------------------------------------------------------ */
/* dense linear algebra                                                */
/* ------------------------------------------------------------------ */

int oracle_lu_det(int n, const double* A, double* logabs, double* sign, double* Ainv) {
    if (n < 0) return -1;
    if (n == 0) {
        *logabs = 0.0;
        *sign = 1.0;
        return 0;
    }
    double* LU = (double*)malloc(sizeof(double) * n * n);
    int* perm = (int*)malloc(sizeof(int) * n);
    memcpy(LU, A, sizeof(double) * n * n);
    for (int i = 0; i < n; ++i) perm[i] = i;
    double sg = 1.0;
    int singular = 0;
    for (int k = 0; k < n; ++k) {
        int piv = k;
        double best = fabs(LU[k * n + k]);
        for (int i = k + 1; i < n; ++i)
            if (fabs(LU[i * n + k]) > best) {
                best = fabs(LU[i * n + k]);
                piv = i;
            }
        if (best == 0.0) {
            singular = 1;
            break;
        }
        if (piv != k) {
            for (int j = 0; j < n; ++j) {
                double t = LU[k * n + j];
                LU[k * n + j] = LU[piv * n + j];
                LU[piv * n + j] = t;
            }
            int t = perm[k];
            perm[k] = perm[piv];
            perm[piv] = t;
            sg = -sg;
        }
        for (int i = k + 1; i < n; ++i) {
            LU[i * n + k] /= LU[k * n + k];
            for (int j = k + 1; j < n; ++j) LU[i * n + j] -= LU[i * n + k] * LU[k * n + j];
        }
    }
    if (singular) {
        *logabs = -INFINITY;
        *sign = 0.0;
        free(LU);
        free(perm);
        return 1;
    }
    double la = 0.0;
    for (int k = 0; k < n; ++k) {
        la += log(fabs(LU[k * n + k]));
        if (LU[k * n + k] < 0) sg = -sg;
    }
    *logabs = la;
    *sign = sg;
    if (Ainv) {
        double* y = (double*)malloc(sizeof(double) * n);
        for (int c = 0; c < n; ++c) {
            /* solve A x = e_c  <=>  L U x = P e_c */
            for (int i = 0; i < n; ++i) y[i] = (perm[i] == c) ? 1.0 : 0.0;
            for (int i = 0; i < n; ++i)
                for (int j = 0; j < i; ++j) y[i] -= LU[i * n + j] * y[j];
            for (int i = n - 1; i >= 0; --i) {
                for (int j = i + 1; j < n; ++j) y[i] -= LU[i * n + j] * y[j];
                y[i] /= LU[i * n + i];
            }
            for (int i = 0; i < n; ++i) Ainv[i * n + c] = y[i];
        }
        free(y);
    }
    free(LU);
    free(perm);
    return 0;
}

/* ------------------------------------------------------------------ */
/* determinant list (single determinant = one entry with weight 1)     */
/* ------------------------------------------------------------------ */

typedef struct {
    int n_det;
    int n_orb;        /* orbitals referenced: 0..n_orb-1 */
    int* orb_up;      /* [n_det][n_up] */
    int* orb_dn;      /* [n_det][n_dn] */
    double* c;        /* [n_det] */
} det_list;

static void bits_to_list(const uint64_t* w, int n_words, int n, int* out) {
    int k = 0;
    for (int b = 0; b < 64 * n_words && k < n; ++b)
        if ((w[b / 64] >> (b % 64)) & 1ULL) out[k++] = b;
}

static void build_dets(const oracle_system* s, det_list* d) {
    const int nu = s->n_up, nd = s->n_dn;
    d->n_det = s->n_det > 0 ? s->n_det : 1;
    d->orb_up = (int*)malloc(sizeof(int) * (size_t)d->n_det * (nu > 0 ? nu : 1));
    d->orb_dn = (int*)malloc(sizeof(int) * (size_t)d->n_det * (nd > 0 ? nd : 1));
    d->c = (double*)malloc(sizeof(double) * d->n_det);
    if (s->n_det == 0) {
        for (int j = 0; j < nu; ++j) d->orb_up[j] = s->occ_up[j];
        for (int j = 0; j < nd; ++j) d->orb_dn[j] = s->occ_dn[j];
        d->c[0] = 1.0;
    } else {
        for (int k = 0; k < d->n_det; ++k) {
            bits_to_list(s->det_up + (size_t)k * s->n_words, s->n_words, nu, d->orb_up + (size_t)k * nu);
            bits_to_list(s->det_dn + (size_t)k * s->n_words, s->n_words, nd, d->orb_dn + (size_t)k * nd);
            d->c[k] = s->ci[k];
        }
    }
    int mx = 0;
    for (size_t q = 0; q < (size_t)d->n_det * nu; ++q)
        if (d->orb_up[q] + 1 > mx) mx = d->orb_up[q] + 1;
    for (size_t q = 0; q < (size_t)d->n_det * nd; ++q)
        if (d->orb_dn[q] + 1 > mx) mx = d->orb_dn[q] + 1;
    d->n_orb = mx;
}

static void free_dets(det_list* d) {
    free(d->orb_up);
    free(d->orb_dn);
    free(d->c);
}

/* ------------------------------------------------------------------ */
/* Jastrow                                                             */
/* ------------------------------------------------------------------ */

static void pade(double a, double b, double r, double* u, double* du, double* d2u, double* d3u) {
    const double q = 1.0 / (1.0 + b * r);
    *u = a * r * q;
    *du = a * q * q;
    *d2u = -2.0 * a * b * q * q * q;
    *d3u = 6.0 * a * b * b * q * q * q * q;
}

/* Three-body term of one nucleus a and one electron pair (i, j), with the
 * coefficients c[n3] of that nucleus: value, and (optionally) its gradient
 * and Laplacian added to gJ, lJ for both electrons.  s(r) = r / (1 + b r),
 * s' = 1 / (1 + b r)^2, s'' = -2 b / (1 + b r)^3; a radial function F(s(r))
 * has grad F = F'(s) s' r_hat and lap F = F''(s) s'^2 + F'(s) (s'' + 2 s' / r). */
static double ipow(double x, int k) {
    double p = 1.0;
    for (int q = 0; q < k; ++q) p *= x;
    return p;
}
static void scaled_dist(double b, const double* ri, const double* rj, double* s, double* s1, double* s2, double u[3],
                        double* r) {
    double d2 = 0.0;
    for (int c = 0; c < 3; ++c) {
        u[c] = ri[c] - rj[c];
        d2 += u[c] * u[c];
    }
    *r = sqrt(d2);
    for (int c = 0; c < 3; ++c) u[c] /= *r;
    const double q = 1.0 / (1.0 + b * *r);
    *s = *r * q;
    *s1 = q * q;
    *s2 = -2.0 * b * q * q * q;
}
static double j3_pair(const oracle_system* s, const double* R, int a, int i, int j, const double* c, double* gJ,
                      double* lJ) {
    double xi, xi1, xi2, ui[3], ri, xj, xj1, xj2, uj[3], rj, y, y1, y2, uy[3], ry;
    scaled_dist(s->b3, R + 3 * i, s->R + 3 * a, &xi, &xi1, &xi2, ui, &ri);
    scaled_dist(s->b3, R + 3 * j, s->R + 3 * a, &xj, &xj1, &xj2, uj, &rj);
    scaled_dist(s->b3, R + 3 * i, R + 3 * j, &y, &y1, &y2, uy, &ry);   /* uy: from j to i */
    double val = 0.0;
    for (int k = 0; k < s->n3; ++k) {
        if (c[k] == 0.0) continue;
        const int m = s->e3[3 * k], n = s->e3[3 * k + 1], o = s->e3[3 * k + 2];
        const double P = ipow(xi, m) * ipow(xj, n) + ipow(xi, n) * ipow(xj, m);
        const double Q = ipow(y, o);
        val += c[k] * P * Q;
        if (!gJ && !lJ) continue;
        /* dP / dx_i, d2P / dx_i^2 and the same in x_j */
        const double Pi = (m ? m * ipow(xi, m - 1) : 0.0) * ipow(xj, n) + (n ? n * ipow(xi, n - 1) : 0.0) * ipow(xj, m);
        const double Pj = ipow(xi, m) * (n ? n * ipow(xj, n - 1) : 0.0) + ipow(xi, n) * (m ? m * ipow(xj, m - 1) : 0.0);
        const double Pii = (m > 1 ? m * (m - 1) * ipow(xi, m - 2) : 0.0) * ipow(xj, n) +
                           (n > 1 ? n * (n - 1) * ipow(xi, n - 2) : 0.0) * ipow(xj, m);
        const double Pjj = ipow(xi, m) * (n > 1 ? n * (n - 1) * ipow(xj, n - 2) : 0.0) +
                           ipow(xi, n) * (m > 1 ? m * (m - 1) * ipow(xj, m - 2) : 0.0);
        const double Q1 = o ? o * ipow(y, o - 1) : 0.0;
        const double Q2 = o > 1 ? o * (o - 1) * ipow(y, o - 2) : 0.0;
        /* electron i: grad = c (Pi Q xi' ui + P Q1 y' uy) */
        double dot_i = 0.0, dot_j = 0.0;
        for (int q = 0; q < 3; ++q) {
            const double gi = c[k] * (Pi * Q * xi1 * ui[q] + P * Q1 * y1 * uy[q]);
            const double gj = c[k] * (Pj * Q * xj1 * uj[q] - P * Q1 * y1 * uy[q]);
            if (gJ) {
                gJ[3 * i + q] += gi;
                gJ[3 * j + q] += gj;
            }
            dot_i += ui[q] * uy[q];
            dot_j += uj[q] * uy[q];
        }
        if (lJ) {
            const double lx_i = xi2 + 2.0 * xi1 / ri, lx_j = xj2 + 2.0 * xj1 / rj, ly = y2 + 2.0 * y1 / ry;
            lJ[i] += c[k] * (Pii * Q * xi1 * xi1 + Pi * Q * lx_i + P * Q2 * y1 * y1 + P * Q1 * ly +
                             2.0 * Pi * Q1 * xi1 * y1 * dot_i);
            lJ[j] += c[k] * (Pjj * Q * xj1 * xj1 + Pj * Q * lx_j + P * Q2 * y1 * y1 + P * Q1 * ly -
                             2.0 * Pj * Q1 * xj1 * y1 * dot_j);
        }
    }
    return val;
}

/* J, grad_i J [N][3], lap_i J [N]. */
static double jastrow(const oracle_system* s, const double* R, double* gJ, double* lJ) {
    const int N = s->n_up + s->n_dn;
    double J = 0.0;
    if (gJ) memset(gJ, 0, sizeof(double) * 3 * N);
    if (lJ) memset(lJ, 0, sizeof(double) * N);
    for (int i = 0; i < N; ++i)
        for (int j = i + 1; j < N; ++j) {
            const int same = (i < s->n_up) == (j < s->n_up);
            const double a = same ? s->a_par : s->a_anti;
            double x[3], r2 = 0.0;
            for (int c = 0; c < 3; ++c) {
                x[c] = R[3 * i + c] - R[3 * j + c];
                r2 += x[c] * x[c];
            }
            const double r = sqrt(r2);
            double u, du, d2u, d3u;
            pade(a, s->b_ee, r, &u, &du, &d2u, &d3u);
            J += u;
            if (gJ)
                for (int c = 0; c < 3; ++c) {
                    gJ[3 * i + c] += du * x[c] / r;
                    gJ[3 * j + c] -= du * x[c] / r;
                }
            if (lJ) {
                lJ[i] += d2u + 2.0 * du / r;
                lJ[j] += d2u + 2.0 * du / r;
            }
        }
    for (int i = 0; i < N; ++i)
        for (int a = 0; a < s->n_nuc; ++a) {
            double x[3], r2 = 0.0;
            for (int c = 0; c < 3; ++c) {
                x[c] = R[3 * i + c] - s->R[3 * a + c];
                r2 += x[c] * x[c];
            }
            const double r = sqrt(r2);
            double u, du, d2u, d3u;
            pade(s->a_en[a], s->b_en, r, &u, &du, &d2u, &d3u);
            J += u;
            if (gJ)
                for (int c = 0; c < 3; ++c) gJ[3 * i + c] += du * x[c] / r;
            if (lJ) lJ[i] += d2u + 2.0 * du / r;
        }
    /* three-body e-e-n terms */
    if (s->n3 > 0) {
        for (int a = 0; a < s->n_nuc; ++a)
            for (int i = 0; i < N; ++i)
                for (int j = i + 1; j < N; ++j)
                    J += j3_pair(s, R, a, i, j, s->c3 + (size_t)a * s->n3, gJ, lJ);
    }
    return J;
}

/* One radial pseudopotential term beta r^(n-2) exp(-alpha r^2). */
static double pp_term(const oracle_system* s, int t, double r) {
    const int k = s->pp_n[t] - 2;
    const double rk = k >= 0 ? ipow(r, k) : 1.0 / ipow(r, -k);
    return s->pp_beta[t] * rk * exp(-s->pp_alpha[t] * r * r);
}

static double potential(const oracle_system* s, const double* R) {
    const int N = s->n_up + s->n_dn;
    double V = 0.0;
    for (int i = 0; i < N; ++i)
        for (int j = i + 1; j < N; ++j) {
            double r2 = 0.0;
            for (int c = 0; c < 3; ++c) r2 += (R[3 * i + c] - R[3 * j + c]) * (R[3 * i + c] - R[3 * j + c]);
            V += 1.0 / sqrt(r2);
        }
    for (int i = 0; i < N; ++i)
        for (int a = 0; a < s->n_nuc; ++a) {
            double r2 = 0.0;
            for (int c = 0; c < 3; ++c)
                r2 += (R[3 * i + c] - s->R[3 * a + c]) * (R[3 * i + c] - s->R[3 * a + c]);
            V -= s->Z[a] / sqrt(r2);
        }
    for (int a = 0; a < s->n_nuc; ++a)
        for (int b = a + 1; b < s->n_nuc; ++b) {
            double r2 = 0.0;
            for (int c = 0; c < 3; ++c) r2 += (s->R[3 * a + c] - s->R[3 * b + c]) * (s->R[3 * a + c] - s->R[3 * b + c]);
            V += s->Z[a] * s->Z[b] / sqrt(r2);
        }
    /* local pseudopotential terms, every electron and every term */
    for (int t = 0; t < s->n_pp; ++t) {
        if (s->pp_l[t] != -1) continue;
        const int a = s->pp_nuc[t];
        for (int i = 0; i < N; ++i) {
            double r2 = 0.0;
            for (int c = 0; c < 3; ++c)
                r2 += (R[3 * i + c] - s->R[3 * a + c]) * (R[3 * i + c] - s->R[3 * a + c]);
            V += pp_term(s, t, sqrt(r2));
        }
    }
    return V;
}

/* ------------------------------------------------------------------ */
/* determinant part: ln|D|, sign, grad_i D/D, lap_i D/D               */
/* ------------------------------------------------------------------ */

/* Orbital values per electron: mo[(i * n_orb + o) * 5 + {v, gx, gy, gz, lap}]. */
static void eval_orbitals(const oracle_system* s, const basis_prep* p, const double* R, int i_begin,
                          int i_end, int n_orb, int order, double* mo) {
    double* bas = (double*)malloc(sizeof(double) * (size_t)p->n_basis * OD_N);
    for (int i = i_begin; i < i_end; ++i) {
        basis_eval(s, p, R + 3 * i, order, bas);
        for (int o = 0; o < n_orb; ++o) {
            double v[5] = {0, 0, 0, 0, 0};
            const double* Co = s->C + (size_t)o * s->n_basis;
            for (int l = 0; l < p->n_basis; ++l) {
                const double* b = bas + (size_t)l * OD_N;
                v[0] += Co[l] * b[OD000];
                if (order >= 1) {
                    v[1] += Co[l] * b[OD100];
                    v[2] += Co[l] * b[OD010];
                    v[3] += Co[l] * b[OD001];
                }
                if (order >= 2) v[4] += Co[l] * (b[OD200] + b[OD020] + b[OD002]);
            }
            memcpy(mo + ((size_t)i * n_orb + o) * 5, v, sizeof(v));
        }
    }
    free(bas);
}

/* One spin block of one determinant: n electrons starting at i0, orbitals
 * orbs[n].  Outputs ln|D|, sign, and per electron grad D/D, lap D/D. */
static int block_det(int n, int i0, const int* orbs, int n_orb, const double* mo, double* logabs,
                     double* sign, double* gD, double* lD, double* A, double* Ainv) {
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) A[i * n + j] = mo[((size_t)(i0 + i) * n_orb + orbs[j]) * 5];
    int st = oracle_lu_det(n, A, logabs, sign, Ainv);
    if (st) return st;
    for (int i = 0; i < n; ++i) {
        double g[3] = {0, 0, 0}, lp = 0.0;
        for (int j = 0; j < n; ++j) {
            const double* m = mo + ((size_t)(i0 + i) * n_orb + orbs[j]) * 5;
            const double ai = Ainv[j * n + i];
            g[0] += m[1] * ai;
            g[1] += m[2] * ai;
            g[2] += m[3] * ai;
            lp += m[4] * ai;
        }
        if (gD) memcpy(gD + 3 * i, g, sizeof(g));
        if (lD) lD[i] = lp;
    }
    return 0;
}

/* Sum over determinants: psi_D = sum_k c_k D_k^up D_k^dn.
 * gD [N][3] = grad_i psi_D / psi_D, lD [N] = lap_i psi_D / psi_D. */
static int det_part(const oracle_system* s, const det_list* d, const double* mo, double* logabs,
                    double* sign, double* gD, double* lD) {
    const int nu = s->n_up, nd = s->n_dn, N = nu + nd;
    const int nmax = nu > nd ? nu : nd;
    double* A = (double*)malloc(sizeof(double) * (nmax * nmax + 1));
    double* Ai = (double*)malloc(sizeof(double) * (nmax * nmax + 1));
    double* la = (double*)malloc(sizeof(double) * d->n_det);
    double* sg = (double*)malloc(sizeof(double) * d->n_det);
    double* g = (double*)malloc(sizeof(double) * (size_t)d->n_det * 3 * N);
    double* lp = (double*)malloc(sizeof(double) * (size_t)d->n_det * N);
    int ok = 0;
    double Lmax = -INFINITY;
    for (int k = 0; k < d->n_det; ++k) {
        double l1, s1, l2, s2;
        int e1 = block_det(nu, 0, d->orb_up + (size_t)k * nu, d->n_orb, mo, &l1, &s1, g + (size_t)k * 3 * N,
                           lp + (size_t)k * N, A, Ai);
        int e2 = block_det(nd, nu, d->orb_dn + (size_t)k * nd, d->n_orb, mo, &l2, &s2,
                           g + (size_t)k * 3 * N + 3 * nu, lp + (size_t)k * N + nu, A, Ai);
        if (e1 || e2 || d->c[k] == 0.0) {
            la[k] = -INFINITY;
            sg[k] = 0.0;
            continue;
        }
        la[k] = l1 + l2;
        sg[k] = s1 * s2;
        if (la[k] > Lmax) Lmax = la[k];
        ok = 1;
    }
    if (!ok) {
        free(A); free(Ai); free(la); free(sg); free(g); free(lp);
        *logabs = -INFINITY;
        *sign = 0.0;
        return 1;
    }
    double S = 0.0;
    if (gD) memset(gD, 0, sizeof(double) * 3 * N);
    if (lD) memset(lD, 0, sizeof(double) * N);
    for (int k = 0; k < d->n_det; ++k) {
        if (sg[k] == 0.0) continue;
        const double rk = d->c[k] * sg[k] * exp(la[k] - Lmax);
        S += rk;
        if (gD)
            for (int q = 0; q < 3 * N; ++q) gD[q] += rk * g[(size_t)k * 3 * N + q];
        if (lD)
            for (int q = 0; q < N; ++q) lD[q] += rk * lp[(size_t)k * N + q];
    }
    if (gD)
        for (int q = 0; q < 3 * N; ++q) gD[q] /= S;
    if (lD)
        for (int q = 0; q < N; ++q) lD[q] /= S;
    *logabs = Lmax + log(fabs(S));
    *sign = S > 0 ? 1.0 : -1.0;
    free(A); free(Ai); free(la); free(sg); free(g); free(lp);
    return S == 0.0;
}

/* ------------------------------------------------------------------ */
/* non-local pseudopotential                                           */
/* ------------------------------------------------------------------ */

/* Legendre polynomial P_l(x), l <= 3. */
static double legendre(int l, double x) {
    switch (l) {
        case 0: return 1.0;
        case 1: return x;
        case 2: return 0.5 * (3.0 * x * x - 1.0);
        default: return 0.5 * (5.0 * x * x * x - 3.0 * x);
    }
}

/* Non-local energy of one walker in the locality approximation:
 *   sum_a sum_{i: r_ia < rcut_a} sum_l v_l(r_ia) (2l + 1)
 *       sum_q w_q P_l(r_hat_ia . d_q) psi(R with r_i -> R_a + r_ia d_q) / psi(R),
 * with d_q the (rotated) quadrature directions.  Every ratio is taken from
 * two full evaluations: the orbital values of all electrons, the
 * determinant(s) by LU and the Jastrow factor, at R and at the moved
 * configuration. */
static double nonlocal_one(const oracle_system* s, const basis_prep* p, const det_list* d, const double* R, int slot) {
    if (s->n_pp == 0) return 0.0;
    const int N = s->n_up + s->n_dn;
    const int n_orb = d->n_orb > 0 ? d->n_orb : 1;
    const size_t mo_sz = (size_t)N * n_orb * 5;
    double* mo = (double*)malloc(sizeof(double) * mo_sz);
    double* mo2 = (double*)malloc(sizeof(double) * mo_sz);
    double* R2 = (double*)malloc(sizeof(double) * 3 * N);
    eval_orbitals(s, p, R, 0, N, d->n_orb, 0, mo);
    double ld0, sd0;
    const int bad = det_part(s, d, mo, &ld0, &sd0, NULL, NULL);
    const double J0 = jastrow(s, R, NULL, NULL);
    double V = 0.0;
    for (int a = 0; a < s->n_nuc && !bad; ++a) {
        int lmax = -1;
        for (int t = 0; t < s->n_pp; ++t)
            if (s->pp_nuc[t] == a && s->pp_l[t] > lmax) lmax = s->pp_l[t];
        if (lmax < 0) continue;
        double rot[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
        if (s->pp_rotate) oracle_pp_rotation(s->pp_seed, s->pp_sweep, (uint32_t)a, s->pp_slot0 + (uint32_t)slot, rot);
        for (int i = 0; i < N; ++i) {
            double x[3], r2 = 0.0;
            for (int c = 0; c < 3; ++c) {
                x[c] = R[3 * i + c] - s->R[3 * a + c];
                r2 += x[c] * x[c];
            }
            const double r = sqrt(r2);
            if (!(r < s->pp_rcut[a])) continue;
            double vl[4] = {0, 0, 0, 0};
            for (int t = 0; t < s->n_pp; ++t)
                if (s->pp_nuc[t] == a && s->pp_l[t] >= 0) vl[s->pp_l[t]] += pp_term(s, t, r);
            for (int q = 0; q < s->pp_nq; ++q) {
                const double* o = s->pp_quad + 3 * q;
                double dq[3], cth = 0.0;
                for (int c = 0; c < 3; ++c) {
                    dq[c] = rot[3 * c] * o[0] + rot[3 * c + 1] * o[1] + rot[3 * c + 2] * o[2];
                    cth += dq[c] * x[c] / r;
                }
                memcpy(R2, R, sizeof(double) * 3 * N);
                for (int c = 0; c < 3; ++c) R2[3 * i + c] = s->R[3 * a + c] + r * dq[c];
                memcpy(mo2, mo, sizeof(double) * mo_sz);
                eval_orbitals(s, p, R2, i, i + 1, d->n_orb, 0, mo2);
                double ld1, sd1;
                if (det_part(s, d, mo2, &ld1, &sd1, NULL, NULL)) continue;   /* psi(R') = 0 */
                const double ratio = sd1 * sd0 * exp(ld1 + jastrow(s, R2, NULL, NULL) - ld0 - J0);
                for (int l = 0; l <= lmax; ++l)
                    V += vl[l] * (2.0 * l + 1.0) * s->pp_qw[q] * legendre(l, cth) * ratio;
            }
        }
    }
    free(mo); free(mo2); free(R2);
    return bad ? NAN : V;
}

/* ------------------------------------------------------------------ */
/* fixed-configuration evaluation                                      */
/* ------------------------------------------------------------------ */

typedef struct {
    const oracle_system* s;
    const basis_prep* p;
    const det_list* d;
    const double* R;
    double *logpsi, *sign, *eloc, *grad, *lap;
} eval_ctx;

static void eval_one(const oracle_system* s, const basis_prep* p, const det_list* d, const double* R, int slot,
                     double* logpsi, double* sign, double* eloc, double* grad, double* lap) {
    const int N = s->n_up + s->n_dn;
    double* mo = (double*)malloc(sizeof(double) * (size_t)N * (d->n_orb > 0 ? d->n_orb : 1) * 5);
    double* gJ = (double*)malloc(sizeof(double) * 3 * (N + 1));
    double* lJ = (double*)malloc(sizeof(double) * (N + 1));
    double* gD = (double*)malloc(sizeof(double) * 3 * (N + 1));
    double* lD = (double*)malloc(sizeof(double) * (N + 1));
    eval_orbitals(s, p, R, 0, N, d->n_orb, 2, mo);
    double ld, sd;
    det_part(s, d, mo, &ld, &sd, gD, lD);
    const double J = jastrow(s, R, gJ, lJ);
    double T = 0.0;
    for (int i = 0; i < N; ++i) {
        double dot = 0.0, gg = 0.0;
        for (int c = 0; c < 3; ++c) {
            dot += gJ[3 * i + c] * gD[3 * i + c];
            gg += gJ[3 * i + c] * gJ[3 * i + c];
        }
        T += -0.5 * (lD[i] + lJ[i] + 2.0 * dot + gg);
        if (grad)
            for (int c = 0; c < 3; ++c) grad[3 * i + c] = gJ[3 * i + c] + gD[3 * i + c];
        if (lap) {
            double dd = 0.0;
            for (int c = 0; c < 3; ++c) dd += gD[3 * i + c] * gD[3 * i + c];
            lap[i] = lJ[i] + lD[i] - dd;
        }
    }
    if (logpsi) *logpsi = J + ld;
    if (sign) *sign = sd;
    if (eloc) *eloc = T + potential(s, R) + nonlocal_one(s, p, d, R, slot);
    free(mo); free(gJ); free(lJ); free(gD); free(lD);
}

static void eval_worker(void* vctx, int w) {
    eval_ctx* c = (eval_ctx*)vctx;
    const int N = c->s->n_up + c->s->n_dn;
    eval_one(c->s, c->p, c->d, c->R + (size_t)w * 3 * N, w, c->logpsi ? c->logpsi + w : NULL,
             c->sign ? c->sign + w : NULL, c->eloc ? c->eloc + w : NULL,
             c->grad ? c->grad + (size_t)w * 3 * N : NULL, c->lap ? c->lap + (size_t)w * N : NULL);
}

int oracle_evaluate(const oracle_system* s, int W, const double* R, double* logpsi, double* sign,
                    double* eloc, double* grad, double* lap, int nthreads) {
    basis_prep p;
    det_list d;
    prep_basis(s, &p);
    build_dets(s, &d);
    eval_ctx c = {s, &p, &d, R, logpsi, sign, eloc, grad, lap};
    parallel_for(W, nthreads, eval_worker, &c);
    free_dets(&d);
    free_basis(&p);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Jastrow parameter derivatives                                       */
/* ------------------------------------------------------------------ */

/* d/db of the Pade function u = a r / (1 + b r): g = -a r^2 / (1 + b r)^2,
 * g' = -2 a r / (1 + b r)^3, g'' = -2 a (1 - 2 b r) / (1 + b r)^4. */
static void pade_db(double a, double b, double r, double* g, double* g1, double* g2) {
    const double q = 1.0 / (1.0 + b * r);
    *g = -a * r * r * q * q;
    *g1 = -2.0 * a * r * q * q * q;
    *g2 = -2.0 * a * (1.0 - 2.0 * b * r) * q * q * q * q;
}

/* B = dJ/db_ee (ee != 0) or dJ/db_en, with grad_i B [N][3] and lap_i B [N]. */
static double jastrow_db(const oracle_system* s, const double* R, int ee, double* gB, double* lB) {
    const int N = s->n_up + s->n_dn;
    double B = 0.0;
    memset(gB, 0, sizeof(double) * 3 * N);
    memset(lB, 0, sizeof(double) * N);
    if (ee) {
        for (int i = 0; i < N; ++i)
            for (int j = i + 1; j < N; ++j) {
                const double a = ((i < s->n_up) == (j < s->n_up)) ? s->a_par : s->a_anti;
                double x[3], r2 = 0.0;
                for (int c = 0; c < 3; ++c) {
                    x[c] = R[3 * i + c] - R[3 * j + c];
                    r2 += x[c] * x[c];
                }
                const double r = sqrt(r2);
                double g, g1, g2;
                pade_db(a, s->b_ee, r, &g, &g1, &g2);
                B += g;
                for (int c = 0; c < 3; ++c) {
                    gB[3 * i + c] += g1 * x[c] / r;
                    gB[3 * j + c] -= g1 * x[c] / r;
                }
                lB[i] += g2 + 2.0 * g1 / r;
                lB[j] += g2 + 2.0 * g1 / r;
            }
    } else {
        for (int i = 0; i < N; ++i)
            for (int a = 0; a < s->n_nuc; ++a) {
                double x[3], r2 = 0.0;
                for (int c = 0; c < 3; ++c) {
                    x[c] = R[3 * i + c] - s->R[3 * a + c];
                    r2 += x[c] * x[c];
                }
                const double r = sqrt(r2);
                double g, g1, g2;
                pade_db(s->a_en[a], s->b_en, r, &g, &g1, &g2);
                B += g;
                for (int c = 0; c < 3; ++c) gB[3 * i + c] += g1 * x[c] / r;
                lB[i] += g2 + 2.0 * g1 / r;
            }
    }
    return B;
}

/* dJ/dp at R for Jastrow parameter q (order a_anti, a_par, b_ee, b_en,
 * a_en[n_nuc], c3[n_nuc][n3]): a linear parameter's is the Jastrow with
 * that parameter set to 1 and every other linear coefficient to 0; b_ee,
 * b_en by jastrow_db.  Scratch: gB [3N], lB [N], unit_en/zero_en [n_nuc],
 * unit_c3/zero_c3 [n_nuc n3]. */
static double jastrow_param(const oracle_system* s, const double* R, int q, double* gB, double* lB, double* zero_en,
                            double* unit_en, double* zero_c3, double* unit_c3) {
    const int nn = s->n_nuc;
    if (q == 2 || q == 3) return jastrow_db(s, R, q == 2, gB, lB);
    oracle_system u = *s;
    u.a_anti = q == 0 ? 1.0 : 0.0;
    u.a_par = q == 1 ? 1.0 : 0.0;
    u.a_en = zero_en;
    u.c3 = zero_c3;
    if (q >= 4 && q < 4 + nn) {
        memset(unit_en, 0, sizeof(double) * nn);
        unit_en[q - 4] = 1.0;
        u.a_en = unit_en;
    }
    if (q >= 4 + nn) {
        memset(unit_c3, 0, sizeof(double) * nn * s->n3);
        unit_c3[q - 4 - nn] = 1.0;
        u.c3 = unit_c3;
    }
    return jastrow(&u, R, gB, lB);
}

/* The non-local energy's Jastrow parameter derivatives, added to dv[P]: the
 * weights and determinant ratios do not depend on the Jastrow, and each
 * ratio psi(R'_p)/psi(R) carries exp(J(R'_p) - J(R)), so
 *   dV_NL/dq = sum_p W_p rho_p (dJ/dq(R'_p) - dJ/dq(R)). */
static void nonlocal_param_deriv(const oracle_system* s, const basis_prep* p, const det_list* d, const double* R,
                                 int slot, int P, double* dv) {
    if (s->n_pp == 0) return;
    const int N = s->n_up + s->n_dn, nn = s->n_nuc;
    double* gB = (double*)malloc(sizeof(double) * 3 * N);
    double* lB = (double*)malloc(sizeof(double) * N);
    double* zero_en = (double*)calloc((size_t)nn + 1, sizeof(double));
    double* unit_en = (double*)calloc((size_t)nn + 1, sizeof(double));
    double* unit_c3 = (double*)calloc((size_t)nn * (s->n3 > 0 ? s->n3 : 1) + 1, sizeof(double));
    double* zero_c3 = (double*)calloc((size_t)nn * (s->n3 > 0 ? s->n3 : 1) + 1, sizeof(double));
    double* B0 = (double*)malloc(sizeof(double) * P);
    double* R2 = (double*)malloc(sizeof(double) * 3 * N);
    double* mo = (double*)malloc(sizeof(double) * (size_t)N * (d->n_orb > 0 ? d->n_orb : 1) * 5);
    for (int q = 0; q < P; ++q) B0[q] = jastrow_param(s, R, q, gB, lB, zero_en, unit_en, zero_c3, unit_c3);
    double l0, s0;
    eval_orbitals(s, p, R, 0, N, d->n_orb, 0, mo);
    const int bad = det_part(s, d, mo, &l0, &s0, NULL, NULL);
    l0 += jastrow(s, R, NULL, NULL);
    for (int a = 0; a < nn && !bad; ++a) {
        int lmax = -1;
        for (int t = 0; t < s->n_pp; ++t)
            if (s->pp_nuc[t] == a && s->pp_l[t] > lmax) lmax = s->pp_l[t];
        if (lmax < 0) continue;
        double rot[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
        if (s->pp_rotate) oracle_pp_rotation(s->pp_seed, s->pp_sweep, (uint32_t)a, s->pp_slot0 + (uint32_t)slot, rot);
        for (int i = 0; i < N; ++i) {
            double x[3], r2 = 0.0;
            for (int c = 0; c < 3; ++c) {
                x[c] = R[3 * i + c] - s->R[3 * a + c];
                r2 += x[c] * x[c];
            }
            const double r = sqrt(r2);
            if (!(r < s->pp_rcut[a])) continue;
            double vl[4] = {0, 0, 0, 0};
            for (int t = 0; t < s->n_pp; ++t)
                if (s->pp_nuc[t] == a && s->pp_l[t] >= 0) vl[s->pp_l[t]] += pp_term(s, t, r);
            for (int qd = 0; qd < s->pp_nq; ++qd) {
                const double* o = s->pp_quad + 3 * qd;
                double dq[3], cth = 0.0;
                for (int c = 0; c < 3; ++c) {
                    dq[c] = rot[3 * c] * o[0] + rot[3 * c + 1] * o[1] + rot[3 * c + 2] * o[2];
                    cth += dq[c] * x[c] / r;
                }
                memcpy(R2, R, sizeof(double) * 3 * N);
                for (int c = 0; c < 3; ++c) R2[3 * i + c] = s->R[3 * a + c] + r * dq[c];
                eval_orbitals(s, p, R2, 0, N, d->n_orb, 0, mo);
                double l1, s1;
                if (det_part(s, d, mo, &l1, &s1, NULL, NULL)) continue;
                const double rho = s1 * s0 * exp(l1 + jastrow(s, R2, NULL, NULL) - l0);
                double W = 0.0;
                for (int l = 0; l <= lmax; ++l) W += vl[l] * (2.0 * l + 1.0) * s->pp_qw[qd] * legendre(l, cth);
                for (int q = 0; q < P; ++q)
                    dv[q] += W * rho *
                             (jastrow_param(s, R2, q, gB, lB, zero_en, unit_en, zero_c3, unit_c3) - B0[q]);
            }
        }
    }
    free(gB); free(lB); free(zero_en); free(unit_en); free(unit_c3); free(zero_c3); free(B0); free(R2); free(mo);
}

typedef struct {
    const oracle_system* s;
    const basis_prep* p;
    const det_list* d;
    const double* R;
    double *dlog, *deloc;
    int P;
} jd_ctx;

static void jd_worker(void* vctx, int w) {
    jd_ctx* cx = (jd_ctx*)vctx;
    const oracle_system* s = cx->s;
    const int N = s->n_up + s->n_dn, nn = s->n_nuc, P = cx->P;
    const double* R = cx->R + (size_t)w * 3 * N;
    double* G = (double*)malloc(sizeof(double) * 3 * N);
    double* gB = (double*)malloc(sizeof(double) * 3 * N);
    double* lB = (double*)malloc(sizeof(double) * N);
    double* zero_en = (double*)calloc((size_t)nn + 1, sizeof(double));
    double* unit_en = (double*)calloc((size_t)nn + 1, sizeof(double));
    double* unit_c3 = (double*)calloc((size_t)nn * (s->n3 > 0 ? s->n3 : 1) + 1, sizeof(double));
    double* zero_c3 = (double*)calloc((size_t)nn * (s->n3 > 0 ? s->n3 : 1) + 1, sizeof(double));
    /* grad_i ln|psi| of the full trial function */
    eval_one(s, cx->p, cx->d, R, w, NULL, NULL, NULL, G, NULL);
    double* dvnl = (double*)calloc((size_t)P + 1, sizeof(double));
    nonlocal_param_deriv(s, cx->p, cx->d, R, w, P, dvnl);
    for (int q = 0; q < P; ++q) {
        double B;
        if (q == 2 || q == 3) {
            B = jastrow_db(s, R, q == 2, gB, lB);
        } else {
            /* a linear parameter: dJ/dp is the Jastrow with that parameter
             * set to 1 and every other linear coefficient to 0 */
            oracle_system u = *s;
            u.a_anti = q == 0 ? 1.0 : 0.0;
            u.a_par = q == 1 ? 1.0 : 0.0;
            u.a_en = zero_en;
            u.c3 = zero_c3;
            if (q >= 4 && q < 4 + nn) {
                memset(unit_en, 0, sizeof(double) * nn);
                unit_en[q - 4] = 1.0;
                u.a_en = unit_en;
            }
            if (q >= 4 + nn) {
                memset(unit_c3, 0, sizeof(double) * nn * s->n3);
                unit_c3[q - 4 - nn] = 1.0;
                u.c3 = unit_c3;
            }
            B = jastrow(&u, R, gB, lB);
        }
        double t = 0.0;
        for (int i = 0; i < N; ++i) {
            double dot = 0.0;
            for (int c = 0; c < 3; ++c) dot += G[3 * i + c] * gB[3 * i + c];
            t += lB[i] + 2.0 * dot;
        }
        cx->dlog[(size_t)w * P + q] = B;
        cx->deloc[(size_t)w * P + q] = -0.5 * t + dvnl[q];
    }
    free(dvnl);
    free(G); free(gB); free(lB); free(zero_en); free(unit_en); free(unit_c3); free(zero_c3);
}

int oracle_jastrow_derivs(const oracle_system* s, int W, const double* R, double* dlog, double* deloc, int nthreads) {
    basis_prep p;
    det_list d;
    prep_basis(s, &p);
    build_dets(s, &d);
    jd_ctx c = {s, &p, &d, R, dlog, deloc, 4 + s->n_nuc + s->n_nuc * s->n3};
    parallel_for(W, nthreads, jd_worker, &c);
    free_dets(&d);
    free_basis(&p);
    return 0;
}

/* ------------------------------------------------------------------ */
/* forward-mode ionic derivatives                                      */
/* ------------------------------------------------------------------ */

/* Hessian slot of (c, c') and the derivative of the Laplacian along c'. */
static int hess_slot(int c, int cp) {
    int m[3] = {0, 0, 0};
    m[c]++;
    m[cp]++;
    return slot_of(m[0], m[1], m[2]);
}

static double dlap(const double* b, int cp) {
    double v = 0.0;
    for (int c = 0; c < 3; ++c) {
        int m[3] = {0, 0, 0};
        m[c] += 2;
        m[cp] += 1;
        v += b[slot_of(m[0], m[1], m[2])];
    }
    return v;
}

/* ------------------------------------------------------------------ */
/* ionic derivatives of the pseudopotential                            */
/* ------------------------------------------------------------------ */

/* d/dr of one radial term: beta exp(-alpha r^2) ((n-2) r^(n-3) - 2 alpha r^(n-1)). */
static double pp_term_dr(const oracle_system* s, int t, double r) {
    const int k = s->pp_n[t] - 2;
    const double rk = k >= 0 ? ipow(r, k) : 1.0 / ipow(r, -k);   /* r^(n-2) */
    return s->pp_beta[t] * exp(-s->pp_alpha[t] * r * r) * rk * ((double)k / r - 2.0 * s->pp_alpha[t] * r);
}

static double legendre_dx(int l, double x) {
    switch (l) {
        case 0: return 0.0;
        case 1: return 1.0;
        case 2: return 3.0 * x;
        default: return 0.5 * (15.0 * x * x - 3.0);
    }
}

/* Explicit nuclear derivatives of ln|psi| at the configuration R (electrons
 * held fixed, every basis function moving with its nucleus), out[3 n_nuc],
 * and grad_e ln|psi| of electron e into ge.  Plain forms: for each
 * determinant block d ln D / dR_bc = sum_ij (A^-1)_ji dA_ij/dR_bc with
 * dA_ij/dR_bc = -sum_{basis l on b} C_{o_j l} d_c Phi_l(r_i); the sum over
 * determinants weighted by c_k D_k / psi_D; the electron-nucleus Jastrow
 * terms -u'(r_ib) (r_i - R_b)_c / r_ib.  Returns nonzero where psi = 0. */
static int dlog_explicit(const oracle_system* s, const basis_prep* p, const det_list* d, const double* R,
                         double* out, int e, double ge[3]) {
    const int nu = s->n_up, nd = s->n_dn, N = nu + nd, nb = p->n_basis, nn = s->n_nuc;
    const int nmax = nu > nd ? nu : nd;
    double* bas = (double*)malloc(sizeof(double) * (size_t)N * nb * OD_N + 1);
    for (int i = 0; i < N; ++i) basis_eval(s, p, R + 3 * i, 1, bas + (size_t)i * nb * OD_N);
    double* mo = (double*)malloc(sizeof(double) * (size_t)N * (d->n_orb > 0 ? d->n_orb : 1) * 5);
    eval_orbitals(s, p, R, 0, N, d->n_orb, 1, mo);
    const int K = d->n_det;
    double* la = (double*)malloc(sizeof(double) * K);
    double* sg = (double*)malloc(sizeof(double) * K);
    double* dla = (double*)calloc((size_t)K * 3 * nn + 1, sizeof(double));
    double* gk = (double*)calloc((size_t)K * 3 + 1, sizeof(double));
    double* A = (double*)malloc(sizeof(double) * (nmax * nmax + 1));
    double* Ai = (double*)malloc(sizeof(double) * (nmax * nmax + 1));
    double Lmax = -INFINITY;
    for (int k = 0; k < K; ++k) {
        la[k] = 0.0;
        sg[k] = 1.0;
        for (int blk = 0; blk < 2; ++blk) {
            const int n = blk == 0 ? nu : nd, i0 = blk == 0 ? 0 : nu;
            const int* orbs = blk == 0 ? d->orb_up + (size_t)k * nu : d->orb_dn + (size_t)k * nd;
            if (n == 0) continue;
            for (int i = 0; i < n; ++i)
                for (int j = 0; j < n; ++j) A[i * n + j] = mo[((size_t)(i0 + i) * d->n_orb + orbs[j]) * 5];
            double lb, sb;
            if (oracle_lu_det(n, A, &lb, &sb, Ai) || sb == 0.0) {
                sg[k] = 0.0;
                break;
            }
            la[k] += lb;
            sg[k] *= sb;
            for (int b = 0; b < nn; ++b)
                for (int c = 0; c < 3; ++c) {
                    double t = 0.0;
                    for (int i = 0; i < n; ++i)
                        for (int j = 0; j < n; ++j) {
                            const double* Cj = s->C + (size_t)orbs[j] * s->n_basis;
                            double dA = 0.0;
                            for (int l = 0; l < nb; ++l)
                                if (p->fn_center[l] == b)
                                    dA -= Cj[l] * bas[((size_t)(i0 + i) * nb + l) * OD_N + OD100 + c];
                            t += Ai[j * n + i] * dA;
                        }
                    dla[(size_t)k * 3 * nn + 3 * b + c] += t;
                }
            if (e >= i0 && e < i0 + n)
                for (int j = 0; j < n; ++j) {
                    const double* m = mo + ((size_t)e * d->n_orb + orbs[j]) * 5;
                    for (int c = 0; c < 3; ++c) gk[3 * k + c] += m[1 + c] * Ai[j * n + (e - i0)];
                }
        }
        if (sg[k] != 0.0 && d->c[k] != 0.0 && la[k] > Lmax) Lmax = la[k];
    }
    double S = 0.0;
    for (int k = 0; k < K; ++k) {
        la[k] = sg[k] == 0.0 ? 0.0 : d->c[k] * sg[k] * exp(la[k] - Lmax);   /* r_k */
        S += la[k];
    }
    const int bad = !(S != 0.0) || !isfinite(S);
    for (int q = 0; q < 3 * nn; ++q) {
        double t = 0.0;
        for (int k = 0; k < K; ++k) t += la[k] * dla[(size_t)k * 3 * nn + q];
        out[q] = bad ? 0.0 : t / S;
    }
    for (int c = 0; c < 3; ++c) {
        double t = 0.0;
        for (int k = 0; k < K; ++k) t += la[k] * gk[3 * k + c];
        ge[c] = bad ? 0.0 : t / S;
    }
    for (int i = 0; i < N; ++i)
        for (int b = 0; b < nn; ++b) {
            double x[3], r2 = 0.0;
            for (int c = 0; c < 3; ++c) {
                x[c] = R[3 * i + c] - s->R[3 * b + c];
                r2 += x[c] * x[c];
            }
            const double r = sqrt(r2);
            double u, du, d2u, d3u;
            pade(s->a_en[b], s->b_en, r, &u, &du, &d2u, &d3u);
            for (int c = 0; c < 3; ++c) out[3 * b + c] += -du * x[c] / r;
        }
    double* gJ = (double*)malloc(sizeof(double) * 3 * (N + 1));
    jastrow(s, R, gJ, NULL);
    for (int c = 0; c < 3; ++c) ge[c] += gJ[3 * e + c];
    free(gJ); free(bas); free(mo); free(la); free(sg); free(dla); free(gk); free(A); free(Ai);
    return bad;
}

/* Nuclear derivatives of the non-local energy of one walker, added to
 * dV[3 n_nuc]: for every point p = (i, a, q) of nonlocal_one with weight
 * W_p = w_q sum_l (2l+1) v_l(r) P_l(cos) and ratio rho_p = psi(R'_p)/psi(R),
 *   d(W_p rho_p)/dR_bc = [b = a] dW_p/dR_ac rho_p
 *       + W_p rho_p (D'_bc - D_bc + [b = a] g'_i . (e_c - d_q x_hat_c)),
 * D and D' the explicit derivatives of ln|psi| at R and at R'_p, g'_i the
 * gradient of ln|psi(R'_p)| in the moved electron, whose position
 * R_a + r d_q follows R_a (dr/dR_a = -x_hat, d cos/dR_a = -(d_q - cos x_hat)/r). */
static void nonlocal_deriv(const oracle_system* s, const basis_prep* p, const det_list* d, const double* R, int slot,
                           double* dV) {
    if (s->n_pp == 0) return;
    const int N = s->n_up + s->n_dn, nn = s->n_nuc;
    double* D0 = (double*)malloc(sizeof(double) * 3 * nn);
    double* D1 = (double*)malloc(sizeof(double) * 3 * nn);
    double* R2 = (double*)malloc(sizeof(double) * 3 * N);
    double g0[3];
    const double v0 = nonlocal_one(s, p, d, R, slot);   /* checks psi(R) != 0 */
    if (!isfinite(v0) || dlog_explicit(s, p, d, R, D0, 0, g0)) {
        for (int q = 0; q < 3 * nn; ++q) dV[q] = NAN;
        free(D0); free(D1); free(R2);
        return;
    }
    double l0, s0;
    {
        double* mo = (double*)malloc(sizeof(double) * (size_t)N * (d->n_orb > 0 ? d->n_orb : 1) * 5);
        eval_orbitals(s, p, R, 0, N, d->n_orb, 0, mo);
        det_part(s, d, mo, &l0, &s0, NULL, NULL);
        free(mo);
    }
    l0 += jastrow(s, R, NULL, NULL);
    for (int a = 0; a < nn; ++a) {
        int lmax = -1;
        for (int t = 0; t < s->n_pp; ++t)
            if (s->pp_nuc[t] == a && s->pp_l[t] > lmax) lmax = s->pp_l[t];
        if (lmax < 0) continue;
        double rot[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
        if (s->pp_rotate) oracle_pp_rotation(s->pp_seed, s->pp_sweep, (uint32_t)a, s->pp_slot0 + (uint32_t)slot, rot);
        for (int i = 0; i < N; ++i) {
            double x[3], r2 = 0.0;
            for (int c = 0; c < 3; ++c) {
                x[c] = R[3 * i + c] - s->R[3 * a + c];
                r2 += x[c] * x[c];
            }
            const double r = sqrt(r2);
            if (!(r < s->pp_rcut[a])) continue;
            double xh[3];
            for (int c = 0; c < 3; ++c) xh[c] = x[c] / r;
            double vl[4] = {0, 0, 0, 0}, dvl[4] = {0, 0, 0, 0};
            for (int t = 0; t < s->n_pp; ++t)
                if (s->pp_nuc[t] == a && s->pp_l[t] >= 0) {
                    vl[s->pp_l[t]] += pp_term(s, t, r);
                    dvl[s->pp_l[t]] += pp_term_dr(s, t, r);
                }
            for (int q = 0; q < s->pp_nq; ++q) {
                const double* o = s->pp_quad + 3 * q;
                double dq[3], cth = 0.0;
                for (int c = 0; c < 3; ++c) {
                    dq[c] = rot[3 * c] * o[0] + rot[3 * c + 1] * o[1] + rot[3 * c + 2] * o[2];
                    cth += dq[c] * xh[c];
                }
                memcpy(R2, R, sizeof(double) * 3 * N);
                for (int c = 0; c < 3; ++c) R2[3 * i + c] = s->R[3 * a + c] + r * dq[c];
                double l1, s1, g1[3];
                {
                    double* mo = (double*)malloc(sizeof(double) * (size_t)N * (d->n_orb > 0 ? d->n_orb : 1) * 5);
                    eval_orbitals(s, p, R2, 0, N, d->n_orb, 0, mo);
                    const int z = det_part(s, d, mo, &l1, &s1, NULL, NULL);
                    free(mo);
                    if (z) continue;   /* psi(R'_p) = 0: the point adds nothing, nor does its derivative */
                }
                l1 += jastrow(s, R2, NULL, NULL);
                const double rho = s1 * s0 * exp(l1 - l0);
                double W = 0.0, dW[3] = {0, 0, 0};
                for (int l = 0; l <= lmax; ++l) {
                    const double f = (2.0 * l + 1.0) * s->pp_qw[q];
                    W += f * vl[l] * legendre(l, cth);
                    for (int c = 0; c < 3; ++c)
                        dW[c] += f * (dvl[l] * legendre(l, cth) * (-xh[c]) +
                                      vl[l] * legendre_dx(l, cth) * (-(dq[c] - cth * xh[c]) / r));
                }
                dlog_explicit(s, p, d, R2, D1, i, g1);
                const double gd = g1[0] * dq[0] + g1[1] * dq[1] + g1[2] * dq[2];
                for (int b = 0; b < nn; ++b)
                    for (int c = 0; c < 3; ++c) {
                        double dl = D1[3 * b + c] - D0[3 * b + c];
                        double t = 0.0;
                        if (b == a) {
                            dl += g1[c] - gd * xh[c];
                            t += dW[c] * rho;
                        }
                        dV[3 * b + c] += t + W * rho * dl;
                    }
            }
        }
    }
    free(D0); free(D1); free(R2);
}

typedef struct {
    const oracle_system* s;
    const basis_prep* p;
    const det_list* d;
    const double* R;
    double *dEL, *dlog;
} force_ctx;

static void propagate_block_deriv(int n, const double* dA, const double* dG, const double* dL, const double* Ainv,
                                  const double* G, const double* L, double* dlogD, double* dgD, double* dlD,
                                  double* dAi, double* tmp);

/* Per determinant and spin block: derivative of ln|D|, grad_i D/D and
 * lap_i D/D with respect to one nuclear coordinate (atom a, direction cp). */
static void block_det_deriv(const oracle_system* s, const basis_prep* p, int n, int i0, const int* orbs,
                            const double* bas /*[N][n_basis][OD_N]*/, int a, int cp, const double* A,
                            const double* Ainv, const double* G /*[3][n][n]*/, const double* L,
                            double* dlogD, double* dgD /*[n][3]*/, double* dlD /*[n]*/, double* work) {
    const int nb = p->n_basis;
    double* dA = work;
    double* dG = dA + n * n;        /* [3][n][n] */
    double* dL = dG + 3 * n * n;
    double* dAi = dL + n * n;
    double* tmp = dAi + n * n;
    const int d1 = cp == 0 ? OD100 : (cp == 1 ? OD010 : OD001);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            const double* Co = s->C + (size_t)orbs[j] * s->n_basis;
            double va = 0.0, vg[3] = {0, 0, 0}, vl = 0.0;
            for (int l = 0; l < nb; ++l) {
                if (p->fn_center[l] != a) continue;
                const double* b = bas + ((size_t)(i0 + i) * nb + l) * OD_N;
                va += Co[l] * b[d1];
                for (int c = 0; c < 3; ++c) vg[c] += Co[l] * b[hess_slot(c, cp)];
                vl += Co[l] * dlap(b, cp);
            }
            /* the basis function moves with the nucleus: d/dR_a = -d/dr */
            dA[i * n + j] = -va;
            for (int c = 0; c < 3; ++c) dG[c * n * n + i * n + j] = -vg[c];
            dL[i * n + j] = -vl;
        }
    (void)A;
    propagate_block_deriv(n, dA, dG, dL, Ainv, G, L, dlogD, dgD, dlD, dAi, tmp);
}

/* Given the derivatives dA, dG [3][n][n], dL of A, of the gradient matrices
 * and of the Laplacian matrix along one direction, the derivatives of
 * ln|D| = ln|det A| (Eq. 3: tr(A^-1 dA)), of grad_i D/D = sum_j G_ij A^-1_ji
 * and of lap_i D/D, with dA^-1 = -A^-1 dA A^-1. */
static void propagate_block_deriv(int n, const double* dA, const double* dG, const double* dL, const double* Ainv,
                                  const double* G, const double* L, double* dlogD, double* dgD, double* dlD,
                                  double* dAi, double* tmp) {
    /* dAinv = -Ainv dA Ainv */
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            double v = 0.0;
            for (int k = 0; k < n; ++k) v += dA[i * n + k] * Ainv[k * n + j];
            tmp[i * n + j] = v;
        }
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            double v = 0.0;
            for (int k = 0; k < n; ++k) v += Ainv[i * n + k] * tmp[k * n + j];
            dAi[i * n + j] = -v;
        }
    double tr = 0.0;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) tr += Ainv[j * n + i] * dA[i * n + j];
    *dlogD = tr;
    for (int i = 0; i < n; ++i) {
        double g[3] = {0, 0, 0}, lp = 0.0;
        for (int j = 0; j < n; ++j) {
            for (int c = 0; c < 3; ++c)
                g[c] += dG[c * n * n + i * n + j] * Ainv[j * n + i] + G[c * n * n + i * n + j] * dAi[j * n + i];
            lp += dL[i * n + j] * Ainv[j * n + i] + L[i * n + j] * dAi[j * n + i];
        }
        for (int c = 0; c < 3; ++c) dgD[3 * i + c] = g[c];
        dlD[i] = lp;
    }
}

static void force_worker(void* vctx, int w) {
    force_ctx* fc = (force_ctx*)vctx;
    const oracle_system* s = fc->s;
    const basis_prep* p = fc->p;
    const det_list* d = fc->d;
    const int nu = s->n_up, nd = s->n_dn, N = nu + nd, nb = p->n_basis, nn = s->n_nuc;
    const double* R = fc->R + (size_t)w * 3 * N;
    const int nmax = nu > nd ? nu : nd;
    const int n2 = nmax * nmax + 1;

    double* bas = (double*)malloc(sizeof(double) * (size_t)N * nb * OD_N + 1);
    for (int i = 0; i < N; ++i) basis_eval(s, p, R + 3 * i, 3, bas + (size_t)i * nb * OD_N);
    double* mo = (double*)malloc(sizeof(double) * (size_t)N * (d->n_orb > 0 ? d->n_orb : 1) * 5);
    eval_orbitals(s, p, R, 0, N, d->n_orb, 2, mo);

    /* per determinant: ln|D_k|, sign, grad/lap D/D, and their derivatives */
    const int K = d->n_det;
    double* la = (double*)malloc(sizeof(double) * K);
    double* sg = (double*)malloc(sizeof(double) * K);
    double* gk = (double*)malloc(sizeof(double) * (size_t)K * 3 * N);
    double* lk = (double*)malloc(sizeof(double) * (size_t)K * N);
    double* dla = (double*)malloc(sizeof(double) * (size_t)K * 3 * nn);
    double* dgk = (double*)malloc(sizeof(double) * (size_t)K * 3 * nn * 3 * N);
    double* dlk = (double*)malloc(sizeof(double) * (size_t)K * 3 * nn * N);
    double* A = (double*)malloc(sizeof(double) * n2);
    double* Ai = (double*)malloc(sizeof(double) * n2);
    double* G = (double*)malloc(sizeof(double) * 3 * n2);
    double* L = (double*)malloc(sizeof(double) * n2);
    double* work = (double*)malloc(sizeof(double) * 8 * n2);
    double* dg1 = (double*)malloc(sizeof(double) * 3 * (nmax + 1));
    double* dl1 = (double*)malloc(sizeof(double) * (nmax + 1));
    double Lmax = -INFINITY;
    for (int k = 0; k < K; ++k) {
        la[k] = 0.0;
        sg[k] = 1.0;
        for (int q = 0; q < 3 * nn; ++q) dla[(size_t)k * 3 * nn + q] = 0.0;
        for (int blk = 0; blk < 2; ++blk) {
            const int n = blk == 0 ? nu : nd;
            const int i0 = blk == 0 ? 0 : nu;
            const int* orbs = blk == 0 ? d->orb_up + (size_t)k * nu : d->orb_dn + (size_t)k * nd;
            double lb, sb;
            int st = block_det(n, i0, orbs, d->n_orb, mo, &lb, &sb, gk + (size_t)k * 3 * N + 3 * i0,
                               lk + (size_t)k * N + i0, A, Ai);
            if (st || sg[k] == 0.0) {
                sg[k] = 0.0;
                continue;
            }
            la[k] += lb;
            sg[k] *= sb;
            if (n == 0) continue;
            for (int i = 0; i < n; ++i)
                for (int j = 0; j < n; ++j) {
                    const double* m = mo + ((size_t)(i0 + i) * d->n_orb + orbs[j]) * 5;
                    for (int c = 0; c < 3; ++c) G[c * n * n + i * n + j] = m[1 + c];
                    L[i * n + j] = m[4];
                }
            for (int a = 0; a < nn; ++a)
                for (int cp = 0; cp < 3; ++cp) {
                    double dl;
                    block_det_deriv(s, p, n, i0, orbs, bas, a, cp, A, Ai, G, L, &dl, dg1, dl1, work);
                    const size_t q = (size_t)k * 3 * nn + 3 * a + cp;
                    dla[q] += dl;
                    for (int i = 0; i < n; ++i) {
                        for (int c = 0; c < 3; ++c) dgk[q * 3 * N + 3 * (i0 + i) + c] = dg1[3 * i + c];
                        dlk[q * N + i0 + i] = dl1[i];
                    }
                }
        }
        if (sg[k] != 0.0 && d->c[k] != 0.0 && la[k] > Lmax) Lmax = la[k];
    }
    /* combine: psi_D / exp(Lmax) = S = sum_k r_k */
    double S = 0.0;
    double* rk = (double*)malloc(sizeof(double) * K);
    for (int k = 0; k < K; ++k) {
        rk[k] = (sg[k] == 0.0) ? 0.0 : d->c[k] * sg[k] * exp(la[k] - Lmax);
        S += rk[k];
    }
    double* gD = (double*)calloc(3 * N + 1, sizeof(double));
    double* lD = (double*)calloc(N + 1, sizeof(double));
    for (int k = 0; k < K; ++k) {
        for (int q = 0; q < 3 * N; ++q) gD[q] += rk[k] * gk[(size_t)k * 3 * N + q] / S;
        for (int q = 0; q < N; ++q) lD[q] += rk[k] * lk[(size_t)k * N + q] / S;
    }
    double* gJ = (double*)malloc(sizeof(double) * 3 * (N + 1));
    double* lJ = (double*)malloc(sizeof(double) * (N + 1));
    jastrow(s, R, gJ, lJ);

    double* dgD = (double*)malloc(sizeof(double) * 3 * (N + 1));
    double* dlD = (double*)malloc(sizeof(double) * (N + 1));
    /* the pseudopotential's non-local energy and its nuclear derivatives */
    double* dVnl = (double*)calloc(3 * nn + 1, sizeof(double));
    nonlocal_deriv(s, p, d, R, w, dVnl);
    for (int a = 0; a < nn; ++a)
        for (int cp = 0; cp < 3; ++cp) {
            /* determinant sum: d ln S and d(grad_i psi_D/psi_D), d(lap_i psi_D/psi_D) */
            double dlnS = 0.0;
            for (int k = 0; k < K; ++k) dlnS += rk[k] * dla[(size_t)k * 3 * nn + 3 * a + cp] / S;
            memset(dgD, 0, sizeof(double) * 3 * N);
            memset(dlD, 0, sizeof(double) * N);
            for (int k = 0; k < K; ++k) {
                if (rk[k] == 0.0) continue;
                const size_t q = (size_t)k * 3 * nn + 3 * a + cp;
                const double f = rk[k] / S;
                const double dr = dla[q] - dlnS; /* d ln(r_k / S) */
                for (int i = 0; i < 3 * N; ++i) dgD[i] += f * (dr * gk[(size_t)k * 3 * N + i] + dgk[q * 3 * N + i]);
                for (int i = 0; i < N; ++i) dlD[i] += f * (dr * lk[(size_t)k * N + i] + dlk[q * N + i]);
            }
            /* electron-nucleus Jastrow and potential terms of nucleus a */
            double dJ = 0.0, dV = 0.0, dT = 0.0;
            for (int i = 0; i < N; ++i) {
                double x[3], r2 = 0.0;
                for (int c = 0; c < 3; ++c) {
                    x[c] = R[3 * i + c] - s->R[3 * a + c];
                    r2 += x[c] * x[c];
                }
                const double r = sqrt(r2);
                double u, du, d2u, d3u;
                pade(s->a_en[a], s->b_en, r, &u, &du, &d2u, &d3u);
                dJ += -du * x[cp] / r;
                double dgJ[3];
                for (int c = 0; c < 3; ++c) {
                    const double H = (d2u - du / r) * x[c] * x[cp] / r2 + (c == cp ? du / r : 0.0);
                    dgJ[c] = -H;
                }
                const double dlJ = -(d3u + 2.0 * d2u / r - 2.0 * du / r2) * x[cp] / r;
                dV += -s->Z[a] * x[cp] / (r2 * r);
                for (int t2 = 0; t2 < s->n_pp; ++t2)   /* local pseudopotential terms of nucleus a */
                    if (s->pp_nuc[t2] == a && s->pp_l[t2] == -1) dV += pp_term_dr(s, t2, r) * (-x[cp] / r);
                double t = dlD[i] + dlJ;
                for (int c = 0; c < 3; ++c)
                    t += 2.0 * dgJ[c] * gD[3 * i + c] + 2.0 * gJ[3 * i + c] * dgD[3 * i + c] +
                         2.0 * gJ[3 * i + c] * dgJ[c];
                dT += -0.5 * t;
            }
            /* nucleus-nucleus repulsion */
            for (int b = 0; b < nn; ++b) {
                if (b == a) continue;
                double x[3], r2 = 0.0;
                for (int c = 0; c < 3; ++c) {
                    x[c] = s->R[3 * a + c] - s->R[3 * b + c];
                    r2 += x[c] * x[c];
                }
                dV += -s->Z[a] * s->Z[b] * x[cp] / (r2 * sqrt(r2));
            }
            fc->dEL[(size_t)w * 3 * nn + 3 * a + cp] = dT + dV + dVnl[3 * a + cp];
            fc->dlog[(size_t)w * 3 * nn + 3 * a + cp] = dJ + dlnS;
        }
    free(bas); free(mo); free(la); free(sg); free(gk); free(lk); free(dla); free(dgk); free(dlk);
    free(A); free(Ai); free(G); free(L); free(work); free(dg1); free(dl1); free(rk); free(gD); free(lD);
    free(gJ); free(lJ); free(dgD); free(dlD); free(dVnl);
}

int oracle_forces(const oracle_system* s, int W, const double* R, double* dEL, double* dlogpsi,
                  int nthreads) {
    /* the ionic derivatives of the three-body term are not written out */
    if (s->n3 > 0) return -9;
    basis_prep p;
    det_list d;
    prep_basis(s, &p);
    build_dets(s, &d);
    force_ctx c = {s, &p, &d, R, dEL, dlogpsi};
    parallel_for(W, nthreads, force_worker, &c);
    free_dets(&d);
    free_basis(&p);
    return 0;
}

/* ------------------------------------------------------------------ */
/* forward-mode electron-coordinate derivatives and the space warp     */
/* ------------------------------------------------------------------ */

/* Derivatives of grad_i J [N][3], lap_i J [N], J and V along coordinate cp
 * of electron e.  Every pair term depends on x = r_p - r_q only; moving
 * electron e changes the offsets of the pairs (e, j) and (e, a) by +e_cp.
 * For u(|x|): d(u' x_c / r)/dx_cp = (u'' - u'/r) x_c x_cp / r^2 + delta_{c,cp} u'/r
 * and d(u'' + 2u'/r)/dx_cp = (u''' + 2u''/r - 2u'/r^2) x_cp / r; the gradient
 * of the partner electron j changes with the opposite sign, its Laplacian
 * with the same sign. */
static void jastrow_pot_deriv_elec(const oracle_system* s, const double* R, int e, int cp, double* dgJ,
                                   double* dlJ, double* dJ, double* dV) {
    const int N = s->n_up + s->n_dn;
    memset(dgJ, 0, sizeof(double) * 3 * N);
    memset(dlJ, 0, sizeof(double) * N);
    *dJ = 0.0;
    *dV = 0.0;
    for (int j = 0; j < N + s->n_nuc; ++j) {
        if (j == e) continue;
        const int nuc = j >= N;
        const double* Rq = nuc ? s->R + 3 * (j - N) : R + 3 * j;
        double x[3], r2 = 0.0;
        for (int c = 0; c < 3; ++c) {
            x[c] = R[3 * e + c] - Rq[c];
            r2 += x[c] * x[c];
        }
        const double r = sqrt(r2);
        double a, b;
        if (nuc) {
            a = s->a_en[j - N];
            b = s->b_en;
        } else {
            a = ((e < s->n_up) == (j < s->n_up)) ? s->a_par : s->a_anti;
            b = s->b_ee;
        }
        double u, du, d2u, d3u;
        pade(a, b, r, &u, &du, &d2u, &d3u);
        for (int c = 0; c < 3; ++c) {
            const double H = (d2u - du / r) * x[c] * x[cp] / r2 + (c == cp ? du / r : 0.0);
            dgJ[3 * e + c] += H;
            if (!nuc) dgJ[3 * j + c] -= H;
        }
        const double D3 = (d3u + 2.0 * d2u / r - 2.0 * du / r2) * x[cp] / r;
        dlJ[e] += D3;
        if (!nuc) dlJ[j] += D3;
        *dJ += du * x[cp] / r;
        /* V_ee = 1/r, V_en = -Z/r */
        *dV += (nuc ? s->Z[j - N] : -1.0) * x[cp] / (r2 * r);
    }
}

typedef struct {
    const oracle_system* s;
    const basis_prep* p;
    const det_list* d;
    const double* R;
    double *gEL, *glog;
} egrad_ctx;

/* grad_e E_L and grad_e ln|psi| of one walker, one electron coordinate at a
 * time: only row e of the spin block holding electron e changes, by the
 * basis derivatives at r_e (all basis functions, d/dr_e), after which the
 * determinant derivatives follow as for a nuclear coordinate. */
static void egrad_worker(void* vctx, int w) {
    egrad_ctx* ec = (egrad_ctx*)vctx;
    const oracle_system* s = ec->s;
    const basis_prep* p = ec->p;
    const det_list* d = ec->d;
    const int nu = s->n_up, nd = s->n_dn, N = nu + nd, nb = p->n_basis;
    const double* R = ec->R + (size_t)w * 3 * N;
    const int nmax = nu > nd ? nu : nd;
    const int n2 = nmax * nmax + 1;
    const int K = d->n_det;

    double* bas = (double*)malloc(sizeof(double) * (size_t)N * nb * OD_N + 1);
    for (int i = 0; i < N; ++i) basis_eval(s, p, R + 3 * i, 3, bas + (size_t)i * nb * OD_N);
    double* mo = (double*)malloc(sizeof(double) * (size_t)N * (d->n_orb > 0 ? d->n_orb : 1) * 5);
    eval_orbitals(s, p, R, 0, N, d->n_orb, 2, mo);

    /* per determinant and block: A^-1, G, L kept for the derivatives */
    double* la = (double*)malloc(sizeof(double) * K);
    double* sg = (double*)malloc(sizeof(double) * K);
    double* gk = (double*)malloc(sizeof(double) * (size_t)K * 3 * N);
    double* lk = (double*)malloc(sizeof(double) * (size_t)K * N);
    double* keep = (double*)malloc(sizeof(double) * (size_t)K * 2 * 5 * n2);
    double* A = (double*)malloc(sizeof(double) * n2);
    double Lmax = -INFINITY;
    for (int k = 0; k < K; ++k) {
        la[k] = 0.0;
        sg[k] = 1.0;
        for (int blk = 0; blk < 2; ++blk) {
            const int n = blk == 0 ? nu : nd;
            const int i0 = blk == 0 ? 0 : nu;
            const int* orbs = blk == 0 ? d->orb_up + (size_t)k * nu : d->orb_dn + (size_t)k * nd;
            double* Ai = keep + ((size_t)k * 2 + blk) * 5 * n2;
            double* G = Ai + n2;
            double* L = G + 3 * n2;
            double lb, sb;
            int st = block_det(n, i0, orbs, d->n_orb, mo, &lb, &sb, gk + (size_t)k * 3 * N + 3 * i0,
                               lk + (size_t)k * N + i0, A, Ai);
            if (st || sg[k] == 0.0) {
                sg[k] = 0.0;
                continue;
            }
            la[k] += lb;
            sg[k] *= sb;
            for (int i = 0; i < n; ++i)
                for (int j = 0; j < n; ++j) {
                    const double* m = mo + ((size_t)(i0 + i) * d->n_orb + orbs[j]) * 5;
                    for (int c = 0; c < 3; ++c) G[c * n * n + i * n + j] = m[1 + c];
                    L[i * n + j] = m[4];
                }
        }
        if (sg[k] != 0.0 && d->c[k] != 0.0 && la[k] > Lmax) Lmax = la[k];
    }
    double S = 0.0;
    double* rk = (double*)malloc(sizeof(double) * K);
    for (int k = 0; k < K; ++k) {
        rk[k] = (sg[k] == 0.0) ? 0.0 : d->c[k] * sg[k] * exp(la[k] - Lmax);
        S += rk[k];
    }
    double* gD = (double*)calloc(3 * N + 1, sizeof(double));
    double* lD = (double*)calloc(N + 1, sizeof(double));
    for (int k = 0; k < K; ++k) {
        for (int q = 0; q < 3 * N; ++q) gD[q] += rk[k] * gk[(size_t)k * 3 * N + q] / S;
        for (int q = 0; q < N; ++q) lD[q] += rk[k] * lk[(size_t)k * N + q] / S;
    }
    double* gJ = (double*)malloc(sizeof(double) * 3 * (N + 1));
    double* lJ = (double*)malloc(sizeof(double) * (N + 1));
    jastrow(s, R, gJ, lJ);

    double* dla = (double*)malloc(sizeof(double) * K);
    double* dgk = (double*)calloc((size_t)K * 3 * N + 1, sizeof(double));
    double* dlk = (double*)calloc((size_t)K * N + 1, sizeof(double));
    double* work = (double*)malloc(sizeof(double) * 8 * n2);
    double* dg1 = (double*)malloc(sizeof(double) * 3 * (nmax + 1));
    double* dl1 = (double*)malloc(sizeof(double) * (nmax + 1));
    double* dgD = (double*)malloc(sizeof(double) * 3 * (N + 1));
    double* dlD = (double*)malloc(sizeof(double) * (N + 1));
    double* dgJ = (double*)malloc(sizeof(double) * 3 * (N + 1));
    double* dlJ = (double*)malloc(sizeof(double) * (N + 1));
    for (int e = 0; e < N; ++e) {
        const int blk = e >= nu;
        const int n = blk ? nd : nu;
        const int i0 = blk ? nu : 0;
        const int ie = e - i0;
        const double* be = bas + (size_t)e * nb * OD_N;
        for (int cp = 0; cp < 3; ++cp) {
            const int d1 = cp == 0 ? OD100 : (cp == 1 ? OD010 : OD001);
            memset(dgk, 0, sizeof(double) * (size_t)K * 3 * N);
            memset(dlk, 0, sizeof(double) * (size_t)K * N);
            for (int k = 0; k < K; ++k) {
                dla[k] = 0.0;
                if (sg[k] == 0.0) continue;
                const int* orbs = blk == 0 ? d->orb_up + (size_t)k * nu : d->orb_dn + (size_t)k * nd;
                const double* Ai = keep + ((size_t)k * 2 + blk) * 5 * n2;
                const double* G = Ai + n2;
                const double* L = G + 3 * n2;
                double* dA = work;
                double* dG = dA + n * n;
                double* dL = dG + 3 * n * n;
                double* dAi = dL + n * n;
                double* tmp = dAi + n * n;
                memset(dA, 0, sizeof(double) * 5 * n * n);
                for (int j = 0; j < n; ++j) {
                    const double* Co = s->C + (size_t)orbs[j] * s->n_basis;
                    double va = 0.0, vg[3] = {0, 0, 0}, vl = 0.0;
                    for (int l = 0; l < nb; ++l) {
                        const double* b = be + (size_t)l * OD_N;
                        va += Co[l] * b[d1];
                        for (int c = 0; c < 3; ++c) vg[c] += Co[l] * b[hess_slot(c, cp)];
                        vl += Co[l] * dlap(b, cp);
                    }
                    dA[ie * n + j] = va;
                    for (int c = 0; c < 3; ++c) dG[c * n * n + ie * n + j] = vg[c];
                    dL[ie * n + j] = vl;
                }
                propagate_block_deriv(n, dA, dG, dL, Ai, G, L, &dla[k], dg1, dl1, dAi, tmp);
                for (int i = 0; i < n; ++i) {
                    for (int c = 0; c < 3; ++c) dgk[(size_t)k * 3 * N + 3 * (i0 + i) + c] = dg1[3 * i + c];
                    dlk[(size_t)k * N + i0 + i] = dl1[i];
                }
            }
            /* determinant sum, as for the nuclear coordinates */
            double dlnS = 0.0;
            for (int k = 0; k < K; ++k) dlnS += rk[k] * dla[k] / S;
            memset(dgD, 0, sizeof(double) * 3 * N);
            memset(dlD, 0, sizeof(double) * N);
            for (int k = 0; k < K; ++k) {
                if (rk[k] == 0.0) continue;
                const double f = rk[k] / S;
                const double dr = dla[k] - dlnS;
                for (int i = 0; i < 3 * N; ++i)
                    dgD[i] += f * (dr * gk[(size_t)k * 3 * N + i] + dgk[(size_t)k * 3 * N + i]);
                for (int i = 0; i < N; ++i) dlD[i] += f * (dr * lk[(size_t)k * N + i] + dlk[(size_t)k * N + i]);
            }
            double dJ, dV;
            jastrow_pot_deriv_elec(s, R, e, cp, dgJ, dlJ, &dJ, &dV);
            double dT = 0.0;
            for (int i = 0; i < N; ++i) {
                double t = dlD[i] + dlJ[i];
                for (int c = 0; c < 3; ++c)
                    t += 2.0 * dgJ[3 * i + c] * gD[3 * i + c] + 2.0 * gJ[3 * i + c] * dgD[3 * i + c] +
                         2.0 * gJ[3 * i + c] * dgJ[3 * i + c];
                dT += -0.5 * t;
            }
            if (ec->gEL) ec->gEL[(size_t)w * 3 * N + 3 * e + cp] = dT + dV;
            if (ec->glog) ec->glog[(size_t)w * 3 * N + 3 * e + cp] = dJ + dlnS;
        }
    }
    free(bas); free(mo); free(la); free(sg); free(gk); free(lk); free(keep); free(A); free(rk); free(gD);
    free(lD); free(gJ); free(lJ); free(dla); free(dgk); free(dlk); free(work); free(dg1); free(dl1);
    free(dgD); free(dlD); free(dgJ); free(dlJ);
}

int oracle_electron_grad(const oracle_system* s, int W, const double* R, double* gEL, double* glog,
                         int nthreads) {
    if (s->n3 > 0 || s->n_pp > 0) return -9;
    basis_prep p;
    det_list d;
    prep_basis(s, &p);
    build_dets(s, &d);
    egrad_ctx c = {s, &p, &d, R, gEL, glog};
    parallel_for(W, nthreads, egrad_worker, &c);
    free_dets(&d);
    free_basis(&p);
    return 0;
}

/* Space-warp weights of Filippi and Umrigar (2000):
 * omega_a(r) = F(|r - R_a|) / sum_b F(|r - R_b|) with F(d) = d^-4, and
 * their gradients, grad F(d) = -4 x / d^6 (x = r - R_a). */
void oracle_warp_weights(const oracle_system* s, const double r[3], double* om, double* gom) {
    const int nn = s->n_nuc;
    double S = 0.0, gS[3] = {0, 0, 0};
    for (int a = 0; a < nn; ++a) {
        double x[3], d2 = 0.0;
        for (int c = 0; c < 3; ++c) {
            x[c] = r[c] - s->R[3 * a + c];
            d2 += x[c] * x[c];
        }
        const double F = 1.0 / (d2 * d2);
        om[a] = F;
        for (int c = 0; c < 3; ++c) {
            gom[3 * a + c] = -4.0 * x[c] * F / d2;
            gS[c] += gom[3 * a + c];
        }
        S += F;
    }
    for (int a = 0; a < nn; ++a) {
        for (int c = 0; c < 3; ++c) gom[3 * a + c] = (gom[3 * a + c] * S - om[a] * gS[c]) / (S * S);
        om[a] /= S;
    }
}

/* Space-warped ionic derivatives.  When nucleus a moves by dR, electron i
 * moves with it by omega_a(r_i) dR, so along coordinate c
 *   dE_L^w / dR_ac      = dE_L/dR_ac + sum_i omega_a(r_i) dE_L/dr_ic,
 *   d ln|psi|^w / dR_ac = d ln|psi|/dR_ac + sum_i omega_a(r_i) d ln|psi|/dr_ic
 *                         + 1/2 sum_i d omega_a(r_i) / dr_ic,
 * the last term being half the derivative of the log Jacobian of the
 * electron map (the sampled density |psi|^2 carries the Jacobian).  Inputs
 * per walker: the unwarped dEL, dlog [n_nuc][3] and the electron gradients
 * gEL, glog [N][3]. */
int oracle_space_warp(const oracle_system* s, int W, const double* R, const double* dEL, const double* dlog,
                      const double* gEL, const double* glog, double* dEL_w, double* dlog_w) {
    const int N = s->n_up + s->n_dn, nn = s->n_nuc;
    double* om = (double*)malloc(sizeof(double) * (nn + 1));
    double* gom = (double*)malloc(sizeof(double) * 3 * (nn + 1));
    for (int w = 0; w < W; ++w) {
        const size_t o = (size_t)w * 3 * nn;
        for (int q = 0; q < 3 * nn; ++q) {
            dEL_w[o + q] = dEL[o + q];
            dlog_w[o + q] = dlog[o + q];
        }
        for (int i = 0; i < N; ++i) {
            const double* r = R + ((size_t)w * N + i) * 3;
            oracle_warp_weights(s, r, om, gom);
            for (int a = 0; a < nn; ++a)
                for (int c = 0; c < 3; ++c) {
                    dEL_w[o + 3 * a + c] += om[a] * gEL[((size_t)w * N + i) * 3 + c];
                    dlog_w[o + 3 * a + c] += om[a] * glog[((size_t)w * N + i) * 3 + c] + 0.5 * gom[3 * a + c];
                }
        }
    }
    free(om);
    free(gom);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Philox4x32-10                                                       */
/* ------------------------------------------------------------------ */

void oracle_philox4x32(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        const uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        c0 = hi1 ^ c1 ^ k0;
        c1 = lo1;
        c2 = hi0 ^ c3 ^ k1;
        c3 = lo0;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static double u01(uint32_t x) { return ((double)x + 0.5) * (1.0 / 4294967296.0); }

/* Stream layout: counter (sweep, electron, walker slot, purpose).
 * purpose 0: three normals by Box-Muller, 1: acceptance uniform,
 * 2: branching uniform (electron field = 0xFFFFFFFF). */
static void draw_normals(uint64_t seed, uint32_t sweep, uint32_t e, uint32_t slot, double chi[3]) {
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    const uint32_t ctr[4] = {sweep, e, slot, 0u};
    uint32_t x[4];
    oracle_philox4x32(ctr, key, x);
    const double r1 = sqrt(-2.0 * log(u01(x[0]))), r2 = sqrt(-2.0 * log(u01(x[2])));
    chi[0] = r1 * cos(2.0 * M_PI * u01(x[1]));
    chi[1] = r1 * sin(2.0 * M_PI * u01(x[1]));
    chi[2] = r2 * cos(2.0 * M_PI * u01(x[3]));
}

static double draw_uniform(uint64_t seed, uint32_t sweep, uint32_t e, uint32_t slot, uint32_t purpose) {
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    const uint32_t ctr[4] = {sweep, e, slot, purpose};
    uint32_t x[4];
    oracle_philox4x32(ctr, key, x);
    return u01(x[0]);
}

/* Uniform random rotation by Shoemake's method ("Uniform random
 * rotations", Graphics Gems III, 1992): three uniforms u1, u2, u3 give the
 * unit quaternion (x, y, z, w) = (sqrt(1-u1) sin 2 pi u2, sqrt(1-u1)
 * cos 2 pi u2, sqrt(u1) sin 2 pi u3, sqrt(u1) cos 2 pi u3); rot is its
 * rotation matrix, row-major.  The uniforms are the first three words of
 * Philox at counter (sweep, nucleus, slot, 3). */
void oracle_pp_rotation(uint64_t seed, uint32_t sweep, uint32_t nucleus, uint32_t slot, double rot[9]) {
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    const uint32_t ctr[4] = {sweep, nucleus, slot, 3u};
    uint32_t v[4];
    oracle_philox4x32(ctr, key, v);
    const double u1 = u01(v[0]), u2 = u01(v[1]), u3 = u01(v[2]);
    const double a = sqrt(1.0 - u1), b = sqrt(u1);
    const double x = a * sin(2.0 * M_PI * u2), y = a * cos(2.0 * M_PI * u2);
    const double z = b * sin(2.0 * M_PI * u3), w = b * cos(2.0 * M_PI * u3);
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

typedef struct {
    const oracle_system* s;
    const basis_prep* p;
    const det_list* d;
    const double* R;
    double* vnl;
} nl_ctx;

static void nl_worker(void* vctx, int w) {
    nl_ctx* c = (nl_ctx*)vctx;
    const int N = c->s->n_up + c->s->n_dn;
    c->vnl[w] = nonlocal_one(c->s, c->p, c->d, c->R + (size_t)w * 3 * N, w);
}

int oracle_nonlocal(const oracle_system* s, int W, const double* R, double* vnl, int nthreads) {
    basis_prep p;
    det_list d;
    prep_basis(s, &p);
    build_dets(s, &d);
    nl_ctx c = {s, &p, &d, R, vnl};
    parallel_for(W, nthreads, nl_worker, &c);
    free_dets(&d);
    free_basis(&p);
    return 0;
}

/* ------------------------------------------------------------------ */
/* particle-by-particle moves                                          */
/* ------------------------------------------------------------------ */

/* ln|psi| (up to the part that does not depend on electron e), its sign
 * and grad_e ln|psi|, all recomputed from scratch.  For a single
 * determinant only the spin block of e is refactorised; for a
 * determinant sum, every determinant. */
static int logpsi_grad_e(const oracle_system* s, const basis_prep* p, const det_list* d, const double* R,
                         int e, double* lnpsi, double* sgn, double g[3], double* scratch_mo) {
    const int nu = s->n_up, nd = s->n_dn, N = nu + nd;
    double gJ[3] = {0, 0, 0};
    double* gJall = (double*)malloc(sizeof(double) * 3 * N);
    const double J = jastrow(s, R, gJall, NULL);
    for (int c = 0; c < 3; ++c) gJ[c] = gJall[3 * e + c];
    free(gJall);
    double ld, sd;
    double gd[3];
    if (d->n_det == 1 && s->n_det == 0) {
        const int up = e < nu;
        const int n = up ? nu : nd, i0 = up ? 0 : nu;
        const int* orbs = up ? d->orb_up : d->orb_dn;
        eval_orbitals(s, p, R, i0, i0 + n, d->n_orb, 1, scratch_mo);
        double* A = (double*)malloc(sizeof(double) * n * n);
        double* Ai = (double*)malloc(sizeof(double) * n * n);
        double* gb = (double*)malloc(sizeof(double) * 3 * n);
        int st = block_det(n, i0, orbs, d->n_orb, scratch_mo, &ld, &sd, gb, NULL, A, Ai);
        for (int c = 0; c < 3; ++c) gd[c] = st ? 0.0 : gb[3 * (e - i0) + c];
        free(A); free(Ai); free(gb);
        if (st) sd = 0.0;
    } else {
        eval_orbitals(s, p, R, 0, N, d->n_orb, 1, scratch_mo);
        double* gD = (double*)malloc(sizeof(double) * 3 * N);
        int st = det_part(s, d, scratch_mo, &ld, &sd, gD, NULL);
        for (int c = 0; c < 3; ++c) gd[c] = st ? 0.0 : gD[3 * e + c];
        free(gD);
        if (st) sd = 0.0;
    }
    *lnpsi = J + ld;
    *sgn = sd;
    for (int c = 0; c < 3; ++c) g[c] = gJ[c] + gd[c];
    return 0;
}

/* Umrigar-Nightingale-Runge (1993) drift cap with a = 1, written in the
 * cancellation-free form 2 / (1 + sqrt(1 + 2 a v^2 tau)). */
static void capped_drift(const double g[3], double tau, double vb[3]) {
    const double v2 = g[0] * g[0] + g[1] * g[1] + g[2] * g[2];
    const double f = 2.0 / (1.0 + sqrt(1.0 + 2.0 * v2 * tau));
    for (int c = 0; c < 3; ++c) vb[c] = f * g[c];
}

typedef struct {
    const oracle_system* s;
    const basis_prep* p;
    const det_list* d;
    double* R;
    double tau;
    uint64_t seed;
    uint32_t sweep;
    long long* n_accept;
} sweep_ctx;

static void sweep_worker(void* vctx, int w) {
    sweep_ctx* c = (sweep_ctx*)vctx;
    const oracle_system* s = c->s;
    const int N = s->n_up + s->n_dn;
    double* R = c->R + (size_t)w * 3 * N;
    double* Rp = (double*)malloc(sizeof(double) * 3 * N);
    double* mo = (double*)malloc(sizeof(double) * (size_t)N * (c->d->n_orb > 0 ? c->d->n_orb : 1) * 5);
    long long acc = 0;
    const double tau = c->tau, st = sqrt(tau);
    for (int e = 0; e < N; ++e) {
        double lp, sg, g[3], vb[3], chi[3];
        logpsi_grad_e(s, c->p, c->d, R, e, &lp, &sg, g, mo);
        capped_drift(g, tau, vb);
        draw_normals(c->seed, c->sweep, (uint32_t)e, (uint32_t)w, chi);
        memcpy(Rp, R, sizeof(double) * 3 * N);
        double rn[3];
        for (int k = 0; k < 3; ++k) rn[k] = R[3 * e + k] + tau * vb[k] + st * chi[k];
        for (int k = 0; k < 3; ++k) Rp[3 * e + k] = rn[k];
        double lpn, sgn, gn[3], vbn[3];
        logpsi_grad_e(s, c->p, c->d, Rp, e, &lpn, &sgn, gn, mo);
        int accept = 0;
        if (sgn == sg && sg != 0.0 && isfinite(lpn)) {
            capped_drift(gn, tau, vbn);
            double fwd = 0.0, bwd = 0.0;
            for (int k = 0; k < 3; ++k) {
                const double f = rn[k] - R[3 * e + k] - tau * vb[k];
                const double b = R[3 * e + k] - rn[k] - tau * vbn[k];
                fwd += f * f;
                bwd += b * b;
            }
            const double lnprob = 2.0 * (lpn - lp) - (bwd - fwd) / (2.0 * tau);
            const double u = draw_uniform(c->seed, c->sweep, (uint32_t)e, (uint32_t)w, 1u);
            accept = (lnprob >= 0.0) || (u < exp(lnprob));
        }
        if (accept) {
            for (int k = 0; k < 3; ++k) R[3 * e + k] = rn[k];
            ++acc;
        }
    }
    if (c->n_accept) c->n_accept[w] += acc;
    free(Rp);
    free(mo);
}

int oracle_vmc(const oracle_system* s, int W, double* R, int n_sweeps, double tau, uint64_t seed,
               uint32_t step0, long long* n_accept, double* eloc_trace, int nthreads) {
    basis_prep p;
    det_list d;
    prep_basis(s, &p);
    build_dets(s, &d);
    /* E_L after the sweep with counter t takes its pseudopotential
     * rotations from counter t + 1 (the counter of the next sweep) */
    oracle_system sl = *s;
    sl.pp_seed = seed;
    sl.pp_slot0 = 0;
    for (int k = 0; k < n_sweeps; ++k) {
        sweep_ctx c = {s, &p, &d, R, tau, seed, step0 + (uint32_t)k, n_accept};
        parallel_for(W, nthreads, sweep_worker, &c);
        if (eloc_trace) {
            sl.pp_sweep = step0 + (uint32_t)k + 1u;
            eval_ctx ec = {&sl, &p, &d, R, NULL, NULL, eloc_trace + (size_t)k * W, NULL, NULL};
            parallel_for(W, nthreads, eval_worker, &ec);
        }
    }
    free_dets(&d);
    free_basis(&p);
    return 0;
}

/* ------------------------------------------------------------------ */
/* DMC                                                                 */
/* ------------------------------------------------------------------ */

int oracle_dmc(const oracle_system* s, int* Wio, int cap, double* R, int n_steps, double tau,
               double e_trial0, uint64_t seed, uint32_t step0, int n_equil, int forces_every,
               double* e_step, int* pop, double* e_trial, double* facc, int nthreads, int fixed_pop) {
    const int N = s->n_up + s->n_dn, nn = s->n_nuc;
    const int W0 = *Wio;
    /* the force sums use the forward-mode derivatives, which do not cover
     * the three-body term */
    if (forces_every > 0 && s->n3 > 0) return -9;
    int W = W0;
    basis_prep p;
    det_list d;
    prep_basis(s, &p);
    build_dets(s, &d);
    const double eps = 0.2 * sqrt((double)N / tau);
    const double g_fb = 10.0;
    double ET = e_trial0;
    double* Eold = (double*)malloc(sizeof(double) * cap);
    double* Enew = (double*)malloc(sizeof(double) * cap);
    double* wgt = (double*)malloc(sizeof(double) * cap);
    double* Rn = (double*)malloc(sizeof(double) * (size_t)cap * 3 * N);
    double* En2 = (double*)malloc(sizeof(double) * cap);
    double* hist = (double*)malloc(sizeof(double) * (n_steps > 0 ? n_steps : 1));
    double* dEL = NULL;
    double* dlg = NULL;
    if (forces_every > 0) {
        dEL = (double*)malloc(sizeof(double) * (size_t)cap * 3 * nn);
        dlg = (double*)malloc(sizeof(double) * (size_t)cap * 3 * nn);
        if (facc) memset(facc, 0, sizeof(double) * (2 + 9 * nn));
    }
    int status = 0;
    /* pseudopotential rotations: counter step0 before the first sweep,
     * t + 1 after the sweep with counter t */
    oracle_system sl = *s;
    sl.pp_seed = seed;
    sl.pp_sweep = step0;
    sl.pp_slot0 = 0;
    {
        eval_ctx ec = {&sl, &p, &d, R, NULL, NULL, Eold, NULL, NULL};
        parallel_for(W, nthreads, eval_worker, &ec);
    }
    for (int k = 0; k < n_steps; ++k) {
        const uint32_t sweep = step0 + (uint32_t)k;
        sweep_ctx sc = {s, &p, &d, R, tau, seed, sweep, NULL};
        parallel_for(W, nthreads, sweep_worker, &sc);
        sl.pp_sweep = sweep + 1u;
        eval_ctx ec = {&sl, &p, &d, R, NULL, NULL, Enew, NULL, NULL};
        parallel_for(W, nthreads, eval_worker, &ec);
        const int do_f = forces_every > 0 && k >= n_equil && (k % forces_every) == 0;
        if (do_f) {
            force_ctx fc = {&sl, &p, &d, R, dEL, dlg};   /* the rotations of this step's E_L */
            parallel_for(W, nthreads, force_worker, &fc);
        }
        double sw = 0.0, swe = 0.0, swc = 0.0;
        for (int w = 0; w < W; ++w) {
            double eo = Eold[w], en = Enew[w];
            if (eo < ET - eps) eo = ET - eps;
            if (eo > ET + eps) eo = ET + eps;
            if (en < ET - eps) en = ET - eps;
            if (en > ET + eps) en = ET + eps;
            wgt[w] = exp(-tau * (0.5 * (eo + en) - ET));
            sw += wgt[w];
            swe += wgt[w] * Enew[w];
            swc += wgt[w] * en;
        }
        const double Ek = swe / sw;
        if (e_step) e_step[k] = Ek;
        /* the trial energy follows the clipped energies that set the weights */
        hist[k] = swc / sw;
        if (do_f && facc) {
            facc[0] += sw;
            facc[1] += swe;
            for (int w = 0; w < W; ++w)
                for (int q = 0; q < 3 * nn; ++q) {
                    facc[2 + q] += wgt[w] * dEL[(size_t)w * 3 * nn + q];
                    facc[2 + 3 * nn + q] += wgt[w] * Enew[w] * dlg[(size_t)w * 3 * nn + q];
                    facc[2 + 6 * nn + q] += wgt[w] * dlg[(size_t)w * 3 * nn + q];
                }
        }
        /* branching: floor(w + u) copies, at most 3, weights reset to 1; or,
         * fixed population, systematic resampling of W0 walkers: a comb of W0
         * teeth with spacing sum(w) / W0 and one offset u; walker w gets the
         * teeth inside its interval [C_w, C_w + w_w) of the cumulative weights */
        int Wn = 0;
        const double du = sw / (double)W0;
        const double uc = draw_uniform(seed, sweep, 0xFFFFFFFFu, 0xFFFFFFFFu, 2u);
        double cum = 0.0;
        for (int w = 0; w < W; ++w) {
            int m;
            if (fixed_pop) {
                const double lo = ceil(cum / du - uc);
                cum += wgt[w];
                m = (int)(ceil(cum / du - uc) - lo);
            } else {
                const double u = draw_uniform(seed, sweep, 0xFFFFFFFFu, (uint32_t)w, 2u);
                m = (int)floor(wgt[w] + u);
                if (m > 3) m = 3;
            }
            for (int t = 0; t < m; ++t) {
                if (Wn >= cap) {
                    status = -5;
                    break;
                }
                memcpy(Rn + (size_t)Wn * 3 * N, R + (size_t)w * 3 * N, sizeof(double) * 3 * N);
                En2[Wn] = Enew[w];
                ++Wn;
            }
            if (status) break;
        }
        if (status || Wn == 0) {
            status = -5;
            break;
        }
        memcpy(R, Rn, sizeof(double) * (size_t)Wn * 3 * N);
        memcpy(Eold, En2, sizeof(double) * Wn);
        W = Wn;
        if (pop) pop[k] = W;
        /* trial energy: mean of the last (up to) 20 clipped step energies,
         * with population feedback of strength 1 / (g tau) */
        const int k0 = k + 1 > 20 ? k + 1 - 20 : 0;
        double est = 0.0;
        for (int q = k0; q <= k; ++q) est += hist[q];
        est /= (double)(k + 1 - k0);
        ET = fixed_pop ? est : est - log((double)W / (double)W0) / (g_fb * tau);
        if (e_trial) e_trial[k] = ET;
    }
    *Wio = W;
    free(Eold); free(Enew); free(wgt); free(Rn); free(En2); free(hist);
    free(dEL); free(dlg);
    free_dets(&d);
    free_basis(&p);
    return status;
}
