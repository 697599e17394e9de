/*
 * CPU FP64 oracle for the walker-batched Slater-Jastrow DMC hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this code: it exists so that tests (and the CPU-baseline leg of the
 * benchmark) can check the CUDA library against a plain, slow and obviously
 * correct restatement of the method.  It shares no code, headers or tables
 * with the CUDA library.
 *
 * What it computes (all in FP64):
 *   - contracted Gaussian basis functions and their derivatives up to third
 *     order (LCAO orbitals phi_i = sum_l C_l^i Phi_l, Eq. 2);
 *   - Slater determinants by LU with partial pivoting, recomputed from
 *     scratch whenever anything moves (A_ij = phi_j(r_i), Sec. "Single
 *     Determinant QMC Forces");
 *   - the Pade Jastrow factor, ln|psi|, its electron gradients and
 *     Laplacians, and the local energy of the Slater-Jastrow (or
 *     multi-determinant) trial function of Eq. 2;
 *   - ionic derivatives of E_L and ln|psi| in forward mode, one nuclear
 *     coordinate at a time, through dlnD/dlambda = tr(A^-1 dA/dlambda)
 *     (Eq. 3) and the derivative of tr(A^-1 B) (Eq. 4);
 *   - particle-by-particle drift-diffusion VMC/DMC with fixed-node
 *     rejection and branching (Eq. 1, Reynolds et al. 1982).
 *
 * Parity status per function is recorded beside each declaration.
 */
#ifndef QMC_ORACLE_H
#define QMC_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int n_nuc;
    const double* Z;          /* [n_nuc] */
    const double* R;          /* [n_nuc][3] bohr */
    int n_up, n_dn;           /* electrons: up block first */
    int n_shell;
    const int* sh_center;     /* [n_shell] */
    const int* sh_l;          /* [n_shell] 0..2 */
    const int* sh_pure;       /* [n_shell] 1 = spherical d */
    const int* sh_nprim;      /* [n_shell] */
    const double* alpha;      /* [sum nprim] */
    const double* coef;       /* [sum nprim] raw weights */
    int n_mo, n_basis;
    const double* C;          /* [n_mo][n_basis] */
    const int* occ_up;        /* [n_up] */
    const int* occ_dn;        /* [n_dn] */
    double a_anti, a_par, b_ee;
    const double* a_en;       /* [n_nuc] */
    double b_en;
    int n_det, n_words;       /* n_det == 0: single determinant from occ_* */
    const uint64_t* det_up;   /* [n_det][n_words] */
    const uint64_t* det_dn;
    const double* ci;         /* [n_det] */
    /* three-body (electron-electron-nucleus) Jastrow: n3 terms, exponents
     * e3 [n3][3] = (m, n, o), coefficients c3 [n_nuc][n3], scale b3; n3 = 0
     * turns it off.  J3 = sum_a sum_{i<j} sum_k c3[a][k] (s_ia^m s_ja^n +
     * s_ia^n s_ja^m) s_ij^o with s(r) = r / (1 + b3 r). */
    int n3;
    const int* e3;
    const double* c3;
    double b3;
    /* semi-local pseudopotential; n_pp = 0 turns it off.  Radial terms
     * pp_beta r^(pp_n - 2) exp(-pp_alpha r^2) of nucleus pp_nuc in channel
     * pp_l: -1 is local (added to -Z/r for every electron), l >= 0 the
     * projector onto angular momentum l (<= 3) about the nucleus, applied to
     * electrons closer than pp_rcut[a] and evaluated by the quadrature rule
     * pp_quad [pp_nq][3] (unit vectors), pp_qw [pp_nq] (weights summing to
     * 1) in the locality approximation.  With pp_rotate != 0 the rule is
     * rotated per (walker slot, nucleus) by a uniform random rotation from
     * Philox with key pp_seed and counter (pp_sweep, nucleus, slot, 3),
     * walker w of a call taking slot pp_slot0 + w; the VMC and DMC drivers
     * set pp_seed and pp_sweep themselves (and use pp_slot0 = 0). */
    int n_pp;
    const int* pp_nuc;
    const int* pp_l;
    const int* pp_n;
    const double* pp_alpha;
    const double* pp_beta;
    const double* pp_rcut;    /* [n_nuc] */
    int pp_nq;
    const double* pp_quad;
    const double* pp_qw;
    int pp_rotate;
    uint64_t pp_seed;
    uint32_t pp_sweep;
    uint32_t pp_slot0;
} oracle_system;

/* Derivative slots per basis function (multi-index order of x,y,z). */
enum { OD000 = 0, OD100, OD010, OD001, OD200, OD110, OD101, OD020, OD011, OD002,
       OD300, OD210, OD201, OD120, OD111, OD102, OD030, OD021, OD012, OD003, OD_N };

int oracle_n_basis(const oracle_system* s);

/* All derivatives of total order <= 3 of every basis function at r.
 * out: [n_basis][20].  Pinned: quadrature norm, central differences. */
int oracle_basis(const oracle_system* s, const double r[3], double* out);

/* ln|det A|, sign(det A) and optionally A^-1 by LU with partial pivoting.
 * A: [n][n] row-major.  Pinned: Leibniz expansion, numpy slogdet. */
int oracle_lu_det(int n, const double* A, double* logabs, double* sign, double* Ainv);

/* Fixed-configuration evaluation for W walkers (R: [W][N][3]).
 * Outputs (any may be NULL): logpsi[W], sign[W], eloc[W], grad[W][N][3]
 * (grad of ln|psi|), lap[W][N] (Laplacian of ln|psi|).  E_L includes the
 * pseudopotential (walker w takes rotation slot w).
 * Pinned: exact hydrogenic E_L, single-Gaussian closed form, finite
 * differences, antisymmetry, cusp cancellation; the pseudopotential by the
 * closed-form projections of an off-centre Gaussian and of determinants of
 * nucleus-centred s and p orbitals. */
int oracle_evaluate(const oracle_system* s, int W, const double* R, double* logpsi, double* sign,
                    double* eloc, double* grad, double* lap, int nthreads);

/* Forward-mode ionic derivatives: dEL[W][n_nuc][3] = dE_L/dR_a,
 * dlogpsi[W][n_nuc][3] = d ln|psi| / dR_a.  Pinned: central differences in
 * the nuclear coordinates, translation identity.  With a pseudopotential
 * the local terms and the non-local energy (quadrature points following
 * their nucleus, rotations as in oracle_evaluate) are differentiated too.
 * Returns -9 for a three-body Jastrow (not derived here). */
int oracle_forces(const oracle_system* s, int W, const double* R, double* dEL, double* dlogpsi,
                  int nthreads);

/* Forward-mode electron-coordinate derivatives: gEL[W][N][3] = dE_L/dr_i,
 * glog[W][N][3] = d ln|psi| / dr_i (either may be NULL).  Pinned: central
 * differences in the electron coordinates, translation identity against
 * oracle_forces. */
int oracle_electron_grad(const oracle_system* s, int W, const double* R, double* gEL, double* glog,
                         int nthreads);

/* Space-warp weights omega_a(r) [n_nuc] and their gradients [n_nuc][3]
 * (Filippi and Umrigar 2000, F(d) = d^-4).  Pinned: partition of unity,
 * central differences. */
void oracle_warp_weights(const oracle_system* s, const double r[3], double* om, double* gom);

/* Space-warped ionic derivatives dEL_w, dlog_w [W][n_nuc][3] from the
 * unwarped ones and the electron gradients.  Pinned: central differences of
 * the warped coordinate map, zero total per configuration, zero for one
 * electron around one nucleus. */
int oracle_space_warp(const oracle_system* s, int W, const double* R, const double* dEL, const double* dlog,
                      const double* gEL, const double* glog, double* dEL_w, double* dlog_w);

/* Jastrow parameter derivatives at fixed configurations (the inputs of a
 * linear-method optimisation step): for the P = 4 + n_nuc + n_nuc n3
 * parameters in the order (a_anti, a_par, b_ee, b_en, a_en[n_nuc],
 * c3[n_nuc][n3]), dlog[W][P] = d ln|psi| / dp and deloc[W][P] = dE_L / dp.
 * With a pseudopotential the non-local energy's dependence (its ratios
 * carry the Jastrow) is included, rotations as in oracle_evaluate.
 * Pinned: central differences of oracle_evaluate in every parameter. */
int oracle_jastrow_derivs(const oracle_system* s, int W, const double* R, double* dlog, double* deloc, int nthreads);

/* The non-local pseudopotential energy alone, vnl[W], and the rotation of
 * the quadrature rule for (slot, nucleus) as a row-major 3x3 matrix (rot
 * may be NULL).  Pinned with oracle_evaluate. */
int oracle_nonlocal(const oracle_system* s, int W, const double* R, double* vnl, int nthreads);
void oracle_pp_rotation(uint64_t seed, uint32_t sweep, uint32_t nucleus, uint32_t slot, double rot[9]);

/* Philox4x32-10 (Salmon et al., SC'11).  Pinned against independent
 * checks (uniformity / moments); parity with the CUDA generator. */
void oracle_philox4x32(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* Particle-by-particle VMC: n_sweeps sweeps at time step tau over W walkers
 * (R updated in place), sweep counter starting at step0.  Outputs (may be
 * NULL): n_accept[W] accepted moves, eloc_trace[n_sweeps][W]. */
int oracle_vmc(const oracle_system* s, int W, double* R, int n_sweeps, double tau, uint64_t seed,
               uint32_t step0, long long* n_accept, double* eloc_trace, int nthreads);

/* DMC with branching.  R: capacity cap walkers, the first *W live on entry
 * and exit.  Per step outputs (may be NULL): e_step[n_steps] (weighted mean
 * E_L before branching), pop[n_steps] (population after branching),
 * e_trial[n_steps].  With forces_every > 0 also accumulates, over steps
 * k >= n_equil with k % forces_every == 0, the weighted sums
 * facc = [sum w, sum w E_L, sum w dE_L/dR (3 n_nuc), sum w E_L dlnpsi/dR
 * (3 n_nuc), sum w dlnpsi/dR (3 n_nuc)].  fixed_pop != 0: the population
 * stays at the entry size W0 by systematic resampling with the branching
 * weights (comb offset from the branching stream, walker field 0xFFFFFFFF)
 * and the trial energy is the clipped-energy mean alone.  Returns 0 or a
 * negative error (-5 population collapse/overflow, -9 forces requested with
 * a three-body Jastrow or a pseudopotential). */
int oracle_dmc(const oracle_system* s, int* W, int cap, double* R, int n_steps, double tau,
               double e_trial0, uint64_t seed, uint32_t step0, int n_equil, int forces_every,
               double* e_step, int* pop, double* e_trial, double* facc, int nthreads, int fixed_pop);

#ifdef __cplusplus
}
#endif
#endif
