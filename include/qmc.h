/*
 * libqmc -- walker-batched Slater-Jastrow diffusion Monte Carlo on one GPU.
 *
 * C ABI of the CUDA library.  The calls follow the statement of the problem
 * in arXiv 2504.07948, Sec. "Quantum Monte Carlo": a molecule (nuclei), a
 * trial wavefunction of the Slater-Jastrow form of Eq. 2,
 *     Psi_T(R) = exp[sum_i J_i(R)] sum_k C_k D_k^up(phi) D_k^dn(phi),
 *     phi_i = sum_l C_l^i Phi_l      (LCAO orbitals over a GTO basis),
 * a population of walkers that is propagated by fixed-node DMC towards the
 * ground state (Eq. 1), the local energy, and the ionic forces obtained from
 * derivatives of determinants (Eqs. 3-4, Sec. "Single Determinant QMC
 * Forces").
 *
 * Conventions for every call:
 *   - Returns a qmc_status (0 = QMC_OK).  No C++ exception crosses the ABI;
 *     qmc_last_error() returns a message for the last failure on a handle.
 *   - Atomic units (bohr, hartree).  Electrons 0 .. n_up-1 are spin up,
 *     n_up .. n_up+n_dn-1 spin down; positions are [W][N][3] row-major
 *     double.
 *   - Input arrays are host pointers, copied into library-owned device
 *     memory; the caller keeps ownership and may free them on return.
 *   - Output arrays are host pointers, or device pointers when on_device is
 *     nonzero (then they must be device memory of the handle's device and
 *     are written in stream order on the handle's stream).
 *   - Every call is synchronous: work it launched has completed on return.
 *   - Any set_* call after walkers exist invalidates them (QMC_ERR_STATE on
 *     the next call that needs walkers, until set_walkers/init_walkers).
 *   - The library owns all device memory it allocates; qmc_destroy frees it.
 */
#ifndef QMC_H
#define QMC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct qmc_ctx* qmc_t;

typedef enum {
    QMC_OK = 0,
    QMC_ERR_ARG = -1,         /* invalid argument (size, pointer, range)          */
    QMC_ERR_CUDA = -2,        /* a CUDA runtime call failed                         */
    QMC_ERR_SINGULAR = -3,    /* a Slater matrix had a zero pivot                   */
    QMC_ERR_NONFINITE = -4,   /* a non-finite local energy or coordinate appeared  */
    QMC_ERR_POPULATION = -5,  /* the DMC population died out or exceeded capacity  */
    QMC_ERR_TIMEOUT = -6,     /* a bounded device wait gave up                      */
    QMC_ERR_STATE = -7,       /* call out of order (e.g. no walkers yet)            */
    QMC_ERR_OOM = -8,         /* device allocation failed                           */
    QMC_ERR_UNSUPPORTED = -9  /* size outside what the kernels support              */
} qmc_status;

enum { QMC_FP64 = 0, QMC_MIXED = 1 };                             /* precision modes */
enum { QMC_EST_VMC = 0, QMC_EST_DMC = 1, QMC_EST_MIXED = 2 };     /* estimators      */
enum { QMC_POP_BRANCH = 0, QMC_POP_FIXED = 1 };                    /* population control */

/* Create a handle on CUDA device `device`.  cuda_stream is a cudaStream_t
 * (e.g. torch.cuda.current_stream().cuda_stream) or NULL for a stream the
 * library creates and owns.  The walker-tiled sweep adds side streams of its
 * own (non-blocking, forked from and joined back into this stream within
 * each call).  Environment variables read here select between equivalent
 * kernel paths (for tests and measurements; the defaults are the fast ones):
 *   QMC_SWEEP_TILED=0          no walker-tiled sweep (the fused delayed sweep)
 *   QMC_SWEEP_TILED_MIN_N=k    tiled sweep from k electrons per spin (96)
 *   QMC_SWEEP_TILED_GROUPS=g   walker groups of the tiled sweep, 1..4 (2)
 *   QMC_FORCE_GEMM_MIN_N=k     GEMM force path from k electrons per spin (65)
 *   QMC_FORCE_GEMM_CUBLAS=1    the mixed GEMM force path's products on cuBLAS
 *   QMC_NLPP_TC=0              u_k of the non-local pass formed in the kernel
 *   QMC_NLPP_TC_MIN_N=k        u_k on the tensor cores from k electrons per spin (64) */
int qmc_create(qmc_t* h, int device, void* cuda_stream);
int qmc_destroy(qmc_t h);
/* Message of the last failure on h (or of the last failed qmc_create when h
 * is NULL).  The pointer stays valid until the next call on h. */
const char* qmc_last_error(qmc_t h);

/* Nuclei and electron counts.  Z: [n_nuc] charges; R: [n_nuc][3] bohr.
 * The nuclear repulsion sum_{a<b} Z_a Z_b / R_ab is part of E_L. */
int qmc_set_system(qmc_t h, int n_nuc, const double* Z, const double* R, int n_up, int n_dn);

/* Move the nuclei (and with them their basis functions) to R [n_nuc][3]
 * without touching the walkers; when walkers exist they are re-evaluated
 * from scratch at the new geometry. */
int qmc_set_nuclei(qmc_t h, const double* R);

/* Contracted Gaussian basis (Sec. "QMC Energy and Wavefunction
 * Evaluation": radial part times angular part per centre).  Per shell:
 * center (nucleus index), l in {0,1,2}, pure (1 = five real solid-harmonic
 * d functions, 0 = six Cartesian d functions), nprim primitives whose
 * exponents alpha and raw weights coef are concatenated in shell order.
 * Function order: s; p = x, y, z; pure d = sqrt3 xy, sqrt3 yz,
 * z^2-(x^2+y^2)/2, sqrt3 xz, sqrt3/2 (x^2-y^2); Cartesian d = xx, xy, xz,
 * yy, yz, zz (xy-type scaled by sqrt3).  Each primitive is normalised with
 * (2a/pi)^(3/4) (4a)^(l/2) / sqrt((2l-1)!!) and the contraction is rescaled
 * to unit norm; shells with a zero exponent keep their raw weights. */
int qmc_set_basis(qmc_t h, int n_shell, const int* center, const int* l, const int* pure, const int* nprim,
                  const double* alpha, const double* coef);

/* LCAO coefficients (Eq. 2): C is [n_mo][n_basis] row-major, orbital j =
 * sum_l C[j][l] Phi_l.  occ_up[n_up], occ_dn[n_dn] select the orbitals of
 * the single (reference) determinant, column order as given. */
int qmc_set_mos(qmc_t h, int n_mo, int n_basis, const double* C, const int* occ_up, const int* occ_dn);

/* Multi-determinant expansion (Eq. 2: sum_k C_k D_k^up D_k^dn), evaluated by
 * the table method of Sec. "Multideterminant QMC Forces".  det_up/det_dn:
 * [n_det][n_words] occupation bit strings (bit b of word b/64 = orbital b),
 * ci[n_det] the coefficients; each determinant's columns are its orbitals in
 * ascending order.  Determinant 0 is the reference: its strings replace the
 * occupation lists of qmc_set_mos.  Every other string must differ from the
 * reference by at most 4 replaced orbitals; at most 64 distinct replacing
 * (virtual) orbitals per spin (QMC_ERR_UNSUPPORTED otherwise).  n_det = 0
 * returns to the single determinant. */
int qmc_set_multidet(qmc_t h, int n_det, int n_words, const uint64_t* det_up, const uint64_t* det_dn,
                     const double* ci);

/* Pade Jastrow J = sum_{i<j} a r_ij/(1 + b_ee r_ij) + sum_{i,a} a_en[a]
 * r_ia/(1 + b_en r_ia), a = a_anti for unlike spins, a_par for like spins. */
int qmc_set_jastrow(qmc_t h, double a_anti, double a_par, double b_ee, const double* a_en, double b_en);

/* Three-body (electron-electron-nucleus) Jastrow factor, the third kind of
 * term of the paper's Jastrow (the paragraph after Eq. 2: one-, two- and
 * three-body terms with up to 40 optimised parameters):
 *   J3 = sum_a sum_{i<j} sum_k coef[a][k] (s_ia^m s_ja^n + s_ia^n s_ja^m) s_ij^o,
 *   s(r) = r / (1 + b3 r),  (m, n, o) = exponents[3k .. 3k+2],
 * added to the Pade terms of qmc_set_jastrow.  Every exponent must be 0 or
 * 2..8, so that neither cusp condition changes (QMC_ERR_ARG otherwise);
 * coef is [n_nuc][n_terms]; n_terms = 0 removes the term.  The three-body
 * term enters qmc_evaluate, qmc_eval_cached (ln|Psi|, gradients, E_L),
 * qmc_jastrow_derivs and the Sherman-Morrison sweep of a single determinant
 * (qmc_vmc, qmc_dmc with delay rank 1: ratios and drifts); delayed updates,
 * determinant expansions, the ionic forces and batches return
 * QMC_ERR_UNSUPPORTED while it is set. */
int qmc_set_jastrow3(qmc_t h, int n_terms, const int* exponents, const double* coef, double b3);

/* Semi-local pseudopotential (the valence Hamiltonian with effective core
 * potentials of Sec. "The SPICE2(+)-ccECP dataset" and Sec. "Quantum Monte
 * Carlo"), in the Gaussian-expansion form: n_terms radial terms
 *   beta[t] r^(n[t] - 2) exp(-alpha[t] r^2)
 * of nucleus nucleus[t] in channel l[t]: -1 is local (added to the -Z/r of
 * qmc_set_system for every electron), 0..3 the projector onto angular
 * momentum l about the nucleus.  The non-local part enters E_L in the
 * locality approximation: for every electron i closer than rcut[a] to
 * nucleus a,
 *   sum_l v_l(r_ia) (2l + 1) sum_q w_q P_l(r_hat_ia . d_q) Psi(r_i -> R_a + r_ia d_q) / Psi,
 * with the quadrature rule quad [n_quad][3] (unit vectors, n_quad <= 192)
 * and weights [n_quad] (summing to 1), rotated per (walker slot, nucleus) by a uniform
 * random rotation when rotate != 0: Shoemake's quaternion from the first
 * three Philox words at counter (sweep, nucleus, slot, 3) under the
 * qmc_set_rng key, the sweep field being the handle's sweep counter when E_L
 * is evaluated (after a sweep, the counter of the next sweep).  rcut is
 * [n_nuc] (bohr; 0 turns a nucleus's non-local part off).  Arrays are host
 * memory, copied.  n_terms = 0 removes the potential.  It enters every E_L
 * (qmc_evaluate, qmc_eval_cached, qmc_vmc, qmc_dmc and their estimators)
 * and the ionic derivatives of E_L: the local terms directly, the non-local
 * energy as rows of the B matrix of Sec. "Single Determinant QMC Forces"
 * (E_L gains tr(B_NL A^-1), B_NL[k][j] = sum over electron k's quadrature
 * points of w_p phi_j(r'_p) times the Jastrow ratio) plus the derivatives
 * of the points, weights and Jastrow ratios with the quadrature points
 * following their nucleus.  Forces with it need a single determinant and
 * no space warp; determinant expansions, batches and space-warped forces
 * return QMC_ERR_UNSUPPORTED while it is set.  qmc_jastrow_derivs carries
 * it (the non-local ratios depend on the Jastrow).  QMC_ERR_ARG on a nucleus out
 * of range, l outside -1..3, n outside 0..8, a non-positive exponent, a
 * negative cutoff or a quadrature point off the unit sphere. */
int qmc_set_pseudopotential(qmc_t h, int n_terms, const int* nucleus, const int* l, const int* n,
                            const double* alpha, const double* beta, const double* rcut, int n_quad,
                            const double* quad, const double* weights, int rotate);

/* Jastrow parameter derivatives at the current walkers (recomputed from
 * scratch), the per-walker inputs of a linear-method optimisation of the
 * Jastrow: for the P = 4 + n_nuc + n_nuc n_terms parameters in the order
 * (a_anti, a_par, b_ee, b_en, a_en[n_nuc], coef[n_nuc][n_terms]),
 *   dlog[W][P]  = d ln|Psi_T| / dp = dJ / dp,
 *   deloc[W][P] = dE_L / dp = -1/2 sum_i (lap_i dJ/dp + 2 grad_i ln|Psi_T| . grad_i dJ/dp),
 * plus, with a pseudopotential, sum_p W_p rho_p (dJ/dp(R'_p) - dJ/dp(R)) over the
 * quadrature points R'_p of the non-local term (weights W_p, ratios rho_p,
 * rotations at the current sweep counter as in qmc_evaluate).
 * Host arrays, or device arrays of the handle's device when on_device. */
int qmc_jastrow_derivs(qmc_t h, double* dlog, double* deloc, int on_device);

/* Precision: QMC_FP64 (everything in double) or QMC_MIXED (basis, orbitals,
 * inverse updates in float; log-determinants, E_L, forces, weights and the
 * periodic recompute in double).  delay_rank in [1, 32]: accepted moves
 * queued before a rank-k (Woodbury) update of the inverse (1 =
 * Sherman-Morrison on every accepted move; QMC_ERR_UNSUPPORTED outside the
 * range; a single-determinant feature, ignored by determinant expansions).
 * recompute_period: sweeps between FP64 recomputes of the inverse (0 =
 * never). */
int qmc_set_precision(qmc_t h, int mode, int delay_rank, int recompute_period);

/* DMC population control (the paper gives the branching projection of Eq. 1
 * but no control scheme).  QMC_POP_BRANCH (default): each walker continues
 * as min(floor(w + u), 3) copies and the trial energy carries the feedback
 * -ln(W / W0) / (10 tau), W0 = population at qmc_set_walkers.
 * QMC_POP_FIXED: the population stays at W0; every step W0 walkers are drawn
 * by systematic resampling with the same weights (one comb offset per step
 * from the branching stream, walker field 0xFFFFFFFF) and the trial energy is
 * the clipped-energy mean alone.  Applies to qmc_dmc and to batches. */
int qmc_set_population_control(qmc_t h, int mode);

/* Counter-based random stream (Philox4x32-10): key = seed, counter =
 * (sweep, electron, walker slot, purpose).  The sweep counter advances by
 * one per VMC sweep or DMC step. */
int qmc_set_rng(qmc_t h, uint64_t seed, uint32_t sweep);

/* Walkers.  set_walkers copies R [W][N][3]; the population capacity for DMC
 * is cap_factor * W (cap_factor >= 1, default 2).  Evaluates the wavefunction
 * from scratch (FP64 inverse).  get_walkers writes R [W][N][3] and weight[W]
 * of the current population (either pointer may be NULL). */
int qmc_set_walkers(qmc_t h, int n_walkers, const double* R, int on_device);
int qmc_set_capacity_factor(qmc_t h, int cap_factor);
/* Draws n_walkers initial walkers on the device and evaluates them as
 * qmc_set_walkers does.  The paper samples walkers from |Psi_T|^2 (Sec.
 * "Quantum Monte Carlo") but states no starting distribution; this one puts
 * round(Z_a) electrons on each nucleus a (in nucleus order; an anion's extra
 * electrons on nucleus 0), gives spin up the even entries of that list and
 * spin down the odd ones (in list order if one spin runs short), and places
 * electron e of walker w at R_a + 0.5 bohr * chi, chi three standard normals
 * of the counter-based stream with key = seed and counter = (0xFFFFFFFE, e,
 * w, 3).  VMC equilibration is the caller's next step.  QMC_ERR_ARG for
 * n_walkers < 1; QMC_ERR_STATE before the system and wavefunction are set. */
int qmc_init_walkers(qmc_t h, int n_walkers, uint64_t seed);
int qmc_get_walkers(qmc_t h, double* R, double* weight, int on_device);
/* Current population size (>= 0) or a negative qmc_status. */
int qmc_n_walkers(qmc_t h);

/* Fixed-configuration evaluation at the current walkers, recomputed from
 * scratch (basis, orbitals, FP64 inverse): logpsi[W] = ln|Psi_T|,
 * sign[W], eloc[W] = local energy, grad[W][N][3] = grad_i ln|Psi_T|.  Any
 * output may be NULL. */
int qmc_evaluate(qmc_t h, double* logpsi, double* sign, double* eloc, double* grad, int on_device);

/* The same outputs from the incrementally maintained state (inverse and
 * orbital-gradient cache as the last sweep left them, in the precision of
 * the current mode), without recomputing: the values the estimators use. */
int qmc_eval_cached(qmc_t h, double* logpsi, double* sign, double* eloc, double* grad, int on_device);

/* Ionic derivatives at the current walkers by the adjoint kernel:
 * dR[a][c] = sum_w g_eloc[w] dE_L/dR_ac + g_logpsi[w] d ln|Psi_T|/dR_ac
 * (g arrays [W]; either may be NULL = zero), per_walker (optional)
 * [W][2][n_nuc][3] = (dE_L/dR, d ln|Psi_T|/dR).  E_L includes the nuclear
 * repulsion, so its derivative carries the ion-ion force. */
int qmc_force_vjp(qmc_t h, const double* g_eloc, const double* g_logpsi, double* dR, double* per_walker,
                  int on_device);

/* Space-warped ionic derivatives (Filippi and Umrigar 2000; the paper adapts
 * the space-warp transformation to its batched force path, Sec. "Single
 * Determinant QMC Forces", and names its finite-difference form the force
 * bottleneck, Sec. "Performance Measurement").  enable = 1: every later
 * per-walker force evaluation of this handle (qmc_force_vjp and the force
 * estimators of qmc_vmc / qmc_dmc) moves each electron i with nucleus a by
 * omega_a(r_i) = |r_i - R_a|^-4 / sum_b |r_i - R_b|^-4, giving
 *   dE_L/dR_a + sum_i omega_a(r_i) dE_L/dr_i and
 *   d ln|Psi_T|/dR_a + sum_i omega_a(r_i) d ln|Psi_T|/dr_i + 1/2 sum_i grad_i omega_a(r_i)
 * (the last term is half the log-Jacobian of the electron map) in place of
 * the plain derivatives.  The estimator's mean is unchanged; per-walker
 * fluctuations from electrons close to a nucleus cancel.  dE_L/dr_i comes
 * from the same adjoint pass (all basis functions moving with the electron)
 * plus the Jastrow and potential terms; two per-walker [N][3] FP64 arrays
 * are allocated on the first warped evaluation.  enable = 0 (default):
 * plain derivatives.  QMC_ERR_ARG for other values.  A batch reads each
 * member's setting when it is created (qmc_batch_create) and warps the
 * forces of those members in its persistent force launches; changing the
 * setting of a member afterwards makes the batch's next call fail with
 * QMC_ERR_STATE. */
int qmc_set_space_warp(qmc_t h, int enable);

/* Variational Monte Carlo: n_sweeps particle-by-particle sweeps with
 * drift-diffusion proposals and fixed-node Metropolis acceptance at time
 * step tau.  eloc_trace (optional) [n_sweeps][W] receives E_L after each
 * sweep; forces_every > 0 accumulates the force estimator every that many
 * sweeps.  Energies feed the QMC_EST_VMC estimator. */
int qmc_vmc(qmc_t h, int n_sweeps, double tau, int forces_every, double* eloc_trace, int on_device);

/* Diffusion Monte Carlo (Eq. 1): n_steps steps of one sweep at tau, local
 * energy, branching with weights exp(-tau[(E_old+E_new)/2 - E_T]) (E
 * clipped to E_T +- 0.2 sqrt(N/tau)), at most 3 copies per walker, and the
 * trial energy fed back from the mean of the last 20 weighted means of the
 * clipped energies, with strength 1/(10 tau) on ln(W/W0).  e_trial: initial E_T.  Steps >= n_equil
 * feed the QMC_EST_DMC estimators; forces every forces_every steps (0 =
 * off).  Per-step host outputs (each optional, [n_steps]): e_step = weighted
 * mean E_L, pop = population after branching, e_trial_out = E_T after the
 * update. */
int qmc_dmc(qmc_t h, int n_steps, double tau, double e_trial, int n_equil, int forces_every, double* e_step,
            int* pop, double* e_trial_out);

/* Trial energy of the population control of Eq. 1 as qmc_dmc updates it
 * after every step: the mean of the last (up to) 20 entries of hist (the
 * weighted means of the clipped local energies of the steps so far), minus
 * ln(pop / pop0) / (10 tau) unless fixed_pop.  Pure host arithmetic (no
 * device work): callers that drive sharded populations use it to check or
 * reproduce the update.  QMC_ERR_ARG for n_hist < 1, tau <= 0 or, without
 * fixed_pop, a non-positive population. */
int qmc_trial_energy(const double* hist, int n_hist, double pop, double pop0, double tau, int fixed_pop,
                     double* e_trial);

/* Walker sharding: one population split over several processes (one GPU
 * each), joined by one exchange per DMC step (Sec. "Quantum Monte Carlo":
 * the walkers of a step are independent; the trial energy and the
 * estimators are properties of the whole population).  When fn is set,
 * qmc_dmc calls it once per step with this rank's step sums
 *   buf = {sum w, sum w E_L, population after branching, sum w clip(E_L),
 *          sum w E_L^2, reference population, [force sums of that step:
 *          sum w, sum w E, sum w dE_L/dR (3 n_nuc), sum w E dln|Psi|/dR,
 *          sum w dln|Psi|/dR, when forces are sampled]},
 * n entries (the same n on every rank), and fn must replace buf in place by
 * the element-wise sum over all ranks (e.g. an all-reduce) and return 0.
 * Every rank then takes its step energy, its trial-energy feedback (global
 * population against the summed reference populations) and its estimator
 * samples from the global sums; branching stays local.  A nonzero return
 * fails the step with QMC_ERR_STATE.  fn = NULL (default) restores the
 * single-process behaviour.  ctx is passed through. */
typedef int (*qmc_reduce_fn)(double* buf, int n, void* ctx);
int qmc_set_step_reduce(qmc_t h, qmc_reduce_fn fn, void* ctx);
/* The reference population W0 of the trial-energy feedback (this rank's
 * share when sharded): pop0 > 0 replaces the population at qmc_set_walkers,
 * so that walkers moved between ranks do not change the summed reference;
 * 0 returns to the default. */
int qmc_set_population_reference(qmc_t h, double pop0);

/* Accumulated estimators (host outputs).  Energy: mean, Flyvbjerg-Petersen
 * blocked standard error, variance of E_L, acceptance ratio.  Forces
 * [n_nuc][3] (Ha/bohr) and their errors: the zero-variance zero-bias form
 * F = -<dE_L/dR> - 2(<E_L dln|Psi|/dR> - <E_L><dln|Psi|/dR>); QMC_EST_MIXED
 * returns 2 F_DMC - F_VMC (Sec. "Performance Measurement"). */
int qmc_get_energy(qmc_t h, int estimator, double* mean, double* stderr_blocked, double* variance,
                   double* acceptance);
int qmc_get_forces(qmc_t h, int estimator, double* F, double* F_err);
/* The zero-variance zero-bias force estimate of qmc_get_forces over the
 * current walkers alone, at their fixed configurations: per-walker ionic
 * derivatives by the adjoint kernel (space-warped when enabled), weighted
 * sums on the device, F [n_nuc][3] (Ha/bohr) =
 *   -<dE_L/dR> - 2 (<E_L dln|Psi|/dR> - <E_L><dln|Psi|/dR>),
 * <x> = sum_w weights[w] x_w / sum_w weights[w].  weights [W] (NULL = all 1)
 * and F are host arrays, or device arrays of the handle's device when
 * on_device.  QMC_ERR_ARG for a null F, negative or non-finite host weights
 * or weights summing to zero.  No estimator samples are recorded. */
int qmc_force_estimate(qmc_t h, const double* weights, double* F, int on_device);
/* Forget accumulated estimator samples. */
int qmc_reset_estimators(qmc_t h);

/* Per-kernel timing.  When enabled, every kernel the library launches is
 * bracketed by CUDA events on the stream it runs on and counted.  family is
 * one of "sweep", "sweep_gemm", "eloc", "nlpp", "force", "branch",
 * "recompute", "reduce" or "all".  The walker-tiled sweep runs its walker
 * groups on several streams: its "sweep" time is the span of the whole
 * sweep on the handle's stream, and "sweep_gemm" the device time of its
 * tensor-core orbital GEMMs, which lies inside that span ("all" adds it
 * once).  total_ms is the summed device time and launches the number of
 * kernels launched since the last reset (either output may be NULL). */
int qmc_set_timing(qmc_t h, int enable);
int qmc_get_timing(qmc_t h, const char* family, double* total_ms, long long* launches);

/* Allocation-free branching step.  The paper has no counterpart: this
 * entry point exists for callers that cannot allocate device memory (a
 * framework that owns every device buffer and passes the library only
 * pointers into its own pool), so it needs no handle and calls no
 * cudaMalloc, cudaFree or allocating library routine.  It computes the same
 * weights and copy counts as qmc_dmc's branching (weights
 * exp(-tau[(E_old+E_new)/2 - E_T]) with energies clipped to E_T +- e_cut,
 * copies = min(floor(w + u), 3), u from the branching stream of `seed` at
 * `sweep`) and writes, instead of moving walkers, the parent map:
 *   parent[j] = index of the walker whose copy occupies new slot j,
 *               for j < stats[2]  (copies of a walker are consecutive and
 *               in walker order; slots beyond are left untouched),
 *   stats[5]  = {sum w, sum w E_new, new population, overflow flag (1 when
 *               the new population exceeds capacity; then parent is not
 *               written), sum w clip(E_new)}.
 * eloc_old, eloc_new [n_walkers], parent [capacity] and stats [5] are device
 * pointers of the current device; the work is enqueued on cuda_stream
 * (NULL = legacy default stream) and the call returns without waiting.
 * Per-walker scratch lives in one fixed device array of the library, sized
 * for at most 65536 walkers (1 MiB, held by every GPU that loads the library
 * until the process exits): more walkers return QMC_ERR_UNSUPPORTED; bad
 * pointers or parameters QMC_ERR_ARG; QMC_ERR_CUDA when a CUDA error from
 * earlier work is already pending (it is left pending for its owner) or a
 * launch fails.  A call made outside stream capture looks up that array's
 * device address in the current context; a call made while cuda_stream is
 * capturing reuses the address the last uncaptured call on this device
 * found (QMC_ERR_STATE if none), so make one call before any capture.  Every
 * call reuses the same scratch (it keeps the last call's contents, and each
 * call overwrites what it reads): calls that may overlap on the GPU, on any
 * streams, race and must be serialised by the caller. */
int qmc_branch_noalloc(int n_walkers, const double* eloc_old, const double* eloc_new, double tau, double e_trial,
                       double e_cut, uint64_t seed, uint32_t sweep, int capacity, int* parent, double* stats,
                       void* cuda_stream);

/* ------------------------------------------------------------------------
 * Batches of independent systems.  The paper runs many molecules at once,
 * one walker population per molecule, and batches walkers on each GPU
 * (Sec. "Quantum Monte Carlo", batched walker evaluation); here systems of
 * different sizes and populations are stepped together on one GPU: every
 * kernel family of a DMC step is one persistent launch over the work items
 * (walkers, walker-electrons, walker-spins) of all systems, scheduled
 * dynamically, largest systems first, and the launches of one step are
 * captured in a CUDA graph and replayed.  Trial energies and populations
 * are updated on the device; estimator samples land in each system's handle
 * as if qmc_dmc had run there (qmc_get_energy / qmc_get_forces on the
 * handle).
 *
 * A batch references its member handles (it does not own them): every
 * member must have walkers, share the device and precision mode, and hold a
 * single determinant; at most 1024 members.  Changing a member's system,
 * wavefunction or precision after qmc_batch_create makes every batch call
 * return QMC_ERR_STATE (create the batch again); setting new walkers is
 * fine.  While a batch call runs, no call may use a member handle.  The
 * recompute period is the smallest positive period of the members.  On a
 * population failure the failing member's walkers are invalidated and the
 * call returns QMC_ERR_POPULATION naming it.
 * ------------------------------------------------------------------------ */
typedef struct qmc_batch* qmc_batch_t;

int qmc_batch_create(qmc_batch_t* b, int n_systems, qmc_t const* systems);
int qmc_batch_destroy(qmc_batch_t b);
const char* qmc_batch_last_error(qmc_batch_t b);

/* Launch configuration by hand: use_graph (0 = plain launches), threads per
 * CTA of the sweep (64, 128 or 256), delayed updates of rank delay_rank
 * (1 = Sherman-Morrison) for members with at least delay_min_electrons
 * electrons of one spin, and a shared-memory budget in bytes up to which a
 * Sherman-Morrison member keeps A^-1 in shared memory during its sweep. */
int qmc_batch_set_options(qmc_batch_t b, int use_graph, int sweep_block, int delay_rank, int delay_min_electrons,
                          int smem_budget);

/* Autotuner: times one batched sweep (at time step tau) per candidate
 * configuration -- sweep CTA size {128, 256} x shared-memory budgets taken
 * from the members' needs, and delayed updates of rank {8, 16, 32} for
 * members with >= 32 electrons per spin -- and keeps the fastest.  The
 * trial sweeps are Metropolis sweeps without branching (they equilibrate
 * the walkers; E_L is refreshed afterwards).  chosen (optional,
 * [4 + n_systems]): CTA size, dynamic shared memory bytes, persistent CTAs,
 * the fastest sweep in microseconds, then per member (caller order)
 * 2 * delay_rank + (1 if A^-1 stays in shared memory). */
int qmc_batch_autotune(qmc_batch_t b, double tau, int* chosen);

/* n_sweeps batched VMC sweeps (equilibration; E_L refreshed every sweep, no
 * estimator samples). */
int qmc_batch_vmc(qmc_batch_t b, int n_sweeps, double tau);

/* n_steps DMC steps of every member as in qmc_dmc, with one initial trial
 * energy per member (e_trial [n_systems], caller order).  Optional host
 * outputs [n_steps][n_systems]: e_step (weighted mean E_L) and pop
 * (population after branching). */
int qmc_batch_dmc(qmc_batch_t b, int n_steps, double tau, const double* e_trial, int n_equil, int forces_every,
                  double* e_step, int* pop);

/* Per-family timing of batch calls (as qmc_set_timing; enabling it runs the
 * steps as plain launches instead of graph replays).  Family "all" returns
 * the summed time and the number of kernels the last batch call launched. */
int qmc_batch_set_timing(qmc_batch_t b, int enable);
int qmc_batch_get_timing(qmc_batch_t b, const char* family, double* total_ms, long long* launches);

/* Batched FP32 GEMM on the tensor cores, the primitive behind the dense
 * products of the adjoint force pass of Eqs. 3-4 in the mixed form:
 *   D_b[m][n] = sum_k A_b[m][k] B_b[n][k]      (b_trans = 0)
 *   D_b[m][n] = sum_k A_b[m][k] B_b[k][n]      (b_trans = 1)
 * for b < batch, row-major operands with row strides lda, ldb, ldd (in
 * elements) and batch strides strideA/B/D (0 shares an operand).  tcgen05
 * MMAs of TF32 operands with the 3xTF32 split (x = hi + lo), FP32
 * accumulation: FP32-level accuracy.  N <= 256.  Device pointers of the
 * current device; enqueued on cuda_stream (NULL = legacy stream) and waited
 * for.  QMC_ERR_ARG on bad sizes, QMC_ERR_TIMEOUT if a bounded wait inside
 * the kernel gave up (the result is then undefined). */
int qmc_tc_gemm(int batch, int M, int N, int K, const float* A, long long strideA, int lda, const float* B,
                long long strideB, int ldb, int b_trans, float* D, long long strideD, int ldd, void* cuda_stream);

/* The same product for operands given already split into TF32 halves,
 *   D[m][n] = sum_k (A_hi + A_lo)[m][k] (B_hi + B_lo)[n][k]
 * (the A_lo B_lo term dropped), where each half is a float whose value is
 * representable in TF32 (1 sign, 8 exponent, 10 mantissa bits), e.g. hi =
 * x rounded to TF32 and lo = (x - hi) rounded to TF32.  This is the form of
 * the walker-tiled sweep's orbital contraction (Eq. 2 for all walkers as
 * one GEMM), whose producer writes the halves directly: TMA moves the tiles
 * straight into the tensor core's 128-byte swizzled layout with no
 * conversion pass.  Row-major [M][K] and [N][K] with row strides lda, ldb
 * (multiples of 4) and 16-byte aligned bases, D [M][ldd]; 1 <= K, N <= 256.
 * Device pointers of the current device; enqueued on cuda_stream and waited
 * for.  QMC_ERR_ARG on bad sizes, QMC_ERR_UNSUPPORTED when the alignment
 * rules do not hold, QMC_ERR_TIMEOUT if a bounded wait inside the kernel
 * gave up. */
int qmc_tc_gemm_split(int M, int N, int K, const float* A_hi, const float* A_lo, int lda, const float* B_hi,
                      const float* B_lo, int ldb, float* D, int ldd, void* cuda_stream);

/* Walker population, RNG position and trial energy to a versioned binary
 * file, and back (the wavefunction itself is not stored). */
int qmc_checkpoint(qmc_t h, const char* path);
int qmc_restore(qmc_t h, const char* path);

#ifdef __cplusplus
}
#endif
#endif
