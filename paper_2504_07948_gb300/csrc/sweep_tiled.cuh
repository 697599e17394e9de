// Scratch of the walker-tiled sweep (k_sweep_tiled.cu), owned by the handle.
// All arrays are walker-major over the W walkers of the launch.
#pragma once

#include "qmc_internal.cuh"

namespace qmc {

constexpr int kTiledMv = 16;   // per-walker move scalars (floats)
constexpr int kTiledMaxShells = 1024;   // the proposal keeps every shell's radial sums in shared memory

struct TiledState {
    int kmax;        // queue capacity = flush period in electrons (multiple of 4)
    int ldv;         // row stride of V and P: max(n_up, n_dn) rounded up to 4
    int nbp;         // row stride of B' and C^T: n_basis rounded up to 4
    float* Bh;       // [W][5][nbp]   basis at r' (value, gradient, Laplacian), TF32 hi half
    float* Bl;       // [W][5][nbp]   and TF32 lo half (x = hi + lo)
    float* Phi;      // [W][5][n]     orbitals at r' (rows of the GEMM output, n of the moving spin)
    float* Cth[2];   // [n_s][nbp]    occupied coefficients per spin, orbital-major, TF32 hi
    float* Ctl[2];   // [n_s][nbp]    and lo halves
    float* ce;       // [W][ldv]      column e of the current inverse
    float* V;        // [W][kmax][ldv] queued orbital rows phi'_m
    float* P;        // [W][kmax][ldv] flush: rows r_m of A0^-T (zero beyond the queue)
    float* Zt;       // [W][n][kmax]  flush: A0^-T V^T
    float* Xt;       // [W][n][kmax]  flush: (K^-1 (Z - E^T))^T
    float2* KinvT;   // [W][kmax][kmax] KinvT[q][m] = (K^-1)_{mq}, double-float (hi, lo)
    float2* tv;      // [W][kmax]     t = K^-1 y of the current move, double-float
    int* rows;       // [W][kmax]     spin-block index of each queued row
    int* dq;         // [W]           queue length
    unsigned* acc;   // [W]           accepted moves of this sweep
    float* mv;       // [W][kTiledMv] r' hi/lo, step, drift at r, Jastrow at r
    double* rn;      // [W][3]        r' in double
    float2* Rp;      // [W][N][3]     positions as hi/lo floats
    const int* fn_shell;   // [n_basis]  shell of each basis function
};

// Pieces of one sweep of every walker (mixed form only; k_sweep_tiled.cu):
// tiled_begin, then per electron e tiled_propose, the orbital GEMM
// (launch_tc_gemm_split on B' and C^T), tiled_accept and, every kmax
// electrons and at the end of each spin block, tiled_flush; tiled_end adds
// the accepted moves to n_acc.  The per-electron pieces take a walker group
// [w0, w0 + nw): groups share no state, so their chains of launches may run
// on different streams.
cudaError_t tiled_begin(const DevWalkers& wk, int W, int N, const TiledState& ts, cudaStream_t st);
cudaError_t tiled_propose(const DevSys& s, const DevWalkers& wk, const TiledState& ts, int w0, int nw, int e,
                          const SweepParams& p, cudaStream_t st);
cudaError_t tiled_accept(const DevSys& s, const DevWalkers& wk, const TiledState& ts, int w0, int nw, int e,
                         const SweepParams& p, cudaStream_t st);
// tiled_accept of electron e and tiled_propose of e + 1 in one launch.
cudaError_t tiled_accept_propose(const DevSys& s, const DevWalkers& wk, const TiledState& ts, int w0, int nw, int e,
                                 const SweepParams& p, cudaStream_t st);
cudaError_t tiled_flush(const DevWalkers& wk, const TiledState& ts, int w0, int nw, int spin, int n, unsigned* err,
                        cudaStream_t st);
cudaError_t tiled_end(const TiledState& ts, int W, unsigned long long* n_acc, cudaStream_t st);
// Ct[spin] from the system's FP32 coefficients.
cudaError_t launch_tiled_coeffs(const DevSys& s, const TiledState& ts, cudaStream_t st);

}  // namespace qmc
