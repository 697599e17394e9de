// Particle-by-particle drift-diffusion sweep with fixed-node Metropolis
// acceptance and Sherman-Morrison inverse updates.
//
// One CTA owns one walker for the whole sweep (all N electron moves), so the
// walker's inverse Slater matrices and orbital gradient/Laplacian cache stay
// in shared memory between moves when they fit; HBM is touched once per
// sweep for them.  Per move the CTA evaluates the basis at the proposed
// position (thread per shell), contracts it with the occupied-orbital
// coefficients, forms the determinant ratio rho = sum_j phi_j(r') A^-1_{je}
// (the column of A^-1 is one contiguous row of the transposed inverse), the
// Jastrow ratio and the new drift, decides acceptance (in double in the FP64
// form, in float in the mixed form) and, when accepted, applies
//   A^-1 <- A^-1 - (A^-1 e_e)(phi'^T A^-1 - e_e^T) / rho
// row by row (one warp per row of the transposed inverse).
#include "sweep_sm.cuh"

namespace qmc {

// kNt threads per CTA: 128 for spins of up to 64 electrons, else 256.  The
// mixed form's 128-thread kernel is held to 72 registers (7 resident CTAs
// per SM); the FP64 form, bound by its FP64 pipe, keeps its registers.
template <typename T, int kNt, bool kJ3 = false>
__global__ void __launch_bounds__(kNt, sizeof(T) == 4 ? (kNt == 128 ? 7 : 3) : (kNt == 128 ? 5 : 2))
    k_sweep(DevSys s, DevWalkers wk, int W, SweepParams p, const int* n_live) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int w = blockIdx.x;
    const int Wl = n_live ? *n_live : W;
    if (w >= Wl) return;
    sweep_walker<T, (kNt > 128), kJ3>(s, wk, w, p, smem);   // 128 threads: n <= 64 only
}

// The sweep of a trial function with the three-body Jastrow (kJ3).
template <typename T, int kNt>
static cudaError_t launch_sweep_j3(const DevSys& s, const DevWalkers& wk, int W, const SweepParams& p,
                                  const int* n_live, size_t smem, cudaStream_t st) {
    cudaError_t e = cudaFuncSetAttribute(k_sweep<T, kNt, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_sweep<T, kNt, true><<<W, kNt, smem, st>>>(s, wk, W, p, n_live);
    return cudaGetLastError();
}

template <typename T>
size_t sweep_smem_bytes(const DevSys& s, int ainv_smem, int g_smem) {
    size_t a, b, c, d, e;
    return sweep_smem_layout<T>(s.N, s.n_basis, s.n_up, s.n_dn, ainv_smem, g_smem, &a, &b, &c, &d, &e);
}

template <typename T>
cudaError_t launch_sweep(const DevSys& s, const DevWalkers& wk, int W, const SweepParams& p, const int* n_live,
                         cudaStream_t st) {
    if (W == 0 || s.N == 0) return cudaSuccess;
    const size_t smem = sweep_smem_bytes<T>(s, p.ainv_smem, p.g_smem);
    const int nmax = s.n_up > s.n_dn ? s.n_up : s.n_dn;
    if (s.n3 > 0)
        return nmax > 64 ? launch_sweep_j3<T, 256>(s, wk, W, p, n_live, smem, st)
                         : launch_sweep_j3<T, 128>(s, wk, W, p, n_live, smem, st);
    if (nmax > 64) {
        cudaError_t e = cudaFuncSetAttribute(k_sweep<T, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_sweep<T, 256><<<W, 256, smem, st>>>(s, wk, W, p, n_live);
    } else {
        cudaError_t e = cudaFuncSetAttribute(k_sweep<T, 128>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_sweep<T, 128><<<W, 128, smem, st>>>(s, wk, W, p, n_live);
    }
    return cudaGetLastError();
}

template size_t sweep_smem_bytes<double>(const DevSys&, int, int);
template size_t sweep_smem_bytes<float>(const DevSys&, int, int);
template cudaError_t launch_sweep<double>(const DevSys&, const DevWalkers&, int, const SweepParams&, const int*,
                                          cudaStream_t);
template cudaError_t launch_sweep<float>(const DevSys&, const DevWalkers&, int, const SweepParams&, const int*,
                                         cudaStream_t);

}  // namespace qmc
