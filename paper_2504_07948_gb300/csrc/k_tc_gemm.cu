// Batched FP32 GEMM on the 5th-generation tensor cores (tcgen05), used for
// the dense products of the adjoint force pass in the mixed form
// (PT = AT B^T, Q = PT AT, M = C AT^T, Y = C Q^T; Eqs. 3-4 pulled back to
// basis space).
//
//   D_b[m][n] = sum_k A_b[m][k] B_b[n][k]     (B_b[k][n] when b_trans)
//
// FP32 accuracy from TF32 units: every operand is split into x_hi =
// round_tf32(x) and x_lo = x - x_hi, and the product is accumulated in FP32
// as A_lo B_hi + A_hi B_lo + A_hi B_hi (the "3xTF32" split; the dropped
// A_lo B_lo term is below FP32 rounding).
//
// One CTA (8 warps) owns a 128-row tile of one batch entry and all N <= 256
// columns: the accumulator is a 128 x N FP32 block in tensor memory.  K is
// consumed in stages of 32: the CTA stages the hi/lo tiles of A and B in
// shared memory in the no-swizzle K-major layout of tcgen05 (core matrices of
// 8 rows x 16 bytes), one thread issues 4 K-steps x 3 MMAs of shape
// 128 x N x 8 and commits them to an mbarrier, and the CTA waits for the
// barrier before overwriting the stage.  Every wait is bounded: on timeout
// the kernel raises kErrTimeout, waits (bounded) for its MMAs once more,
// frees its tensor memory and returns.
#include "qmc_internal.cuh"

namespace qmc {

namespace {

constexpr int kTcM = 128;     // rows per CTA = UMMA M
constexpr int kTcK = 32;      // K per shared-memory stage
constexpr int kTcMaxN = 256;  // UMMA N limit
constexpr unsigned kTcSpin = 1u << 24;   // mbarrier polls before giving up

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Offset (in floats) of element (r, k) of a [rows][kTcK] tile in the
// no-swizzle K-major layout: core matrix (r / 8, k / 4) holds 8 rows of 4
// consecutive k (16 bytes each, 128 bytes per core matrix); core matrices
// adjacent in K are 128 bytes apart (leading byte offset), adjacent 8-row
// groups kTcK / 4 * 128 = 1024 bytes apart (stride byte offset).
__device__ __forceinline__ int tile_off(int r, int k) {
    return ((r >> 3) * (kTcK / 4) + (k >> 2)) * 32 + (r & 7) * 4 + (k & 3);
}
constexpr uint32_t kLBO = 128;
constexpr uint32_t kSBO = (kTcK / 4) * 128;

// Shared-memory matrix descriptor of tcgen05 (no swizzle): start address,
// leading and stride byte offsets (all >> 4) and the descriptor version 1.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((kLBO >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((kSBO >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Instruction descriptor of kind::tf32: FP32 accumulator, TF32 A and B, both
// K-major, shape M x N.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ float tf32_hi(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accum) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}"
        :
        : "r"(tmem), "l"(a), "l"(b), "r"(idesc), "r"(accum));
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t phase) {
    for (unsigned it = 0; it < kTcSpin; ++it) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(bar), "r"(phase)
            : "memory");
        if (ok) return true;
    }
    return false;
}

// Stages rows [r0, r0 + nrows) x k [k0, k0 + kTcK) of a row-major operand
// (element (r, k) at X[r * ld + k], or X[k * ld + r] when trans) as hi / lo
// tiles; zero outside [0, R) x [0, K).  Each thread issues kVec loads before
// it converts and stores any of them, so a stage's loads overlap.  The
// thread-to-element maps make every shared-memory store conflict-free: a
// store's bank is fixed by (r mod 8, k mod 4) within a core matrix.
//  - plain (vec): 16-byte loads of 4 consecutive k; lane pairs read the 32
//    contiguous bytes of one row (full sectors), 16 rows per warp, and a
//    warp's stores fall into the four wavefronts 512 bytes need;
//  - trans or unaligned: scalar loads, lane -> (r mod 8, k mod 4), so a warp
//    covers all 32 banks and reads 8 consecutive r (32 bytes) per k.
constexpr int kVec = 8;
__device__ __forceinline__ void split_store(float x, float* hi, float* lo, int o) {
    const float h = tf32_hi(x);
    hi[o] = h;
    lo[o] = x - h;
}
__device__ __forceinline__ void stage(const float* X, int ld, int trans, int R, int K, int r0, int nrows, int k0,
                                      float* hi, float* lo, bool vec) {
    if (vec && !trans) {
        const int nv = nrows * (kTcK / 4);      // float4 per tile
        for (int v0 = threadIdx.x; v0 < nv; v0 += kVec * blockDim.x) {
            float4 x[kVec];
#pragma unroll
            for (int u = 0; u < kVec; ++u) {
                const int v = v0 + u * blockDim.x;
                x[u] = make_float4(0.f, 0.f, 0.f, 0.f);
                const int rest = v >> 1, r = rest % nrows, k = 8 * (rest / nrows) + 4 * (v & 1);
                const int gr = r0 + r, gk = k0 + k;
                if (v < nv && gr < R && gk < K) x[u] = *reinterpret_cast<const float4*>(X + (size_t)gr * ld + gk);
            }
#pragma unroll
            for (int u = 0; u < kVec; ++u) {
                const int v = v0 + u * blockDim.x;
                if (v >= nv) continue;
                const int rest = v >> 1;
                const int o = tile_off(rest % nrows, 8 * (rest / nrows) + 4 * (v & 1));
                float4 h, l;
                h.x = tf32_hi(x[u].x);
                h.y = tf32_hi(x[u].y);
                h.z = tf32_hi(x[u].z);
                h.w = tf32_hi(x[u].w);
                l.x = x[u].x - h.x;
                l.y = x[u].y - h.y;
                l.z = x[u].z - h.z;
                l.w = x[u].w - h.w;
                *reinterpret_cast<float4*>(hi + o) = h;
                *reinterpret_cast<float4*>(lo + o) = l;
            }
        }
        return;
    }
    const int ne = nrows * kTcK, rb = nrows / 8;   // nrows is a multiple of 8
    for (int e0 = threadIdx.x; e0 < ne; e0 += kVec * blockDim.x) {
        float x[kVec];
#pragma unroll
        for (int u = 0; u < kVec; ++u) {
            const int e = e0 + u * blockDim.x;
            const int rest = e >> 5;
            const int r = 8 * (rest % rb) + (e & 7), k = 4 * (rest / rb) + ((e >> 3) & 3);
            const int gr = r0 + r, gk = k0 + k;
            x[u] = 0.f;
            if (e < ne && gr < R && gk < K) x[u] = trans ? X[(size_t)gk * ld + gr] : X[(size_t)gr * ld + gk];
        }
#pragma unroll
        for (int u = 0; u < kVec; ++u) {
            const int e = e0 + u * blockDim.x;
            if (e >= ne) continue;
            const int rest = e >> 5;
            split_store(x[u], hi, lo, tile_off(8 * (rest % rb) + (e & 7), 4 * (rest / rb) + ((e >> 3) & 3)));
        }
    }
}

__global__ void __launch_bounds__(256) k_tc_gemm(int M, int N, int K, const float* __restrict__ A, long long sA,
                                                 int lda, const float* __restrict__ B, long long sB, int ldb,
                                                 int b_trans, float* __restrict__ D, long long sD, int ldd,
                                                 unsigned* err) {
    extern __shared__ __align__(128) float sm[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t s_tmem;
    const int Np = (N + 15) & ~15;              // UMMA N: multiple of 16
    uint32_t ncol = 32;
    while ((int)ncol < Np) ncol <<= 1;          // tensor-memory columns (power of two)
    float* Ahi = sm;
    float* Alo = Ahi + kTcM * kTcK;
    float* Bhi = Alo + kTcM * kTcK;
    float* Blo = Bhi + Np * kTcK;
    const int b = blockIdx.y, m0 = blockIdx.x * kTcM;
    const float* Ab = A + (size_t)b * sA;
    const float* Bb = B + (size_t)b * sB;
    float* Db = D + (size_t)b * sD;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                     "r"(ncol));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar)));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = s_tmem;
    const uint32_t idesc = idesc_tf32(kTcM, Np);
    uint32_t phase = 0;
    bool ok = true;
    const int n_stage = (K + kTcK - 1) / kTcK;
    const bool va = (K % 4 == 0) && (lda % 4 == 0) && ((uintptr_t)Ab % 16 == 0);
    const bool vb = (K % 4 == 0) && (ldb % 4 == 0) && ((uintptr_t)Bb % 16 == 0);
    for (int s = 0; s < n_stage && ok; ++s) {
        stage(Ab, lda, 0, M, K, m0, kTcM, s * kTcK, Ahi, Alo, va);
        stage(Bb, ldb, b_trans, N, K, 0, Np, s * kTcK, Bhi, Blo, vb);
        // make the generic-proxy stores visible to the tensor core's reads
        asm volatile("fence.proxy.async.shared::cta;");
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;");
        if (threadIdx.x == 0) {
            const uint32_t ah = smem_u32(Ahi), al = smem_u32(Alo), bh = smem_u32(Bhi), bl = smem_u32(Blo);
#pragma unroll
            for (int kk = 0; kk < kTcK / 8; ++kk) {
                const uint32_t o = kk * 2 * kLBO;   // 8 K = two core matrices along K
                const uint32_t acc0 = (s > 0 || kk > 0) ? 1u : 0u;
                mma_tf32(tmem, smem_desc(al + o), smem_desc(bh + o), idesc, acc0);
                mma_tf32(tmem, smem_desc(ah + o), smem_desc(bl + o), idesc, 1u);
                mma_tf32(tmem, smem_desc(ah + o), smem_desc(bh + o), idesc, 1u);
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                smem_u32(&bar)));
        }
        // every thread polls; the CTA proceeds only if all saw the barrier
        ok = __syncthreads_and(mbar_wait(smem_u32(&bar), phase) ? 1 : 0) != 0;
        phase ^= 1u;
        asm volatile("tcgen05.fence::after_thread_sync;");
    }
    if (!ok) {
        if (threadIdx.x == 0) atomicOr(err, kErrTimeout);
        mbar_wait(smem_u32(&bar), phase ^ 1u);   // the MMAs still in flight, bounded
    } else if (n_stage > 0) {
        // Accumulator row m0 + 32 (warp % 4) + lane lives in TMEM lane
        // 32 (warp % 4) + lane; warps w and w + 4 take alternate 32-column
        // chunks.  A chunk goes TMEM -> registers (lane = row) -> a padded
        // 32 x 33 shared tile (the stages are free now) -> global by rows, so
        // every warp store writes 128 contiguous bytes of one row instead of
        // 32 rows' worth of 4-byte pieces.
        const int q4 = warp & 3;
        const uint32_t taddr = tmem + ((uint32_t)(q4 * 32) << 16);
        float* buf = sm + warp * (32 * 33);
        for (int c0 = (warp >> 2) * 32; c0 < Np; c0 += 64) {
            uint32_t r[32];
#pragma unroll
            for (int g = 0; g < 4; ++g) {
                if (c0 + 8 * g < Np)
                    asm volatile(
                        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                        : "=r"(r[8 * g]), "=r"(r[8 * g + 1]), "=r"(r[8 * g + 2]), "=r"(r[8 * g + 3]),
                          "=r"(r[8 * g + 4]), "=r"(r[8 * g + 5]), "=r"(r[8 * g + 6]), "=r"(r[8 * g + 7])
                        : "r"(taddr + (uint32_t)(c0 + 8 * g)));
            }
            asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
            for (int j = 0; j < 32; ++j) buf[lane * 33 + j] = __uint_as_float(r[j]);
            __syncwarp();
            const int col = c0 + lane;
            for (int rr = 0; rr < 32; ++rr) {
                const int row = m0 + q4 * 32 + rr;
                if (row < M && col < N) Db[(size_t)row * ldd + col] = buf[rr * 33 + lane];
            }
            __syncwarp();
        }
    } else if (warp < 4) {
        const int row = m0 + warp * 32 + lane;   // K = 0: D = 0
        if (row < M)
            for (int j = 0; j < N; ++j) Db[(size_t)row * ldd + j] = 0.f;
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncol));
}

}  // namespace

size_t tc_gemm_smem_bytes(int N) {
    const int Np = (N + 15) & ~15;
    const size_t stages = sizeof(float) * 2 * (size_t)(kTcM + Np) * kTcK;
    const size_t epilogue = sizeof(float) * 8 * 32 * 33;   // eight 32 x 33 transpose tiles
    return stages > epilogue ? stages : epilogue;
}

cudaError_t launch_tc_gemm(int batch, int M, int N, int K, const float* A, long long sA, int lda, const float* B,
                           long long sB, int ldb, int b_trans, float* D, long long sD, int ldd, unsigned* err,
                           cudaStream_t st) {
    if (batch <= 0 || M <= 0 || N <= 0) return cudaSuccess;
    if (N > kTcMaxN || K < 0) return cudaErrorInvalidValue;
    const size_t smem = tc_gemm_smem_bytes(N);
    cudaError_t e = cudaFuncSetAttribute(k_tc_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_tc_gemm<<<dim3((M + kTcM - 1) / kTcM, batch), 256, smem, st>>>(M, N, K, A, sA, lda, B, sB, ldb, b_trans, D, sD,
                                                                     ldd, err);
    return cudaGetLastError();
}

}  // namespace qmc
