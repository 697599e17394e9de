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
#include <cuda.h>

#include <mutex>

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

static cudaError_t launch_tc_gemm_staged(int batch, int M, int N, int K, const float* A, long long sA, int lda,
                                         const float* B, long long sB, int ldb, int b_trans, float* D, long long sD,
                                         int ldd, unsigned* err, cudaStream_t st) {
    if (batch <= 0 || M <= 0 || N <= 0) return cudaSuccess;
    if (N > kTcMaxN || K < 0) return cudaErrorInvalidValue;
    const size_t smem = tc_gemm_smem_bytes(N);
    cudaError_t e = cudaFuncSetAttribute(k_tc_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_tc_gemm<<<dim3((M + kTcM - 1) / kTcM, batch), 256, smem, st>>>(M, N, K, A, sA, lda, B, sB, ldb, b_trans, D, sD,
                                                                     ldd, err);
    return cudaGetLastError();
}


namespace {

// ---------------------------------------------------------------------
// Pipelined persistent form: TMA loads, warp-specialised staging, tcgen05
// MMAs, double-buffered accumulators.
//
// The staged kernel above serialises load -> split -> MMA -> wait for
// every K stage and launches one CTA per output tile, so the tensor pipe
// idles while a CTA loads and every tile pays the CTA's set-up.  Here
// grid-stride CTAs (as many as fit on the GPU) walk the tiles (batch entry,
// 128-row block) and the roles run concurrently on rings that continue
// from one tile to the next:
//   warp 0    one thread issues cp.async.bulk.tensor loads of raw FP32 tiles
//             (A: 128 rows x 16 k; B: N rows x 16 k, or 16 k x N when B is
//             given [K][N]) into kRaw raw buffers, completion counted on an
//             mbarrier by bytes;
//   warps 4-7 split each raw tile into TF32 hi / lo tiles (lo rounded to
//             nearest) in the no-swizzle K-major core-matrix layout of
//             tcgen05 (kConv buffers), release the raw buffer and mark the
//             converted one full;
//   warp 1    one thread issues the 2 K-steps x 3 MMAs (lo*hi, hi*lo, hi*hi)
//             of a converted stage into the tile's accumulator (two 128 x N
//             FP32 blocks of tensor memory, alternating by tile) and
//             commits them to the stage's "empty" barrier; after a tile's
//             last stage a commit marks that accumulator full;
//   warps 8-11 drain a full accumulator (tcgen05.ld, TMEM lane = row),
//             release it for the tile after next, apply D = alpha A B^T +
//             beta D and write rows through a padded shared-memory
//             transpose (every warp store covers 128 contiguous bytes),
//             while the other roles already work on the next tile.
// Every mbarrier wait is bounded.  A role that gives up sets kErrTimeout
// and a shared abort flag that makes the other roles skip their remaining
// waits; before the CTA frees its tensor memory the MMA thread waits
// (bounded) for the MMAs it issued and the load thread for its loads.
// ---------------------------------------------------------------------
constexpr int kPK = 16;       // K per stage
constexpr int kRaw = 3;       // raw (TMA) buffers
constexpr int kConv = 2;      // converted (hi / lo) buffers
constexpr unsigned kPSpin = 1u << 22;

__device__ __forceinline__ int ptile_off(int r, int k) {   // [rows][kPK] core-matrix layout, floats
    return ((r >> 3) * (kPK / 4) + (k >> 2)) * 32 + (r & 7) * 4 + (k & 3);
}
constexpr uint32_t kPLBO = 128;                // K-adjacent core matrices
constexpr uint32_t kPSBO = (kPK / 4) * 128;    // 8-row groups

__device__ __forceinline__ uint64_t psmem_desc(uint32_t saddr) {
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((kPLBO >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((kPSBO >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
// Bounded wait for the completion of phase `parity`; false once the abort
// flag is set or after kPSpin polls (then the flag and kErrTimeout are set).
__device__ __forceinline__ bool pwait(uint32_t bar, uint32_t parity, volatile int* abort_flag, unsigned* err) {
    for (unsigned it = 0; it < kPSpin; ++it) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
        if (ok) return true;
        if ((it & 255) == 255 && *abort_flag) return false;
    }
    *abort_flag = 1;
    atomicOr(err, kErrTimeout);
    return false;
}
// The same wait without the abort flag (the final drains).
__device__ __forceinline__ void pdrain(uint32_t bar, uint32_t parity) {
    for (unsigned it = 0; it < kPSpin; ++it) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
        if (ok) return;
    }
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int x, int y, int z, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
            dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(bar)
        : "memory");
}

__device__ __forceinline__ float4 split_hi4(float4 x) {
    return make_float4(tf32_hi(x.x), tf32_hi(x.y), tf32_hi(x.z), tf32_hi(x.w));
}
// lo = round_tf32(x - hi): the tensor core reads only the TF32 bits of an
// operand, so the remainder is rounded to nearest here instead of being cut
// short (a one-sided error that would add up along K).
__device__ __forceinline__ float4 split_lo4(float4 x, float4 h) {
    return make_float4(tf32_hi(x.x - h.x), tf32_hi(x.y - h.y), tf32_hi(x.z - h.z), tf32_hi(x.w - h.w));
}

struct PipeSmem {   // byte offsets of the dynamic shared memory
    uint32_t rawA, rawB, convA, convB, epi, raw_bytes, conv_bytes, total;
};
__host__ __device__ inline PipeSmem pipe_layout(int Np) {
    PipeSmem L;
    const uint32_t ra = kTcM * kPK * 4, rb = (uint32_t)Np * kPK * 4;
    L.raw_bytes = ra + rb;
    L.conv_bytes = 2 * (ra + rb);
    L.rawA = 0;
    L.rawB = ra;
    L.convA = kRaw * L.raw_bytes;
    L.convB = L.convA + 2 * ra;
    L.epi = kRaw * L.raw_bytes + kConv * L.conv_bytes;
    L.total = L.epi + 4 * 32 * 33 * 4;
    return L;
}

// D_b = alpha A_b B_b^T + beta D_b: A through tmA (dims K, M, batch), B
// through tmB (dims K, N, batch; or N, K, batch when b_trans).
__global__ void __launch_bounds__(384, 1)
    k_tc_gemm_pipe(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, int M, int N, int K,
                   int batch, int b_trans, int a_batched, int b_batched, float alpha, float beta,
                   float* __restrict__ D, long long sD, int ldd, unsigned* err) {
    extern __shared__ __align__(1024) unsigned char psm[];
    __shared__ __align__(8) uint64_t bar_raw_full[kRaw], bar_raw_empty[kRaw], bar_conv_full[kConv],
        bar_conv_empty[kConv], bar_acc_full[2], bar_acc_empty[2], bar_drain;
    __shared__ uint32_t s_tmem;
    __shared__ int s_abort;
    const int Np = (N + 15) & ~15;
    uint32_t ncol = 32;
    while ((int)ncol < Np) ncol <<= 1;
    const PipeSmem L = pipe_layout(Np);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n_stage = (K + kPK - 1) / kPK;
    const int mt = (M + kTcM - 1) / kTcM, n_tiles = mt * batch;
    // tiles of this CTA: blockIdx.x, + gridDim.x, ...
    const int my_tiles = blockIdx.x < n_tiles ? (n_tiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    const uint32_t sbase = smem_u32(psm);
    volatile int* abort_flag = &s_abort;

    if (threadIdx.x == 0) {
        for (int i = 0; i < kRaw; ++i) {
            mbar_init(smem_u32(&bar_raw_full[i]), 1);
            mbar_init(smem_u32(&bar_raw_empty[i]), 4);
        }
        for (int i = 0; i < kConv; ++i) {
            mbar_init(smem_u32(&bar_conv_full[i]), 4);
            mbar_init(smem_u32(&bar_conv_empty[i]), 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(smem_u32(&bar_acc_full[i]), 1);
            mbar_init(smem_u32(&bar_acc_empty[i]), 4);
        }
        mbar_init(smem_u32(&bar_drain), 1);
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmA)) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmB)) : "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                     "r"(2 * ncol));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = s_tmem;

    if (warp == 0) {
        // ---- loads ------------------------------------------------------
        if (lane == 0) {
            int g = 0;   // global stage counter of this CTA
            bool ok = true;
            for (int i = 0; i < my_tiles && ok; ++i) {
                const int tile = (int)blockIdx.x + i * (int)gridDim.x;
                const int b = tile / mt, m0 = (tile - b * mt) * kTcM;
                for (int s = 0; s < n_stage; ++s, ++g) {
                    const int slot = g % kRaw;
                    if (g >= kRaw && !pwait(smem_u32(&bar_raw_empty[slot]), ((g / kRaw) - 1) & 1, abort_flag, err)) {
                        ok = false;
                        break;
                    }
                    const uint32_t full = smem_u32(&bar_raw_full[slot]);
                    mbar_expect_tx(full, L.raw_bytes);
                    const uint32_t dst = sbase + slot * L.raw_bytes;
                    const int k0 = s * kPK;
                    tma_load_3d(dst + L.rawA, &tmA, k0, m0, a_batched ? b : 0, full);
                    if (b_trans)
                        tma_load_3d(dst + L.rawB, &tmB, 0, k0, b_batched ? b : 0, full);
                    else
                        tma_load_3d(dst + L.rawB, &tmB, k0, 0, b_batched ? b : 0, full);
                }
            }
            // every load this thread issued has landed before the CTA exits
            for (int q = (g > kRaw ? g - kRaw : 0); q < g; ++q) pdrain(smem_u32(&bar_raw_full[q % kRaw]), (q / kRaw) & 1);
        }
    } else if (warp == 1) {
        // ---- MMAs -------------------------------------------------------
        if (lane == 0) {
            const uint32_t idesc = idesc_tf32(kTcM, Np);
            int g = 0;
            bool ok = true;
            for (int i = 0; i < my_tiles && ok; ++i) {
                const int a = i & 1;
                if (i >= 2 && !pwait(smem_u32(&bar_acc_empty[a]), ((i >> 1) - 1) & 1, abort_flag, err)) break;
                asm volatile("tcgen05.fence::after_thread_sync;");
                const uint32_t acc = tmem + (uint32_t)(a * ncol);
                for (int s = 0; s < n_stage; ++s, ++g) {
                    const int slot = g % kConv;
                    if (!pwait(smem_u32(&bar_conv_full[slot]), (g / kConv) & 1, abort_flag, err)) {
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;");
                    const uint32_t ca = sbase + L.convA + slot * L.conv_bytes;
                    const uint32_t ah = ca, al = ca + kTcM * kPK * 4;
                    const uint32_t cb = sbase + L.convB + slot * L.conv_bytes;
                    const uint32_t bh = cb, bl = cb + (uint32_t)Np * kPK * 4;
#pragma unroll
                    for (int kk = 0; kk < kPK / 8; ++kk) {
                        const uint32_t o = kk * 2 * kPLBO;
                        mma_tf32(acc, psmem_desc(al + o), psmem_desc(bh + o), idesc, (s > 0 || kk > 0) ? 1u : 0u);
                        mma_tf32(acc, psmem_desc(ah + o), psmem_desc(bl + o), idesc, 1u);
                        mma_tf32(acc, psmem_desc(ah + o), psmem_desc(bh + o), idesc, 1u);
                    }
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                        smem_u32(&bar_conv_empty[slot])));
                }
                if (ok)
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                        smem_u32(&bar_acc_full[a])));
            }
            // the MMAs issued so far have completed before tensor memory is freed
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                smem_u32(&bar_drain)));
            pdrain(smem_u32(&bar_drain), 0);
        }
    } else if (warp >= 4 && warp < 8) {
        // ---- split into hi / lo -----------------------------------------
        const int t = threadIdx.x - 128;      // 0..127
        const int q = t & 7;                  // lane within a quarter warp
        int g = 0;
        bool ok = true;
        for (int i = 0; i < my_tiles && ok; ++i) {
            for (int s = 0; s < n_stage; ++s, ++g) {
                const int rs = g % kRaw, cs = g % kConv;
                ok = pwait(smem_u32(&bar_raw_full[rs]), (g / kRaw) & 1, abort_flag, err);
                if (ok && g >= kConv) ok = pwait(smem_u32(&bar_conv_empty[cs]), ((g / kConv) - 1) & 1, abort_flag, err);
                if (!ok) break;
                const float* rA = reinterpret_cast<const float*>(psm + rs * L.raw_bytes + L.rawA);
                const float* rB = reinterpret_cast<const float*>(psm + rs * L.raw_bytes + L.rawB);
                float* aH = reinterpret_cast<float*>(psm + L.convA + cs * L.conv_bytes);
                float* aL = aH + kTcM * kPK;
                float* bH = reinterpret_cast<float*>(psm + L.convB + cs * L.conv_bytes);
                float* bL = bH + Np * kPK;
                // A: thread t owns row t; its four 16-byte chunks are visited
                // in a rotated order so a quarter warp's reads spread over the banks
#pragma unroll
                for (int j = 0; j < kPK / 4; ++j) {
                    const int kq = (q + j) & 3;
                    const float4 x = *reinterpret_cast<const float4*>(rA + t * kPK + 4 * kq);
                    const float4 h = split_hi4(x);
                    const int o = ptile_off(t, 4 * kq);
                    *reinterpret_cast<float4*>(aH + o) = h;
                    *reinterpret_cast<float4*>(aL + o) = split_lo4(x, h);
                }
                if (!b_trans) {
                    for (int r = t; r < Np; r += 128)
#pragma unroll
                        for (int j = 0; j < kPK / 4; ++j) {
                            const int kq = (q + j) & 3;
                            const float4 x = *reinterpret_cast<const float4*>(rB + r * kPK + 4 * kq);
                            const float4 h = split_hi4(x);
                            const int o = ptile_off(r, 4 * kq);
                            *reinterpret_cast<float4*>(bH + o) = h;
                            *reinterpret_cast<float4*>(bL + o) = split_lo4(x, h);
                        }
                } else {
                    // raw B is [kPK][Np] (n contiguous): thread -> n
                    for (int r = t; r < Np; r += 128)
#pragma unroll
                        for (int kq = 0; kq < kPK / 4; ++kq) {
                            const float4 x = make_float4(rB[(4 * kq) * Np + r], rB[(4 * kq + 1) * Np + r],
                                                         rB[(4 * kq + 2) * Np + r], rB[(4 * kq + 3) * Np + r]);
                            const float4 h = split_hi4(x);
                            const int o = ptile_off(r, 4 * kq);
                            *reinterpret_cast<float4*>(bH + o) = h;
                            *reinterpret_cast<float4*>(bL + o) = split_lo4(x, h);
                        }
                }
                // generic-proxy stores -> visible to the tensor core's reads
                asm volatile("fence.proxy.async.shared::cta;");
                __syncwarp();
                if (lane == 0) {
                    mbar_arrive(smem_u32(&bar_raw_empty[rs]));
                    mbar_arrive(smem_u32(&bar_conv_full[cs]));
                }
            }
        }
    } else if (warp >= 8) {
        // ---- epilogue ---------------------------------------------------
        const int q4 = warp & 3;
        float* buf = reinterpret_cast<float*>(psm + L.epi) + q4 * (32 * 33);
        for (int i = 0; i < my_tiles; ++i) {
            const int a = i & 1;
            if (!pwait(smem_u32(&bar_acc_full[a]), (i >> 1) & 1, abort_flag, err)) break;
            asm volatile("tcgen05.fence::after_thread_sync;");
            const int tile = (int)blockIdx.x + i * (int)gridDim.x;
            const int b = tile / mt, m0 = (tile - b * mt) * kTcM;
            const uint32_t taddr = tmem + (uint32_t)(a * ncol) + ((uint32_t)(q4 * 32) << 16);
            float* Db = D + (size_t)b * sD;
            for (int c0 = 0; c0 < Np; c0 += 32) {
                uint32_t r[32];
#pragma unroll
                for (int gq = 0; gq < 4; ++gq) {
                    if (c0 + 8 * gq < Np)
                        asm volatile(
                            "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                            : "=r"(r[8 * gq]), "=r"(r[8 * gq + 1]), "=r"(r[8 * gq + 2]), "=r"(r[8 * gq + 3]),
                              "=r"(r[8 * gq + 4]), "=r"(r[8 * gq + 5]), "=r"(r[8 * gq + 6]), "=r"(r[8 * gq + 7])
                            : "r"(taddr + (uint32_t)(c0 + 8 * gq)));
                    else
#pragma unroll
                        for (int u = 0; u < 8; ++u) r[8 * gq + u] = 0u;
                }
                asm volatile("tcgen05.wait::ld.sync.aligned;");
                if (c0 + 32 >= Np) {
                    // the accumulator is read out: free it for the tile after next
                    asm volatile("tcgen05.fence::before_thread_sync;");
                    __syncwarp();
                    if (lane == 0) mbar_arrive(smem_u32(&bar_acc_empty[a]));
                }
#pragma unroll
                for (int j = 0; j < 32; ++j) buf[lane * 33 + j] = __uint_as_float(r[j]);
                __syncwarp();
                const int col = c0 + lane;
                if (beta != 0.f) {
                    // all 32 old values in flight before any store (the
                    // compiler cannot prove D and the tile do not alias)
                    float old[32];
#pragma unroll
                    for (int rr = 0; rr < 32; ++rr) {
                        const int row = m0 + q4 * 32 + rr;
                        old[rr] = (row < M && col < N) ? Db[(size_t)row * ldd + col] : 0.f;
                    }
#pragma unroll
                    for (int rr = 0; rr < 32; ++rr) {
                        const int row = m0 + q4 * 32 + rr;
                        if (row < M && col < N)
                            Db[(size_t)row * ldd + col] = alpha * buf[rr * 33 + lane] + beta * old[rr];
                    }
                } else {
                    for (int rr = 0; rr < 32; ++rr) {
                        const int row = m0 + q4 * 32 + rr;
                        if (row < M && col < N) Db[(size_t)row * ldd + col] = alpha * buf[rr * 33 + lane];
                    }
                }
                __syncwarp();
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * ncol));
}

using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static std::once_flag once;
    static EncodeTiledFn fn = nullptr;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
        else
            cudaGetLastError();
    });
    return fn;
}

// 3-D FP32 tensor map over rows of `inner` elements (row stride ld), `outer`
// rows per batch entry (batch stride sbatch elements, or 1 entry when
// sbatch == 0), box {box_inner, box_outer, 1}; out-of-range elements read 0.
bool make_map(CUtensorMap* m, const float* base, int inner, int outer, int ld, long long sbatch, int batch,
              int box_inner, int box_outer) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    const int nb = sbatch == 0 ? 1 : batch;
    cuuint64_t dims[3] = {(cuuint64_t)inner, (cuuint64_t)outer, (cuuint64_t)nb};
    cuuint64_t strides[2] = {(cuuint64_t)ld * 4, (cuuint64_t)(sbatch == 0 ? (long long)ld * outer : sbatch) * 4};
    cuuint32_t box[3] = {(cuuint32_t)box_inner, (cuuint32_t)box_outer, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(base), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}


// ---------------------------------------------------------------------
// Pre-split form: D = A B^T with both operands already given as TF32 hi /
// lo pairs (x = hi + lo, each a TF32-exact float), so TMA loads land in the
// MMA's layout and nothing else touches the operands.  128-byte swizzled
// K-major tiles (TMA SWIZZLE_128B, UMMA layout type 2): a stage is 32 k of
// A_hi, A_lo, B_hi, B_lo (rows of 128 bytes, 8-row atoms of 1024 bytes);
// the four 8-k MMA steps of a stage advance the descriptors' start address
// by 32 bytes inside the swizzle atom.  Roles: warp 0 issues the loads of a
// ring of up to kSStages slots, warp 1 the MMAs (committed to the stage's "empty"
// barrier), warps 2-5 drain the accumulator (TMEM lane quadrant = warp % 4).
// ---------------------------------------------------------------------
constexpr int kSK = 32;
constexpr int kSStages = 4;   // ring slots at most (fewer when a stage is large)

__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)1 << 16;                      // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(1024 >> 4) << 32;            // 8-row atoms 1024 bytes apart
    d |= (uint64_t)1 << 46;                      // descriptor version
    d |= (uint64_t)2 << 61;                      // 128-byte swizzle
    return d;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

struct SplitSmem {
    uint32_t a_bytes, b_bytes, stage_bytes, slots, total;
};
// As many ring slots (2..kSStages) as fit the 227 KB a CTA may use, less
// the static barriers and the 1024-byte alignment slack.
__host__ __device__ inline SplitSmem split_layout(int Np) {
    SplitSmem L;
    L.a_bytes = kTcM * kSK * 4;
    L.b_bytes = (uint32_t)Np * kSK * 4;
    L.stage_bytes = 2 * (L.a_bytes + L.b_bytes);
    uint32_t slots = (232448u - 2048u - 1024u) / L.stage_bytes;
    if (slots > (uint32_t)kSStages) slots = kSStages;
    if (slots < 2u) slots = 2u;
    L.slots = slots;
    L.total = slots * L.stage_bytes + 1024;
    return L;
}

__global__ void __launch_bounds__(192, 1)
    k_tc_gemm_split(const __grid_constant__ CUtensorMap tAh, const __grid_constant__ CUtensorMap tAl,
                    const __grid_constant__ CUtensorMap tBh, const __grid_constant__ CUtensorMap tBl, int M, int N,
                    int K, float* __restrict__ D, int ldd, unsigned* err) {
    extern __shared__ unsigned char ssm_raw[];
    __shared__ __align__(8) uint64_t bar_full[kSStages], bar_empty[kSStages], bar_acc, bar_drain;
    __shared__ uint32_t s_tmem;
    __shared__ int s_abort;
    const int Np = (N + 15) & ~15;
    uint32_t ncol = 32;
    while ((int)ncol < Np) ncol <<= 1;
    const SplitSmem L = split_layout(Np);
    const uint32_t sraw = smem_u32(ssm_raw);
    const uint32_t sbase = (sraw + 1023u) & ~1023u;      // 1024-byte aligned stages
    unsigned char* ssm = ssm_raw + (sbase - sraw);
    const int m0 = blockIdx.x * kTcM;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n_stage = (K + kSK - 1) / kSK;
    volatile int* abort_flag = &s_abort;
    if (threadIdx.x == 0) {
        for (int i = 0; i < (int)L.slots; ++i) {
            mbar_init(smem_u32(&bar_full[i]), 1);
            mbar_init(smem_u32(&bar_empty[i]), 1);
        }
        mbar_init(smem_u32(&bar_acc), 1);
        mbar_init(smem_u32(&bar_drain), 1);
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tAh)) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tAl)) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tBh)) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tBl)) : "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                     "r"(ncol));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = s_tmem;
    if (warp == 0) {
        if (lane == 0) {
            int issued = 0;
            for (int s = 0; s < n_stage; ++s) {
                const int slot = s % (int)L.slots;
                if (s >= (int)L.slots &&
                    !pwait(smem_u32(&bar_empty[slot]), ((s / (int)L.slots) - 1) & 1, abort_flag, err))
                    break;
                const uint32_t full = smem_u32(&bar_full[slot]);
                mbar_expect_tx(full, L.stage_bytes);
                const uint32_t st = sbase + slot * L.stage_bytes;
                const int k0 = s * kSK;
                tma_load_2d(st, &tAh, k0, m0, full);
                tma_load_2d(st + L.a_bytes, &tAl, k0, m0, full);
                tma_load_2d(st + 2 * L.a_bytes, &tBh, k0, 0, full);
                tma_load_2d(st + 2 * L.a_bytes + L.b_bytes, &tBl, k0, 0, full);
                ++issued;
            }
            for (int s = (issued > (int)L.slots ? issued - (int)L.slots : 0); s < issued; ++s)
                pdrain(smem_u32(&bar_full[s % (int)L.slots]), (s / (int)L.slots) & 1);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t idesc = idesc_tf32(kTcM, Np);
            int done = 0;
            for (int s = 0; s < n_stage; ++s) {
                const int slot = s % (int)L.slots;
                if (!pwait(smem_u32(&bar_full[slot]), (s / (int)L.slots) & 1, abort_flag, err)) break;
                asm volatile("tcgen05.fence::after_thread_sync;");
                const uint32_t ah = sbase + slot * L.stage_bytes, al = ah + L.a_bytes;
                const uint32_t bh = ah + 2 * L.a_bytes, bl = bh + L.b_bytes;
#pragma unroll
                for (int kk = 0; kk < kSK / 8; ++kk) {
                    const uint32_t o = kk * 32;   // 8 TF32 = 32 bytes along the swizzled row
                    mma_tf32(tmem, sw128_desc(al + o), sw128_desc(bh + o), idesc, (s > 0 || kk > 0) ? 1u : 0u);
                    mma_tf32(tmem, sw128_desc(ah + o), sw128_desc(bl + o), idesc, 1u);
                    mma_tf32(tmem, sw128_desc(ah + o), sw128_desc(bh + o), idesc, 1u);
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                    smem_u32(&bar_empty[slot])));
                ++done;
            }
            if (done == n_stage)
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                    smem_u32(&bar_acc)));
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                smem_u32(&bar_drain)));
            pdrain(smem_u32(&bar_drain), 0);
        }
    } else {
        // epilogue warps 2..5: TMEM lane quadrant warp % 4
        bool ok = n_stage > 0 && pwait(smem_u32(&bar_acc), 0, abort_flag, err);
        asm volatile("tcgen05.fence::after_thread_sync;");
        if (ok) {
            const int q4 = warp & 3;
            const uint32_t taddr = tmem + ((uint32_t)(q4 * 32) << 16);
            // every MMA has completed, so the stage buffers are free: one
            // padded 32 x 33 transpose tile per warp
            float* buf = reinterpret_cast<float*>(ssm) + q4 * (32 * 33);
            for (int c0 = 0; c0 < Np; c0 += 32) {
                uint32_t r[32];
#pragma unroll
                for (int g = 0; g < 4; ++g) {
                    if (c0 + 8 * g < Np)
                        asm volatile(
                            "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                            : "=r"(r[8 * g]), "=r"(r[8 * g + 1]), "=r"(r[8 * g + 2]), "=r"(r[8 * g + 3]),
                              "=r"(r[8 * g + 4]), "=r"(r[8 * g + 5]), "=r"(r[8 * g + 6]), "=r"(r[8 * g + 7])
                            : "r"(taddr + (uint32_t)(c0 + 8 * g)));
                    else
#pragma unroll
                        for (int u = 0; u < 8; ++u) r[8 * g + u] = 0u;
                }
                asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
                for (int j = 0; j < 32; ++j) buf[lane * 33 + j] = __uint_as_float(r[j]);
                __syncwarp();
                const int col = c0 + lane;
                for (int rr = 0; rr < 32; ++rr) {
                    const int row = m0 + q4 * 32 + rr;
                    if (row < M && col < N) D[(size_t)row * ldd + col] = buf[rr * 33 + lane];
                }
                __syncwarp();
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncol));
}

// 2-D FP32 tensor map, rows of `inner` elements (row stride ld), box
// {32, box_rows}, 128-byte swizzle.
bool make_map_sw128(CUtensorMap* m, const float* base, int inner, int rows, int ld, int box_rows) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)ld * 4};
    cuuint32_t box[2] = {(cuuint32_t)kSK, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

// Whether the pipelined kernel can take these operands: TMA needs 16-byte
// aligned bases, row strides and batch strides.
static bool pipe_ok(int K, const float* A, long long sA, int lda, const float* B, long long sB, int ldb) {
    const auto al16 = [](const void* p) { return ((uintptr_t)p & 15) == 0; };
    return K > 0 && al16(A) && al16(B) && lda % 4 == 0 && ldb % 4 == 0 && sA % 4 == 0 && sB % 4 == 0 &&
           encode_fn() != nullptr;
}

cudaError_t launch_tc_gemm_ab(int batch, int M, int N, int K, float alpha, const float* A, long long sA, int lda,
                              const float* B, long long sB, int ldb, int b_trans, float beta, float* D, long long sD,
                              int ldd, unsigned* err, cudaStream_t st) {
    if (batch <= 0 || M <= 0 || N <= 0) return cudaSuccess;
    if (N > kTcMaxN || K < 0) return cudaErrorInvalidValue;
    if (!pipe_ok(K, A, sA, lda, B, sB, ldb)) return cudaErrorNotSupported;
    const int Np = (N + 15) & ~15;
    alignas(64) CUtensorMap ta, tb;
    if (!make_map(&ta, A, K, M, lda, sA, batch, kPK, kTcM)) return cudaErrorNotSupported;
    const bool ok_b = b_trans ? make_map(&tb, B, N, K, ldb, sB, batch, Np, kPK)
                              : make_map(&tb, B, K, N, ldb, sB, batch, kPK, Np);
    if (!ok_b) return cudaErrorNotSupported;
    const PipeSmem L = pipe_layout(Np);
    cudaError_t e = cudaFuncSetAttribute(k_tc_gemm_pipe, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.total);
    if (e != cudaSuccess) return e;
    // persistent: as many CTAs as are resident at once (tensor memory: two
    // accumulators of up to 256 columns each fit one CTA per SM at N > 128)
    static int n_sm[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!n_sm[dev] && cudaDeviceGetAttribute(&n_sm[dev], cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return cudaErrorInvalidDevice;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tc_gemm_pipe, 384, L.total);
    if (e != cudaSuccess) return e;
    uint32_t ncol = 32;
    while ((int)ncol < Np) ncol <<= 1;
    const int tmem_fit = (int)(512 / (2 * ncol));
    per_sm = per_sm < tmem_fit ? per_sm : tmem_fit;
    if (per_sm < 1) per_sm = 1;
    const long long tiles = (long long)((M + kTcM - 1) / kTcM) * batch;
    const int grid = (int)(tiles < (long long)n_sm[dev] * per_sm ? tiles : (long long)n_sm[dev] * per_sm);
    k_tc_gemm_pipe<<<grid, 384, L.total, st>>>(ta, tb, M, N, K, batch, b_trans, sA != 0, sB != 0, alpha, beta, D, sD,
                                             ldd, err);
    return cudaGetLastError();
}

// The pipelined kernel where TMA can describe the operands, else the staged
// one (unaligned rows or bases, K = 0).
cudaError_t launch_tc_gemm(int batch, int M, int N, int K, const float* A, long long sA, int lda, const float* B,
                           long long sB, int ldb, int b_trans, float* D, long long sD, int ldd, unsigned* err,
                           cudaStream_t st) {
    if (batch > 0 && M > 0 && N > 0 && N <= kTcMaxN && pipe_ok(K, A, sA, lda, B, sB, ldb)) {
        const cudaError_t e =
            launch_tc_gemm_ab(batch, M, N, K, 1.f, A, sA, lda, B, sB, ldb, b_trans, 0.f, D, sD, ldd, err, st);
        if (e != cudaErrorNotSupported) return e;
    }
    return launch_tc_gemm_staged(batch, M, N, K, A, sA, lda, B, sB, ldb, b_trans, D, sD, ldd, err, st);
}


bool tc_split_plan(TcSplitPlan* p, int M, int N, int K, const float* Ah, const float* Al, int lda, const float* Bh,
                   const float* Bl, int ldb) {
    const auto al16 = [](const void* q) { return ((uintptr_t)q & 15) == 0; };
    if (M <= 0 || N <= 0 || N > kTcMaxN || K <= 0 || lda % 4 || ldb % 4 || !al16(Ah) || !al16(Al) || !al16(Bh) ||
        !al16(Bl))
        return false;
    const int Np = (N + 15) & ~15;
    p->M = M;
    p->N = N;
    p->K = K;
    return make_map_sw128(reinterpret_cast<CUtensorMap*>(p->map[0]), Ah, K, M, lda, kTcM) &&
           make_map_sw128(reinterpret_cast<CUtensorMap*>(p->map[1]), Al, K, M, lda, kTcM) &&
           make_map_sw128(reinterpret_cast<CUtensorMap*>(p->map[2]), Bh, K, N, ldb, Np) &&
           make_map_sw128(reinterpret_cast<CUtensorMap*>(p->map[3]), Bl, K, N, ldb, Np);
}

size_t tc_split_smem_bytes(int N) { return split_layout((N + 15) & ~15).total; }

cudaError_t tc_split_prepare(int N) {
    return cudaFuncSetAttribute(k_tc_gemm_split, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)tc_split_smem_bytes(N));
}

cudaError_t launch_tc_gemm_split(const TcSplitPlan& p, float* D, int ldd, unsigned* err, cudaStream_t st) {
    const CUtensorMap* m = reinterpret_cast<const CUtensorMap*>(p.map[0]);
    k_tc_gemm_split<<<(p.M + kTcM - 1) / kTcM, 192, tc_split_smem_bytes(p.N), st>>>(m[0], m[1], m[2], m[3], p.M, p.N,
                                                                                     p.K, D, ldd, err);
    return cudaGetLastError();
}

}  // namespace qmc
