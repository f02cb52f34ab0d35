// Tensor-core Gram product for the correlation integral (the one dense
// contraction of the path): P_ij = hi_i.hi_j + hi_i.lo_j + lo_i.hi_j over one
// K-chunk, bf16 operands, FP32 accumulation in tensor memory.
//
// Blackwell (sm_100 family) structure, written with inline PTX:
//   * TMA (cp.async.bulk.tensor) loads 128-row x 64-column bf16 tiles of the
//     hi and lo parts of both pattern sets into 128-byte-swizzled shared
//     memory, three stages deep, completion tracked by mbarriers;
//   * one elected thread issues tcgen05.mma (M = N = 128, K = 16, kind::f16
//     with bf16 inputs, FP32 accumulator in TMEM) and frees each stage with
//     tcgen05.commit;
//   * four warps read the 128 x 128 FP32 accumulator back with tcgen05.ld
//     (warp w owns TMEM lanes 32w..32w+31) and store the chunk partials.
// Every mbarrier wait is bounded: on timeout the kernel raises ST_TIMEOUT in
// the status word, skips its epilogue, frees its TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <mutex>
#include "common.cuh"

namespace rdcil {

static constexpr int TC_BM = 128, TC_BN = 128, TC_BK = 64, TC_STAGES = 3;
static constexpr int TC_TILE_BYTES = TC_BM * TC_BK * 2;              // 16 KiB
static constexpr int TC_STAGE_BYTES = 4 * TC_TILE_BYTES;             // A hi, A lo, B hi, B lo
static constexpr int TC_SMEM = TC_STAGES * TC_STAGE_BYTES + 1024 + 256;
static constexpr uint32_t TC_WAIT_LIMIT = 1u << 22;                  // bounded spin (~seconds)

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for the phase with the given parity to complete.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
    for (uint32_t it = 0; it < TC_WAIT_LIMIT; ++it)
        if (mbar_try(bar, parity)) return true;
    return false;
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *tm, int c0, int c1, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
        "[%4];" ::"r"(smem_u32(dst)),
        "l"((uint64_t)tm), "r"(c0), "r"(c1), "r"(smem_u32(bar))
        : "memory");
}

// Shared-memory matrix descriptor, K-major operand in the 128-byte swizzle
// layout: start address >> 4 (bits 0-13), leading byte offset (unused for
// swizzled K-major, set to 1), stride byte offset = 1024 B between 8-row
// groups (bits 32-45), descriptor version 1 (bits 46-47), swizzle mode
// 128B = 2 (bits 61-63).
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t addr) {
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFF);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// Instruction descriptor, kind::f16: FP32 accumulator (bits 4-5 = 1), A and
// B bf16 (bits 7-9 = 1, bits 10-12 = 1), both K-major, N >> 3 at bits
// 17-22, M >> 4 at bits 24-28.
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int q = 0; q < 16; ++q) v[q] = __uint_as_float(r[q]);
}

// grid: (ceil(n2/128), ceil(n1/128), nchunk); block: 128 threads.
// Rows 0..n1-1 of the hi/lo arrays are set 1, rows n1..n1+n2-1 set 2.
__global__ void __launch_bounds__(128, 1)
gram_tc_kernel(const __grid_constant__ CUtensorMap tm_hi, const __grid_constant__ CUtensorMap tm_lo, int n1, int n2,
               int dp, int kc, float *__restrict__ Ppart, uint32_t *__restrict__ status) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t *full = (uint64_t *)(smem + TC_STAGES * TC_STAGE_BYTES);
    uint64_t *empty = full + TC_STAGES;
    uint64_t *done = empty + TC_STAGES;
    uint32_t *tslot = (uint32_t *)(done + 1);
    __shared__ int s_fail;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int i0 = blockIdx.y * TC_BM, j0 = blockIdx.x * TC_BN;
    const int k_begin = blockIdx.z * kc;
    const int k_end = min(dp, k_begin + kc);
    const int nk = (k_end - k_begin) / TC_BK;

    if (threadIdx.x == 0) {
        for (int s = 0; s < TC_STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(done, 1);
        s_fail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(TC_BN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tslot;
    int issued = 0;   // stages handed to TMA by the producer

    if (threadIdx.x == 0) {
        // ---- producer: TMA loads ----
        for (int it = 0; it < nk; ++it) {
            const int s = it % TC_STAGES;
            const uint32_t ph = (uint32_t)(it / TC_STAGES) & 1u;
            if (!mbar_wait(&empty[s], ph ^ 1u)) { s_fail = 1; break; }
            uint8_t *st = smem + s * TC_STAGE_BYTES;
            mbar_expect_tx(&full[s], TC_STAGE_BYTES);
            const int k = k_begin + it * TC_BK;
            tma_load_2d(st, &tm_hi, k, i0, &full[s]);
            tma_load_2d(st + TC_TILE_BYTES, &tm_lo, k, i0, &full[s]);
            tma_load_2d(st + 2 * TC_TILE_BYTES, &tm_hi, k, n1 + j0, &full[s]);
            tma_load_2d(st + 3 * TC_TILE_BYTES, &tm_lo, k, n1 + j0, &full[s]);
            issued = it + 1;
        }
    } else if (threadIdx.x == 32) {
        // ---- MMA issuer ----
        constexpr uint32_t idesc = idesc_bf16_f32(TC_BM, TC_BN);
        bool ok = true;
        for (int it = 0; it < nk && ok; ++it) {
            const int s = it % TC_STAGES;
            const uint32_t ph = (uint32_t)(it / TC_STAGES) & 1u;
            if (!mbar_wait(&full[s], ph)) { s_fail = 1; ok = false; break; }
            fence_after();
            const uint32_t base = smem_u32(smem + s * TC_STAGE_BYTES);
#pragma unroll
            for (int kk = 0; kk < TC_BK / 16; ++kk) {
                const uint32_t off = kk * 32;   // 16 bf16 = 32 bytes along K inside the swizzle atom
                const uint64_t ah = smem_desc_sw128(base + off);
                const uint64_t al = smem_desc_sw128(base + TC_TILE_BYTES + off);
                const uint64_t bh = smem_desc_sw128(base + 2 * TC_TILE_BYTES + off);
                const uint64_t bl = smem_desc_sw128(base + 3 * TC_TILE_BYTES + off);
                mma_bf16(tmem, ah, bh, idesc, (it | kk) ? 1u : 0u);
                mma_bf16(tmem, ah, bl, idesc, 1u);
                mma_bf16(tmem, al, bh, idesc, 1u);
            }
            mma_commit(&empty[s]);   // stage free once these MMAs have read it
        }
        mma_commit(done);            // accumulator complete
    }
    __syncwarp();

    // ---- epilogue: TMEM -> registers -> partials ----
    const bool ok = mbar_wait(done, 0);
    fence_after();
    // block-uniform decision: tcgen05.ld below is warp-collective
    const int good = __syncthreads_and(ok ? 1 : 0) && !s_fail;
    if (good) {
        const int i = i0 + warp * 32 + lane;
        float *out = Ppart + (int64_t)blockIdx.z * n1 * n2;
#pragma unroll 1
        for (int c = 0; c < TC_BN; c += 16) {
            float v[16];
            tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c, v);
            if (i < n1) {
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    const int j = j0 + c + q;
                    if (j < n2) out[(int64_t)i * n2 + j] = v[q];
                }
            }
        }
    }
    if (threadIdx.x == 0 && !good) {
        atomicOr(status, (unsigned)ST_TIMEOUT);
        // let the copies already in flight land before the block's shared
        // memory is released (bounded)
        for (int it = 0; it < issued; ++it) mbar_wait(&full[it % TC_STAGES], (uint32_t)(it / TC_STAGES) & 1u);
    }
    fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_BN) : "memory");
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    });
    return fn;
}

static bool make_map(CUtensorMap *m, const void *base, int64_t rows, int64_t dp) {
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {(cuuint64_t)dp, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)dp * 2};
    cuuint32_t box[2] = {(cuuint32_t)TC_BK, (cuuint32_t)TC_BM};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// Preconditions (checked): hi/lo 16-byte aligned, dp a multiple of 64, kc a
// multiple of 64.
rd_status launch_gram_tc(const void *hi, const void *lo, int64_t n1, int64_t n2, int64_t dp, int64_t kc,
                         int64_t nchunk, float *Ppart, uint32_t *status, cudaStream_t s) {
    if ((((uintptr_t)hi | (uintptr_t)lo) & 15) || (dp % TC_BK) || (kc % TC_BK) || n1 < 1 || n2 < 1)
        return RD_ERR_INVALID_ARG;
    if (n1 + n2 > 0x7FFFFFFF || dp > 0x7FFFFFFF) return RD_ERR_UNSUPPORTED;
    CUtensorMap mh, ml;
    if (!make_map(&mh, hi, n1 + n2, dp) || !make_map(&ml, lo, n1 + n2, dp)) return RD_ERR_CUDA;
    static bool attr = false;
    if (!attr) {
        RD_CUDA_TRY(cudaFuncSetAttribute(gram_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM));
        attr = true;
    }
    dim3 grid((unsigned)((n2 + TC_BN - 1) / TC_BN), (unsigned)((n1 + TC_BM - 1) / TC_BM), (unsigned)nchunk);
    gram_tc_kernel<<<grid, 128, TC_SMEM, s>>>(mh, ml, (int)n1, (int)n2, (int)dp, (int)kc, Ppart, status);
    note_launch();
    return cuda_status(cudaGetLastError());
}

}  // namespace rdcil
