// Tensor-core Gram product for the correlation integral (the one dense
// contraction of the path), in one of two forms:
//   three products  P_ij = hi_i.hi_j + hi_i.lo_j + lo_i.hi_j (tight: only
//                   lo.lo is dropped),
//   one product     P_ij = hi_i.hi_j (a third of the MMA work and half the
//                   operand bytes; the caller's bound covers the dropped
//                   cross terms by Cauchy-Schwarz on the parts' norms),
// bf16 operands, FP32 accumulation in tensor memory, accumulated over K
// chunks whose partials are summed with compensation.
//
// Blackwell (sm_100 family) structure, written with inline PTX:
//   * TMA (cp.async.bulk.tensor) loads 128-row x 64-column bf16 tiles of the
//     hi (and lo) parts of both pattern sets into 128-byte-swizzled shared
//     memory, three stages of four tiles (six of two for one product) deep,
//     completion tracked by mbarriers;
//   * one elected thread issues tcgen05.mma (M = N = 128, K = 16, kind::f16
//     with bf16 inputs, FP32 accumulator in TMEM) into two alternating TMEM
//     accumulators, one K chunk each (the chunk length bounds the FP32
//     accumulation error), and frees each stage with tcgen05.commit;
//   * four drain warps read each finished chunk back with tcgen05.ld (one
//     load per 32 columns), hand the accumulator back at once and add the
//     chunk into FP32 running sums held in registers (128 per thread, one
//     output row each), while the tensor core fills the other accumulator;
//     after the segment's last chunk they store the sums once.  A plain
//     running sum of the segment's chunk partials errs by at most
//     (chunks - 1) 2^-24 of their magnitudes; the caller's bound carries
//     that term.  (Keeping a compensated hi/lo sum in TMEM instead costs
//     five tensor-memory accesses per 32 columns and chunk, and those stall
//     the tensor core: 0.200 ms against 0.165 on 2 x 1024 x 32768.)
// One CTA per (output tile, K segment); the segments of all tiles run
// concurrently and in step along K, so each bf16 tile is fetched from HBM
// about once and re-read from L2 by the CTAs that share it.
// Every mbarrier wait is bounded: on timeout the kernel raises ST_TIMEOUT in
// the status word, skips its epilogue, frees its TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <mutex>
#include "common.cuh"
#include "tma.cuh"
#include "tc.cuh"

namespace rdcil {

static constexpr int TC_BM = 128, TC_BN = 128, TC_BK = 64;
static constexpr int TC_TILE_BYTES = TC_BM * TC_BK * 2;              // 16 KiB
// per product count: tiles per stage (A hi, A lo, B hi, B lo / A hi, B hi)
// and stages, 192 KiB of operands either way
template <int NP> struct GramShape {
    static constexpr int TILES = NP == 3 ? 4 : 2;
    static constexpr int STAGES = NP == 3 ? 3 : 6;
    static constexpr int STAGE_BYTES = TILES * TC_TILE_BYTES;
    static_assert(NP == 1 || NP == 3, "one or three products");
    static_assert((2 * STAGES + 5) * 8 + 4 <= 256, "barrier area");
};
static constexpr int TC_SMEM = 3 * 4 * TC_TILE_BYTES + 1024 + 256;
static_assert(GramShape<1>::STAGES * GramShape<1>::STAGE_BYTES == 3 * 4 * TC_TILE_BYTES, "same operand area");
static constexpr uint32_t TC_WAIT_LIMIT = MBAR_WAIT_LIMIT;           // bounded spin (~seconds)
static constexpr uint32_t TC_TMEM_COLS = 2 * TC_BN;                  // two accumulators

// One CTA per (output tile t, K segment s): grid = ntiles * S, block = 192
// threads.  Tile t covers set-1 rows 128*(t / ntj) and set-2 rows
// 128*(t % ntj) (rows 0..n1-1 of the hi/lo arrays are set 1, rows
// n1..n1+n2-1 set 2).  Segment s covers the 64-column K steps
// [s*n64/S, (s+1)*n64/S).
//   warp 0    TMA producer (one lane)
//   warp 1    MMA issuer (one lane): K chunks of at most cs steps, each
//             accumulated from zero into TMEM accumulator (chunk & 1)
//   warps 2-5 drain: add each finished chunk into FP32 running sums in
//             registers (thread = output row, 128 columns), and after the
//             last chunk of the segment store the sums of the valid pairs
//             to Ppart[s * n1 * n2 + i * n2 + j].
// TMEM columns: [0,128) and [128,256) accumulators; warp w may access TMEM
// lanes 32 (w % 4) .. +31 (rows).  NP = 1 never reads tm_lo.
template <int NP>
__global__ void __launch_bounds__(192, 1)
gram_tc_kernel(const __grid_constant__ CUtensorMap tm_hi, const __grid_constant__ CUtensorMap tm_lo, int n1, int n2,
               int dp, int ntj, int S, int cs, float *__restrict__ Ppart, uint32_t *__restrict__ status,
               uint32_t spin) {
    constexpr int TC_STAGES = GramShape<NP>::STAGES, TC_STAGE_BYTES = GramShape<NP>::STAGE_BYTES;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t *full = (uint64_t *)(smem + TC_STAGES * TC_STAGE_BYTES);
    uint64_t *empty = full + TC_STAGES;
    uint64_t *accf = empty + TC_STAGES;     // [2] chunk accumulated (MMA commit)
    uint64_t *acce = accf + 2;              // [2] accumulator drained (4 drain warps)
    uint64_t *mdone = acce + 2;             // every MMA issued by this CTA has completed
    uint32_t *tslot = (uint32_t *)(mdone + 1);
    __shared__ int s_fail;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int t = blockIdx.x / S, sgm = blockIdx.x - (blockIdx.x / S) * S;
    const int i0 = (t / ntj) * TC_BM, j0 = (t % ntj) * TC_BN;
    const int n64 = dp / TC_BK;
    const int k_lo = (int)((int64_t)sgm * n64 / S), k_hi = (int)((int64_t)(sgm + 1) * n64 / S);
    const int nst = k_hi - k_lo;                           // K steps of this segment (>= 1)
    const int nch = (nst + cs - 1) / cs;                   // chunks of this segment

    if (threadIdx.x == 0) {
        for (int q = 0; q < TC_STAGES; ++q) {
            mbar_init(&full[q], 1);
            mbar_init(&empty[q], 1);
        }
        for (int q = 0; q < 2; ++q) {
            mbar_init(&accf[q], 1);
            mbar_init(&acce[q], 4);
        }
        mbar_init(mdone, 1);
        s_fail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(TC_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tslot;
    int issued = 0;   // stages handed to TMA by the producer

    if (threadIdx.x == 0) {
        // ---- producer: TMA loads of the whole segment ----
        for (int it = 0; it < nst; ++it) {
            const int q = it % TC_STAGES;
            const uint32_t ph = (uint32_t)(it / TC_STAGES) & 1u;
            if (!mbar_wait(&empty[q], ph ^ 1u, spin)) { s_fail = 1; break; }
            uint8_t *st = smem + q * TC_STAGE_BYTES;
            mbar_expect_tx(&full[q], TC_STAGE_BYTES);
            const int k = (k_lo + it) * TC_BK;
            if (NP == 3) {
                tma_load_2d(st, &tm_hi, k, i0, &full[q]);
                tma_load_2d(st + TC_TILE_BYTES, &tm_lo, k, i0, &full[q]);
                tma_load_2d(st + 2 * TC_TILE_BYTES, &tm_hi, k, n1 + j0, &full[q]);
                tma_load_2d(st + 3 * TC_TILE_BYTES, &tm_lo, k, n1 + j0, &full[q]);
            } else {
                tma_load_2d(st, &tm_hi, k, i0, &full[q]);
                tma_load_2d(st + TC_TILE_BYTES, &tm_hi, k, n1 + j0, &full[q]);
            }
            issued = it + 1;
        }
    } else if (threadIdx.x == 32) {
        // ---- MMA issuer ----
        constexpr uint32_t idesc = idesc_bf16_f32(TC_BM, TC_BN);
        bool ok = true;
        int it = 0;
        for (int c = 0; c < nch && ok; ++c) {
            const int buf = c & 1;
            if (c >= 2 && !mbar_wait(&acce[buf], (uint32_t)((c >> 1) - 1) & 1u, spin)) { s_fail = 1; break; }
            fence_after();
            const uint32_t dacc = tmem + (uint32_t)(buf * TC_BN);
            const int it_end = min(nst, (c + 1) * cs);
            for (int first = 1; it < it_end; ++it, first = 0) {
                const int q = it % TC_STAGES;
                const uint32_t ph = (uint32_t)(it / TC_STAGES) & 1u;
                if (!mbar_wait(&full[q], ph, spin)) { s_fail = 1; ok = false; break; }
                fence_after();
                const uint32_t base = smem_u32(smem + q * TC_STAGE_BYTES);
#pragma unroll
                for (int kk = 0; kk < TC_BK / 16; ++kk) {
                    const uint32_t off = kk * 32;   // 16 bf16 = 32 bytes along K inside the swizzle atom
                    if (NP == 3) {
                        const uint64_t ah = smem_desc_sw128(base + off);
                        const uint64_t al = smem_desc_sw128(base + TC_TILE_BYTES + off);
                        const uint64_t bh = smem_desc_sw128(base + 2 * TC_TILE_BYTES + off);
                        const uint64_t bl = smem_desc_sw128(base + 3 * TC_TILE_BYTES + off);
                        mma_bf16(dacc, ah, bh, idesc, (first && kk == 0) ? 0u : 1u);
                        mma_bf16(dacc, ah, bl, idesc, 1u);
                        mma_bf16(dacc, al, bh, idesc, 1u);
                    } else {
                        const uint64_t ah = smem_desc_sw128(base + off);
                        const uint64_t bh = smem_desc_sw128(base + TC_TILE_BYTES + off);
                        mma_bf16(dacc, ah, bh, idesc, (first && kk == 0) ? 0u : 1u);
                    }
                }
                mma_commit(&empty[q]);   // stage free once these MMAs have read it
            }
            if (ok) mma_commit(&accf[buf]);   // chunk complete in accumulator buf
        }
        // whatever happened above, let every MMA this CTA issued finish before
        // its shared memory and tensor memory are released
        mma_commit(mdone);
        if (!mbar_wait(mdone, 0)) s_fail = 1;
    } else if (warp >= 2) {
        // ---- drain: FP32 running sums of the chunk partials ----
        const int qd = warp & 3;                                   // TMEM lane quarter
        const uint32_t lrow = (uint32_t)(qd * 32) << 16;
        const int row = qd * 32 + lane;
        float sum[TC_BN];
#pragma unroll
        for (int k = 0; k < TC_BN; ++k) sum[k] = 0.f;
        bool drained = true;
        for (int c = 0; c < nch; ++c) {
            const int buf = c & 1;
            const bool got = mbar_wait(&accf[buf], (uint32_t)(c >> 1) & 1u, spin);
            // warp-uniform: tcgen05.ld below is warp-collective
            if (!__all_sync(0xffffffffu, got)) { s_fail = 1; drained = false; break; }
            fence_after();
#pragma unroll
            for (int cb = 0; cb < TC_BN; cb += 32) {
                float a[32];
                tmem_ld32(tmem + lrow + (uint32_t)(buf * TC_BN + cb), a);
#pragma unroll
                for (int k = 0; k < 32; ++k) sum[cb + k] += a[k];
            }
            fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acce[buf]);   // accumulator buf may be overwritten
        }
        const int i = i0 + row;
        if (drained && i < n1) {
            float *out = Ppart + (int64_t)sgm * n1 * n2 + (int64_t)i * n2 + j0;
            if ((n2 & 3) == 0 && j0 + TC_BN <= n2) {
#pragma unroll
                for (int k = 0; k < TC_BN; k += 4)
                    *reinterpret_cast<float4 *>(out + k) = make_float4(sum[k], sum[k + 1], sum[k + 2], sum[k + 3]);
            } else {
#pragma unroll
                for (int k = 0; k < TC_BN; ++k)
                    if (j0 + k < n2) out[k] = sum[k];
            }
        }
    }
    __syncwarp();

    fence_before();
    const int bad = __syncthreads_or(s_fail);
    if (threadIdx.x == 0 && bad) {
        atomicOr(status, (unsigned)ST_TIMEOUT);
        // let the copies still in flight (at most the last TC_STAGES issued;
        // earlier ones were waited for by the MMA issuer before their stage
        // was refilled) land before the block's shared memory is released
        for (int it = issued > TC_STAGES ? issued - TC_STAGES : 0; it < issued; ++it)
            mbar_wait(&full[it % TC_STAGES], (uint32_t)(it / TC_STAGES) & 1u);
    }
    __syncthreads();
    fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS)
                     : "memory");
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

// Preconditions (checked): hi (and lo for three products) 16-byte aligned,
// dp a multiple of 64, 1 <= S <= dp / 64, cs >= 1 (K steps of 64 per
// accumulator chunk), np_ 1 or 3.  Ppart holds S * n1 * n2 floats
// (16-byte aligned).
static uint32_t g_spin_limit = TC_WAIT_LIMIT;
void set_gram_spin_limit(uint32_t n) { g_spin_limit = n ? n : TC_WAIT_LIMIT; }

rd_status launch_gram_tc(const void *hi, const void *lo, int64_t n1, int64_t n2, int64_t dp, int64_t S, int64_t cs,
                         int np_, float *Ppart, uint32_t *status, cudaStream_t s) {
    if (np_ != 1 && np_ != 3) return RD_ERR_INVALID_ARG;
    if (np_ == 1) lo = hi;   // not read
    if ((((uintptr_t)hi | (uintptr_t)lo | (uintptr_t)Ppart) & 15) || (dp % TC_BK) || n1 < 1 || n2 < 1 || S < 1 ||
        S > dp / TC_BK || cs < 1 || cs > dp / TC_BK)
        return RD_ERR_INVALID_ARG;
    if (n1 + n2 > 0x7FFFFFFF || dp > 0x7FFFFFFF) return RD_ERR_UNSUPPORTED;
    const int64_t nti = (n1 + TC_BM - 1) / TC_BM, ntj = (n2 + TC_BN - 1) / TC_BN;
    if (nti * ntj * S > 0x7FFFFFFF) return RD_ERR_UNSUPPORTED;
    CUtensorMap mh, ml;
    if (!make_map(&mh, hi, n1 + n2, dp) || !make_map(&ml, lo, n1 + n2, dp)) return RD_ERR_CUDA;
    auto kern = np_ == 3 ? gram_tc_kernel<3> : gram_tc_kernel<1>;
    {
        rd_status ast = smem_attr(kern, TC_SMEM);
        if (ast) return ast;
    }
    kern<<<(unsigned)(nti * ntj * S), 192, TC_SMEM, s>>>(mh, ml, (int)n1, (int)n2, (int)dp, (int)ntj, (int)S,
                                                         (int)cs, Ppart, status, g_spin_limit);
    note_launch();
    return cuda_status(cudaGetLastError());
}

}  // namespace rdcil
