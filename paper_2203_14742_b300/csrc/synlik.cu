// Synthetic-likelihood statistics over resampled set pairs.
//
// Paper (arXiv 2203.14742): bootstrap resampling with replacement of each
// set, Alg. 5 step 2.1 (appendix A) and Alg. 6 steps 2.1-2.2; mean and
// covariance of the CIL vector, Alg. 1 step 3; cost eq. (cil:CF) and
// eq. (cil:CF_synth), reported with the Gaussian log-likelihood.
//
// bootstrap_kernel: one CTA per (row block, resample, problem).  Indices
//   come from the counter-based SplitMix64 stream; the per-radius counts of
//   the resampled pair set are accumulated with warp ballot + popc over the
//   stored bin indices K_ij and summed with integer atomics.
// stats_kernel: one CTA per problem.  Mean and covariance are the exact
//   rationals of the integer counts, formed with integer sums and rounded
//   once; Cholesky of the active block column by column (rows of a column in
//   parallel); log-determinant, Mahalanobis term and log-likelihood (M <= 32).
#include "common.cuh"

namespace rdcil {

static constexpr int SYN_MAX_M = 96;   // components of the (concatenated) CIL vector

__device__ __forceinline__ uint32_t lemire_index(uint64_t seed, uint64_t ctr, uint32_t n) {
    return (uint32_t)__umul64hi(splitmix64_at(seed, ctr), (uint64_t)n);
}

// One CTA per (row block, resample, problem).  The resampled column indices
// J (n2 of them, < 65536) are staged in shared memory; each warp walks the
// resampled rows a of its block (I[a] drawn per row, warp-uniform) and the
// columns in steps of 32, gathering K = bins[I[a]][J[b]] (the source row is
// reused from L1) and counting K > k for every radius with one ballot and
// popc per 32 pairs.  Counts meet in shared memory, then in Y (int64)
// through integer atomics, so the result does not depend on the order.
__global__ void __launch_bounds__(256) bootstrap_kernel(const uint8_t *__restrict__ bins, int nf, int n1, int n2,
                                                        int M, int T, uint64_t seed, int RB,
                                                        unsigned long long *__restrict__ Y) {
    extern __shared__ uint16_t sJ[];
    __shared__ unsigned int cnt[SYN_MAX_M];
    const int rb = blockIdx.x, t = blockIdx.y, p = blockIdx.z;
    const uint64_t sp = seed + (uint64_t)p;
    for (int b = threadIdx.x; b < n2; b += blockDim.x)
        sJ[b] = (uint16_t)lemire_index(sp, (((uint64_t)t * 2u + 1u) << 32) | (uint64_t)b, (uint32_t)n2);
    const int Mt = nf * M;
    for (int k = threadIdx.x; k < Mt; k += blockDim.x) cnt[k] = 0u;
    __syncthreads();
    const int a0 = (int)((int64_t)rb * n1 / RB), a1 = (int)((int64_t)(rb + 1) * n1 / RB);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const int64_t np = (int64_t)n1 * n2;
    for (int f = 0; f < nf; ++f) {
        const uint8_t *B = bins + ((int64_t)p * nf + f) * np;
        unsigned int c[32];
#pragma unroll
        for (int k = 0; k < 32; ++k) c[k] = 0u;
        for (int a = a0 + warp; a < a1; a += nw) {
            const uint32_t r = lemire_index(sp, (((uint64_t)t * 2u + 0u) << 32) | (uint64_t)a, (uint32_t)n1);
            const uint8_t *row = B + (int64_t)r * n2;
            for (int b0 = 0; b0 < n2; b0 += 32) {
                const int b = b0 + lane;
                const int K = b < n2 ? (int)__ldg(row + sJ[b]) : 0;
#pragma unroll
                for (int k = 0; k < 32; ++k)
                    if (k < M) c[k] += (unsigned)__popc(__ballot_sync(0xffffffffu, K > k));
            }
        }
        if (lane == 0) {
#pragma unroll
            for (int k = 0; k < 32; ++k)
                if (k < M && c[k]) atomicAdd(&cnt[f * M + k], c[k]);
        }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < Mt; k += blockDim.x)
        if (cnt[k]) atomicAdd(&Y[((int64_t)p * T + t) * Mt + k], (unsigned long long)cnt[k]);
}

__global__ void stats_kernel(const int64_t *__restrict__ Yall, int M, int T, int64_t np,
                             const double *__restrict__ y_obs_all, double *__restrict__ mu_all,
                             double *__restrict__ cov_all, double *__restrict__ chol_all,
                             double *__restrict__ scal_all, uint8_t *__restrict__ active_all,
                             int32_t *__restrict__ status_all) {
    const int p = blockIdx.x;
    const int64_t *Y = Yall + (int64_t)p * T * M;
    // M components: S, mu, cov, L, act, idx in dynamic shared memory
    extern __shared__ double smem_d[];
    double *mu = smem_d, *cov = mu + M, *L = cov + M * M;
    long long *S = reinterpret_cast<long long *>(L + M * M);
    int *act = reinterpret_cast<int *>(S + M), *idx = act + M;
    __shared__ int s_ma, s_st;
    const int tid = threadIdx.x;
    // mean: S_k / (T n_pairs), S_k an exact integer sum
    for (int k = tid; k < M; k += blockDim.x) {
        long long sum = 0;
        int same = 1;
        const long long y0 = Y[k];
        for (int t = 0; t < T; ++t) {
            const long long yy = Y[(int64_t)t * M + k];
            sum += yy;
            same &= (yy == y0);
        }
        S[k] = sum;
        mu[k] = __ddiv_rn(__ll2double_rn(sum), __dmul_rn((double)T, (double)np));
        act[k] = same ? 0 : 1;
    }
    __syncthreads();
    // covariance: (T P_kl - S_k S_l) / (T (T-1) n_pairs^2), exact integers,
    // each rounded to FP64 once, then one division
    const double dden = __ll2double_rn((long long)T * (long long)(T - 1) * np * np);
    for (int e = tid; e < M * M; e += blockDim.x) {
        const int k = e / M, l = e - k * M;
        if (l >= k) {
            long long P = 0;
            for (int t = 0; t < T; ++t) P += Y[(int64_t)t * M + k] * Y[(int64_t)t * M + l];
            const long long num = (long long)T * P - S[k] * S[l];
            cov[e] = __ddiv_rn(__ll2double_rn(num), dden);
        }
        L[e] = 0.0;
    }
    __syncthreads();
    for (int e = tid; e < M * M; e += blockDim.x) {
        const int k = e / M, l = e - k * M;
        if (l < k) cov[e] = cov[l * M + k];
    }
    if (tid == 0) {
        int ma = 0;
        for (int k = 0; k < M; ++k)
            if (act[k]) idx[ma++] = k;
        s_ma = ma;
        s_st = RD_OK;
    }
    __syncthreads();
    const int ma = s_ma;
    // Cholesky of the active block, column by column; every entry is the
    // same sequence of operations as row-by-row Cholesky-Banachiewicz
    // (inner sums in increasing k), so the factor is identical
    for (int j = 0; j < ma; ++j) {
        if (tid == 0) {
            double s = cov[idx[j] * M + idx[j]];
            for (int k = 0; k < j; ++k) s = __dsub_rn(s, __dmul_rn(L[j * M + k], L[j * M + k]));
            if (!(s > 0.0)) s_st = RD_ERR_NOT_PD;
            else L[j * M + j] = __dsqrt_rn(s);
        }
        __syncthreads();
        if (s_st != RD_OK) break;
        for (int i = j + 1 + tid; i < ma; i += blockDim.x) {
            double s = cov[idx[i] * M + idx[j]];
            for (int k = 0; k < j; ++k) s = __dsub_rn(s, __dmul_rn(L[i * M + k], L[j * M + k]));
            L[i * M + j] = __ddiv_rn(s, L[j * M + j]);
        }
        __syncthreads();
    }
    if (tid == 0) {
        const int st = s_st;
        const double nan = __longlong_as_double(0x7ff8000000000000ll);
        double logdet = nan, f = nan, ll = nan;
        if (st == RD_OK) {
            double ld = 0.0;
            for (int i = 0; i < ma; ++i) ld = __dadd_rn(ld, log(L[i * M + i]));
            logdet = 2.0 * ld;
            if (y_obs_all) {
                const double *yo = y_obs_all + (int64_t)p * M;
                double z[SYN_MAX_M];
                double ff = 0.0;
                for (int i = 0; i < ma; ++i) {
                    double s = __dsub_rn(yo[idx[i]], mu[idx[i]]);
                    for (int k = 0; k < i; ++k) s = __dsub_rn(s, __dmul_rn(L[i * M + k], z[k]));
                    z[i] = __ddiv_rn(s, L[i * M + i]);
                    ff = __dadd_rn(ff, __dmul_rn(z[i], z[i]));
                }
                f = ff;
                // log(2 pi) correctly rounded
                ll = -0.5 * (ff + logdet + (double)ma * 1.8378770664093453);
            }
        }
        double *sc = scal_all + (int64_t)p * 4;
        sc[0] = logdet; sc[1] = f; sc[2] = ll; sc[3] = (double)ma;
        status_all[p] = st;
    }
    __syncthreads();
    for (int e = tid; e < M * M; e += blockDim.x) {
        cov_all[(int64_t)p * M * M + e] = cov[e];
        chol_all[(int64_t)p * M * M + e] = L[e];
    }
    for (int k = tid; k < M; k += blockDim.x) {
        mu_all[(int64_t)p * M + k] = mu[k];
        active_all[(int64_t)p * M + k] = (uint8_t)act[k];
    }
}

}  // namespace rdcil

using namespace rdcil;

extern "C" rd_status synlik_stats_multi(const uint8_t *d_bins, int32_t n_feat, int64_t n1, int64_t n2, int32_t M,
                                        int32_t T, uint64_t seed, int32_t n_problems, const double *d_y_obs,
                                        int64_t *d_Y, double *d_mu, double *d_cov, double *d_chol, double *d_scalars,
                                        uint8_t *d_active, int32_t *d_status, void *stream) {
    if (!d_bins || !d_Y || !d_mu || !d_cov || !d_chol || !d_scalars || !d_active || !d_status)
        return RD_ERR_INVALID_ARG;
    if (n1 < 1 || n2 < 1 || n1 + n2 > 49152 || M < 1 || M > 32 || T < 2 || T > 65535 || n_problems < 1 ||
        n_problems > 65535 || n_feat < 1 || n_feat * M > SYN_MAX_M)
        return RD_ERR_INVALID_ARG;
    // the exact covariance numerators T P_kl - S_k S_l stay in 64 bits
    double np = (double)n1 * (double)n2;
    if ((double)T * (double)T * np * np >= 4.6e18) return RD_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const int Mt0 = n_feat * M;
    RD_CUDA_TRY(cudaMemsetAsync(d_Y, 0, sizeof(int64_t) * (size_t)n_problems * T * Mt0, s));
    const size_t smem = (size_t)n2 * sizeof(uint16_t);
    if (smem > 48 * 1024) {
        static size_t set = 0;
        if (smem > set) {
            RD_CUDA_TRY(cudaFuncSetAttribute(bootstrap_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem));
            set = smem;
        }
    }
    // row blocks per resample: about eight CTAs of 256 threads per SM over
    // the whole launch, at least one row per warp
    int64_t RB = (8 * 148 + (int64_t)T * n_problems - 1) / ((int64_t)T * n_problems);
    if (RB > (n1 + 7) / 8) RB = (n1 + 7) / 8;
    if (RB < 1) RB = 1;
    dim3 g((unsigned)RB, (unsigned)T, (unsigned)n_problems);
    bootstrap_kernel<<<g, 256, smem, s>>>(d_bins, n_feat, (int)n1, (int)n2, M, T, seed, (int)RB,
                                         reinterpret_cast<unsigned long long *>(d_Y));
    note_launch();
    const int Mt = n_feat * M;
    const size_t smem2 = sizeof(double) * ((size_t)Mt + 2 * (size_t)Mt * Mt) + sizeof(long long) * Mt +
                         2 * sizeof(int) * Mt;
    if (smem2 > 48 * 1024) {
        static size_t set2 = 0;
        if (smem2 > set2) {
            RD_CUDA_TRY(cudaFuncSetAttribute(stats_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem2));
            set2 = smem2;
        }
    }
    stats_kernel<<<(unsigned)n_problems, 256, smem2, s>>>(d_Y, Mt, T, n1 * n2, d_y_obs, d_mu, d_cov, d_chol,
                                                          d_scalars, d_active, d_status);
    note_launch();
    return cuda_status(cudaGetLastError());
}

extern "C" rd_status synlik_stats(const uint8_t *d_bins, int64_t n1, int64_t n2, int32_t M, int32_t T,
                                  uint64_t seed, int32_t n_problems, const double *d_y_obs, int64_t *d_Y,
                                  double *d_mu, double *d_cov, double *d_chol, double *d_scalars,
                                  uint8_t *d_active, int32_t *d_status, void *stream) {
    return synlik_stats_multi(d_bins, 1, n1, n2, M, T, seed, n_problems, d_y_obs, d_Y, d_mu, d_cov, d_chol,
                              d_scalars, d_active, d_status, stream);
}
