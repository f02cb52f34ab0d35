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
// (The workspace form synlik_stats_ws counts on the tensor cores instead,
//   boot_tc.cu, and runs bootstrap_kernel only as its fallback.)
// moments_kernel: one CTA per (chunk of resamples, problem): the integer
//   sums S_k, P_kl of the counts (64-bit atomics, exact in any order).
// stats_kernel: one CTA per problem.  Mean and covariance are the exact
//   rationals of the integer counts, rounded once; right-looking Cholesky
//   of the active block (each entry's terms in the plain definition's
//   order); log-determinant, Mahalanobis term and log-likelihood.
#include "common.cuh"

namespace rdcil {

// tensor-core bootstrap counts (boot_tc.cu)
size_t boot_workspace_bytes(int64_t n1, int64_t n2, int M, int T, int nf, int P);
void boot_set_mult_limit(int n);
rd_status launch_bootstrap_tc(const uint8_t *bins, int nf, int64_t n1, int64_t n2, int M, int T, uint64_t seed,
                              int P, int64_t *Y, void *work, size_t work_bytes, const uint32_t **flag_out,
                              cudaStream_t s);

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
                                                        unsigned long long *__restrict__ Y,
                                                        const uint32_t *__restrict__ only_if) {
    if (only_if && *(volatile const uint32_t *)only_if == 0u) return;   // the tensor cores counted
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

// Integer moments of the counts, split over chunks of MO_T resamples (one
// CTA per (chunk, problem)); partial sums meet in 64-bit atomics, exact in
// any order.  Accumulators (cleared by the caller), reusing the outputs:
//   mu_all  as uint64 [P][M]:     S_k  = sum_t Y[t][k]
//   cov_all as uint64 [P][M][M]:  P_kl = sum_t Y[t][k] Y[t][l]  (k <= l)
//   chol_all as uint64 [P][M][M], first M words: some Y[t][k] != Y[0][k]
static constexpr int MO_T = 32;

__global__ void moments_kernel(const int64_t *__restrict__ Yall, int M, int T, double *__restrict__ mu_all,
                               double *__restrict__ cov_all, double *__restrict__ chol_all) {
    __shared__ long long sy[MO_T * SYN_MAX_M];
    const int c = blockIdx.x, p = blockIdx.y;
    const int64_t *Y = Yall + (int64_t)p * T * M;
    const int t0 = c * MO_T, nt = min(MO_T, T - t0);
    for (int e = threadIdx.x; e < nt * M; e += blockDim.x) sy[e] = Y[(int64_t)t0 * M + e];
    __syncthreads();
    unsigned long long *S = reinterpret_cast<unsigned long long *>(mu_all) + (int64_t)p * M;
    unsigned long long *P = reinterpret_cast<unsigned long long *>(cov_all) + (int64_t)p * M * M;
    unsigned long long *D = reinterpret_cast<unsigned long long *>(chol_all) + (int64_t)p * M * M;
    for (int e = threadIdx.x; e < M * M; e += blockDim.x) {
        const int k = e / M, l = e - k * M;
        if (l < k) continue;
        long long acc = 0;
        for (int t = 0; t < nt; ++t) acc += sy[t * M + k] * sy[t * M + l];
        if (acc) atomicAdd(&P[e], (unsigned long long)acc);
    }
    for (int k = threadIdx.x; k < M; k += blockDim.x) {
        long long sum = 0;
        int diff = 0;
        const long long y0 = Y[k];
        for (int t = 0; t < nt; ++t) {
            sum += sy[t * M + k];
            diff |= (sy[t * M + k] != y0);
        }
        if (sum) atomicAdd(&S[k], (unsigned long long)sum);
        if (diff) atomicOr(&D[k], 1ull);
    }
}

__global__ void moments_clear_kernel(int M, int P, double *__restrict__ mu_all, double *__restrict__ cov_all,
                                     double *__restrict__ chol_all) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x, e0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (int64_t e = e0; e < (int64_t)P * M; e += stride) mu_all[e] = 0.0;
    for (int64_t e = e0; e < (int64_t)P * M * M; e += stride) {
        cov_all[e] = 0.0;
        chol_all[e] = 0.0;
    }
}

// One CTA per problem.  Mean mu_k = S_k / (T n_pairs) and covariance
// (T P_kl - S_k S_l) / (T (T-1) n_pairs^2), every integer converted to FP64
// once, then one division; active[k] = some count differs.  Cholesky of the
// active block right-looking: at step k the column k is finished (sqrt,
// divisions) and every later entry subtracts L_ik L_jk, so each entry
// subtracts its terms in increasing k, as in the row-by-row
// Cholesky-Banachiewicz of the plain definition, and the factor is the
// same; the forward solve for f likewise.
__global__ void stats_kernel(int M, int T, int64_t np, const double *__restrict__ y_obs_all,
                             double *__restrict__ mu_all, double *__restrict__ cov_all,
                             double *__restrict__ chol_all, double *__restrict__ scal_all,
                             uint8_t *__restrict__ active_all, int32_t *__restrict__ status_all,
                             const uint32_t *__restrict__ timed_out) {
    const int p = blockIdx.x;
    // M components: mu, cov, L, r/z, logs (double); S (int64); act, idx (int)
    extern __shared__ double smem_d[];
    double *mu = smem_d, *cov = mu + M, *L = cov + M * M, *r = L + M * M, *lg = r + M;
    long long *S = reinterpret_cast<long long *>(lg + M);
    int *act = reinterpret_cast<int *>(S + M), *idx = act + M;
    __shared__ int s_ma, s_st;
    const int tid = threadIdx.x;
    const unsigned long long *Su = reinterpret_cast<const unsigned long long *>(mu_all) + (int64_t)p * M;
    const unsigned long long *Pu = reinterpret_cast<const unsigned long long *>(cov_all) + (int64_t)p * M * M;
    const unsigned long long *Du = reinterpret_cast<const unsigned long long *>(chol_all) + (int64_t)p * M * M;
    for (int k = tid; k < M; k += blockDim.x) {
        S[k] = (long long)Su[k];
        act[k] = Du[k] ? 1 : 0;
    }
    for (int e = tid; e < M * M; e += blockDim.x) {
        const int k = e / M, l = e - k * M;
        L[e] = 0.0;
        if (l >= k) cov[e] = __longlong_as_double((long long)Pu[e]);   // raw P_kl bits for now
    }
    __syncthreads();
    const double dden = __ll2double_rn((long long)T * (long long)(T - 1) * np * np);
    for (int e = tid; e < M * M; e += blockDim.x) {
        const int k = e / M, l = e - k * M;
        if (l >= k) {
            const long long P = __double_as_longlong(cov[e]);
            const long long num = (long long)T * P - S[k] * S[l];
            cov[e] = __ddiv_rn(__ll2double_rn(num), dden);
        }
    }
    for (int k = tid; k < M; k += blockDim.x)
        mu[k] = __ddiv_rn(__ll2double_rn(S[k]), __dmul_rn((double)T, (double)np));
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
    // the active block, lower triangle, into L (updated in place)
    for (int e = tid; e < ma * ma; e += blockDim.x) {
        const int i = e / ma, j = e - i * ma;
        if (j <= i) L[i * M + j] = cov[idx[i] * M + idx[j]];
    }
    __syncthreads();
    for (int k = 0; k < ma; ++k) {
        if (tid == 0) {
            const double sd = L[k * M + k];
            if (!(sd > 0.0)) s_st = RD_ERR_NOT_PD;
            else L[k * M + k] = __dsqrt_rn(sd);
        }
        __syncthreads();
        if (s_st != RD_OK) break;
        const double lkk = L[k * M + k];
        for (int i = k + 1 + tid; i < ma; i += blockDim.x) L[i * M + k] = __ddiv_rn(L[i * M + k], lkk);
        __syncthreads();
        const int R = ma - k - 1;
        for (int e = tid; e < R * R; e += blockDim.x) {
            const int i = k + 1 + e / R, j = k + 1 + e % R;
            if (j <= i) L[i * M + j] = __dsub_rn(L[i * M + j], __dmul_rn(L[i * M + k], L[j * M + k]));
        }
        __syncthreads();
    }
    const int st = (timed_out && *timed_out) ? RD_ERR_TIMEOUT : s_st;
    const double nan = __longlong_as_double(0x7ff8000000000000ll);
    double logdet = nan, f = nan, ll = nan;
    if (s_st == RD_OK) {
        for (int i = tid; i < ma; i += blockDim.x) lg[i] = log(L[i * M + i]);
        const double *yo = y_obs_all ? y_obs_all + (int64_t)p * M : nullptr;
        if (yo)
            for (int i = tid; i < ma; i += blockDim.x) r[i] = __dsub_rn(yo[idx[i]], mu[idx[i]]);
        __syncthreads();
        if (yo) {
            for (int k = 0; k < ma; ++k) {
                if (tid == 0) r[k] = __ddiv_rn(r[k], L[k * M + k]);   // z_k
                __syncthreads();
                const double zk = r[k];
                for (int i = k + 1 + tid; i < ma; i += blockDim.x)
                    r[i] = __dsub_rn(r[i], __dmul_rn(L[i * M + k], zk));
                __syncthreads();
            }
        }
        if (tid == 0) {
            double ld = 0.0;
            for (int i = 0; i < ma; ++i) ld = __dadd_rn(ld, lg[i]);
            logdet = 2.0 * ld;
            if (yo) {
                double ff = 0.0;
                for (int i = 0; i < ma; ++i) ff = __dadd_rn(ff, __dmul_rn(r[i], r[i]));
                f = ff;
                // log(2 pi) correctly rounded
                ll = -0.5 * (ff + logdet + (double)ma * 1.8378770664093453);
            }
        }
    }
    __syncthreads();
    if (tid == 0) {
        double *sc = scal_all + (int64_t)p * 4;
        sc[0] = logdet; sc[1] = f; sc[2] = ll; sc[3] = (double)ma;
        status_all[p] = st;
    }
    for (int e = tid; e < M * M; e += blockDim.x) {
        const int i = e / M, j = e - i * M;
        // the factor occupies the leading ma x ma lower triangle
        chol_all[(int64_t)p * M * M + e] = (s_st == RD_OK && i < ma && j <= i) ? L[e] : 0.0;
        cov_all[(int64_t)p * M * M + e] = cov[e];
    }
    for (int k = tid; k < M; k += blockDim.x) {
        mu_all[(int64_t)p * M + k] = mu[k];
        active_all[(int64_t)p * M + k] = (uint8_t)act[k];
    }
}

}  // namespace rdcil

using namespace rdcil;

static rd_status synlik_check(int32_t n_feat, int64_t n1, int64_t n2, int32_t M, int32_t T, int32_t n_problems) {
    if (n1 < 1 || n2 < 1 || n1 + n2 > 49152 || M < 1 || M > 32 || T < 2 || T > 65535 || n_problems < 1 ||
        n_problems > 65535 || n_feat < 1 || n_feat * M > SYN_MAX_M)
        return RD_ERR_INVALID_ARG;
    // the exact covariance numerators T P_kl - S_k S_l stay in 64 bits
    double np = (double)n1 * (double)n2;
    if ((double)T * (double)T * np * np >= 4.6e18) return RD_ERR_INVALID_ARG;
    return RD_OK;
}

// SIMT bootstrap counts into Y (cleared by the caller); with only_if, the
// kernel counts only when *only_if is non-zero.
static rd_status launch_bootstrap_simt(const uint8_t *d_bins, int32_t n_feat, int64_t n1, int64_t n2, int32_t M,
                                       int32_t T, uint64_t seed, int32_t n_problems, int64_t *d_Y,
                                       const uint32_t *only_if, cudaStream_t s) {
    const size_t smem = (size_t)n2 * sizeof(uint16_t);
    if (smem > 48 * 1024) {
        {   // the size varies with the problem and the attribute is per device: set it per call
            RD_CUDA_TRY(cudaFuncSetAttribute(bootstrap_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem));
        }
    }
    // row blocks per resample: about eight CTAs of 256 threads per SM over
    // the whole launch, at least one row per warp
    int64_t RB = (8 * 148 + (int64_t)T * n_problems - 1) / ((int64_t)T * n_problems);
    if (RB > (n1 + 7) / 8) RB = (n1 + 7) / 8;
    if (RB < 1) RB = 1;
    dim3 g((unsigned)RB, (unsigned)T, (unsigned)n_problems);
    bootstrap_kernel<<<g, 256, smem, s>>>(d_bins, n_feat, (int)n1, (int)n2, M, T, seed, (int)RB,
                                         reinterpret_cast<unsigned long long *>(d_Y), only_if);
    note_launch();
    return cuda_status(cudaGetLastError());
}

static rd_status launch_stats(const int64_t *d_Y, int32_t Mt, int32_t T, int64_t np, int32_t n_problems,
                              const double *d_y_obs, double *d_mu, double *d_cov, double *d_chol, double *d_scalars,
                              uint8_t *d_active, int32_t *d_status, const uint32_t *timed_out, cudaStream_t s) {
    const size_t smem2 = sizeof(double) * (3 * (size_t)Mt + 2 * (size_t)Mt * Mt) + sizeof(long long) * Mt +
                         2 * sizeof(int) * Mt;
    if (smem2 > 48 * 1024) {
        {
            RD_CUDA_TRY(cudaFuncSetAttribute(stats_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem2));
        }
    }
    moments_clear_kernel<<<64, 256, 0, s>>>(Mt, n_problems, d_mu, d_cov, d_chol);
    note_launch();
    moments_kernel<<<dim3((unsigned)((T + MO_T - 1) / MO_T), (unsigned)n_problems), 256, 0, s>>>(
        d_Y, Mt, T, d_mu, d_cov, d_chol);
    note_launch();
    // 512 threads: the FP64 pipe is narrow and long-latency, and more
    // independent trailing-update products in flight hide it (same-box A/B
    // at 96 components, 1000 resamples, us per statistics call: 128 threads
    // 720, 256 540, 512 497, 1024 503)
    stats_kernel<<<(unsigned)n_problems, 512, smem2, s>>>(Mt, T, np, d_y_obs, d_mu, d_cov, d_chol, d_scalars,
                                                          d_active, d_status, timed_out);
    note_launch();
    return cuda_status(cudaGetLastError());
}

extern "C" rd_status synlik_stats_multi(const uint8_t *d_bins, int32_t n_feat, int64_t n1, int64_t n2, int32_t M,
                                        int32_t T, uint64_t seed, int32_t n_problems, const double *d_y_obs,
                                        int64_t *d_Y, double *d_mu, double *d_cov, double *d_chol, double *d_scalars,
                                        uint8_t *d_active, int32_t *d_status, void *stream) {
    if (!d_bins || !d_Y || !d_mu || !d_cov || !d_chol || !d_scalars || !d_active || !d_status)
        return RD_ERR_INVALID_ARG;
    rd_status st = synlik_check(n_feat, n1, n2, M, T, n_problems);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const int Mt = n_feat * M;
    RD_CUDA_TRY(cudaMemsetAsync(d_Y, 0, sizeof(int64_t) * (size_t)n_problems * T * Mt, s));
    st = launch_bootstrap_simt(d_bins, n_feat, n1, n2, M, T, seed, n_problems, d_Y, nullptr, s);
    if (st) return st;
    return launch_stats(d_Y, Mt, T, n1 * n2, n_problems, d_y_obs, d_mu, d_cov, d_chol, d_scalars, d_active,
                        d_status, nullptr, s);
}

static int64_t g_tc_min_pairs = (int64_t)1 << 22;

extern "C" void synlik_set_tc_min_pairs(int64_t n) { g_tc_min_pairs = n < 0 ? ((int64_t)1 << 22) : n; }

extern "C" void synlik_set_tc_mult_limit(int32_t n) { boot_set_mult_limit(n); }

extern "C" rd_status synlik_workspace_size(int64_t n1, int64_t n2, int32_t M, int32_t T, int32_t n_feat,
                                           int32_t n_problems, size_t *bytes) {
    if (!bytes) return RD_ERR_INVALID_ARG;
    rd_status st = synlik_check(n_feat, n1, n2, M, T, n_problems);
    if (st) return st;
    *bytes = boot_workspace_bytes(n1, n2, M, T, n_feat, n_problems);
    return RD_OK;
}

extern "C" rd_status synlik_stats_ws(const uint8_t *d_bins, int32_t n_feat, int64_t n1, int64_t n2, int32_t M,
                                     int32_t T, uint64_t seed, int32_t n_problems, const double *d_y_obs,
                                     int64_t *d_Y, double *d_mu, double *d_cov, double *d_chol, double *d_scalars,
                                     uint8_t *d_active, int32_t *d_status, void *d_work, size_t work_bytes,
                                     void *stream) {
    if (!d_bins || !d_Y || !d_mu || !d_cov || !d_chol || !d_scalars || !d_active || !d_status || !d_work)
        return RD_ERR_INVALID_ARG;
    rd_status st = synlik_check(n_feat, n1, n2, M, T, n_problems);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const int Mt = n_feat * M;
    RD_CUDA_TRY(cudaMemsetAsync(d_Y, 0, sizeof(int64_t) * (size_t)n_problems * T * Mt, s));
    // small problems (under g_tc_min_pairs resampled pairs per feature and
    // problem): the SIMT kernel is faster than the tensor-core set-up
    if ((double)n1 * (double)n2 * (double)T < (double)g_tc_min_pairs) {
        st = launch_bootstrap_simt(d_bins, n_feat, n1, n2, M, T, seed, n_problems, d_Y, nullptr, s);
        if (st) return st;
        return launch_stats(d_Y, Mt, T, n1 * n2, n_problems, d_y_obs, d_mu, d_cov, d_chol, d_scalars, d_active,
                            d_status, nullptr, s);
    }
    const uint32_t *flag = nullptr;
    st = launch_bootstrap_tc(d_bins, n_feat, n1, n2, M, T, seed, n_problems, d_Y, d_work, work_bytes, &flag, s);
    if (st) return st;
    st = launch_bootstrap_simt(d_bins, n_feat, n1, n2, M, T, seed, n_problems, d_Y, flag, s);
    if (st) return st;
    return launch_stats(d_Y, Mt, T, n1 * n2, n_problems, d_y_obs, d_mu, d_cov, d_chol, d_scalars, d_active,
                        d_status, flag + 1, s);
}

extern "C" rd_status synlik_stats(const uint8_t *d_bins, int64_t n1, int64_t n2, int32_t M, int32_t T,
                                  uint64_t seed, int32_t n_problems, const double *d_y_obs, int64_t *d_Y,
                                  double *d_mu, double *d_cov, double *d_chol, double *d_scalars,
                                  uint8_t *d_active, int32_t *d_status, void *stream) {
    return synlik_stats_multi(d_bins, 1, n1, n2, M, T, seed, n_problems, d_y_obs, d_Y, d_mu, d_cov, d_chol,
                              d_scalars, d_active, d_status, stream);
}
