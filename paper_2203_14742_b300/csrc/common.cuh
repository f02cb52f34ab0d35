// Internal declarations shared by the CUDA translation units of librdcil.
#pragma once
#include <atomic>
#include <cstdint>
#include <cstddef>
#include <cuda_runtime.h>
#include "../../include/rdcil.h"

namespace rdcil {

// Device status word bits (the handle's status word is an OR of these).
enum : uint32_t {
    ST_NONFINITE = 1u,
    ST_TIMEOUT = 2u,
    ST_STEPFAIL = 4u,
};

// SplitMix64 (Steele, Lea & Flood 2014): output number i of the stream that
// starts at state `seed` is the Stafford variant-13 finaliser applied to
// seed + (i+1)*0x9E3779B97F4A7C15.
__host__ __device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t i) {
    uint64_t z = seed + (i + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Device copy of one group plus derived FP32 coefficients.
struct GroupDev {
    int32_t model, G, n_real, flags;
    int64_t n_steps, field_offset;
    double dt;
    double p[6];
    double noise_lo, noise_hi;
    uint64_t seed;
    int64_t real_base;   // index of this group's first realisation overall
};

struct Handle {
    int device;
    int32_t n_groups;
    int64_t n_real_total;
    GroupDev *h_groups;       // host copy
    GroupDev *d_groups;       // device copy
    uint32_t *d_status;       // device status word
    // adjoint scratch (checkpoints + per-segment trajectory + lambda)
    float *d_ckpt;
    size_t ckpt_floats;
    double *d_adj_scratch;
    size_t adj_scratch_doubles;
    // adjoint scratch (adjoint.cu) and the persistent batch plan (stepper.cu)
    void *plan;
    void *batch;
    int32_t schedule;         // 0 auto, 1 one launch per group, 2 one persistent launch
    // streaming stepper (groups that are not resident, stream.cu)
    float *d_stream_tmp;      // the other HBM buffer of the ping-pong
    double *d_stream_part;    // residual partial sums
    int32_t stream_depth;     // Euler steps fused per launch (1, 2, 4 or 8)
    // step tables, formed in rd_init on the handle's device in one
    // allocation at d_tables (null when no group can use them): the
    // stabilised RK2 coefficients and stability bounds, and the cosine-basis
    // tables of the semi-implicit stepper per G = 32, 64, 128 (full products,
    // even/odd split; G = 128 has the even/odd table only)
    void *d_tables;
    float4 *d_rkc_tab;
    double *d_rkc_beta;
    float *d_imex_tab[3];
    float *d_imex_eo_tab[3];
    size_t table_bytes;
};

// Step tables a handle holds for its groups (rd_init allocates and fills
// them; tables_release frees them).
struct TableNeeds {
    bool rkc;          // some group can run the stabilised RK2
    bool imex[3];      // some group can run the semi-implicit stepper at G = 32 / 64 / 128
};
TableNeeds table_needs(const GroupDev *groups, int n_groups);
size_t table_bytes(const TableNeeds &n);
rd_status tables_create(Handle &h, cudaStream_t s);
void tables_release(Handle &h);

inline rd_status cuda_status(cudaError_t e) {
    return e == cudaSuccess ? RD_OK : RD_ERR_CUDA;
}

#define RD_CUDA_TRY(expr)                                  \
    do {                                                   \
        cudaError_t _e = (expr);                           \
        if (_e != cudaSuccess) return RD_ERR_CUDA;         \
    } while (0)

// Count of kernels this library has launched (its own kernels only).
void note_launch();

// Raise kernel `kern`'s dynamic shared-memory limit to `bytes` on the
// current device.  The attribute belongs to a (kernel, device) pair, so it
// is set the first time each pair needs it (api.cu keeps the record).
rd_status smem_attr_of(const void *kern, int bytes);
template <class K>
rd_status smem_attr(K kern, int bytes) {
    return smem_attr_of(reinterpret_cast<const void *>(kern), bytes);
}

// ---- launchers implemented in the kernel translation units --------------
rd_status launch_init_fields(const GroupDev &g, float *fields, cudaStream_t s);
rd_status launch_init_all(const GroupDev *groups, int n_groups, float *fields, cudaStream_t s);
rd_status launch_integrate_group(const GroupDev &g, float *fields, int64_t steps,
                                 double *residual, uint32_t *status, cudaStream_t s);
rd_status launch_integrate_reference(const GroupDev &g, float *fields, float *tmp,
                                     int64_t steps, cudaStream_t s);
rd_status launch_integrate_plain(const GroupDev &g, float *fields, float *tmp, int64_t steps, cudaStream_t s);
rd_status launch_integrate_f64(const GroupDev &g, double *fields, double *tmp, int64_t steps,
                               cudaStream_t s);
rd_status launch_record_group(const GroupDev &g, float *fields, float *traj, int64_t steps,
                              cudaStream_t s);
rd_status launch_integrate_variant(const GroupDev &g, float *fields, int64_t steps, double *residual,
                                   uint32_t *status, cudaStream_t s, int vi);
rd_status batch_plan_create(const GroupDev *groups, int n_groups, void **out);
rd_status batch_plan_set_group(void *plan, int i, const GroupDev &g, cudaStream_t s);
void batch_plan_free(void *plan);
rd_status launch_batch(void *plan, float *fields, int64_t steps_override, double *residual, uint32_t *status,
                       cudaStream_t s);
void set_variant_choice(int model, int G, int vi);
int get_variant_choice(int model, int G);
int n_variants();
bool group_is_resident(const GroupDev &g);
rd_status stream_reserve(Handle &h);
void stream_release(Handle &h);
rd_status launch_stream_group(const Handle &h, const GroupDev &g, float *fields, int64_t steps, double *residual,
                              cudaStream_t s);
void set_gram_spin_limit(uint32_t n);
bool variant_shape(int G, int vi, int *packed, int *TY, int *TX);
bool rkc_supported(const GroupDev &g);
bool rkc1d_supported(const GroupDev &g);
rd_status launch_rkc1d_group(const GroupDev &g, const float4 *tab, const double *beta, float *fields,
                             const rd_rkc_opts &o, int64_t *stats,
                             double *residual, uint32_t *status, cudaStream_t s);
rd_status launch_rdode_init(const GroupDev &g, float *fields, cudaStream_t s);
int rkc_n_variants();
bool rkc_set_variant(int G, int v);
int rkc_get_variant(int G);
rd_status launch_rkc_group(const GroupDev &g, const float4 *tab, const double *beta, float *fields,
                           const rd_rkc_opts &o, int64_t *stats, double *residual,
                           uint32_t *status, cudaStream_t s);
bool imex_supported(const GroupDev &g);
int imex_table_index(int G);   // 0, 1, 2 for G = 32, 64, 128; -1 otherwise
int imex_n_variants();
bool imex_set_variant(int G, int v);
int imex_get_variant(int G);
rd_status launch_imex_group(const GroupDev &g, const float *tab, const float *eo_tab, float *fields, double *residual,
                            uint32_t *status, cudaStream_t s);
rd_status rkc_tables_fill(float4 *tab, double *beta, cudaStream_t s);
size_t rkc_table_bytes();
rd_status imex_tables_fill(int G, float *tab, float *eo_tab, cudaStream_t s);
size_t imex_table_floats(int G);
size_t imex_eo_table_floats(int G);

}  // namespace rdcil

// the opaque handle of the C ABI
struct rd_handle {
    rdcil::Handle h;
};
