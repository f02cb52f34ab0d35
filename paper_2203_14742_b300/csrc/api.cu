// C ABI entry points: handle management, argument validation, dispatch.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>
#include "common.cuh"

using namespace rdcil;

namespace rdcil {
rd_status adjoint_reserve(Handle &h);
void adjoint_release(Handle &h);
}  // namespace rdcil

// True if the handle holds a group of the 1-D model, which only
// rd_integrate_rkc integrates.
static bool has_rdode(const Handle &h) {
    for (int32_t i = 0; i < h.n_groups; ++i)
        if (h.h_groups[i].model == RD_RDODE) return true;
    return false;
}

static rd_status validate_groups(const rd_group *groups, int32_t n_groups) {
    if (!groups || n_groups < 1) return RD_ERR_INVALID_ARG;
    std::vector<std::pair<int64_t, int64_t>> iv;
    for (int32_t i = 0; i < n_groups; ++i) {
        const rd_group &g = groups[i];
        if (g.model != RD_FHN && g.model != RD_GM && g.model != RD_DIFF && g.model != RD_BZ && g.model != RD_RDODE)
            return RD_ERR_INVALID_ARG;
        if (g.model == RD_RDODE) {
            // 1-D: 32, 64, 128 or 256 nodes, no flags
            if ((g.G != 32 && g.G != 64 && g.G != 128 && g.G != 256) || g.flags) return RD_ERR_INVALID_ARG;
        }
        // resident stepper: G = 32, 64, 128; streaming stepper: any multiple of
        // 4 from 8 to 4096
        if (g.G < 8 || g.G > 4096 || (g.G & 3)) return RD_ERR_INVALID_ARG;
        const bool resident = !(g.flags & RD_GROUP_STREAM) && (g.G == 32 || g.G == 64 || g.G == 128);
        if ((g.flags & RD_GROUP_ADJOINT) && !resident) return RD_ERR_UNSUPPORTED;
        if (g.flags & ~(RD_GROUP_ADJOINT | RD_GROUP_STREAM)) return RD_ERR_INVALID_ARG;
        if (g.n_real < 1 || g.n_steps < 0 || g.field_offset < 0 || (g.field_offset & 3)) return RD_ERR_INVALID_ARG;
        if (!(g.dt > 0.0) || !std::isfinite(g.dt)) return RD_ERR_INVALID_ARG;
        for (double p : g.params)
            if (!std::isfinite(p)) return RD_ERR_INVALID_ARG;
        if (g.model == RD_GM && !(g.params[3] != 0.0)) return RD_ERR_INVALID_ARG;
        if (g.model == RD_BZ && !(g.params[2] != 0.0)) return RD_ERR_INVALID_ARG;
        if (!(g.noise_lo <= g.noise_hi)) return RD_ERR_INVALID_ARG;
        int64_t len = (int64_t)g.n_real * 2 * g.G * (g.model == RD_RDODE ? 1 : g.G);
        iv.emplace_back(g.field_offset, g.field_offset + len);
    }
    std::sort(iv.begin(), iv.end());
    for (size_t i = 1; i < iv.size(); ++i)
        if (iv[i].first < iv[i - 1].second) return RD_ERR_INVALID_ARG;
    return RD_OK;
}

extern "C" rd_status rd_init(const rd_group *groups, int32_t n_groups, float *d_fields, void *stream,
                             rd_handle **out) {
    if (!out || !d_fields || ((uintptr_t)d_fields & 15)) return RD_ERR_INVALID_ARG;
    *out = nullptr;
    rd_status st = validate_groups(groups, n_groups);
    if (st) return st;
    rd_handle *hh = new (std::nothrow) rd_handle();
    if (!hh) return RD_ERR_OOM;
    Handle &h = hh->h;
    if (cudaGetDevice(&h.device) != cudaSuccess) { delete hh; return RD_ERR_CUDA; }
    h.n_groups = n_groups;
    h.h_groups = new (std::nothrow) GroupDev[n_groups];
    if (!h.h_groups) { delete hh; return RD_ERR_OOM; }
    int64_t base = 0;
    for (int32_t i = 0; i < n_groups; ++i) {
        const rd_group &g = groups[i];
        GroupDev &d = h.h_groups[i];
        d.model = g.model; d.G = g.G; d.n_real = g.n_real; d.flags = g.flags;
        d.n_steps = g.n_steps; d.field_offset = g.field_offset; d.dt = g.dt;
        for (int k = 0; k < 6; ++k) d.p[k] = g.params[k];
        d.noise_lo = g.noise_lo; d.noise_hi = g.noise_hi; d.seed = g.seed;
        d.real_base = base;
        base += g.n_real;
    }
    h.n_real_total = base;
    if (cudaMalloc(&h.d_groups, sizeof(GroupDev) * n_groups) != cudaSuccess ||
        cudaMalloc(&h.d_status, sizeof(uint32_t)) != cudaSuccess) {
        rd_free(hh);
        return RD_ERR_OOM;
    }
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaMemcpyAsync(h.d_groups, h.h_groups, sizeof(GroupDev) * n_groups, cudaMemcpyHostToDevice, s) !=
            cudaSuccess ||
        cudaMemsetAsync(h.d_status, 0, sizeof(uint32_t), s) != cudaSuccess) {
        rd_free(hh);
        return RD_ERR_CUDA;
    }
    st = adjoint_reserve(h);
    if (st) { rd_free(hh); return st; }
    st = stream_reserve(h);
    if (st) { rd_free(hh); return st; }
    st = batch_plan_create(h.h_groups, n_groups, &h.batch);
    if (st) { rd_free(hh); return st; }
    st = tables_create(h, s);
    if (st) { rd_free(hh); return st; }
    st = launch_init_all(h.h_groups, n_groups, d_fields, s);
    if (st) { rd_free(hh); return st; }
    // the group table is read by the host copy only after this point; make
    // sure the pageable source of the async copy is no longer needed
    if (cudaStreamSynchronize(s) != cudaSuccess) { rd_free(hh); return RD_ERR_CUDA; }
    *out = hh;
    return RD_OK;
}

// ---------------------------------------------------------------------------
// step tables of the handle (formed once in rd_init, on the handle's device)
// ---------------------------------------------------------------------------
TableNeeds rdcil::table_needs(const GroupDev *groups, int n_groups) {
    TableNeeds n{false, {false, false, false}};
    for (int i = 0; i < n_groups; ++i) {
        n.rkc |= rkc_supported(groups[i]);
        if (imex_supported(groups[i])) n.imex[imex_table_index(groups[i].G)] = true;
    }
    return n;
}

static size_t up256(size_t b) { return (b + 255) / 256 * 256; }

size_t rdcil::table_bytes(const TableNeeds &n) {
    size_t b = n.rkc ? up256(rkc_table_bytes()) : 0;
    for (int gi = 0; gi < 3; ++gi)
        if (n.imex[gi]) {
            const int G = 32 << gi;
            b += up256(sizeof(float) * imex_table_floats(G)) + up256(sizeof(float) * imex_eo_table_floats(G));
        }
    return b;
}

rd_status rdcil::tables_create(Handle &h, cudaStream_t s) {
    const TableNeeds n = table_needs(h.h_groups, h.n_groups);
    const size_t bytes = table_bytes(n);
    h.table_bytes = 0;
    if (bytes == 0) return RD_OK;
    char *base = nullptr;
    if (cudaMalloc(&base, bytes) != cudaSuccess) return RD_ERR_OOM;
    h.d_tables = base;
    h.table_bytes = bytes;
    size_t off = 0;
    if (n.rkc) {
        h.d_rkc_tab = (float4 *)(base + off);
        h.d_rkc_beta = (double *)(base + off + sizeof(float4) * (size_t)(RD_RKC_S_MAX + 1) * (RD_RKC_S_MAX + 1));
        off += up256(rkc_table_bytes());
        rd_status st = rkc_tables_fill(h.d_rkc_tab, h.d_rkc_beta, s);
        if (st) return st;
    }
    for (int gi = 0; gi < 3; ++gi) {
        if (!n.imex[gi]) continue;
        const int G = 32 << gi;
        const size_t full = sizeof(float) * imex_table_floats(G);
        h.d_imex_tab[gi] = full ? (float *)(base + off) : nullptr;
        off += up256(full);
        h.d_imex_eo_tab[gi] = (float *)(base + off);
        off += up256(sizeof(float) * imex_eo_table_floats(G));
        rd_status st = imex_tables_fill(G, h.d_imex_tab[gi], h.d_imex_eo_tab[gi], s);
        if (st) return st;
    }
    return RD_OK;
}

void rdcil::tables_release(Handle &h) {
    if (h.d_tables) cudaFree(h.d_tables);
    h.d_tables = nullptr;
    h.d_rkc_tab = nullptr;
    h.d_rkc_beta = nullptr;
    for (int gi = 0; gi < 3; ++gi) h.d_imex_tab[gi] = h.d_imex_eo_tab[gi] = nullptr;
    h.table_bytes = 0;
}

extern "C" rd_status rd_tables_size(const rd_group *groups, int32_t n_groups, size_t *bytes) {
    if (!bytes) return RD_ERR_INVALID_ARG;
    rd_status st = validate_groups(groups, n_groups);
    if (st) return st;
    std::vector<GroupDev> gd(n_groups);
    for (int32_t i = 0; i < n_groups; ++i) {
        gd[i] = GroupDev{};
        gd[i].model = groups[i].model;
        gd[i].G = groups[i].G;
        gd[i].flags = groups[i].flags;
    }
    *bytes = table_bytes(table_needs(gd.data(), n_groups));
    return RD_OK;
}

extern "C" size_t rd_handle_table_bytes(const rd_handle *hh) { return hh ? hh->h.table_bytes : 0; }

extern "C" rd_status rd_set_params(rd_handle *hh, int32_t group, const double *params, void *stream) {
    if (!hh || !params) return RD_ERR_INVALID_ARG;
    Handle &h = hh->h;
    if (group < 0 || group >= h.n_groups) return RD_ERR_INVALID_ARG;
    GroupDev &g = h.h_groups[group];
    for (int k = 0; k < 6; ++k)
        if (!std::isfinite(params[k])) return RD_ERR_INVALID_ARG;
    if (g.model == RD_GM && !(params[3] != 0.0)) return RD_ERR_INVALID_ARG;
    if (g.model == RD_BZ && !(params[2] != 0.0)) return RD_ERR_INVALID_ARG;
    for (int k = 0; k < 6; ++k) g.p[k] = params[k];
    cudaStream_t s = (cudaStream_t)stream;
    // pageable source: the copy is staged before the call returns
    RD_CUDA_TRY(cudaMemcpyAsync(h.d_groups + group, &g, sizeof(GroupDev), cudaMemcpyHostToDevice, s));
    return batch_plan_set_group(h.batch, group, g, s);
}

extern "C" rd_status rd_set_seed(rd_handle *hh, int32_t group, uint64_t seed) {
    if (!hh || group < 0 || group >= hh->h.n_groups) return RD_ERR_INVALID_ARG;
    hh->h.h_groups[group].seed = seed;   // read on the host by every initial-state launch
    return RD_OK;
}

extern "C" rd_status rd_reinit(rd_handle *hh, float *d_fields, void *stream) {
    if (!hh || !d_fields || ((uintptr_t)d_fields & 15)) return RD_ERR_INVALID_ARG;
    return launch_init_all(hh->h.h_groups, hh->h.n_groups, d_fields, (cudaStream_t)stream);
}

extern "C" rd_status rd_set_stream_depth(rd_handle *hh, int32_t depth) {
    if (!hh || (depth != 1 && depth != 2 && depth != 4 && depth != 8)) return RD_ERR_INVALID_ARG;
    hh->h.stream_depth = depth;
    return RD_OK;
}

extern "C" int32_t rd_get_stream_depth(const rd_handle *hh) { return hh ? hh->h.stream_depth : -1; }

extern "C" rd_status rd_set_schedule(rd_handle *hh, int32_t mode) {
    if (!hh || mode < 0 || mode > 2) return RD_ERR_INVALID_ARG;
    hh->h.schedule = mode;
    return RD_OK;
}

extern "C" rd_status rd_integrate_batch(rd_handle *hh, float *d_fields, int64_t steps_override, double *d_residual,
                                        void *stream) {
    if (!hh || !d_fields || ((uintptr_t)d_fields & 15)) return RD_ERR_INVALID_ARG;
    Handle &h = hh->h;
    if (has_rdode(h)) return RD_ERR_UNSUPPORTED;
    cudaStream_t s = (cudaStream_t)stream;
    int n_res = 0;
    for (int32_t i = 0; i < h.n_groups; ++i) n_res += group_is_resident(h.h_groups[i]) ? 1 : 0;
    const bool persistent = h.schedule == 2 || (h.schedule == 0 && n_res > 1);
    if (persistent && n_res > 0) {
        rd_status st = launch_batch(h.batch, d_fields, steps_override, d_residual, h.d_status, s);
        if (st) return st;
    }
    for (int32_t i = 0; i < h.n_groups; ++i) {
        const GroupDev &g = h.h_groups[i];
        int64_t steps = steps_override >= 0 ? steps_override : g.n_steps;
        rd_status st = RD_OK;
        if (!group_is_resident(g))
            st = launch_stream_group(h, g, d_fields, steps, d_residual, s);
        else if (!persistent)
            st = launch_integrate_group(g, d_fields, steps, d_residual, h.d_status, s);
        if (st) return st;
    }
    return RD_OK;
}

extern "C" rd_status rd_integrate_reference(rd_handle *hh, float *d_fields, float *d_tmp, int64_t steps_override,
                                            void *stream) {
    if (!hh || !d_fields || !d_tmp) return RD_ERR_INVALID_ARG;
    Handle &h = hh->h;
    if (has_rdode(h)) return RD_ERR_UNSUPPORTED;
    for (int32_t i = 0; i < h.n_groups; ++i) {
        const GroupDev &g = h.h_groups[i];
        int64_t steps = steps_override >= 0 ? steps_override : g.n_steps;
        rd_status st = launch_integrate_reference(g, d_fields, d_tmp, steps, (cudaStream_t)stream);
        if (st) return st;
    }
    return RD_OK;
}

extern "C" rd_status rd_integrate_plain(rd_handle *hh, float *d_fields, float *d_tmp, int64_t steps_override,
                                        void *stream) {
    if (!hh || !d_fields || !d_tmp) return RD_ERR_INVALID_ARG;
    Handle &h = hh->h;
    if (has_rdode(h)) return RD_ERR_UNSUPPORTED;
    for (int32_t i = 0; i < h.n_groups; ++i) {
        const GroupDev &g = h.h_groups[i];
        int64_t steps = steps_override >= 0 ? steps_override : g.n_steps;
        rd_status st = launch_integrate_plain(g, d_fields, d_tmp, steps, (cudaStream_t)stream);
        if (st) return st;
    }
    return RD_OK;
}

extern "C" rd_status rd_integrate_f64(rd_handle *hh, double *d_fields64, double *d_tmp64, int64_t steps_override,
                                      void *stream) {
    if (!hh || !d_fields64 || !d_tmp64) return RD_ERR_INVALID_ARG;
    Handle &h = hh->h;
    if (has_rdode(h)) return RD_ERR_UNSUPPORTED;
    for (int32_t i = 0; i < h.n_groups; ++i) {
        const GroupDev &g = h.h_groups[i];
        int64_t steps = steps_override >= 0 ? steps_override : g.n_steps;
        rd_status st = launch_integrate_f64(g, d_fields64, d_tmp64, steps, (cudaStream_t)stream);
        if (st) return st;
    }
    return RD_OK;
}

extern "C" rd_status rd_integrate_rkc(rd_handle *hh, float *d_fields, const rd_rkc_opts *opts, int64_t *d_stats,
                                      double *d_residual, void *stream) {
    if (!hh || !d_fields || !opts) return RD_ERR_INVALID_ARG;
    const rd_rkc_opts &o = *opts;
    if (!(o.h0 > 0.0) || !std::isfinite(o.h0)) return RD_ERR_INVALID_ARG;
    if (o.s_fixed != 0 && (o.s_fixed < 2 || o.s_fixed > RD_RKC_S_MAX)) return RD_ERR_INVALID_ARG;
    if (o.s_fixed == 0) {
        if (!(o.rtol >= 0.0) || !(o.atol >= 0.0) || !(o.rtol + o.atol > 0.0)) return RD_ERR_INVALID_ARG;
        if (o.s_max < 2 || o.s_max > RD_RKC_S_MAX || o.max_attempts < 1) return RD_ERR_INVALID_ARG;
        if (!std::isfinite(o.t_end)) return RD_ERR_INVALID_ARG;
    } else if (o.n_fixed < 0) {
        return RD_ERR_INVALID_ARG;
    }
    Handle &h = hh->h;
    for (int gi = 0; gi < h.n_groups; ++gi)
        if (!rkc_supported(h.h_groups[gi])) return RD_ERR_UNSUPPORTED;
    cudaStream_t s = (cudaStream_t)stream;
    for (int gi = 0; gi < h.n_groups; ++gi) {
        rd_status st = launch_rkc_group(h.h_groups[gi], h.d_rkc_tab, h.d_rkc_beta, d_fields, o, d_stats, d_residual,
                                        h.d_status, s);
        if (st != RD_OK) return st;
    }
    return RD_OK;
}

extern "C" rd_status rd_integrate_imex(rd_handle *hh, float *d_fields, double *d_residual, void *stream) {
    if (!hh || !d_fields) return RD_ERR_INVALID_ARG;
    Handle &h = hh->h;
    for (int gi = 0; gi < h.n_groups; ++gi)
        if (!imex_supported(h.h_groups[gi])) return RD_ERR_UNSUPPORTED;
    cudaStream_t s = (cudaStream_t)stream;
    for (int gi = 0; gi < h.n_groups; ++gi) {
        const int gi2 = imex_table_index(h.h_groups[gi].G);
        rd_status st = launch_imex_group(h.h_groups[gi], h.d_imex_tab[gi2], h.d_imex_eo_tab[gi2], d_fields,
                                         d_residual, h.d_status, s);
        if (st != RD_OK) return st;
    }
    return RD_OK;
}

extern "C" int32_t rd_imex_n_variants(void) { return imex_n_variants(); }
extern "C" rd_status rd_imex_set_variant(int32_t G, int32_t variant) {
    return imex_set_variant(G, variant) ? RD_OK : RD_ERR_INVALID_ARG;
}
extern "C" int32_t rd_imex_get_variant(int32_t G) { return imex_get_variant(G); }

extern "C" int32_t rd_rkc_n_variants(void) { return rkc_n_variants(); }
extern "C" rd_status rd_rkc_set_variant(int32_t G, int32_t variant) {
    return rkc_set_variant(G, variant) ? RD_OK : RD_ERR_INVALID_ARG;
}
extern "C" int32_t rd_rkc_get_variant(int32_t G) { return rkc_get_variant(G); }

extern "C" rd_status rd_sync_status(rd_handle *hh, void *stream) {
    if (!hh) return RD_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    uint32_t v = 0;
    if (cudaMemcpyAsync(&v, hh->h.d_status, sizeof(v), cudaMemcpyDeviceToHost, s) != cudaSuccess) return RD_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return RD_ERR_CUDA;
    if (cudaMemsetAsync(hh->h.d_status, 0, sizeof(uint32_t), s) != cudaSuccess) return RD_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return RD_ERR_CUDA;
    if (v & ST_TIMEOUT) return RD_ERR_TIMEOUT;
    if (v & ST_NONFINITE) return RD_ERR_NONFINITE;
    if (v & ST_STEPFAIL) return RD_ERR_STEPSIZE;
    return RD_OK;
}

extern "C" int64_t rd_n_real_total(const rd_handle *hh) { return hh ? hh->h.n_real_total : -1; }

extern "C" void rd_free(rd_handle *hh) {
    if (!hh) return;
    Handle &h = hh->h;
    adjoint_release(h);
    stream_release(h);
    tables_release(h);
    batch_plan_free(h.batch);
    if (h.d_groups) cudaFree(h.d_groups);
    if (h.d_status) cudaFree(h.d_status);
    delete[] h.h_groups;
    delete hh;
}

extern "C" const char *rd_status_str(rd_status s) {
    switch (s) {
        case RD_OK: return "ok";
        case RD_ERR_INVALID_ARG: return "invalid argument";
        case RD_ERR_CUDA: return "CUDA error";
        case RD_ERR_NOT_PD: return "covariance not positive definite";
        case RD_ERR_TIMEOUT: return "device wait timed out";
        case RD_ERR_NONFINITE: return "non-finite field";
        case RD_ERR_UNSUPPORTED: return "unsupported configuration";
        case RD_ERR_OOM: return "out of device memory";
        case RD_ERR_STEPSIZE: return "adaptive step control gave up";
        default: return "unknown status";
    }
}

#include <atomic>
#include <map>
#include <mutex>
rd_status rdcil::smem_attr_of(const void *kern, int bytes) {
    static std::mutex mu;
    static std::map<std::pair<const void *, int>, int> done;   // (kernel, device) -> bytes set
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return RD_ERR_CUDA;
    std::lock_guard<std::mutex> lock(mu);
    auto it = done.find({kern, dev});
    if (it != done.end() && it->second >= bytes) return RD_OK;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) != cudaSuccess)
        return RD_ERR_CUDA;
    done[{kern, dev}] = bytes;
    return RD_OK;
}

static std::atomic<uint64_t> g_launches{0};
void rdcil::note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

extern "C" uint64_t rd_kernel_launches(void) { return g_launches.load(); }

extern "C" void rd_set_spin_limit(uint32_t polls) { set_gram_spin_limit(polls); }

// ---------------------------------------------------------------------------
// tile-shape variants and the autotuner
// ---------------------------------------------------------------------------
extern "C" int32_t rd_n_variants(void) { return n_variants(); }

extern "C" rd_status rd_variant_shape(int32_t G, int32_t variant, int32_t *shape) {
    int pk, ty, tx;
    if (!shape || !variant_shape(G, variant, &pk, &ty, &tx)) return RD_ERR_INVALID_ARG;
    shape[0] = pk;
    shape[1] = ty;
    shape[2] = tx;
    return RD_OK;
}

extern "C" rd_status rd_set_variant(int32_t model, int32_t G, int32_t variant) {
    if (model < 0 || model > 3 || (G != 32 && G != 64 && G != 128) || variant < 0 || variant >= n_variants())
        return RD_ERR_INVALID_ARG;
    set_variant_choice(model, G, variant);
    return RD_OK;
}

extern "C" int32_t rd_get_variant(int32_t model, int32_t G) {
    if (model < 0 || model > 3 || (G != 32 && G != 64 && G != 128)) return -1;
    return get_variant_choice(model, G);
}

extern "C" rd_status rd_autotune(rd_handle *hh, float *d_fields, int64_t steps, void *stream, int32_t *chosen) {
    if (!hh || !d_fields || steps < 1) return RD_ERR_INVALID_ARG;
    Handle &h = hh->h;
    if (has_rdode(h)) return RD_ERR_UNSUPPORTED;
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    RD_CUDA_TRY(cudaEventCreate(&e0));
    RD_CUDA_TRY(cudaEventCreate(&e1));
    rd_status st = RD_OK;
    for (int model = 0; model < 4 && st == RD_OK; ++model)
        for (int G : {32, 64, 128}) {
            // the largest group of this (model, G) class stands for the class
            int best_g = -1;
            for (int i = 0; i < h.n_groups; ++i)
                if (h.h_groups[i].model == model && h.h_groups[i].G == G && group_is_resident(h.h_groups[i]) &&
                    (best_g < 0 || h.h_groups[i].n_real > h.h_groups[best_g].n_real))
                    best_g = i;
            if (best_g < 0) continue;
            const GroupDev &g = h.h_groups[best_g];
            float best_ms = 1e30f;
            int best_v = get_variant_choice(model, G);
            for (int v = 0; v < n_variants() && st == RD_OK; ++v) {
                st = launch_integrate_variant(g, d_fields, steps, nullptr, h.d_status, s, v);   // warm
                if (st) break;
                float ms = 1e30f;
                for (int rep = 0; rep < 2 && st == RD_OK; ++rep) {
                    cudaEventRecord(e0, s);
                    st = launch_integrate_variant(g, d_fields, steps, nullptr, h.d_status, s, v);
                    cudaEventRecord(e1, s);
                    if (cudaEventSynchronize(e1) != cudaSuccess) { st = RD_ERR_CUDA; break; }
                    float t = 0.f;
                    cudaEventElapsedTime(&t, e0, e1);
                    ms = t < ms ? t : ms;
                }
                if (ms < best_ms) { best_ms = ms; best_v = v; }
            }
            set_variant_choice(model, G, best_v);
            if (chosen) chosen[model * 3 + (G == 32 ? 0 : G == 64 ? 1 : 2)] = best_v;
        }
    // streaming groups: the temporal depth, timed on the largest of them
    int best_s = -1;
    for (int i = 0; i < h.n_groups; ++i)
        if (!group_is_resident(h.h_groups[i]) &&
            (best_s < 0 || (double)h.h_groups[i].n_real * h.h_groups[i].G * h.h_groups[i].G >
                               (double)h.h_groups[best_s].n_real * h.h_groups[best_s].G * h.h_groups[best_s].G))
            best_s = i;
    if (best_s >= 0 && st == RD_OK) {
        const GroupDev &g = h.h_groups[best_s];
        float best_ms = 1e30f;
        int best_d = h.stream_depth;
        for (int d : {1, 2, 4, 8}) {
            h.stream_depth = d;
            st = launch_stream_group(h, g, d_fields, steps, nullptr, s);   // warm
            if (st) break;
            cudaEventRecord(e0, s);
            st = launch_stream_group(h, g, d_fields, steps, nullptr, s);
            cudaEventRecord(e1, s);
            if (st || cudaEventSynchronize(e1) != cudaSuccess) { st = st ? st : RD_ERR_CUDA; break; }
            float t = 0.f;
            cudaEventElapsedTime(&t, e0, e1);
            if (t < best_ms) { best_ms = t; best_d = d; }
        }
        h.stream_depth = best_d;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st) return st;
    // the tuning runs advanced the fields: restore the initial states
    return rd_reinit(hh, d_fields, stream);
}
