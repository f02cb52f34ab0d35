// One evaluation of the synthetic-likelihood cost f(theta) with
// bootstrapping (Alg. 6; Sec. 3.3 eq. CIL_synth_kl, eq. cil:CF_synth):
//   1. simulate the N_syn patterns of one group at its parameter vector
//      (fresh initial states if asked, then the group's integrator);
//   2. split them (reading: one fixed partition) into s^1 = realisations
//      0..N_set-1 and s^2 = the other N_syn - N_set;
//   3. multi-feature correlation integral of s^1 against s^2 (Alg. 2 step
//      2.2): per feature the radii (the chosen law) and the bin matrix;
//   4. the data vector y~(theta) = C(R, s_data, s^2) with those radii
//      (eq. CIL_synth);
//   5. the bootstrap over resampled (s^1, s^2) pairs, the mean and
//      covariance of the concatenated vector, its Cholesky factor and the
//      cost at y~ (Alg. 6 steps 2-3 and 5).
// Host code only: every step is one of the library's own launches, in
// stream order, into caller-owned memory (no allocation, no synchronise).
#include <cstring>
#include "common.cuh"

using namespace rdcil;

namespace {

struct ScilPlan {
    const GroupDev *g;
    int64_t n_syn, n_set, n_rest, d_pat, ld_pat;
    int K;
    size_t off_mcil, mcil_bytes, off_bins_syn, off_bins_data, off_counts_syn, off_counts_data, off_radii_tmp,
        off_C_syn, off_nex, off_syn, syn_bytes, total;
};

size_t up256(size_t b) { return (b + 255) / 256 * 256; }

rd_status plan_of(const Handle &h, const scil_spec &sp, int64_t n_data, ScilPlan *P) {
    if (sp.group < 0 || sp.group >= h.n_groups) return RD_ERR_INVALID_ARG;
    const GroupDev &g = h.h_groups[sp.group];
    if (g.model == RD_RDODE) return RD_ERR_UNSUPPORTED;
    if (sp.n_species != 1 && sp.n_species != 2) return RD_ERR_INVALID_ARG;
    if (sp.features < 1 || sp.features > 63 || sp.M < 1 || sp.M > 32) return RD_ERR_INVALID_ARG;
    if (sp.law < 0 || sp.law > 2 || (sp.law == 0 && !(sp.b > 1.0))) return RD_ERR_INVALID_ARG;
    if (sp.integrator != 0 && sp.integrator != 1) return RD_ERR_INVALID_ARG;
    if (sp.n_set < 1 || sp.n_set >= g.n_real || n_data < 1 || sp.T < 2) return RD_ERR_INVALID_ARG;
    P->g = &g;
    P->n_syn = g.n_real;
    P->n_set = sp.n_set;
    P->n_rest = g.n_real - sp.n_set;
    P->d_pat = (int64_t)sp.n_species * g.G * g.G;
    P->ld_pat = 2ll * g.G * g.G;
    P->K = __builtin_popcount((unsigned)sp.features);
    if (P->K * sp.M > 96) return RD_ERR_INVALID_ARG;
    size_t m1 = 0, m2 = 0, sy = 0;
    rd_status st = mcil_workspace_size_rect(P->n_set, P->n_rest, g.G, g.G, sp.n_species, sp.features, sp.scale, sp.M,
                                            &m1);
    if (st) return st;
    st = mcil_workspace_size_rect(n_data, P->n_rest, g.G, g.G, sp.n_species, sp.features, sp.scale, sp.M, &m2);
    if (st) return st;
    st = synlik_workspace_size(P->n_set, P->n_rest, sp.M, sp.T, P->K, 1, &sy);
    if (st) return st;
    size_t off = 0;
    auto take = [&](size_t b) {
        const size_t o = off;
        off += up256(b);
        return o;
    };
    P->mcil_bytes = m1 > m2 ? m1 : m2;
    P->off_mcil = take(P->mcil_bytes);   // both correlation integrals, one after the other
    P->off_bins_syn = take((size_t)P->K * P->n_set * P->n_rest);
    P->off_bins_data = take((size_t)P->K * n_data * P->n_rest);
    P->off_counts_syn = take(sizeof(int64_t) * P->K * sp.M);
    P->off_counts_data = take(sizeof(int64_t) * P->K * sp.M);
    P->off_radii_tmp = take(sizeof(double) * P->K * (sp.M + 1));
    P->off_C_syn = take(sizeof(double) * P->K * sp.M);
    P->off_nex = take(sizeof(int64_t) * 2);
    P->syn_bytes = sy;
    P->off_syn = take(sy);
    P->total = off;
    return RD_OK;
}

}  // namespace

extern "C" rd_status scil_workspace_size(const rd_handle *hh, const scil_spec *spec, int64_t n_data, size_t *bytes) {
    if (!hh || !spec || !bytes) return RD_ERR_INVALID_ARG;
    ScilPlan P;
    rd_status st = plan_of(hh->h, *spec, n_data, &P);
    if (st) return st;
    *bytes = P.total;
    return RD_OK;
}

extern "C" rd_status scil_evaluate(rd_handle *hh, float *d_fields, const scil_spec *spec, const float *d_data,
                                   int64_t ld_data, int64_t n_data, double *d_radii, double *d_y_data,
                                   int64_t *d_Y, double *d_mu, double *d_cov, double *d_chol, double *d_scalars,
                                   uint8_t *d_active, int32_t *d_status, int64_t *d_n_exact, void *d_work,
                                   size_t work_bytes, void *stream) {
    if (!hh || !d_fields || !spec || !d_data || !d_radii || !d_y_data || !d_Y || !d_mu || !d_cov || !d_chol ||
        !d_scalars || !d_active || !d_status || !d_work)
        return RD_ERR_INVALID_ARG;
    if (((uintptr_t)d_work & 255) || ((uintptr_t)d_fields & 15)) return RD_ERR_INVALID_ARG;
    Handle &h = hh->h;
    const scil_spec &sp = *spec;
    ScilPlan P;
    rd_status st = plan_of(h, sp, n_data, &P);
    if (st) return st;
    if (P.total > work_bytes || ld_data < P.d_pat) return RD_ERR_INVALID_ARG;
    const GroupDev &g = *P.g;
    cudaStream_t s = (cudaStream_t)stream;
    char *w = (char *)d_work;

    // 1. simulate the N_syn patterns at theta
    if (sp.reinit) {
        st = launch_init_fields(g, d_fields, s);
        if (st) return st;
    }
    if (sp.integrator == 0) {
        st = group_is_resident(g) ? launch_integrate_group(g, d_fields, g.n_steps, nullptr, h.d_status, s)
                                  : launch_stream_group(h, g, d_fields, g.n_steps, nullptr, s);
    } else {
        if (!rkc_supported(g)) return RD_ERR_UNSUPPORTED;
        st = launch_rkc_group(g, h.d_rkc_tab, h.d_rkc_beta, d_fields, sp.rkc, nullptr, nullptr, h.d_status, s);
    }
    if (st) return st;

    // 2-3. s^1 = realisations 0..N_set-1, s^2 = the rest; radii and bins
    const float *S1 = d_fields + g.field_offset, *S2 = S1 + P.n_set * P.ld_pat;
    uint8_t *bins_syn = (uint8_t *)(w + P.off_bins_syn), *bins_data = (uint8_t *)(w + P.off_bins_data);
    int64_t *cnt_syn = (int64_t *)(w + P.off_counts_syn), *cnt_data = (int64_t *)(w + P.off_counts_data);
    int64_t *nex = d_n_exact ? d_n_exact : (int64_t *)(w + P.off_nex);
    double *C_syn = (double *)(w + P.off_C_syn);
    void *mw = w + P.off_mcil;
    switch (sp.law) {
        case 0:
            st = mcil_features_rect(S1, P.ld_pat, P.n_set, S2, P.ld_pat, P.n_rest, g.G, g.G, sp.n_species,
                                    sp.features, sp.scale, sp.b, sp.M, d_radii, bins_syn, cnt_syn, C_syn, nex, mw,
                                    P.mcil_bytes, stream);
            break;
        case 1:
            st = mcil_features_linear_rect(S1, P.ld_pat, P.n_set, S2, P.ld_pat, P.n_rest, g.G, g.G, sp.n_species,
                                           sp.features, sp.scale, sp.M, d_radii, bins_syn, cnt_syn, C_syn, nex, mw,
                                           P.mcil_bytes, stream);
            break;
        default:
            st = mcil_features_fitted_rect(S1, P.ld_pat, P.n_set, S2, P.ld_pat, P.n_rest, g.G, g.G, sp.n_species,
                                           sp.features, sp.scale, sp.M, d_radii, bins_syn, cnt_syn, C_syn, nex, mw,
                                           P.mcil_bytes, stream);
    }
    if (st) return st;

    // 4. y~ = C(R, s_data, s^2) with the radii of step 3
    st = mcil_features_given_rect(d_data, ld_data, n_data, S2, P.ld_pat, P.n_rest, g.G, g.G, sp.n_species,
                                  sp.features, sp.scale, sp.M, d_radii, (double *)(w + P.off_radii_tmp), bins_data,
                                  cnt_data, d_y_data, nex + 1, mw, P.mcil_bytes, stream);
    if (st) return st;

    // 5. bootstrap of (s^1, s^2), mean, covariance, Cholesky, cost at y~
    return synlik_stats_ws(bins_syn, P.K, P.n_set, P.n_rest, sp.M, sp.T, sp.seed, 1, d_y_data, d_Y, d_mu, d_cov,
                           d_chol, d_scalars, d_active, d_status, w + P.off_syn, P.syn_bytes, stream);
}
