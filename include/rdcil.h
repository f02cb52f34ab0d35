/*
 * rdcil.h — C ABI of the B300-native Correlation Integral Likelihood hot path.
 *
 * Paper: A. Kazarnikov, R. Scheichl, H. Haario and A. Marciniak-Czochra,
 * "A Bayesian Approach to Modelling Biological Pattern Formation with
 * Limited Data", arXiv 2203.14742.  The calls follow the paper's statement of the problem:
 * simulate N patterns at a parameter vector from random initial states
 * (Sec. 2.1, Sec. 4.1), compare two pattern sets by the correlation sum at a
 * ladder of radii (eq. eCDF, eq. CIL), and estimate the mean and covariance
 * of the resulting vector over resampled set pairs to evaluate the cost
 * (Alg. 1 step 3, Alg. 5, eq. cil:CF, eq. cil:CF_synth).
 *
 * Conventions for every call
 *  - Pointers named d_* are CUDA device pointers on the current device, owned
 *    by the caller, contiguous, and must stay valid until the stream work
 *    that uses them has finished.  Host pointers are named without d_.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Every call only enqueues work and returns; nothing is
 *    synchronised unless the call's comment says so.
 *  - Argument errors are returned before any work is enqueued.  Errors that
 *    can only be seen on the device (non-finite fields, a non-positive-
 *    definite covariance) are written to the device status outputs named in
 *    each call, or to the handle's status word read by rd_sync_status.
 *  - No call throws; no call allocates device memory except rd_init.
 *  - Thread-compatible: one handle per host thread.
 */
#ifndef RDCIL_H
#define RDCIL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t rd_status;
#define RD_OK 0
#define RD_ERR_INVALID_ARG 1
#define RD_ERR_CUDA 2
#define RD_ERR_NOT_PD 3
#define RD_ERR_TIMEOUT 4
#define RD_ERR_NONFINITE 5
#define RD_ERR_UNSUPPORTED 6
#define RD_ERR_OOM 7
#define RD_ERR_STEPSIZE 8   /* adaptive step control gave up (rd_integrate_rkc) */

/* Reaction kinetics (Sec. 4.1), species order (u, v):
 *  RD_FHN  FitzHugh-Nagumo, eq. (introduction:0) with u = membrane potential
 *          w, v = recovery variable v, mu = 1:
 *            u_t = Du Lap u + u - u^3 - v,   v_t = Dv Lap v + eps (u - a v)
 *          params = (Du, Dv, eps, a); equilibrium (0, 0).
 *  RD_GM   Gierer-Meinhardt, eq. (gmSystem) with u = activator, v =
 *          inhibitor, mu_w = 1, mu = mu_v and an overall rate rho:
 *            u_t = Du Lap u + rho (u^2/v - mu u),  v_t = Dv Lap v + rho (u^2 - v)
 *          params = (Du, Dv, rho, mu); equilibrium (1/mu, 1/mu^2).
 *  RD_DIFF pure diffusion (reaction off), params = (Du, Dv, -, -); a
 *          degenerate case with closed-form solutions, used for checks.
 *  RD_BZ   the Brusselator ("BZ" in the paper's Table 1), eq. (bzSystem)
 *          with u = v, v = w:
 *            u_t = Du Lap u + A - (B+1) u + u^2 v,  v_t = Dv Lap v + B u - u^2 v
 *          params = (Du, Dv, A, B); equilibrium (A, B/A).
 *  RD_RDODE the 1-D reaction-diffusion-ODE model, Sec. 4.3 eq. (rdode), a
 *          non-diffusing u coupled to a diffusing w on G nodes of (0, 1),
 *          h = 1/(G-1), zero flux:
 *            u_t = -u - u w + m1 u^2/(1 + k u^2),
 *            w_t = D w_xx - m3 w - u w + m2 u^2/(1 + k u^2)
 *          params = (unused, D, m1, m2, m3, k); a realisation is
 *          [species u, w][x] (2*G floats); G = 32, 64, 128 or 256.
 *          Initial state (Sec. 4.3): u = uniform noise U(noise_lo, noise_hi)
 *          per node (SplitMix64 output number (r*2)*G + x of the group's
 *          stream, FP64 lo + (hi - lo) U), smoothed by RD_RDODE_SMOOTH passes
 *          of the 3-node moving average ((u_{x-1} + u_x) + u_{x+1}) / 3 with
 *          ghost = edge node, in FP64, rounded once to FP32; w = 0.  Only
 *          rd_integrate_rkc integrates it (explicit Euler would need
 *          dt < h^2/(2D), the paper integrates it with ROCK2). */
#define RD_FHN 0
#define RD_GM 1
#define RD_DIFF 2
#define RD_BZ 3
#define RD_RDODE 4
#define RD_RDODE_SMOOTH 10

/* group flags */
#define RD_GROUP_ADJOINT 1   /* reserve checkpoint memory for rd_adjoint */
#define RD_GROUP_STREAM 2    /* use the streaming stepper even where the resident one fits */

/* One parameter group: n_real realisations of one model on one G x G grid
 * with one parameter vector and one step count (a theta of Alg. 3/6 step 1).
 * Fields of realisation r live at d_fields + field_offset + r*2*G*G as
 * [species u, v][y][x] float32, row-major.  field_offset must be a multiple
 * of 4 floats (16-byte rows).  G: a multiple of 4 from 8 to 4096 (32, 64
 * and 128 run on the resident stepper, others on the streaming stepper, see
 * rd_set_stream_depth).  dt must be below
 * the explicit stability limit (h^2 / (4 max(Du, Dv)), h = 1/(G-1)); the
 * library does not check stability, but a blow-up is reported as
 * RD_ERR_NONFINITE.  RD_RDODE groups are 1-D: G nodes, realisation r at
 * d_fields + field_offset + r*2*G as [species u, w][x]; flags must be 0;
 * rd_integrate_batch, rd_integrate_reference, rd_integrate_f64,
 * rd_autotune and rd_adjoint return RD_ERR_UNSUPPORTED for a handle that
 * holds one. */
typedef struct rd_group {
    int32_t model;          /* RD_FHN / RD_GM / RD_DIFF / RD_BZ / RD_RDODE */
    int32_t G;              /* grid side (RD_RDODE: node count) */
    int32_t n_real;         /* realisations in this group (>= 1) */
    int32_t flags;          /* RD_GROUP_* */
    int64_t n_steps;        /* explicit Euler steps for rd_integrate_batch */
    int64_t field_offset;   /* floats from d_fields to realisation 0 */
    double dt;              /* time step */
    double params[6];       /* see the model list above (unused slots 0) */
    double noise_lo;        /* initial state = equilibrium + U(noise_lo, noise_hi) */
    double noise_hi;
    uint64_t seed;          /* counter-based noise stream of this group */
} rd_group;

typedef struct rd_handle rd_handle;

/* rd_init — plan a batch of groups and write their random initial states
 * (Sec. 4.1: homogeneous equilibrium plus small uniform noise).
 *
 * Initial value of (realisation r, species s, node c) of a group:
 *   U = (SplitMix64 output number ((r*2+s)*G*G + c) of stream group.seed
 *        >> 11) * 2^-53,
 *   value = float( x0_s + (noise_lo + (noise_hi - noise_lo) * U) )
 * evaluated in FP64 without fused multiply-add and rounded once to FP32.
 *
 * groups/n_groups: host array, copied (may be freed after the call).
 * d_fields: device float32 array holding every group's fields.
 * out: receives the handle; the handle owns the device copy of the group
 *   table, the status word, the step tables of rd_tables_size and (for
 *   RD_GROUP_ADJOINT groups) checkpoint memory.  Release with rd_free.
 * Returns RD_ERR_INVALID_ARG for an unsupported G, model, n_real < 1,
 * misaligned field_offset, dt <= 0 or overlapping groups; RD_ERR_OOM when
 * the handle's device memory cannot be allocated. */
rd_status rd_init(const rd_group *groups, int32_t n_groups, float *d_fields,
                  void *stream, rd_handle **out);

/* rd_tables_size — device bytes of the step tables rd_init forms for this
 * group list (host-only; no GPU needed): the stabilised RK2 coefficients
 * and stability bounds when some group can run rd_integrate_rkc (about
 * 1 MB), and the cosine-basis tables of rd_integrate_imex per grid side
 * 32, 64 or 128 present.  rd_init allocates and fills them once, on the current
 * device, so rd_integrate_rkc and rd_integrate_imex allocate nothing and
 * never synchronise (safe inside stream capture from the first call).
 * RD_ERR_INVALID_ARG as rd_init for an invalid group list.
 * rd_handle_table_bytes — the bytes a handle holds (0 for a null handle). */
rd_status rd_tables_size(const rd_group *groups, int32_t n_groups, size_t *bytes);
size_t rd_handle_table_bytes(const rd_handle *h);

/* rd_set_params — replace the parameter vector (theta, params[6] host
 * array, the layout of rd_group.params) of group `group` for every later
 * call on the handle (integration, adjoint).  The initial states are not
 * rewritten.  Enqueues the update on `stream` (a pageable host-to-device
 * copy: not for use inside stream capture).  RD_ERR_INVALID_ARG for a bad
 * group index or a parameter rd_init would refuse. */
rd_status rd_set_params(rd_handle *h, int32_t group, const double *params, void *stream);

/* rd_set_seed — replace the noise stream (rd_group.seed) of group `group`
 * for later rd_reinit / initial-state writes (fresh random initial states
 * per cost evaluation, Sec. 2.2: the likelihood is stochastic through them).
 * Host-side only; RD_ERR_INVALID_ARG for a bad group index. */
rd_status rd_set_seed(rd_handle *h, int32_t group, uint64_t seed);

/* rd_reinit — write the initial states again (same rule as rd_init) into
 * d_fields, for a handle created earlier.  No allocation. */
rd_status rd_reinit(rd_handle *h, float *d_fields, void *stream);

/* rd_integrate_batch — explicit Euler for every realisation of every group
 * (Sec. 5.1, method of lines App. B.1.1):
 *   w <- w + dt * F(w),  F = D * Lap_h(w) + R(w),
 *   Lap_h(w)_{y,x} = (w_{y,x+1} + w_{y,x-1} + w_{y+1,x} + w_{y-1,x} - 4 w_{y,x}) (G-1)^2
 * with mirrored Neumann ghosts (ghost = adjacent edge node).  FP32 state.
 * steps_override < 0: each group advances its own n_steps; >= 0: every
 *   group advances steps_override steps.
 * d_residual (nullable): [n_real_total][2] float64, the steady-state residual
 *   of the final state per realisation in group order: max |F| and
 *   sqrt(mean F^2) over both species, F evaluated in FP64 from the FP32
 *   state (the L-infinity criterion of Sec. 5.1).
 * A realisation whose final state is not finite sets RD_ERR_NONFINITE in the
 * handle's status word.  Integrating n then m steps equals integrating n+m. */
rd_status rd_integrate_batch(rd_handle *h, float *d_fields, int64_t steps_override,
                             double *d_residual, void *stream);

/* rd_set_schedule — how rd_integrate_batch launches the batch:
 *   0 (default) automatic: one persistent launch when the handle holds more
 *     than one group, otherwise one launch of the autotuned tile variant;
 *   1 one launch per group (tile variant per (model, G));
 *   2 one persistent launch for all groups: 256-thread CTAs, one per SM,
 *     pulling (group, realisation) items longest first from a device queue,
 *     so mixed models, grid sizes and step counts share the GPU.
 * All schedules give bit-identical fields; the residual's RMS is summed in
 * an order that follows the tiling and agrees to FP64 rounding. */
rd_status rd_set_schedule(rd_handle *h, int32_t mode);

/* Groups whose grid is not 32, 64 or 128 (or that carry RD_GROUP_STREAM)
 * run on the streaming stepper: one CTA per (32 x 64 tile, realisation)
 * loads the tile and a halo by TMA, advances it `depth` Euler steps in
 * shared memory (temporal blocking) and writes it back, ping-ponging
 * between d_fields and a handle-owned buffer (the result always ends in
 * d_fields).  Per node the arithmetic equals the resident stepper's, so a
 * group gives bit-identical fields on either.  They are not in the
 * persistent launch, and rd_adjoint does not support them.
 * rd_set_stream_depth: steps fused per launch, 1, 2, 4 (default) or 8.
 * rd_get_stream_depth: the current depth (-1 for a null handle). */
rd_status rd_set_stream_depth(rd_handle *h, int32_t depth);
int32_t rd_get_stream_depth(const rd_handle *h);

/* rd_integrate_reference — the plain path the batched stepper is measured
 * against: one realisation per launch, one Euler step per launch, state
 * round-tripping through global memory.  Same arithmetic contract as
 * rd_integrate_batch for FP32 (results agree to FP32 rounding, not bit for
 * bit: GM and BZ nodes go through their deviation form per step).  d_tmp:
 * caller scratch of 2*G*G floats of the largest group.
 * rd_integrate_plain — the same plain step with every realisation of a
 * group in one launch (one Euler step per launch, state through global
 * memory): the fields equal rd_integrate_reference's bit for bit.  d_tmp:
 * caller scratch of 2*G*G*n_real floats of the largest group.  Groups of
 * more than 65535 realisations: RD_ERR_UNSUPPORTED. */
rd_status rd_integrate_reference(rd_handle *h, float *d_fields, float *d_tmp,
                                 int64_t steps_override, void *stream);
rd_status rd_integrate_plain(rd_handle *h, float *d_fields, float *d_tmp,
                             int64_t steps_override, void *stream);

/* rd_integrate_f64 — the same Euler recursion on a float64 copy of the
 * fields (layout as d_fields, offsets in doubles), in the operation order
 *   Lap = ((((w_{x+1} + w_{x-1}) + w_{y+1}) + w_{y-1}) - 4 w) * (G-1)^2,
 *   F = D*Lap + R(w),  w <- w + dt*F
 * with every operation rounded separately (no fused multiply-add), so it
 * reproduces a plain FP64 evaluation of that order bit for bit.  d_tmp64:
 * caller scratch of the same size as d_fields64.  For checking only (FP64
 * is slow on this GPU). */
rd_status rd_integrate_f64(rd_handle *h, double *d_fields64, double *d_tmp64,
                           int64_t steps_override, void *stream);

/* ------------------------------------------------------------------------
 * Stabilised explicit second-order Runge-Kutta integration (App. B.2).
 *
 * The paper integrates the RD systems with ROCK2: stages by a three-term
 * recurrence, the stage number s from h times a Gershgorin bound of the
 * Jacobian's spectral radius, a weighted RMS error norm and a predictive
 * step-size controller with eta = 0.8.  ROCK2's recurrence coefficients are
 * not printed in the paper; this library uses the same family's member with
 * closed-form coefficients, the second-order Runge-Kutta-Chebyshev method
 * (damping 2/13), with T_j the Chebyshev polynomials of the first kind:
 *   w0 = 1 + (2/13)/s^2,  w1 = T_s'(w0)/T_s''(w0),
 *   b_j = T_j''(w0)/T_j'(w0)^2 (b_0 = b_1 = b_2),  a_j = 1 - b_j T_j(w0),
 *   Y_0 = w_n,  Y_1 = Y_0 + b_1 w1 h F(Y_0),
 *   Y_j = (1-mu_j-nu_j) Y_0 + mu_j Y_{j-1} + nu_j Y_{j-2}
 *         + mt_j h F(Y_{j-1}) + gt_j h F(Y_0),   j = 2..s,
 *   mu_j = 2 b_j w0/b_{j-1}, nu_j = -b_j/b_{j-2}, mt_j = 2 b_j w1/b_{j-1},
 *   gt_j = -a_{j-1} mt_j,   w_{n+1} = Y_s,
 * stable for h rho <= beta(s) = (1 + w0)/w1 (about 0.65 s^2).
 * Step control (adaptive mode), per realisation:
 *   rho   = max over nodes of the Gershgorin row sums of dF/dw at w_n (a node
 *           with n in-domain neighbours: |-n D (G-1)^2 + df/du| +
 *           n D (G-1)^2 + |df/dv|, likewise the v row);
 *   s     = the smallest s >= 2 with h rho <= beta(s); above s_max the step
 *           is cut to beta(s_max)/rho;
 *   est   = (12 (w_n - w_{n+1}) + 6 h (F(w_n) + F(w_{n+1}))) / 15;
 *   err   = sqrt(mean (est / (atol + rtol max(|w_n|, |w_{n+1}|)))^2), accept
 *           when err <= 1;
 *   h_new = fac h, fac = 0.8 err^(-1/3) (h_n/h_{n-1}) (err_{n-1}/err)^(1/3)
 *           after two consecutive accepted steps, 0.8 err^(-1/3) otherwise,
 *           err floored at 1e-10, fac in [0.1, 10] and <= 1 right after a
 *           rejection; the last step ends exactly at t_end.
 * FP32 state, FP64 control.  Groups must have G = 32, 64 or 128 (or be
 * RD_RDODE groups; RD_ERR_UNSUPPORTED otherwise, nothing is launched):
 * one CTA per realisation for G <= 64, one cluster of 4 CTAs for G = 128
 * (distributed shared memory for the rows between them).
 */
#define RD_RKC_S_MAX 256

typedef struct rd_rkc_opts {
    double t_end;          /* > 0: every group integrates from 0 to t_end;
                              <= 0: each group to its own dt * n_steps */
    double h0;             /* first trial step (adaptive) / the step (fixed), > 0 */
    double rtol, atol;     /* error weights (adaptive), >= 0, not both 0 */
    int32_t s_max;         /* stage limit, 2 .. RD_RKC_S_MAX (adaptive) */
    int32_t s_fixed;       /* 0: adaptive; 2 .. RD_RKC_S_MAX: fixed mode, n_fixed
                              steps of size h0 with s_fixed stages, no error
                              control (t_end, rtol, atol, s_max ignored) */
    int64_t n_fixed;       /* steps of the fixed mode, >= 0 */
    int64_t max_attempts;  /* attempted steps per realisation before giving up, >= 1 */
} rd_rkc_opts;

/* rd_integrate_rkc — integrate every realisation of every group in place
 * (d_fields as for rd_integrate_batch), one CTA per realisation running its
 * own step control on the device, groups launched in order on `stream`.
 * opts: host struct, read during the call.
 * d_stats (nullable): device int64 [n_real_total][4] = accepted steps,
 *   rejected steps, RHS evaluations (1 + the sum of s over all attempts),
 *   largest s used.
 * d_residual (nullable): as for rd_integrate_batch.
 * A realisation whose control gives up (more than max_attempts attempts, or
 * h below 1e-12 t_end) sets RD_ERR_STEPSIZE, one whose error or state turns
 * non-finite RD_ERR_NONFINITE, in the status word (rd_sync_status); its
 * state is left where it stopped.  Returns RD_ERR_INVALID_ARG for a bad
 * option, RD_ERR_UNSUPPORTED for a group it cannot run. */
rd_status rd_integrate_rkc(rd_handle *h, float *d_fields, const rd_rkc_opts *opts, int64_t *d_stats,
                           double *d_residual, void *stream);

/* rd_integrate_imex — semi-implicit (IMEX) Euler in place: every
 * realisation of every group takes its group's n_steps steps of size dt,
 *   (I - dt D_s L_h) w_s^{n+1} = w_s^n + dt R_s(u^n, v^n),   s = u, v,
 * diffusion implicit (L_h the 5-point Laplacian with mirrored Neumann
 * ghosts, App. B.1.1), reaction explicit (Sec. 4.1 kinetics).  Sec. 5.1 and
 * App. B.2 contrast explicit stepping with implicit stepping through linear
 * solves; here the solve is exact up to rounding, through the orthonormal
 * cosine (DCT-II) basis that diagonalises L_h, so dt is not bound by the
 * diffusive limit h^2 / (4 D) (the reaction still bounds it).
 * d_fields as for rd_integrate_batch; d_residual (nullable) as for
 * rd_integrate_batch, of the final state.  One CTA per realisation at
 * G = 32 and 64; at G = 128 one cluster of four CTAs per realisation (rows
 * split four ways, the transforms along y through distributed shared
 * memory).  Groups in order on `stream`.  Models RD_FHN, RD_GM, RD_DIFF,
 * RD_BZ on G = 32, 64 or 128; RD_ERR_UNSUPPORTED (nothing launched) for
 * any other group in h.  A
 * non-finite final state sets RD_ERR_NONFINITE in the status word when a
 * residual is asked for.  Precision: FP32 state and products; the
 * transform tables are formed in FP64 and rounded once. */
rd_status rd_integrate_imex(rd_handle *h, float *d_fields, double *d_residual, void *stream);

/* Output tiles of the rd_integrate_imex products (outputs per thread,
 * TM x TN): 0 = 4x4 (G = 64: 512 threads), 1 = 8x4, 2 = 4x8 (256),
 * 3 = 8x8 (128); G = 32 has a quarter of the threads.  Every tile runs the same
 * FMA chains, so the fields are bit-identical; the choice (per G,
 * process-wide) is a speed knob.  4 = the even/odd split: with the spectrum
 * ordered (even, odd) each product is two half-length sums over
 * Y[k] +- Y[G-1-k] (the cosine basis's symmetry), half the FMAs, its own
 * rounding (same tolerance, not bit-identical to 0-3); the default at both
 * G (256 threads at G = 64).  G = 128 has the even/odd cluster kernel
 * alone (no knob).  rd_imex_set_variant returns RD_ERR_INVALID_ARG for
 * another G or an unknown variant; rd_imex_get_variant returns -1 for
 * another G. */
int32_t rd_imex_n_variants(void);
rd_status rd_imex_set_variant(int32_t G, int32_t variant);
int32_t rd_imex_get_variant(int32_t G);

/* Tile shapes of the rd_integrate_rkc kernel (nodes per thread, TY x TX):
 * G = 32: 0 = 2x1 (512 threads, default), 1 = 4x1 (256), 2 = 2x2 (256);
 * G = 64: 0 = 4x2 (512 threads), 1 = 4x4 (256, default), 2 = 2x4 (512).
 * Per node every shape runs the same arithmetic, so a fixed schedule gives
 * bit-identical fields; in adaptive mode the error norm is summed in an
 * order that follows the tiling, so its last bits, and through the step
 * sizes the fields, may differ between shapes (a given shape is
 * deterministic).  The choice (per G, process-wide) is a speed knob.  rd_rkc_set_variant returns RD_ERR_INVALID_ARG for
 * another G or an unknown variant; rd_rkc_get_variant returns -1 for
 * another G. */
int32_t rd_rkc_n_variants(void);
rd_status rd_rkc_set_variant(int32_t G, int32_t variant);
int32_t rd_rkc_get_variant(int32_t G);

/* Tile-shape variants of the resident stepper.  Every variant performs the
 * same per-node arithmetic in the same order, so all give bit-identical
 * fields; the choice (per model and G, process-wide) only affects speed.
 * rd_n_variants: number of variants (indices 0..n-1, 0 = default).
 * rd_set_variant / rd_get_variant: choose / read the variant of (model, G).
 * rd_variant_shape: the tile shape of variant `variant` at grid side G
 *   (32, 64 or 128): shape = host int32[3] receiving {kind (0 = separate u
 *   and v tiles, 1 = float2 (u, v) tiles, 2 = separate tiles kept in TY + 1
 *   rotating row slots, which saves a register copy per node and step,
 *   3 = float2 (u, v) tiles in rotating row slots, whose neighbour sums are
 *   paired adds), TY, TX}.  RD_ERR_INVALID_ARG for an unknown G or variant or a null
 *   shape.
 * rd_autotune: time every variant on the largest group of each (model, G)
 *   class present in h for `steps` Euler steps, keep the fastest (and, if
 *   h holds streaming groups, the fastest temporal depth on the largest of
 *   them), then re-initialise d_fields (rd_reinit).  Synchronous.  chosen (nullable,
 *   host int32[12]) receives the choice per [model][G index 32/64/128]. */
int32_t rd_n_variants(void);
rd_status rd_set_variant(int32_t model, int32_t G, int32_t variant);
int32_t rd_get_variant(int32_t model, int32_t G);
rd_status rd_variant_shape(int32_t G, int32_t variant, int32_t *shape);
rd_status rd_autotune(rd_handle *h, float *d_fields, int64_t steps, void *stream, int32_t *chosen);

/* rd_sync_status — synchronise `stream`, read and clear the handle's device
 * status word.  Returns RD_OK, RD_ERR_NONFINITE, RD_ERR_TIMEOUT, or
 * RD_ERR_CUDA when the stream itself reported an error. */
rd_status rd_sync_status(rd_handle *h, void *stream);

/* rd_n_real_total — total realisations over all groups of the handle. */
int64_t rd_n_real_total(const rd_handle *h);

void rd_free(rd_handle *h);

/* rd_kernel_launches — number of CUDA kernels this library has launched in
 * this process so far (its own kernels only; memset/memcpy not counted). */
uint64_t rd_kernel_launches(void);

/* rd_set_spin_limit — testing hook for the failure path (the paper has no
 * counterpart).  The tensor-core Gram kernel's pipeline waits on its
 * mbarriers poll at most `polls` times before the kernel gives up, flags a
 * timeout (cil_features then reports *d_n_rechecked = -2) and returns with
 * its copies and tensor-core work drained; 0 restores the default (about
 * 4 million polls, seconds).  A tiny limit makes the waits run out on
 * purpose, so a test can check that the timeout is reported and that the
 * context stays usable.  Process-wide; not thread-safe against concurrent
 * CIL calls. */
void rd_set_spin_limit(uint32_t polls);

const char *rd_status_str(rd_status s);

/* ------------------------------------------------------------------------
 * Correlation integral (eq. eCDF, eq. CIL, Sec. 2.1).
 *
 * Pattern i of set 1 is the d floats at d_X1 + i*ld1 (likewise set 2), so a
 * set can be read straight out of the field array: one species of
 * realisation r is d = G*G floats at offset r*2*G*G, both species d = 2*G*G.
 *
 * Definitions (both sides of every comparison use them exactly):
 *   d2_ij = the real number sum_{t=0}^{d-1} (x_t - y_t)^2 of the FP32 inputs,
 *           rounded once to the nearest double (ties to even).  The paper
 *           defines the distance on the reals; this value depends on no
 *           evaluation order.  Patterns must be finite (a non-finite element
 *           makes d2 NaN and the pair's bin unspecified);
 *   R0    = sqrt(max_ij d2_ij)  (largest cross-set distance, Sec. 2.1);
 *   R_k   = R_{k-1} / b, k = 1..M (power law R0 b^-k), FP64;
 *   K_ij  = #{k : d2_ij < R_k * R_k}  (strict '<' of eq. eCDF);
 *   counts[k-1] = #{(i,j) : K_ij >= k} = n1*n2 * C(R_k).
 * d_radii_in (nullable): if given, the M radii R_1..R_M are taken from it
 *   (b ignored) and R0 is not computed (radii_out[0] = NaN).
 * Outputs: d_radii_out[M+1] = (R0, R_1..R_M); d_bins[n1*n2] uint8 K_ij
 *   (row i, column j); d_counts[M] int64; d_C (nullable) float64[M], the
 *   correlation integral vector C(R_k) = counts[k-1] / (n1 n2) (eq. CIL);
 *   d_n_rechecked (nullable) int64: pairs whose distance had to be
 *   evaluated exactly; -2 if the tensor-core stage timed out (a bounded
 *   wait expired; outputs invalid), -1 if an approximate interval
 *   straddled a threshold that the exact pass did not foresee (outputs
 *   invalid; not expected to occur).
 *
 * Method: the patterns are centred and split into bf16 hi + lo parts; a
 * tensor-core Gram product (FP32 accumulation; hi.hi + hi.lo + lo.hi, or
 * hi.hi alone when asked, see cil_set_gram_products) gives
 * d2 ~ |x|^2 + |y|^2 - 2 x.y for every pair together with a rigorous error
 * bound; pairs whose bound straddles a threshold (or the maximum) are
 * re-bounded by FP32 error-free sums and, if still undecided, evaluated
 * exactly (integer fixed-point accumulation of every x^2, y^2 and -2xy,
 * then one rounding), so K_ij and the counts equal the definition bit for
 * bit.
 * Limits: 1 <= n1, n2 <= 65535; 1 <= d <= 2^28; 1 <= M <= 32; b > 1.
 * d_work: caller scratch of cil_workspace_size bytes (256-byte aligned). */
rd_status cil_workspace_size(int64_t n1, int64_t n2, int64_t d, size_t *bytes);
rd_status cil_features(const float *d_X1, int64_t ld1, int64_t n1,
                       const float *d_X2, int64_t ld2, int64_t n2, int64_t d,
                       const double *d_radii_in, double b, int32_t M,
                       double *d_radii_out, uint8_t *d_bins, int64_t *d_counts,
                       double *d_C, int64_t *d_n_rechecked, void *d_work, size_t work_bytes,
                       void *stream);

/* cil_features_linear — the same correlation integral with the linear radii
 * law of Sec. 2.1 / Sec. 3.2 (Table 1 uses it for the MC and RD-ODE models):
 *   R0 = sqrt(max_ij d2_ij), R_min = sqrt(min_ij d2_ij) (the largest and the
 *   smallest cross-set distance, both from d2 as defined above),
 *   h = (R0 - R_min) / M,  R_k = R0 - k h  (k = 1..M),
 * every operation FP64 rounded to nearest.  Bins and counts exactly as for
 * cil_features (K_ij = #{k : d2_ij < R_k * R_k}); d_radii_out[0] = R0,
 * d_radii_out[M] = R_M.  The smallest distance is found exactly like the
 * largest (tier-1 bounds, error-free tier 2, exact tier 3 for the
 * candidates left).  Arguments, workspace and limits as for cil_features
 * (no b). */
rd_status cil_features_linear(const float *d_X1, int64_t ld1, int64_t n1,
                              const float *d_X2, int64_t ld2, int64_t n2, int64_t d, int32_t M,
                              double *d_radii_out, uint8_t *d_bins, int64_t *d_counts,
                              double *d_C, int64_t *d_n_rechecked, void *d_work, size_t work_bytes,
                              void *stream);

/* cil_features_fitted — the same correlation integral with the power law
 * whose decay is fitted to the range of the distances (Sec. 2.1, Sec. 3.2;
 * Table 1 uses it for the FHN, GM and BZ models): R0 and R_min the largest
 * and the smallest cross-set distance (from d2), b > 1 with
 * R_M / R0 = b^-M, R_k = R_{k-1} / b.  The paper gives the condition, not
 * how b is computed; here b is the smallest double whose M-th power, formed
 * as M - 1 sequential products rounded to nearest, reaches R0 / R_min,
 * found by halving [1, R0 / R_min] (mid = lo + (hi - lo) * 0.5, every
 * operation rounded to nearest) until the ends are adjacent doubles; b = 1
 * when R_min = R0 and b = +inf (every R_k = 0) when R_min = 0.  Bins and
 * counts as for cil_features; d_radii_out[0] = R0.  Arguments, workspace
 * and limits as for cil_features (no b). */
rd_status cil_features_fitted(const float *d_X1, int64_t ld1, int64_t n1,
                              const float *d_X2, int64_t ld2, int64_t n2, int64_t d, int32_t M,
                              double *d_radii_out, uint8_t *d_bins, int64_t *d_counts,
                              double *d_C, int64_t *d_n_rechecked, void *d_work, size_t work_bytes,
                              void *stream);

/* cil_features_static — cil_features for callers that cannot allocate
 * device memory on their hot path (cudaMalloc may synchronise the whole
 * device; some host applications own all device memory through their own
 * pool and forbid plug-in allocations).  The paper has no counterpart: this
 * is a deployment variant.  Same arguments, definitions and outputs as
 * cil_features, but no workspace: the scratch is one 16 MiB file-scope
 * device array that every GPU loading the library holds until the process
 * exits.  Limits: n1, n2 <= 128, d <= 8192 (RD_ERR_INVALID_ARG otherwise).
 * The first call on a device looks up the array's device address (with
 * that device current); make that first call before any stream capture.
 * Every call shares the one array: calls whose GPU work overlaps (other
 * streams, other host threads) race and must be serialised by the caller.
 * The call allocates nothing (no cudaMalloc/cudaFree, no allocating
 * library routine); it clears what it needs cleared itself. */
rd_status cil_features_static(const float *d_X1, int64_t ld1, int64_t n1,
                              const float *d_X2, int64_t ld2, int64_t n2, int64_t d,
                              const double *d_radii_in, double b, int32_t M,
                              double *d_radii_out, uint8_t *d_bins, int64_t *d_counts,
                              double *d_C, int64_t *d_n_rechecked, void *stream);

/* cil_debug_approx — checking entry point: for every pair, the approximate
 * d2 (A, from the centred bf16 hi/lo tensor-core Gram) and the rigorous
 * bound m with |A - d2| <= m that cil_features relies on, before any exact
 * evaluation.  d_A, d_m: float64 [n1*n2].  Same workspace as cil_features. */
rd_status cil_debug_approx(const float *d_X1, int64_t ld1, int64_t n1,
                           const float *d_X2, int64_t ld2, int64_t n2, int64_t d,
                           double *d_A, double *d_m, void *d_work, size_t work_bytes,
                           void *stream);

/* cil_gram_only — benchmarking entry point: re-run only the tensor-core Gram
 * stage on a workspace already packed by cil_features or cil_debug_approx
 * with the same (n1, n2, d) and product count.  *flops (host, nullable)
 * receives the FLOPs of the launch: (3 or 1) bf16 products x 2 x n1 x n2 x
 * d_padded. */
rd_status cil_gram_only(int64_t n1, int64_t n2, int64_t d, void *d_work, size_t work_bytes,
                        double *flops, void *stream);

/* cil_set_gram_products — the tensor-core Gram's form, process-wide, for
 * every correlation integral (cil_*, mcil_*, scil_evaluate) started after
 * the call: 3 = hi.hi + hi.lo + lo.hi (only lo.lo dropped: the tightest
 * interval, the fewest pairs re-evaluated), 1 = hi.hi alone (a third of the
 * tensor-core work and half its operand bytes; the dropped cross terms are
 * bounded by Cauchy-Schwarz, |hi_i| |lo_j| + |lo_i| |hi_j|, about 2^-8 of
 * |x_i| |x_j|, so more pairs near the radii are re-evaluated one by one:
 * worth it only when the distances sit far from the thresholds), 0 = the
 * default (three).  Results are identical in every form (the bounds are
 * rigorous and every undecided pair is re-evaluated); only the time
 * changes.  RD_ERR_INVALID_ARG for another value.
 * cil_gram_products — the form a correlation integral of (n1, n2, d) takes
 * under the current setting (1 or 3; -1 for sizes below 1).  Host only. */
rd_status cil_set_gram_products(int32_t mode);
int32_t cil_gram_products(int64_t n1, int64_t n2, int64_t d);

/* cil_queue_lengths — checking entry point: after a cil_features* call on
 * d_work with the same (n1, n2, d), the number of pairs that call sent to
 * tier 2 (FP32 error-free re-evaluation: their tier-1 interval met a
 * threshold or could hold the maximum) and to tier 3 (exact), as two int64
 * written to d_out (device), in stream order. */
rd_status cil_queue_lengths(int64_t n1, int64_t n2, int64_t d, const void *d_work, size_t work_bytes,
                            int64_t *d_out, void *stream);

/* cil_features_exact — the same outputs with every pair evaluated exactly
 * (no Gram product, no bounds).  Slow; for checking. */
/* cil_exact_d2 — checking entry point: d_out[e] = d2 (as defined above) of
 * pattern d_pairs[2e] of set 1 and pattern d_pairs[2e+1] of set 2, for
 * e < n_pairs (int64 index pairs, device memory; no bounds check of the
 * indices, which must lie inside the sets).  The same exact evaluation as
 * the correlation integral's last tier.  RD_ERR_INVALID_ARG for d outside
 * 1..2^28, ld < d or n_pairs < 0. */
rd_status cil_exact_d2(const float *d_X1, int64_t ld1, const float *d_X2, int64_t ld2, int64_t d,
                       const int64_t *d_pairs, int64_t n_pairs, double *d_out, void *stream);

rd_status cil_features_exact(const float *d_X1, int64_t ld1, int64_t n1,
                             const float *d_X2, int64_t ld2, int64_t n2, int64_t d,
                             const double *d_radii_in, double b, int32_t M,
                             double *d_radii_out, uint8_t *d_bins, int64_t *d_counts,
                             double *d_C, void *d_work, size_t work_bytes, void *stream);

/* ------------------------------------------------------------------------
 * Synthetic-likelihood statistics over resampled set pairs
 * (Alg. 5 step 2 / Alg. 6 step 2: resample each set with replacement;
 * Alg. 1 step 3: mean and covariance; eq. cil:CF / cil:CF_synth: cost).
 *
 * n_problems independent problems, packed back to back: problem p reads
 * d_bins + p*n1*n2 and d_y_obs + p*M, writes d_Y + p*T*M, d_mu + p*M,
 * d_cov + p*M*M, d_chol + p*M*M, d_scalars + p*4, d_active + p*M,
 * d_status + p.
 *
 * Resample t (0 <= t < T) of problem p draws set-1 index a (a < n1) as
 *   floor(SplitMix64 output number (((t*2+0) << 32) | a) of stream
 *         seed + p  *  n1 / 2^64)
 * (Lemire's multiply-shift), set-2 index b with ((t*2+1) << 32) | b.
 * Y[t][k-1] = sum_a sum_b [K_{I_a J_b} >= k]   (int64)
 * y_t = Y_t / (n1 n2);  mu = (1/T) sum_t y_t;
 * cov = (1/(T-1)) sum_t (y_t - mu)(y_t - mu)^T,
 * both formed exactly from the integer counts and rounded once:
 *   mu_k = S_k / (T n1 n2),  cov_kl = (T P_kl - S_k S_l) / (T (T-1) (n1 n2)^2)
 *   with S_k = sum_t Y[t][k], P_kl = sum_t Y[t][k] Y[t][l] (64-bit integers;
 *   numerator and denominator each converted to FP64 with rounding to
 *   nearest, then one FP64 division);
 * active[k] = 0 iff Y[t][k] is the same for every t;
 * chol = lower Cholesky factor of the active block of cov, packed into the
 *   leading M_act x M_act corner (rest zero);
 * scalars = (logdet, f, loglik, M_act) with logdet = 2 sum log L_ii,
 *   f = |L^-1 (y_obs - mu)_act|^2, loglik = -(f + logdet + M_act log 2pi)/2
 *   (f and loglik NaN when d_y_obs is NULL);
 * status[p] = RD_OK or RD_ERR_NOT_PD (active block not positive definite).
 * Limits: n1 + n2 <= 49152; 1 <= M <= 32; 2 <= T <= 65535; n_problems <= 65535;
 * (T n1 n2)^2 < 4.6e18.  Violations return RD_ERR_INVALID_ARG. */
rd_status synlik_stats(const uint8_t *d_bins, int64_t n1, int64_t n2, int32_t M,
                       int32_t T, uint64_t seed, int32_t n_problems,
                       const double *d_y_obs, int64_t *d_Y, double *d_mu,
                       double *d_cov, double *d_chol, double *d_scalars,
                       uint8_t *d_active, int32_t *d_status, void *stream);

/* synlik_stats_multi — the same statistics of a concatenated feature
 * vector (the multi-feature CIL of Sec. 3.1 / Alg. 2 with the bootstrap of
 * Alg. 5): d_bins is uint8 [n_problems][n_feat][n1][n2] (one bin matrix
 * per feature, e.g. from mcil_features); every resample draws one pair of
 * index sets (as above, stream seed + p) and counts it under every
 * feature, so d_Y is [n_problems][T][n_feat*M] with component f*M + k-1
 * the count of feature f at radius k; all other outputs as above with
 * n_feat*M components.  synlik_stats is the case n_feat = 1.
 * Limits as above and 1 <= n_feat*M <= 96. */
rd_status synlik_stats_multi(const uint8_t *d_bins, int32_t n_feat, int64_t n1, int64_t n2,
                             int32_t M, int32_t T, uint64_t seed, int32_t n_problems,
                             const double *d_y_obs, int64_t *d_Y, double *d_mu, double *d_cov,
                             double *d_chol, double *d_scalars, uint8_t *d_active,
                             int32_t *d_status, void *stream);

/* synlik_workspace_size / synlik_stats_ws — synlik_stats_multi with a
 * caller workspace (d_work, 256-byte aligned, synlik_workspace_size bytes),
 * which lets the bootstrap counts run on the tensor cores.  Same arguments,
 * definitions, outputs and limits as synlik_stats_multi; Y is identical.
 * Per resample the counts are the bilinear form
 *   Y[t][k-1] = sum_i c1[i] sum_j [K_ij >= k] c2[j]
 * with c1, c2 the multiplicities of the drawn indices (Alg. 5 step 2.1,
 * Alg. 6 steps 2.1-2.2): a product of the 0/1 matrices [K >= k] with the
 * multiplicities on tcgen05 (bf16 operands, FP32 accumulation; every value
 * is an integer below 2^24, so it is exact), then integer sums.  A
 * multiplicity above 256 (bf16's exact integer range; not expected in
 * practice) makes the call count with the SIMT kernel of
 * synlik_stats_multi instead, and so do problems under 2^22 resampled
 * pairs (n1 n2 T; synlik_set_tc_min_pairs changes the bound, process-wide,
 * a negative value restores it), where that kernel is faster.  status[p] =
 * RD_ERR_TIMEOUT if a bounded wait of the tensor-core stage gave up
 * (outputs invalid). */
rd_status synlik_workspace_size(int64_t n1, int64_t n2, int32_t M, int32_t T, int32_t n_feat,
                                int32_t n_problems, size_t *bytes);
void synlik_set_tc_min_pairs(int64_t n);
/* synlik_set_tc_mult_limit — the multiplicity above which synlik_stats_ws
 * counts with the SIMT kernel instead of the tensor cores (process-wide;
 * default and maximum 256, bf16's exact integer range; values outside
 * 1..256 restore the default).  A lower limit exercises that path. */
void synlik_set_tc_mult_limit(int32_t n);
rd_status synlik_stats_ws(const uint8_t *d_bins, int32_t n_feat, int64_t n1, int64_t n2,
                          int32_t M, int32_t T, uint64_t seed, int32_t n_problems,
                          const double *d_y_obs, int64_t *d_Y, double *d_mu, double *d_cov,
                          double *d_chol, double *d_scalars, uint8_t *d_active,
                          int32_t *d_status, void *d_work, size_t work_bytes, void *stream);

/* ------------------------------------------------------------------------
 * Multi-feature correlation integral (Sec. 3.1, Alg. 2 step 2.2; min-max
 * scaled data, Sec. 4).
 *
 * Patterns are n_species (1 or 2) fields of G x G floats, contiguous per
 * pattern: pattern i of set 1 starts at d_X1 + i*ld1 (likewise set 2), so
 * one or both species of a realisation are read in place from the field
 * array.  h = 1/(G-1), g = G-1.  The derivative patterns are forward
 * differences of each field, rounded to FP32 once (Dx: G x (G-1) values
 * s[y][x+1] - s[y][x], Dy: (G-1) x G values s[y+1][x] - s[y][x]).  With
 * q0, qx, qy the squared distances of the patterns and of their Dx and Dy
 * patterns as cil_features defines d2 (the exact real sum of squared
 * differences rounded once to the nearest double), and m0, mx, my the
 * maxima of |difference| with each difference in FP64 (rounded to nearest,
 * as in the squared distance), feature f (bit f of `features`) is the FP64
 * expression (every operation rounded to nearest, no FMA)
 *   0 L2      (eq. norm:L2)         squared value  q0
 *   1 Linf    (eq. norm:Linf)       value          m0
 *   2 W12     (eq. norm:W12)        squared value  (h^2 q0 + qx) + qy
 *   3 W12'    (eq. norm:W12prime)   value          (h sqrt(q0) + sqrt(qx)) + sqrt(qy)
 *   4 W1inf   (eq. norm:W1inf)      value          max(m0, max(g mx, g my))
 *   5 W1inf'  (eq. norm:W1infprime) value          (m0 + g mx) + g my
 * (h = 1/g and h^2 = 1/(g*g) rounded to nearest).  The L2 feature is the
 * plain Euclidean distance of cil_features (same bins and counts).  A
 * squared feature is decided like cil_features (R0 = sqrt(max), K = #{k :
 * V < R_k * R_k}); a value feature directly (R0 = max V, K = #{k : V <
 * R_k}); R_k = R_{k-1} / b, all in FP64.
 * scale != 0: every species of every pattern is first min-max scaled,
 *   s -> fl32(((double)s - min) / (max - min)) in FP64 (0 where max == min).
 * Outputs, for the K = popcount(features) selected features in ascending
 * order: d_radii_out [K][M+1] (R0, R_1..R_M); d_bins uint8 [K][n1][n2];
 * d_counts int64 [K][M]; d_C (nullable) float64 [K*M], the concatenated
 * correlation integral vector (counts / (n1 n2)); d_n_exact (nullable)
 * int64: pairs evaluated exactly (-2 if a tensor-core stage
 * timed out; outputs invalid).  Bins and counts equal the definition bit
 * for bit: squared distances come from the tensor-core Gram with rigorous
 * intervals, maxima from an FP32 pass (whose rounding is within 2^-23 of
 * the maximum), and every pair whose interval may hold a maximum or meets
 * a threshold is re-bounded (FP32 error-free sums, exact maxima) and if
 * still undecided evaluated exactly.
 * Workspace: d_work (256-byte aligned) of mcil_workspace_size bytes.
 * Limits: 1 <= n1, n2 <= 65535; 2 <= G <= 4096; n_species * G * G <= 2^28;
 * 1 <= M <= 32; b > 1; 1 <= features <= 63. */
rd_status mcil_workspace_size(int64_t n1, int64_t n2, int32_t G, int32_t n_species,
                              int32_t features, int32_t scale, int32_t M, size_t *bytes);
rd_status mcil_features(const float *d_X1, int64_t ld1, int64_t n1, const float *d_X2,
                        int64_t ld2, int64_t n2, int32_t G, int32_t n_species, int32_t features,
                        int32_t scale, double b, int32_t M, double *d_radii_out, uint8_t *d_bins,
                        int64_t *d_counts, double *d_C, int64_t *d_n_exact, void *d_work,
                        size_t work_bytes, void *stream);

/* mcil_workspace_size_rect / mcil_features_rect — the same on fields of Gy
 * x Gx nodes per species (a pattern is n_species * Gy * Gx floats;
 * 1 <= Gy <= 4096, 2 <= Gx <= 4096), h = 1/(Gx-1), g = Gx-1.  Gy = 1 gives
 * the 1-D patterns of the reaction-diffusion-ODE model (Sec. 4.3): no y
 * differences, so qy = my = 0 and the features are the 1-D discrete norms
 * up to a constant factor per feature (which leaves the bins unchanged).
 * Sec. 5.2 takes the derivative-based norms of that model on w alone: call
 * once with both species for L2 and Linf and once with the w rows for the
 * W features.  mcil_features(G) = mcil_features_rect(Gy = Gx = G). */
rd_status mcil_workspace_size_rect(int64_t n1, int64_t n2, int32_t Gy, int32_t Gx, int32_t n_species,
                                   int32_t features, int32_t scale, int32_t M, size_t *bytes);
rd_status mcil_features_rect(const float *d_X1, int64_t ld1, int64_t n1, const float *d_X2,
                             int64_t ld2, int64_t n2, int32_t Gy, int32_t Gx, int32_t n_species,
                             int32_t features, int32_t scale, double b, int32_t M, double *d_radii_out,
                             uint8_t *d_bins, int64_t *d_counts, double *d_C, int64_t *d_n_exact,
                             void *d_work, size_t work_bytes, void *stream);

/* mcil_features_linear_rect — mcil_features_rect with the linear radii law
 * of Sec. 2.1 / Sec. 3.2 per feature (Table 1 pairs it with the MC and
 * RD-ODE models): R0 as above, R_min = sqrt(min V) for a squared feature
 * and min V for a value feature (min over all n1 n2 pairs), h = (R0 -
 * R_min) / M, R_k = R0 - k h, every operation FP64 rounded to nearest
 * (k h first, then the subtraction).  The smallest value of each feature
 * is found exactly like the largest: the pairs whose interval may hold it
 * are re-bounded and, if still undecided, evaluated exactly.  Bins, counts, outputs, workspace (mcil_workspace_size_rect) and
 * limits as for mcil_features_rect; no b. */
rd_status mcil_features_linear_rect(const float *d_X1, int64_t ld1, int64_t n1, const float *d_X2,
                                    int64_t ld2, int64_t n2, int32_t Gy, int32_t Gx, int32_t n_species,
                                    int32_t features, int32_t scale, int32_t M, double *d_radii_out,
                                    uint8_t *d_bins, int64_t *d_counts, double *d_C, int64_t *d_n_exact,
                                    void *d_work, size_t work_bytes, void *stream);

/* mcil_features_fitted_rect — mcil_features_rect with the power law fitted
 * to each feature's range (Sec. 2.1 / Sec. 3.2): R0 and R_min as for
 * mcil_features_linear_rect, b the fitted decay of cil_features_fitted
 * (the smallest double whose sequentially rounded M-th power reaches
 * R0 / R_min), R_k = R_{k-1} / b.  Everything else as for
 * mcil_features_rect; no b. */
rd_status mcil_features_fitted_rect(const float *d_X1, int64_t ld1, int64_t n1, const float *d_X2,
                                    int64_t ld2, int64_t n2, int32_t Gy, int32_t Gx, int32_t n_species,
                                    int32_t features, int32_t scale, int32_t M, double *d_radii_out,
                                    uint8_t *d_bins, int64_t *d_counts, double *d_C, int64_t *d_n_exact,
                                    void *d_work, size_t work_bytes, void *stream);

/* ------------------------------------------------------------------------
 * Synthetic correlation integral likelihood with bootstrapping (Alg. 6,
 * Sec. 3.3): one evaluation of the cost f(theta) as one call.
 *
 *   1. simulate the N_syn = n_real patterns of group `group` at its
 *      parameter vector (rd_set_params): with reinit, first the initial
 *      states of that group (rd_reinit's rule, the group's seed,
 *      rd_set_seed), then integrator 0 = explicit Euler (the group's n_steps
 *      of dt, rd_integrate_batch's arithmetic) or 1 = the adaptive
 *      stabilised RK2 of rd_integrate_rkc with `rkc`;
 *   2. (reading of "from the remaining patterns") one fixed partition:
 *      s^1 = realisations 0..n_set-1, s^2 = realisations n_set..N_syn-1;
 *   3. the multi-feature correlation integral of s^1 against s^2 (as
 *      mcil_features_rect / _linear_rect / _fitted_rect for law 0 / 1 / 2,
 *      the power law taking b): d_radii [K][M+1] and the bin matrices;
 *   4. y~(theta) = C(R_m, s_data, s^2) (eq. CIL_synth) with those radii:
 *      d_y_data [K*M], the concatenated vector;
 *   5. the bootstrap (Alg. 6 step 2, each part resampled with replacement
 *      at its own size, synlik_stats_multi's index rule with stream seed),
 *      T resamples: d_Y [T][K*M] counts, d_mu, d_cov, d_chol [K*M][K*M],
 *      d_scalars = (logdet, f, loglik, M_act) with f = (y~ - mu)^T
 *      Sigma^-1 (y~ - mu) on the active block (eq. cil:CF_synth),
 *      d_active, d_status [1] as synlik_stats_ws.
 * K = popcount(features).  Patterns: n_species = 1 (u only, G*G floats of
 * each realisation) or 2 (both species, 2*G*G); data pattern i at d_data +
 * i*ld_data with the same layout (ld_data >= n_species*G*G).  d_fields is
 * the handle's field array (the group's patterns are read in place and
 * left integrated).  d_n_exact (nullable) int64[2]: pairs evaluated exactly
 * in steps 3 and 4 (-2: a tensor-core stage timed out).  d_work: caller
 * scratch of scil_workspace_size bytes (256-byte aligned).  Asynchronous on
 * `stream`, no allocation, no synchronisation.  Limits: 1 <= n_set <
 * N_syn, n_data >= 1, T >= 2, K*M <= 96 and those of the calls above;
 * RD_ERR_UNSUPPORTED for an RD_RDODE group. */
typedef struct scil_spec {
    int32_t group;        /* the group simulated at theta */
    int32_t integrator;   /* 0 explicit Euler, 1 adaptive stabilised RK2 */
    rd_rkc_opts rkc;      /* integrator 1 */
    int64_t n_set;        /* N_set: size of s^1 */
    int32_t n_species;    /* 1 or 2 */
    int32_t features;     /* bit f = feature f of mcil_features */
    int32_t scale;        /* nonzero: min-max scaled patterns (Sec. 4) */
    int32_t law;          /* 0 power law with b, 1 linear, 2 power law fitted to the range */
    double b;             /* law 0 */
    int32_t M;            /* radii per feature */
    int32_t T;            /* n_CIL resamples */
    uint64_t seed;        /* resampling stream */
    int32_t reinit;       /* nonzero: write fresh initial states first */
    int32_t pad;
} scil_spec;

rd_status scil_workspace_size(const rd_handle *h, const scil_spec *spec, int64_t n_data, size_t *bytes);
rd_status scil_evaluate(rd_handle *h, float *d_fields, const scil_spec *spec, const float *d_data,
                        int64_t ld_data, int64_t n_data, double *d_radii, double *d_y_data, int64_t *d_Y,
                        double *d_mu, double *d_cov, double *d_chol, double *d_scalars, uint8_t *d_active,
                        int32_t *d_status, int64_t *d_n_exact, void *d_work, size_t work_bytes, void *stream);

/* mcil_features_given_rect — mcil_features_rect with given radii:
 * d_radii_in [K][M+1] per selected feature (R0 first, copied to
 * d_radii_out and not used; R_1..R_M), thresholds R_k * R_k for the squared
 * features and R_k for the others, bins and counts as mcil_features_rect
 * (the data vector of Alg. 6 step 5, eq. CIL_synth).  No b. */
rd_status mcil_features_given_rect(const float *d_X1, int64_t ld1, int64_t n1, const float *d_X2,
                                   int64_t ld2, int64_t n2, int32_t Gy, int32_t Gx, int32_t n_species,
                                   int32_t features, int32_t scale, int32_t M, const double *d_radii_in,
                                   double *d_radii_out, uint8_t *d_bins, int64_t *d_counts, double *d_C,
                                   int64_t *d_n_exact, void *d_work, size_t work_bytes, void *stream);

/* ------------------------------------------------------------------------
 * Adjoint: gradient of a sigmoid-smoothed correlation integral with respect
 * to the four parameters of one group (the paper itself is gradient-free;
 * this serves proposal construction only, the likelihood keeps the exact
 * indicator counts of eq. eCDF).
 *
 *   C_k  = (1/(n1 n2)) sum_ij sigma((R_k - d_ij)/tau_k),  tau_k = tau_frac R_k,
 *   L    = sum_k cot_k C_k,
 * d_ij the Euclidean distance of the patterns (species_mask bit 0 = u,
 * bit 1 = v, concatenated) of realisations set1[i] and set2[j] of the group
 * after n_steps Euler steps from d_fields0 (the group's initial states,
 * same layout as d_fields, held fixed).  Radii are held fixed.
 * Reverse mode of the FP32 Euler recursion: the forward pass stores a
 * checkpoint every ceil(sqrt(n_steps)) steps, the reverse pass recomputes
 * each segment from its checkpoint and runs
 *   lambda_n = lambda_{n+1} + dt J_F(w_n)^T lambda_{n+1},
 *   g       += dt (dF/dtheta(w_n))^T lambda_{n+1}   (accumulated in FP64).
 * Outputs: d_C[M] (float64, nullable), d_grad[4] (float64).  Forward
 * only: with d_cotangent and d_grad both NULL the call integrates once
 * (no checkpoints, no reverse sweep) and writes d_C (then required).
 * Requires the group to carry RD_GROUP_ADJOINT (checkpoints reserved at
 * rd_init).  set1/set2 are host arrays of realisation indices.
 * Synchronous with respect to the host only through stream order. */
rd_status rd_adjoint(rd_handle *h, int32_t group, const float *d_fields0,
                     int32_t species_mask, const int32_t *d_set1, int64_t n1,
                     const int32_t *d_set2, int64_t n2, const double *d_radii,
                     int32_t M, double tau_frac, const double *d_cotangent,
                     double *d_C, double *d_grad, void *stream);

#ifdef __cplusplus
}
#endif
#endif
