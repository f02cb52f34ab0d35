"""GPU parity of the stabilised second-order Runge-Kutta integrator
(App. B.2, Chebyshev coefficients) against the oracle.

Fixed schedule (h, s given): the GPU runs the same recurrence as the oracle
in FP32 (on the increments D_j = Y_j - Y_0), the oracle in FP64 on the
stages themselves; held to the field tolerance max|gpu - oracle| /
max|oracle| <= 1e-5 per realisation and species, and the RHS count exactly.

Adaptive: the step-control decisions (accept, s, h) are taken from FP32
fields on the GPU and FP64 fields in the oracle.  The GPU forms every RHS
evaluation of a step as F(Y_0) + dF(increment) and holds the state
compensated, so its error estimate is not disturbed by rounding-level
stiff modes and it takes the oracle's schedule; a decision could still
part at an exact boundary, so the counts are compared to within one step,
the fields to the oracle's result when the schedules agree, and the
accuracy against an accurate reference in every case.
"""
import numpy as np
import pytest
import torch

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

FIELD_TOL = 1e-5


@pytest.fixture(scope="module")
def p():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2203_14742_b300 as pk
    return pk


def rel_err(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    num = np.abs(a - b).reshape(a.shape[0], 2, -1).max(-1)
    den = np.abs(b).reshape(b.shape[0], 2, -1).max(-1)
    return float((num / np.maximum(den, 1e-300)).max())


def stage_count(beta_target):
    s = 2
    while oracle.rkc_beta(s) < beta_target:
        s += 1
    return s


def sim_of(p, model, G, n, par, noise, seed, dt=2 ** -10, steps=0):
    return p.Simulation([p.Group(model, G, n, par, dt, steps, noise, seed)])


# (model, G, n_real, params, noise, h, n_steps)
FIXED = [
    (W.FHN, 64, 3, W.FHN_THETA0, (-0.05, 0.05), 0.2, 50),
    (W.FHN, 64, 2, (2.9e-4, 0.048, 9.7, 0.93), (-0.05, 0.05), 0.05, 100),
    (W.FHN, 32, 4, (2.8e-4, 0.05, 10.0, 0.95), (-0.05, 0.05), 0.5, 30),
    (W.GM, 64, 3, (2.5e-4, 0.01, 1.0, 0.52), (0.0, 0.01), 0.5, 60),
    (W.GM, 32, 2, W.GM_THETA0, (0.0, 0.01), 1.0, 40),
    (W.BZ, 64, 3, W.BZ_THETA0, (0.0, 0.01), 0.05, 80),
    (W.BZ, 32, 2, (1.6e-3, 1.32e-2, 4.4, 7.1), (0.0, 0.01), 0.05, 60),
    (W.DIFF, 64, 2, (3e-3, 1e-3), (-1.0, 1.0), 0.02, 40),
    # G = 128: one realisation per 4-CTA cluster
    (W.FHN, 128, 2, (2.8e-4, 0.05, 10.0, 0.97), (-0.05, 0.05), 0.05, 20),
    (W.GM, 128, 3, (2.5e-4, 0.01, 1.0, 0.48), (0.0, 0.01), 0.5, 20),
    (W.BZ, 128, 2, W.BZ_THETA0, (0.0, 0.01), 0.02, 20),
    (W.DIFF, 128, 2, (3e-3, 1e-3), (-1.0, 1.0), 0.01, 10),
]


@pytest.mark.parametrize("case", FIXED)
def test_fixed_schedule_parity(p, case):
    model, G, n, par, noise, h, nst = case
    seed = 0x5151 + G + model
    sim = sim_of(p, model, G, n, par, noise, seed)
    w0 = sim.group_fields(0).cpu().numpy()
    rho = max(oracle.gershgorin(model, par, w.astype(np.float64)) for w in w0)
    s = stage_count(1.1 * h * rho)
    st, _ = sim.integrate_rkc(h, s_fixed=s, n_fixed=nst)
    assert sim.sync_status() == 0
    got = sim.group_fields(0).cpu().numpy()
    ref = oracle.rkc_fixed(model, par, h, s, nst, w0)
    assert rel_err(got, ref) <= FIELD_TOL
    st = st.cpu().numpy()
    assert (st[:, 0] == nst).all() and (st[:, 1] == 0).all()
    assert (st[:, 2] == 1 + nst * s).all() and (st[:, 3] == s).all()


@pytest.mark.parametrize("s", [2, 3, 9, 40])
def test_eigenmode_amplification(p, s):
    # pure diffusion of DCT-II modes (exact eigenvectors of the mirrored-ghost
    # Laplacian): one step multiplies each by R_s(h lambda)
    G = 64
    Du, Dv = 1e-3, 4e-3
    sim = sim_of(p, W.DIFF, G, 2, (Du, Dv), (0.0, 0.0), 1)
    x = np.arange(G)
    modes = [((1, 0), (0, 3)), ((63, 62), (20, 45))]
    w = np.zeros((2, 2, G, G))
    for r, ((k, l), (k2, l2)) in enumerate(modes):
        w[r, 0] = np.outer(np.cos(np.pi * l * (x + 0.5) / G), np.cos(np.pi * k * (x + 0.5) / G))
        w[r, 1] = np.outer(np.cos(np.pi * l2 * (x + 0.5) / G), np.cos(np.pi * k2 * (x + 0.5) / G))
    sim.group_fields(0).copy_(torch.from_numpy(w.astype(np.float32)))
    w32 = w.astype(np.float32).astype(np.float64)
    c = oracle.rkc_coef(s)
    h = 0.95 * c["beta"] / (8 * (G - 1) ** 2 * Dv)
    sim.integrate_rkc(h, s_fixed=s, n_fixed=1)
    got = sim.group_fields(0).cpu().numpy()
    ref = oracle.rkc_fixed(W.DIFF, (Du, Dv), h, s, 1, w32)
    assert np.abs(got - ref).max() <= 2e-6


def test_homogeneous_state_and_mass(p):
    G = 64
    sim = sim_of(p, W.FHN, G, 2, W.FHN_THETA0, (0.0, 0.0), 3)
    sim.integrate_rkc(0.2, s_fixed=23, n_fixed=10)
    assert np.all(sim.group_fields(0).cpu().numpy() == 0.0)
    sim = sim_of(p, W.DIFF, G, 2, (2e-3, 7e-3), (0.0, 1.0), 4)
    m0 = sim.group_fields(0).double().sum(dim=(2, 3)).cpu().numpy()
    sim.integrate_rkc(0.02, s_fixed=12, n_fixed=20)
    m1 = sim.group_fields(0).double().sum(dim=(2, 3)).cpu().numpy()
    np.testing.assert_allclose(m1, m0, rtol=2e-6)


@pytest.mark.parametrize("model,G,par,noise,h0", [
    (W.FHN, 64, W.FHN_THETA0, (-0.05, 0.05), 0.013),
    (W.GM, 64, W.GM_THETA0, (0.0, 0.01), 0.3),
    (W.BZ, 32, W.BZ_THETA0, (0.0, 0.01), 0.0021),
])
def test_single_step_stage_rule(p, model, G, par, noise, h0):
    # one accepted step to t_end = h0: s is the smallest with h0 rho <= beta(s)
    # (a loose tolerance: the iid initial noise puts stiff modes into the
    # error estimate, which would otherwise reject the first trials)
    sim = sim_of(p, model, G, 3, par, noise, 21)
    w0 = sim.group_fields(0).cpu().numpy()
    st, _ = sim.integrate_rkc(h0, t_end=h0, rtol=1.0, atol=1.0)
    assert sim.sync_status() == 0
    st = st.cpu().numpy()
    for r in range(3):
        rho = oracle.gershgorin(model, par, w0[r].astype(np.float64))
        s_ref = stage_count(h0 * rho)
        # not at a boundary (else the FP32 rho may decide either way)
        assert abs(h0 * rho - oracle.rkc_beta(s_ref)) > 1e-4 * h0 * rho
        assert abs(h0 * rho - oracle.rkc_beta(s_ref - 1)) > 1e-4 * h0 * rho or s_ref == 2
        assert tuple(st[r]) == (1, 0, 1 + s_ref, s_ref)
    ref, ost, failed = oracle.rkc_adaptive(model, par, h0, h0, 1.0, 1.0, w0)
    assert failed == 0 and (ost == st).all()
    assert rel_err(sim.group_fields(0).cpu().numpy(), ref) <= FIELD_TOL


def test_forced_rejection_matches(p):
    # a first trial step far too long for the tolerance is rejected, then
    # the run proceeds; counts agree with the oracle's
    G = 32
    par = W.FHN_THETA0
    sim = sim_of(p, W.FHN, G, 2, par, (-0.05, 0.05), 8)
    w0 = sim.group_fields(0).cpu().numpy()
    st, _ = sim.integrate_rkc(2.0, t_end=2.0, rtol=1e-4, atol=1e-4)
    assert sim.sync_status() == 0
    st = st.cpu().numpy()
    ref, ost, failed = oracle.rkc_adaptive(W.FHN, par, 2.0, 2.0, 1e-4, 1e-4, w0)
    assert failed == 0
    assert (st[:, 1] >= 1).all() and (ost[:, 1] >= 1).all()
    assert np.abs(st[:, 0] - ost[:, 0]).max() <= 1
    assert np.abs(st[:, 1] - ost[:, 1]).max() <= 1
    assert rel_err(sim.group_fields(0).cpu().numpy(), ref) <= 1e-3


@pytest.mark.parametrize("model,G,par,noise,T,tol", [
    (W.FHN, 64, W.FHN_THETA0, (-0.05, 0.05), 10000 * 2 ** -10, 1e-5),
    (W.FHN, 64, W.FHN_THETA0, (-0.05, 0.05), 10000 * 2 ** -10, 1e-7),
    (W.GM, 64, (2.5e-4, 0.01, 1.0, 0.52), (0.0, 0.01), 40.0, 1e-6),
    (W.BZ, 64, W.BZ_THETA0, (0.0, 0.01), 10.0, 1e-7),
    (W.FHN, 32, (2.8e-4, 0.05, 10.0, 0.95), (-0.05, 0.05), 2000 * 2 ** -8, 1e-6),
    (W.GM, 128, (2.5e-4, 0.01, 1.0, 0.48), (0.0, 0.01), 10.0, 1e-5),
    (W.FHN, 128, (2.8e-4, 0.05, 10.0, 0.97), (-0.05, 0.05), 2.0, 1e-6),
])
def test_adaptive_run_against_oracle(p, model, G, par, noise, T, tol):
    n = 2
    sim = sim_of(p, model, G, n, par, noise, 77)
    w0 = sim.group_fields(0).cpu().numpy()
    st, _ = sim.integrate_rkc(1e-3, t_end=T, rtol=tol, atol=tol)
    assert sim.sync_status() == 0
    got = sim.group_fields(0).cpu().numpy()
    st = st.cpu().numpy()
    mine, ost, failed = oracle.rkc_adaptive(model, par, T, 1e-3, tol, tol, w0)
    assert failed == 0
    # accurate reference: the oracle at a 100x tighter tolerance
    acc, _, _ = oracle.rkc_adaptive(model, par, T, 1e-3, tol / 100, tol / 100, w0)
    e_gpu, e_orc = rel_err(got, acc), rel_err(mine, acc)
    assert e_gpu <= 1.05 * e_orc + 1e-6
    # the FP32 run takes the FP64 run's schedule (its error estimate is not
    # disturbed by rounding-level stiff modes) and so lands on its result
    assert np.abs(st[:, 0] - ost[:, 0]).max() <= 1
    assert np.abs(st[:, 1] - ost[:, 1]).max() <= 1
    assert np.abs(st[:, 2] - ost[:, 2]).max() <= 0.02 * ost[:, 2].max()
    if (st == ost).all():
        assert rel_err(got, mine) <= FIELD_TOL


def test_split_horizon_mixed_groups(p):
    # two groups of different models and grids in one call, each to its own
    # horizon dt * n_steps; per-group results equal separate calls
    ga = p.Group(W.FHN, 64, 2, W.FHN_THETA0, 2 ** -10, 2048, (-0.05, 0.05), 5)
    gb = p.Group(W.BZ, 32, 3, W.BZ_THETA0, 2 ** -8, 512, (0.0, 0.01), 6)
    both = p.Simulation([ga, gb])
    st, _ = both.integrate_rkc(1e-3, rtol=1e-5, atol=1e-5)
    assert both.sync_status() == 0
    st = st.cpu().numpy()
    for i, g in enumerate((ga, gb)):
        one = p.Simulation([g])
        s1, _ = one.integrate_rkc(1e-3, rtol=1e-5, atol=1e-5)
        assert torch.equal(one.group_fields(0), both.group_fields(i))
        lo = 0 if i == 0 else 2
        assert (s1.cpu().numpy() == st[lo:lo + g.n_real]).all()


def test_residual_output(p):
    sim = sim_of(p, W.FHN, 64, 2, W.FHN_THETA0, (-0.05, 0.05), 12)
    _, res = sim.integrate_rkc(0.2, s_fixed=23, n_fixed=5, residual=True)
    got = sim.group_fields(0).cpu().numpy().astype(np.float64)
    ref = oracle.residual(W.FHN, W.FHN_THETA0, got)
    np.testing.assert_allclose(res.cpu().numpy(), ref, rtol=1e-12)


def test_step_control_failure_is_reported(p):
    # the attempt limit runs out (host-set limit, no device fault)
    sim = sim_of(p, W.FHN, 32, 2, W.FHN_THETA0, (-0.05, 0.05), 13)
    sim.integrate_rkc(1e-3, t_end=10.0, max_attempts=3)
    assert sim.sync_status() == 8                     # RD_ERR_STEPSIZE
    # the context stays usable
    sim.reinit()
    sim.integrate_rkc(1e-3, t_end=0.01)
    assert sim.sync_status() == 0


def test_unstable_fixed_step_reports_nonfinite(p):
    sim = sim_of(p, W.FHN, 32, 1, W.FHN_THETA0, (-0.05, 0.05), 14)
    sim.integrate_rkc(5.0, s_fixed=2, n_fixed=200)
    assert sim.sync_status() == 5
    sim.reinit()
    sim.integrate_rkc(0.1, s_fixed=12, n_fixed=2)
    assert sim.sync_status() == 0


def test_argument_checks(p):
    sim = sim_of(p, W.FHN, 32, 1, W.FHN_THETA0, (-0.05, 0.05), 15)
    for kw in (dict(h0=0.0), dict(h0=1e-3, s_fixed=1), dict(h0=1e-3, s_fixed=300),
               dict(h0=1e-3, rtol=0.0, atol=0.0), dict(h0=1e-3, s_max=1), dict(h0=1e-3, max_attempts=0),
               dict(h0=1e-3, s_fixed=4, n_fixed=-1)):
        with pytest.raises(p.RdError) as e:
            sim.integrate_rkc(**kw)
        assert e.value.status == 1
    big = p.Simulation([p.Group(W.FHN, 256, 1, W.FHN_THETA0, 2 ** -12, 1, (-0.05, 0.05), 1)])
    with pytest.raises(p.RdError) as e:
        big.integrate_rkc(1e-3)
    assert e.value.status == 6


@pytest.mark.parametrize("model,G,par,noise", [
    (W.FHN, 64, W.FHN_THETA0, (-0.05, 0.05)),
    (W.GM, 32, W.GM_THETA0, (0.0, 0.01)),
    (W.BZ, 64, W.BZ_THETA0, (0.0, 0.01)),
])
def test_tile_shapes(p, model, G, par, noise):
    # Per node every shape runs the same arithmetic: a fixed schedule gives
    # bit-identical fields.  The adaptive error norm is summed in an order
    # that follows the tiling, so its last bits (and through h the fields)
    # may differ; the runs must still agree to the field tolerance.
    fixed, adaptive = [], []
    try:
        for v in range(p.lib().rd_rkc_n_variants()):
            p.rkc_set_variant(G, v)
            assert p.rkc_get_variant(G) == v
            sim = sim_of(p, model, G, 3, par, noise, 31)
            sim.integrate_rkc(0.05, s_fixed=12, n_fixed=20)
            fixed.append(sim.group_fields(0).clone())
            sim.reinit()
            st, _ = sim.integrate_rkc(1e-3, t_end=2.0, rtol=1e-5, atol=1e-5)
            assert sim.sync_status() == 0
            adaptive.append((sim.group_fields(0).cpu().numpy(), st.cpu().numpy()))
    finally:
        p.rkc_set_variant(G, 1 if G == 64 else 0)
    for f in fixed[1:]:
        assert torch.equal(f, fixed[0])
    for f, st in adaptive[1:]:
        assert rel_err(f, adaptive[0][0]) <= 1e-4
        assert np.abs(st[:, 0] - adaptive[0][1][:, 0]).max() <= 2
