"""GPU parity of the initial state and the Euler steppers against the oracle.

Tolerances.  The FP64 GPU path evaluates the same operation sequence as the
oracle with every operation rounded separately, so it must agree bit for
bit.  The FP32 path is held to the stated field tolerance: per realisation
and species, max_cell |gpu - oracle| / max_cell |oracle| <= 1e-5.
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
    """max over realisations and species of max|a-b| / max|b|."""
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    num = np.abs(a - b).reshape(a.shape[0], 2, -1).max(-1)
    den = np.abs(b).reshape(b.shape[0], 2, -1).max(-1)
    return float((num / np.maximum(den, 1e-300)).max())


def mkgroup(p, model, G, n_real, params, dt, steps, noise, seed):
    return p.Group(model, G, n_real, params, dt, steps, noise, seed)


CASES = [
    (W.FHN, 32, 5, (2.8e-4, 0.05, 10.0, 0.95), 2 ** -8, (-0.05, 0.05)),
    (W.FHN, 64, 3, (2.9e-4, 0.048, 9.7, 0.93), 2 ** -10, (-0.05, 0.05)),
    (W.GM, 64, 3, (2.5e-4, 0.01, 1.0, 0.52), 2 ** -8, (0.0, 0.01)),
    (W.GM, 128, 2, (2.5e-4, 0.01, 1.0, 0.48), 2 ** -10, (0.0, 0.01)),
    (W.FHN, 128, 2, (2.8e-4, 0.05, 10.0, 0.97), 2 ** -12, (-0.05, 0.05)),
    (W.DIFF, 64, 2, (3e-3, 1e-3), 2 ** -12, (-1.0, 1.0)),
    (W.BZ, 64, 3, W.BZ_THETA0, 2 ** -8, (0.0, 0.01)),
    (W.BZ, 32, 4, (1.6e-3, 1.32e-2, 4.4, 7.1), 2 ** -8, (0.0, 0.01)),
]


@pytest.mark.parametrize("case", CASES)
def test_initial_state_bit_exact(p, case):
    model, G, n, par, dt, noise = case
    seed = 0x1234 + G
    sim = p.Simulation([mkgroup(p, model, G, n, par, dt, 0, noise, seed)])
    got = sim.group_fields(0).cpu().numpy()
    ref = oracle.init_fields(model, G, n, par, noise[0], noise[1], seed)
    assert np.array_equal(got, ref)


def test_initial_state_multi_group_offsets(p):
    gs = [mkgroup(p, W.FHN, 32, 3, (2.8e-4, 0.05, 10, 0.95), 2 ** -8, 0, (-0.05, 0.05), 11),
          mkgroup(p, W.GM, 64, 2, (2.5e-4, 0.01, 1, 0.5), 2 ** -8, 0, (0, 0.01), 12),
          mkgroup(p, W.FHN, 128, 1, (2.8e-4, 0.05, 10, 0.95), 2 ** -12, 0, (-0.05, 0.05), 13)]
    sim = p.Simulation(gs)
    for i, g in enumerate(gs):
        ref = oracle.init_fields(g.model, g.G, g.n_real, g.params, g.noise[0], g.noise[1], g.seed)
        assert np.array_equal(sim.group_fields(i).cpu().numpy(), ref)


def test_initial_state_many_groups_and_new_seeds(p):
    """More groups than one initial-state launch takes (120), every model,
    an RD-ODE group among them; then new seeds for some groups and a
    re-initialisation: every group's state equals the oracle's for the seed
    it holds at that moment."""
    models = [(W.FHN, (2.8e-4, 0.05, 10.0, 0.95), (-0.05, 0.05)),
              (W.GM, (2.5e-4, 0.01, 1.0, 0.52), (0.0, 0.01)),
              (W.BZ, W.BZ_THETA0, (0.0, 0.01)),
              (W.DIFF, (3e-3, 1e-3), (-1.0, 1.0))]
    gs = []
    for i in range(125):
        model, par, noise = models[i % 4]
        gs.append(mkgroup(p, model, 32 if i % 3 else 64, 1 + i % 2, par, 2 ** -10, 0, noise, 1000 + 7 * i))
    gs.insert(61, p.Group(W.RDODE, 64, 2, W.RDODE_THETA0, 1e-3, 0, (0.0, 2.0), 555))

    def check(sim, seeds):
        for i, g in enumerate(gs):
            got = sim.group_fields(i).cpu().numpy()
            if g.model == W.RDODE:
                ref = oracle.rdode_init(g.G, g.n_real, g.noise[0], g.noise[1], seeds[i], 10)
            else:
                ref = oracle.init_fields(g.model, g.G, g.n_real, g.params, g.noise[0], g.noise[1], seeds[i])
            assert np.array_equal(got, ref), i

    sim = p.Simulation(gs)
    seeds = [g.seed for g in gs]
    check(sim, seeds)
    for i in (0, 61, 119, 120, 125):
        seeds[i] = seeds[i] + 99991
        assert p.lib().rd_set_seed(sim.handle, i, seeds[i]) == 0
    sim.reinit()
    torch.cuda.synchronize()
    check(sim, seeds)


@pytest.mark.parametrize("case", CASES)
def test_f64_path_bit_exact(p, case):
    model, G, n, par, dt, noise = case
    steps = 60 if G == 128 else 150
    sim = p.Simulation([mkgroup(p, model, G, n, par, dt, steps, noise, 77)])
    f64 = sim.fields.to(torch.float64)
    sim.integrate_f64(f64)
    got = f64.view(n, 2, G, G).cpu().numpy()
    ref = oracle.step(model, par, dt, steps,
                      oracle.init_fields(model, G, n, par, noise[0], noise[1], 77).astype(np.float64))
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("case", CASES)
def test_fp32_resident_within_tolerance(p, case):
    model, G, n, par, dt, noise = case
    steps = {32: 600, 64: 400, 128: 200}[G]
    sim = p.Simulation([mkgroup(p, model, G, n, par, dt, steps, noise, 99)])
    f0 = sim.group_fields(0).cpu().numpy().astype(np.float64)
    res = sim.integrate()
    assert sim.sync_status() == 0
    got = sim.group_fields(0).cpu().numpy()
    ref = oracle.step(model, par, dt, steps, f0)
    assert rel_err(got, ref) <= FIELD_TOL
    # residual: FP64 RHS of the final FP32 state against the oracle's residual
    # of its own FP64 state.  F is Lipschitz in the state with constant
    # L_F <= 8 max(Du, Dv) (G-1)^2 + |dR/dw|, so both the max and the RMS of F
    # may differ by at most L_F * max|gpu - oracle state|.
    rr = oracle.residual(model, par, ref)
    r = res.cpu().numpy()
    dw = np.abs(got.astype(np.float64) - ref).max()
    umax = np.abs(ref).max()
    k = abs(par[2]) if len(par) > 2 else 0.0
    LF = 8 * max(par[0], par[1]) * (G - 1) ** 2 + 4 * (1 + k) * (1 + umax) ** 2
    assert np.all(np.abs(r - rr) <= LF * dw * 1.01 + 1e-12), (r, rr, LF * dw)


@pytest.mark.parametrize("case", CASES[:4])
def test_residual_of_initial_state(p, case):
    """With zero steps both sides see the same FP32 state: the FP64 residuals
    agree to rounding."""
    model, G, n, par, dt, noise = case
    sim = p.Simulation([mkgroup(p, model, G, n, par, dt, 0, noise, 5)])
    res = sim.integrate().cpu().numpy()
    ref = oracle.residual(model, par, oracle.init_fields(model, G, n, par, noise[0], noise[1], 5))
    assert np.allclose(res, ref, rtol=1e-12, atol=0)


@pytest.mark.parametrize("model,G,par,dt,noise", [
    (W.FHN, 64, (2.8e-4, 0.05, 10.0, 0.95), 2 ** -10, (-0.05, 0.05)),
    (W.GM, 64, (2.5e-4, 0.01, 1.0, 0.52), 2 ** -8, (0.0, 0.01)),
    (W.BZ, 32, (1.6e-3, 1.32e-2, 4.4, 7.1), 2 ** -8, (0.0, 0.01)),
    (W.GM, 128, (2.5e-4, 0.01, 1.0, 0.48), 2 ** -10, (0.0, 0.01)),
])
def test_reference_path_agrees(p, model, G, par, dt, noise):
    """The plain paths (one realisation per launch, and the whole group per
    launch) agree with the oracle like the resident stepper, and with each
    other bit for bit (same per-node arithmetic)."""
    g = mkgroup(p, model, G, 3, par, dt, 301, noise, 3)
    a = p.Simulation([g])
    b = p.Simulation([g])
    c = p.Simulation([g])
    a.integrate()
    b.integrate_reference()
    c.integrate_plain()
    torch.cuda.synchronize()
    ref = oracle.step(model, par, dt, 301, oracle.init_fields(model, G, 3, par, noise[0], noise[1], 3)
                      .astype(np.float64))
    assert rel_err(a.group_fields(0).cpu().numpy(), ref) <= FIELD_TOL
    assert rel_err(b.group_fields(0).cpu().numpy(), ref) <= FIELD_TOL
    assert torch.equal(b.fields, c.fields)


def test_split_integration_is_bit_identical(p):
    par = (2.9e-4, 0.05, 10.0, 0.95)
    g = mkgroup(p, W.FHN, 64, 2, par, 2 ** -10, 0, (-0.05, 0.05), 8)
    a = p.Simulation([g])
    b = p.Simulation([g])
    a.integrate(steps=250)
    b.integrate(steps=100)
    b.integrate(steps=150)
    assert torch.equal(a.fields, b.fields)


@pytest.mark.parametrize("model,par,x0", [(W.FHN, (2.8e-4, 0.05, 10.0, 1.0), (0.0, 0.0)),
                                          (W.GM, (2.5e-4, 0.01, 1.0, 0.5), (2.0, 4.0)),
                                          (W.BZ, (1.6e-3, 1.32e-2, 2.0, 3.0), (2.0, 1.5))])
def test_equilibrium_fixed_point(p, model, par, x0):
    sim = p.Simulation([mkgroup(p, model, 64, 2, par, 2 ** -10, 500, (0.0, 0.0), 1)])
    f0 = sim.fields.clone()
    assert float(f0[0]) == x0[0]
    sim.integrate()
    assert torch.equal(sim.fields, f0)


def test_pure_diffusion_conserves_mass(p):
    sim = p.Simulation([mkgroup(p, W.DIFF, 64, 2, (3e-3, 1e-3), 2 ** -12, 2000, (-1, 1), 21)])
    m0 = sim.group_fields(0).double().sum(dim=(2, 3))
    sim.integrate()
    m1 = sim.group_fields(0).double().sum(dim=(2, 3))
    # FP32 rounding of 4096 cells per step over 2000 steps
    assert torch.allclose(m0, m1, rtol=0, atol=2e-2)


def test_unstable_step_reports_nonfinite(p):
    # dt far above the explicit diffusion limit blows up; reported, no fault
    sim = p.Simulation([mkgroup(p, W.DIFF, 32, 1, (1.0, 1.0), 1e-2, 400, (-1, 1), 2)])
    sim.integrate()
    assert sim.sync_status() == 5


def test_c2_full_size_error_curve(p):
    """c2 (FHN 64x64, 128 realisations, 10^4 steps) against the FP64 oracle on
    a sample of 8 realisations, at increasing step counts up to the full
    horizon."""
    cfg = W.config("c2")
    g = cfg["groups"][0]
    sim = p.Simulation([p.Group.from_dict(g)])
    f0 = sim.group_fields(0)[:8].cpu().numpy().astype(np.float64)
    done = 0
    errs = {}
    ref = f0
    for target in (500, 2000, 5000, 10000):
        sim.integrate(steps=target - done)
        ref = oracle.step(g["model"], g["params"], g["dt"], target - done, ref)
        done = target
        errs[target] = rel_err(sim.group_fields(0)[:8].cpu().numpy(), ref)
    print("c2 field error by step:", errs)
    assert all(e <= FIELD_TOL for e in errs.values()), errs


@pytest.mark.parametrize("model,G,par,dt,noise", [
    (W.FHN, 64, (2.8e-4, 0.05, 10.0, 0.95), 2 ** -10, (-0.05, 0.05)),
    (W.GM, 128, (2.5e-4, 0.01, 1.0, 0.47), 2 ** -10, (0.0, 0.01)),
    (W.FHN, 128, (2.8e-4, 0.05, 10.0, 0.95), 2 ** -13, (-0.05, 0.05)),
    (W.BZ, 128, W.BZ_THETA0, 2 ** -11, (0.0, 0.01)),
    (W.FHN, 32, (2.8e-4, 0.05, 10.0, 0.95), 2 ** -8, (-0.05, 0.05)),
    (W.BZ, 64, W.BZ_THETA0, 2 ** -8, (0.0, 0.01)),
])
def test_tile_variants_bit_identical(p, model, G, par, dt, noise):
    """Tile shape only changes data movement: every variant gives the same bits."""
    L = p.lib()
    keep = L.rd_get_variant(model, G)
    outs = []
    try:
        for v in range(L.rd_n_variants()):
            assert L.rd_set_variant(model, G, v) == 0
            sim = p.Simulation([mkgroup(p, model, G, 3, par, dt, 150, noise, 41)])
            sim.integrate()
            outs.append(sim.fields.clone())
    finally:
        L.rd_set_variant(model, G, keep)
    assert torch.isfinite(outs[0]).all()    # within the explicit step limit of the case
    for o in outs[1:]:
        assert torch.equal(o, outs[0])


def test_autotune_restores_initial_state(p):
    g = mkgroup(p, W.FHN, 64, 4, (2.8e-4, 0.05, 10.0, 0.95), 2 ** -10, 100, (-0.05, 0.05), 5)
    sim = p.Simulation([g])
    f0 = sim.fields.clone()
    chosen = sim.autotune(steps=50)
    assert 0 <= chosen[0 * 3 + 1] < p.lib().rd_n_variants()
    assert torch.equal(sim.fields, f0)


def test_c3_sample_gm128_full_horizon(p):
    """c3 (GM 128x128, 2*10^4 steps, dt 2^-10): two realisations against the
    FP64 oracle over the full horizon."""
    cfg = W.config("c3")
    g = dict(cfg["groups"][0])
    g["n_real"] = 2
    sim = p.Simulation([p.Group.from_dict(g)])
    f0 = sim.group_fields(0).cpu().numpy().astype(np.float64)
    sim.integrate()
    ref = oracle.step(g["model"], g["params"], g["dt"], g["n_steps"], f0)
    err = rel_err(sim.group_fields(0).cpu().numpy(), ref)
    print("c3 GM 128 full-horizon field error", err)
    assert err <= FIELD_TOL


def test_c6_sample_bz64_full_horizon(p):
    """c6 (Brusselator 64x64, 25600 steps of 2^-8, T = 100 as in Table 1): two
    realisations against the FP64 oracle over the full horizon."""
    cfg = W.config("c6")
    g = dict(cfg["groups"][0])
    g["n_real"] = 2
    sim = p.Simulation([p.Group.from_dict(g)])
    f0 = sim.group_fields(0).cpu().numpy().astype(np.float64)
    res = sim.integrate()
    assert sim.sync_status() == 0
    ref = oracle.step(g["model"], g["params"], g["dt"], g["n_steps"], f0)
    err = rel_err(sim.group_fields(0).cpu().numpy(), ref)
    print("c6 BZ 64 full-horizon field error", err, "residual", res.cpu().numpy())
    assert err <= FIELD_TOL


def mixed_groups(p, steps_scale=1.0):
    def st(n):
        return max(1, int(n * steps_scale))
    return [mkgroup(p, W.FHN, 64, 5, (2.8e-4, 0.05, 10.0, 0.95), 2 ** -10, st(300), (-0.05, 0.05), 101),
            mkgroup(p, W.GM, 128, 3, (2.5e-4, 0.01, 1.0, 0.52), 2 ** -10, st(200), (0.0, 0.01), 102),
            mkgroup(p, W.FHN, 32, 7, (2.9e-4, 0.05, 9.5, 0.93), 2 ** -8, st(400), (-0.05, 0.05), 103),
            mkgroup(p, W.GM, 64, 4, (2.5e-4, 0.01, 1.0, 0.47), 2 ** -8, st(250), (0.0, 0.01), 104),
            mkgroup(p, W.FHN, 128, 2, (2.8e-4, 0.05, 10.0, 0.97), 2 ** -12, st(150), (-0.05, 0.05), 105),
            mkgroup(p, W.DIFF, 64, 2, (3e-3, 1e-3), 2 ** -12, st(100), (-1.0, 1.0), 106),
            mkgroup(p, W.BZ, 64, 3, W.BZ_THETA0, 2 ** -8, st(300), (0.0, 0.01), 107)]


def test_persistent_batch_bit_identical_to_per_group(p):
    gs = mixed_groups(p)
    a = p.Simulation(gs)
    b = p.Simulation(gs)
    a.set_schedule(1)          # one launch per group
    b.set_schedule(2)          # one persistent launch
    ra = a.integrate()
    rb = b.integrate()
    assert a.sync_status() == 0 and b.sync_status() == 0
    assert torch.equal(a.fields, b.fields)
    # the max of |F| is order-free; the RMS sum follows the tiling's order
    assert torch.equal(ra[:, 0], rb[:, 0])
    assert torch.allclose(ra[:, 1], rb[:, 1], rtol=1e-13, atol=0)


def test_persistent_batch_against_oracle(p):
    gs = mixed_groups(p)
    sim = p.Simulation(gs)     # more than one group: automatic schedule is persistent
    f0 = [sim.group_fields(i).cpu().numpy().astype(np.float64) for i in range(len(gs))]
    sim.integrate()
    for i, g in enumerate(gs):
        ref = oracle.step(g.model, g.params, g.dt, g.n_steps, f0[i])
        assert rel_err(sim.group_fields(i).cpu().numpy(), ref) <= FIELD_TOL, i


def test_c4_mixed_batch_slice(p):
    """c4: 64 parameter vectors x 128 realisations, FHN and GM at 64^2 and
    128^2 in one persistent launch (steps shortened to 2 %); one realisation
    of every eighth group checked against the oracle."""
    cfg = W.config("c4", steps_scale=0.02)
    gs = [p.Group.from_dict(g) for g in cfg["groups"]]
    sim = p.Simulation(gs)
    picks = list(range(0, len(gs), 8))
    f0 = {i: sim.group_fields(i)[:1].cpu().numpy().astype(np.float64) for i in picks}
    res = sim.integrate()
    assert sim.sync_status() == 0
    assert torch.isfinite(res).all()
    for i in picks:
        g = gs[i]
        ref = oracle.step(g.model, g.params, g.dt, g.n_steps, f0[i])
        assert rel_err(sim.group_fields(i)[:1].cpu().numpy(), ref) <= FIELD_TOL, i
