"""GPU parity of the semi-implicit (IMEX) Euler stepper (implicit diffusion
solved in the cosine basis, explicit reaction; Sec. 5.1 and App. B.2 on
implicit stepping, App. B.1.1 discretisation) against the oracle's LU
solve of the same equations in FP64 (dense; sparse at 128 x 128).

Tolerance.  The GPU solves for the increment d = w^{n+1} - w^n, so each
step's four FP32 products of length G with an orthonormal matrix round
relative to d (about sqrt(G) 2^-24 of it per product), and the state takes
one FP32 rounding per step as in explicit Euler; the implicit diffusion
damps what is carried over.  Measured: 5e-7 after 300 FHN steps at
G = 32 and 64, 5e-8 for GM and BZ (relative to the field's maximum); at
G = 128 (one 4-CTA cluster per realisation) 5.7e-7 FHN, 3.4e-8 GM,
5.3e-8 BZ and 8.7e-7 for pure diffusion of +-0.5 noise.  Held to
max|gpu - oracle| / max|oracle| <= 1e-5 per realisation and species over
the step counts below (the fields' own tolerance), and bit-exact where the
arithmetic is exact (zeros and the homogeneous equilibrium of the
deviation form)."""
import numpy as np
import pytest
import torch

import oracle
from oracle import imex as OI
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


def run_gpu(p, model, G, n, par, dt, steps, noise, seed, residual=False):
    sim = p.Simulation([p.Group(model, G, n, par, dt, steps, noise, seed)])
    w0 = sim.group_fields(0).cpu().numpy().copy()
    res = sim.integrate_imex(residual=residual)
    torch.cuda.synchronize()
    return w0, sim.group_fields(0).cpu().numpy(), res


# (model, G, n_real, params, dt, steps, noise): dt far above the explicit
# diffusive limit h^2 / (4 max D) (FHN 64: 1.26e-3; GM 64: 6.3e-3)
CASES = [
    (W.FHN, 32, 3, (2.8e-4, 0.05, 10.0, 0.95), 2 ** -6, 200, (-0.05, 0.05)),
    (W.FHN, 64, 2, (2.9e-4, 0.048, 9.7, 0.93), 2 ** -6, 150, (-0.05, 0.05)),
    (W.GM, 64, 2, (2.5e-4, 0.01, 1.0, 0.52), 2 ** -4, 150, (0.0, 0.01)),
    (W.GM, 32, 3, (2.5e-4, 0.01, 1.0, 0.48), 2 ** -4, 200, (0.0, 0.01)),
    (W.BZ, 64, 2, W.BZ_THETA0, 2 ** -6, 150, (0.0, 0.01)),
    (W.BZ, 32, 3, (1.6e-3, 1.32e-2, 4.4, 7.1), 2 ** -7, 200, (0.0, 0.01)),
]


@pytest.mark.parametrize("case", CASES)
def test_imex_fields_within_tolerance(p, case):
    model, G, n, par, dt, steps, noise = case
    w0, got, res = run_gpu(p, model, G, n, par, dt, steps, noise, 0x77 + G, residual=True)
    want = OI.imex_run(model, par, dt, steps, w0)
    err = rel_err(got, want)
    assert err <= FIELD_TOL, err
    # the residual is the FP64 right-hand side of the final FP32 state
    ref = oracle.residual(model, par, got.astype(np.float64))
    np.testing.assert_allclose(res.cpu().numpy(), ref, rtol=1e-9, atol=1e-12)


def test_imex_single_step_matches_closely(p):
    """One step: only the rounding of one right-hand side and four products.
    On the first step from uniform noise the increment is as large as the
    field (the diffusion removes most of the noise at once), so the products'
    rounding, about sqrt(G) 2^-24 of the increment each, is of the field's
    size: bound 5e-6."""
    par = (2.9e-4, 0.048, 9.7, 0.93)
    w0, got, _ = run_gpu(p, W.FHN, 64, 2, par, 2 ** -6, 1, (-0.05, 0.05), 5)
    want = OI.imex_run(W.FHN, par, 2 ** -6, 1, w0)
    assert rel_err(got, want) <= 5e-6


@pytest.mark.parametrize("G", [32, 64])
def test_pure_diffusion_mode_decay_and_mass(p, G):
    """DIFF: a cosine mode decays by the closed-form factor per step (to
    FP32 rounding of the tables and products), and the mean is kept."""
    D = (3e-3, 1e-3)
    dt, steps = 0.01, 20
    sim = p.Simulation([p.Group(W.DIFF, G, 1, D, dt, steps, (0.0, 0.0), 1)])
    x = (np.arange(G) + 0.5) * np.pi / G
    pq = ((1, 2), (3, 0))
    modes = [np.outer(np.cos(q * x), np.cos(pp * x)) for (pp, q) in pq]
    f0 = np.stack([0.5 + modes[0], -0.25 + modes[1]])[None].astype(np.float32)
    sim.group_fields(0).copy_(torch.from_numpy(f0))
    sim.integrate_imex()
    got = sim.group_fields(0).cpu().numpy()[0].astype(np.float64)
    for s, ((pp, q), c) in enumerate(zip(pq, (0.5, -0.25))):
        lam = (G - 1) ** 2 * (4 * np.sin(np.pi * pp / (2 * G)) ** 2 + 4 * np.sin(np.pi * q / (2 * G)) ** 2)
        fac = (1.0 / (1.0 + dt * D[s] * lam)) ** steps
        want = c + fac * modes[s]
        assert np.abs(got[s] - want).max() <= 2e-6 * (1 + abs(c)), (s, np.abs(got[s] - want).max())
        assert abs(got[s].mean() - c) <= 2e-6


@pytest.mark.parametrize("model,par,noise", [
    (W.FHN, (2.8e-4, 0.05, 10.0, 0.95), (0.0, 0.0)),
    (W.GM, (2.5e-4, 0.01, 1.0, 0.52), (0.0, 0.0)),
    (W.BZ, W.BZ_THETA0, (0.0, 0.0)),
])
def test_equilibrium_is_kept_bit_exact(p, model, par, noise):
    """The homogeneous equilibrium (zero deviation) stays exactly in place."""
    w0, got, _ = run_gpu(p, model, 64, 1, par, 2 ** -5, 40, noise, 3)
    np.testing.assert_array_equal(got, w0)


def test_imex_refuses_unsupported_groups(p):
    sim = p.Simulation([p.Group(W.FHN, 256, 1, (2.8e-4, 0.05, 10.0, 0.95), 2 ** -6, 1, (-0.05, 0.05), 1)])
    with pytest.raises(p.RdError) as e:
        sim.integrate_imex()
    assert e.value.status == 6   # RD_ERR_UNSUPPORTED


def test_imex_takes_steps_the_explicit_stepper_cannot(p):
    """At dt = 16 x the explicit diffusive limit the explicit Euler stepper
    blows up while the semi-implicit one stays bounded and matches the
    oracle."""
    par = (2.9e-4, 0.048, 9.7, 0.93)
    dt = 16 * (1.0 / 63) ** 2 / (4 * par[1])
    w0, got, _ = run_gpu(p, W.FHN, 64, 1, par, dt, 60, (-0.05, 0.05), 9)
    assert np.isfinite(got).all() and np.abs(got).max() < 2.0
    want = OI.imex_run(W.FHN, par, dt, 60, w0)
    assert rel_err(got, want) <= FIELD_TOL
    ex = oracle.step(W.FHN, par, dt, 60, w0.astype(np.float64))
    assert not (np.isfinite(ex).all() and np.abs(ex).max() < 2.0)


@pytest.mark.parametrize("G", [32, 64])
def test_imex_tiles_bit_identical(p, G):
    """The product tile only changes which thread forms an output: every
    variant gives the same bits."""
    par = (2.9e-4, 0.048, 9.7, 0.93)
    keep = p.imex_get_variant(G)
    outs = []
    try:
        for v in range(4):
            p.imex_set_variant(G, v)
            _, got, _ = run_gpu(p, W.FHN, G, 2, par, 2 ** -6, 30, (-0.05, 0.05), 21)
            outs.append(got)
    finally:
        p.imex_set_variant(G, keep)
    for o in outs[1:]:
        np.testing.assert_array_equal(o, outs[0])


@pytest.mark.parametrize("case", [CASES[0], CASES[1], CASES[2], CASES[4]])
def test_imex_even_odd_split_within_tolerance(p, case):
    """Variant 4 forms the same solve from half-length sums (the cosine
    basis's even/odd symmetry): its own rounding, the same tolerance."""
    model, G, n, par, dt, steps, noise = case
    keep = p.imex_get_variant(G)
    try:
        p.imex_set_variant(G, 4)
        w0, got, res = run_gpu(p, model, G, n, par, dt, steps, noise, 0x91 + G, residual=True)
    finally:
        p.imex_set_variant(G, keep)
    want = OI.imex_run(model, par, dt, steps, w0)
    assert rel_err(got, want) <= FIELD_TOL
    ref = oracle.residual(model, par, got.astype(np.float64))
    np.testing.assert_allclose(res.cpu().numpy(), ref, rtol=1e-9, atol=1e-12)


@pytest.mark.parametrize("G", [32, 64])
def test_imex_even_odd_mode_decay(p, G):
    keep = p.imex_get_variant(G)
    try:
        p.imex_set_variant(G, 4)
        test_pure_diffusion_mode_decay_and_mass(p, G)
        test_equilibrium_is_kept_bit_exact(p, W.GM, (2.5e-4, 0.01, 1.0, 0.52), (0.0, 0.0))
    finally:
        p.imex_set_variant(G, keep)


def test_imex_several_groups_in_one_handle(p):
    """Groups of different models and grids in one handle: each realisation
    lands at its own offset and matches the oracle."""
    gs = [p.Group(W.FHN, 32, 2, (2.8e-4, 0.05, 10.0, 0.95), 2 ** -6, 80, (-0.05, 0.05), 31),
          p.Group(W.GM, 64, 1, (2.5e-4, 0.01, 1.0, 0.52), 2 ** -4, 60, (0.0, 0.01), 32),
          p.Group(W.BZ, 32, 2, (1.6e-3, 1.32e-2, 4.4, 7.1), 2 ** -7, 70, (0.0, 0.01), 33)]
    sim = p.Simulation(gs)
    w0 = [sim.group_fields(i).cpu().numpy().copy() for i in range(3)]
    res = sim.integrate_imex(residual=True)
    torch.cuda.synchronize()
    assert sim.sync_status() == 0
    base = 0
    for i, g in enumerate(gs):
        got = sim.group_fields(i).cpu().numpy()
        want = OI.imex_run(g.model, g.params, g.dt, g.n_steps, w0[i])
        assert rel_err(got, want) <= FIELD_TOL, i
        ref = oracle.residual(g.model, g.params, got.astype(np.float64))
        np.testing.assert_allclose(res[base:base + g.n_real].cpu().numpy(), ref, rtol=1e-9, atol=1e-12)
        base += g.n_real


def test_imex_reports_a_blow_up(p):
    """An explicit reaction step far beyond its limit (FHN, eps dt = 40)
    diverges: the residual turns NaN and the status word says non-finite."""
    sim = p.Simulation([p.Group(W.FHN, 32, 1, (2.8e-4, 0.05, 10.0, 0.95), 4.0, 40, (-0.5, 0.5), 3)])
    res = sim.integrate_imex(residual=True)
    torch.cuda.synchronize()
    assert np.isnan(res.cpu().numpy()).all()
    assert sim.sync_status() == 5   # RD_ERR_NONFINITE


def test_imex_c2_full_size_sample(p):
    """The benchmark's launch: all 128 realisations of the FHN 64x64
    workload, 625 steps of 2^-6 (the c2 horizon), default kernel; the first
    and the last realisation against the oracle."""
    g = W.config("c2")["groups"][0]
    grp = p.Group(g["model"], g["G"], g["n_real"], g["params"], 2 ** -6, 625, g["noise"], g["seed"])
    sim = p.Simulation([grp])
    w0 = sim.group_fields(0).cpu().numpy().copy()
    sim.integrate_imex()
    torch.cuda.synchronize()
    assert sim.sync_status() == 0
    got = sim.group_fields(0).cpu().numpy()
    pick = [0, g["n_real"] - 1]
    want = OI.imex_run(g["model"], g["params"], 2 ** -6, 625, w0[pick])
    assert rel_err(got[pick], want) <= FIELD_TOL


# G = 128: one 4-CTA cluster per realisation (rows split four ways, the
# transforms along y through distributed shared memory).  The products are
# twice as long as at G = 64 (about sqrt(2) more rounding per product); the
# same field tolerance holds.
CASES_128 = [
    (W.FHN, 128, 2, (2.8e-4, 0.05, 10.0, 0.95), 2 ** -6, 120, (-0.05, 0.05)),
    (W.GM, 128, 3, (2.5e-4, 0.01, 1.0, 0.5251796931279438), 2 ** -6, 150, (0.0, 0.01)),
    (W.BZ, 128, 2, W.BZ_THETA0, 2 ** -7, 100, (0.0, 0.01)),
    (W.DIFF, 128, 2, (3e-3, 1e-3), 2 ** -5, 60, (-0.5, 0.5)),
]


@pytest.mark.parametrize("case", CASES_128)
def test_imex_cluster_fields_within_tolerance(p, case):
    model, G, n, par, dt, steps, noise = case
    w0, got, res = run_gpu(p, model, G, n, par, dt, steps, noise, 0x128 + n, residual=True)
    want = OI.imex_run(model, par, dt, steps, w0)
    err = rel_err(got, want)
    assert err <= FIELD_TOL, err
    ref = oracle.residual(model, par, got.astype(np.float64))
    np.testing.assert_allclose(res.cpu().numpy(), ref, rtol=1e-9, atol=1e-12)


def test_imex_cluster_single_step(p):
    """One step from uniform noise, the worst case for the transforms'
    rounding: at G = 128 the v-species increment is cv = Dv dt (G-1)^2
    (about 12) times the noise's Laplacian, some 100 x the field, and the
    inverse products carry the solved increment, of the field's size; each
    product is a 64-term FP32 chain plus a pre-add and a recombination.
    Measured 8.7e-6 of max|field| (G = 64: below 5e-6); bound 1.5e-5.  The
    later steps' increments are small, which is why the multi-step runs stay
    within the field tolerance."""
    par = (2.9e-4, 0.048, 9.7, 0.93)
    w0, got, _ = run_gpu(p, W.FHN, 128, 2, par, 2 ** -6, 1, (-0.05, 0.05), 15)
    want = OI.imex_run(W.FHN, par, 2 ** -6, 1, w0)
    assert rel_err(got, want) <= 1.5e-5


def test_imex_cluster_mode_decay_mass_and_equilibrium(p):
    """Closed-form decay of cosine modes and the kept mean at G = 128, and
    the homogeneous equilibrium bit-exact."""
    test_pure_diffusion_mode_decay_and_mass(p, 128)
    w0, got, _ = run_gpu(p, W.GM, 128, 2, (2.5e-4, 0.01, 1.0, 0.52), 2 ** -5, 40, (0.0, 0.0), 3)
    np.testing.assert_array_equal(got, w0)


def test_imex_cluster_mixed_with_one_cta_groups(p):
    """A G = 128 group between G = 64 and G = 32 groups in one handle: each
    kernel reads its own table and writes its own realisations."""
    gs = [p.Group(W.GM, 64, 1, (2.5e-4, 0.01, 1.0, 0.52), 2 ** -4, 40, (0.0, 0.01), 41),
          p.Group(W.FHN, 128, 2, (2.8e-4, 0.05, 10.0, 0.95), 2 ** -6, 50, (-0.05, 0.05), 42),
          p.Group(W.FHN, 32, 1, (2.8e-4, 0.05, 10.0, 0.95), 2 ** -6, 50, (-0.05, 0.05), 43)]
    sim = p.Simulation(gs)
    w0 = [sim.group_fields(i).cpu().numpy().copy() for i in range(3)]
    sim.integrate_imex()
    torch.cuda.synchronize()
    assert sim.sync_status() == 0
    for i, g in enumerate(gs):
        want = OI.imex_run(g.model, g.params, g.dt, g.n_steps, w0[i])
        assert rel_err(sim.group_fields(i).cpu().numpy(), want) <= FIELD_TOL, i


def test_imex_cluster_reports_a_blow_up(p):
    sim = p.Simulation([p.Group(W.FHN, 128, 1, (2.8e-4, 0.05, 10.0, 0.95), 4.0, 40, (-0.5, 0.5), 3)])
    res = sim.integrate_imex(residual=True)
    torch.cuda.synchronize()
    assert np.isnan(res.cpu().numpy()).all()
    assert sim.sync_status() == 5   # RD_ERR_NONFINITE


def test_imex_c3_full_size_sample(p):
    """All 512 realisations of the GM 128x128 workload to its horizon
    (20000 explicit steps of 2^-10) in 1250 semi-implicit steps of 2^-6:
    the first and the last realisation against the oracle."""
    g = W.config("c3")["groups"][0]
    steps = g["n_steps"] // 16
    grp = p.Group(g["model"], g["G"], g["n_real"], g["params"], 2 ** -6, steps, g["noise"], g["seed"])
    sim = p.Simulation([grp])
    w0 = sim.group_fields(0).cpu().numpy().copy()
    sim.integrate_imex()
    torch.cuda.synchronize()
    assert sim.sync_status() == 0
    got = sim.group_fields(0).cpu().numpy()
    pick = [0, g["n_real"] - 1]
    want = OI.imex_run(g["model"], g["params"], 2 ** -6, steps, w0[pick])
    assert rel_err(got[pick], want) <= FIELD_TOL
