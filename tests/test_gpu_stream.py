"""The streaming stepper (grids the resident stepper cannot hold, or groups
flagged stream=True): bit-identical to the resident stepper where both
apply, at every temporal depth and for step counts that are not multiples of
it; within the field tolerance of the FP64 oracle on larger and ragged grids;
FP64 residual, status and mixed batches."""
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


RES_CASES = [
    (W.FHN, 64, (2.8e-4, 0.05, 10.0, 0.95), 2 ** -10, (-0.05, 0.05)),
    (W.GM, 128, (2.5e-4, 0.01, 1.0, 0.47), 2 ** -10, (0.0, 0.01)),
    (W.BZ, 64, W.BZ_THETA0, 2 ** -8, (0.0, 0.01)),
    (W.FHN, 32, (2.8e-4, 0.05, 10.0, 0.95), 2 ** -8, (-0.05, 0.05)),
]


@pytest.mark.parametrize("case", RES_CASES)
@pytest.mark.parametrize("depth", [1, 2, 4, 8])
def test_stream_bit_identical_to_resident(p, case, depth):
    model, G, par, dt, noise = case
    for steps in (37, 1, 0):
        a = p.Simulation([p.Group(model, G, 3, par, dt, steps, noise, 61)])
        b = p.Simulation([p.Group(model, G, 3, par, dt, steps, noise, 61, stream=True)])
        b.set_stream_depth(depth)
        ra = a.integrate()
        rb = b.integrate()
        assert a.sync_status() == 0 and b.sync_status() == 0
        assert torch.equal(a.fields, b.fields), steps
        assert torch.equal(ra[:, 0], rb[:, 0])
        assert torch.allclose(ra[:, 1], rb[:, 1], rtol=1e-13, atol=0)


@pytest.mark.parametrize("model,G,par,dt,noise,steps", [
    (W.FHN, 256, (2.8e-4, 0.05, 10.0, 0.95), 2 ** -14, (-0.05, 0.05), 300),
    (W.FHN, 200, (2.8e-4, 0.05, 10.0, 0.95), 2 ** -14, (-0.05, 0.05), 257),
    (W.GM, 200, (2.5e-4, 0.01, 1.0, 0.5), 2 ** -12, (0.0, 0.01), 203),
    (W.BZ, 100, W.BZ_THETA0, 2 ** -10, (0.0, 0.01), 190),
    (W.FHN, 12, (2.8e-3, 0.05, 10.0, 0.95), 2 ** -8, (-0.05, 0.05), 101),
])
@pytest.mark.parametrize("depth", [1, 4, 8])
def test_stream_against_oracle(p, model, G, par, dt, noise, steps, depth):
    sim = p.Simulation([p.Group(model, G, 2, par, dt, steps, noise, 91)])
    sim.set_stream_depth(depth)
    f0 = sim.group_fields(0).cpu().numpy().astype(np.float64)
    res = sim.integrate()
    assert sim.sync_status() == 0
    ref = oracle.step(model, par, dt, steps, f0)
    assert rel_err(sim.group_fields(0).cpu().numpy(), ref) <= FIELD_TOL
    assert torch.isfinite(res).all()


@pytest.mark.parametrize("G", [12, 100, 200])
def test_stream_initial_state_f64_and_residual(p, G):
    par, dt, noise = (2.8e-4, 0.05, 10.0, 0.95), 2 ** -14, (-0.05, 0.05)
    sim = p.Simulation([p.Group(W.FHN, G, 2, par, dt, 0, noise, 7)])
    f0 = sim.group_fields(0).cpu().numpy()
    assert np.array_equal(f0, oracle.init_fields(W.FHN, G, 2, par, noise[0], noise[1], 7))
    res = sim.integrate().cpu().numpy()
    assert np.allclose(res, oracle.residual(W.FHN, par, f0.astype(np.float64)), rtol=1e-12, atol=0)
    f64 = sim.fields.to(torch.float64)
    sim.integrate_f64(f64, steps=40)
    ref = oracle.step(W.FHN, par, dt, 40, f0.astype(np.float64))
    assert np.array_equal(f64.view(2, 2, G, G).cpu().numpy(), ref)


def test_mixed_resident_and_streaming_groups(p):
    gs = [p.Group(W.FHN, 64, 3, (2.8e-4, 0.05, 10.0, 0.95), 2 ** -10, 120, (-0.05, 0.05), 1),
          p.Group(W.GM, 200, 2, (2.5e-4, 0.01, 1.0, 0.5), 2 ** -12, 90, (0.0, 0.01), 2),
          p.Group(W.FHN, 32, 4, (2.8e-4, 0.05, 10.0, 0.95), 2 ** -8, 150, (-0.05, 0.05), 3),
          p.Group(W.BZ, 64, 2, W.BZ_THETA0, 2 ** -8, 77, (0.0, 0.01), 4, stream=True)]
    sim = p.Simulation(gs)
    f0 = [sim.group_fields(i).cpu().numpy().astype(np.float64) for i in range(len(gs))]
    res = sim.integrate()
    assert sim.sync_status() == 0
    assert torch.isfinite(res).all()
    for i, g in enumerate(gs):
        ref = oracle.step(g.model, g.params, g.dt, g.n_steps, f0[i])
        assert rel_err(sim.group_fields(i).cpu().numpy(), ref) <= FIELD_TOL, i


def test_stream_nonfinite_reported(p):
    sim = p.Simulation([p.Group(W.DIFF, 200, 1, (1.0, 1.0), 1e-2, 200, (-1, 1), 2)])
    res = sim.integrate()
    assert sim.sync_status() == 5
    assert torch.isnan(res).all()


def test_adjoint_not_offered_on_streaming_groups(p):
    with pytest.raises(Exception):
        p.Simulation([p.Group(W.FHN, 200, 2, (2.8e-4, 0.05, 10.0, 0.95), 2 ** -14, 10, (-0.05, 0.05), 1,
                              adjoint=True)])


def test_autotune_picks_a_depth_and_restores_state(p):
    gs = [p.Group(W.FHN, 256, 4, (2.8e-4, 0.05, 10.0, 0.95), 2 ** -14, 40, (-0.05, 0.05), 3),
          p.Group(W.FHN, 64, 2, (2.8e-4, 0.05, 10.0, 0.95), 2 ** -10, 40, (-0.05, 0.05), 4)]
    sim = p.Simulation(gs)
    f0 = sim.fields.clone()
    sim.autotune(steps=16)
    assert p.lib().rd_get_stream_depth(sim.handle) in (1, 2, 4, 8)
    assert torch.equal(sim.fields, f0)
