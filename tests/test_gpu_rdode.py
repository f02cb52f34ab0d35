"""GPU parity of the 1-D reaction-diffusion-ODE model (Sec. 4.3, eq. rdode):
initial state bit-exact, fixed-schedule stabilised RK2 within the field
tolerance of the FP64 oracle, adaptive runs to Table 1's t = 50 against the
oracle's accuracy and its far-from-equilibrium pattern, residual output,
and the calls that do not take the 1-D model."""
import numpy as np
import pytest
import torch

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

FIELD_TOL = 1e-5
P0 = W.RDODE_THETA0


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


def sim_of(p, N, n, par=P0, seed=9, noise=(0.0, 2.0), T=50.0):
    return p.Simulation([p.Group(W.RDODE, N, n, par, T / 1024, 1024, noise, seed)])


@pytest.mark.parametrize("N", [32, 64, 128, 256])
def test_initial_state_bit_exact(p, N):
    sim = sim_of(p, N, 7, seed=0x77 + N)
    got = sim.group_fields(0).cpu().numpy()
    ref = oracle.rdode_init(N, 7, 0.0, 2.0, 0x77 + N, 10)
    assert got.shape == (7, 2, N)
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("N,h,nst", [(64, 2e-3, 100), (32, 5e-3, 60), (128, 1e-3, 50), (256, 2e-4, 40)])
def test_fixed_schedule_parity(p, N, h, nst):
    sim = sim_of(p, N, 5, seed=N)
    w0 = sim.group_fields(0).cpu().numpy()
    rho = max(oracle.gershgorin(W.RDODE, P0, w.astype(np.float64)) for w in w0)
    s = 2
    while oracle.rkc_beta(s) < 1.1 * h * rho:
        s += 1
    st, _ = sim.integrate_rkc(h, s_fixed=s, n_fixed=nst)
    assert sim.sync_status() == 0
    got = sim.group_fields(0).cpu().numpy()
    ref = oracle.rkc_fixed(W.RDODE, P0, h, s, nst, w0)
    assert rel_err(got, ref) <= FIELD_TOL
    st = st.cpu().numpy()
    assert (st[:, 0] == nst).all() and (st[:, 2] == 1 + nst * s).all() and (st[:, 3] == s).all()


def test_adaptive_run_to_t50(p):
    # Table 1: t in [0, 50]; the GPU's result is as close to an accurate
    # reference as the oracle's own at the same tolerance, and the
    # far-from-equilibrium pattern (which nodes sit on the high branch) is
    # the same
    N, n, tol = 64, 4, 1e-6
    sim = sim_of(p, N, n, seed=123)
    w0 = sim.group_fields(0).cpu().numpy()
    st, res = sim.integrate_rkc(1e-3, t_end=50.0, rtol=tol, atol=tol, residual=True)
    assert sim.sync_status() == 0
    got = sim.group_fields(0).cpu().numpy()
    mine, ost, failed = oracle.rkc_adaptive(W.RDODE, P0, 50.0, 1e-3, tol, tol, w0)
    acc, _, _ = oracle.rkc_adaptive(W.RDODE, P0, 50.0, 1e-3, tol / 100, tol / 100, w0)
    assert failed == 0
    assert rel_err(got, acc) <= 2.0 * rel_err(mine, acc) + 1e-5
    assert np.array_equal(got[:, 0] > 1.0, acc[:, 0] > 1.0)
    st = st.cpu().numpy()
    assert np.abs(st[:, 0] - ost[:, 0]).max() <= max(3, 0.05 * ost[:, 0].max())
    if (st[:, :2] == ost[:, :2]).all():
        assert rel_err(got, mine) <= 1e-4
    # the stored FP32 state cannot do better than the rounding of w, which
    # the stiff diffusion turns into |F| up to D (N-1)^2 * 4 * ulp(w) / 2
    floor = P0[1] * (N - 1) ** 2 * 4 * np.abs(got[:, 1]).max() * 2.0 ** -24
    assert (res.cpu().numpy()[:, 0] < 2 * floor).all()


def test_residual_output(p):
    N = 64
    sim = sim_of(p, N, 3, seed=5)
    _, res = sim.integrate_rkc(2e-3, s_fixed=30, n_fixed=20, residual=True)
    got = sim.group_fields(0).cpu().numpy().astype(np.float64)
    ref = np.array([[np.abs(F).max(), np.sqrt((F ** 2).mean())]
                    for F in (oracle.rdode_rhs(P0, w) for w in got)])
    np.testing.assert_allclose(res.cpu().numpy(), ref, rtol=1e-12)


def test_c7_sample(p):
    # the c7 workload (200 realisations, own parameter draw) to t = 50;
    # a sample of realisations against the oracle's accuracy
    cfg = W.config("c7")
    gd = cfg["groups"][0]
    sim = p.Simulation([p.Group.from_dict(gd)])
    idx = [0, 57, 199]
    w0 = sim.group_fields(0)[idx].cpu().numpy()
    tol = cfg["rkc_tol"]
    st, _ = sim.integrate_rkc(1e-3, rtol=tol, atol=tol)
    assert sim.sync_status() == 0
    got = sim.group_fields(0)[idx].cpu().numpy()
    T = gd["dt"] * gd["n_steps"]
    assert T == 50.0
    mine, _, failed = oracle.rkc_adaptive(W.RDODE, gd["params"], T, 1e-3, tol, tol, w0)
    acc, _, _ = oracle.rkc_adaptive(W.RDODE, gd["params"], T, 1e-3, tol / 100, tol / 100, w0)
    assert failed == 0
    assert rel_err(got, acc) <= 2.0 * rel_err(mine, acc) + 1e-5
    assert (st.cpu().numpy()[:, 0] > 0).all()


def test_2d_only_calls_refuse_the_1d_model(p):
    sim = sim_of(p, 64, 2)
    with pytest.raises(p.RdError) as e:
        sim.integrate()
    assert e.value.status == 6
    with pytest.raises(p.RdError) as e:
        sim.integrate_f64(torch.zeros(sim.total_floats, dtype=torch.float64, device="cuda"))
    assert e.value.status == 6
    with pytest.raises(p.RdError) as e:
        sim.autotune(steps=2)
    assert e.value.status == 6
    # a mixed handle: the 2-D group still runs through rd_integrate_rkc
    both = p.Simulation([p.Group(W.FHN, 32, 2, W.FHN_THETA0, 2 ** -8, 64, (-0.05, 0.05), 1),
                         p.Group(W.RDODE, 64, 2, P0, 1e-3, 100, (0.0, 2.0), 2)])
    st, _ = both.integrate_rkc(1e-3, rtol=1e-5, atol=1e-5)
    assert both.sync_status() == 0
    assert (st.cpu().numpy()[:, 0] > 0).all()


def test_invalid_1d_groups(p):
    for G, flags in ((48, 0), (512, 0), (64, 1)):
        g = p.Group(W.RDODE, G, 1, P0, 1e-3, 1, (0.0, 2.0), 1, adjoint=bool(flags))
        with pytest.raises(p.RdError) as e:
            p.Simulation([g])
        assert e.value.status == 1
