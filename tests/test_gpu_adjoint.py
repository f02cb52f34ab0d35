"""GPU adjoint (smoothed-CIL gradient) against the oracle's FP64 discrete
adjoint, which the CPU suite pins to central finite differences.

Tolerances: the GPU runs the forward and reverse recursions in FP32 (FP64
only for the parameter accumulators), the oracle in FP64.  A distance error
dd moves C_k by at most max(sigma')/tau_k * dd = dd / (4 tau_k) =
5 dd / R_k, so with field errors within the 1e-5 field tolerance and
d <= R_0 the smoothed integral may differ by 5e-5 * R_0 / R_M absolute at
most; the test uses 5e-5 absolute plus 1e-4 relative.  The gradient is
compared at 2e-3 relative to its largest component (FP32 rounding of lambda
through every reverse step).
"""
import numpy as np
import pytest
import torch

import oracle
import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def p():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2203_14742_b300 as pk
    return pk


def problem(p, model, G, n_real, par, dt, steps, noise, seed, mask, M=6, shrink=1.15):
    g = p.Group(model, G, n_real, par, dt, steps, noise, seed, adjoint=True)
    sim = p.Simulation([g])
    f0 = sim.fields.clone()
    w0 = f0.view(n_real, 2, G, G).cpu().numpy().astype(np.float64)
    half = n_real // 2
    set1, set2 = list(range(half)), list(range(half, n_real))
    wN = oracle.step(model, par, dt, steps, w0)
    X = oracle.patterns(wN, mask)
    d = np.sqrt(((X[:half, None, :] - X[None, half:, :]) ** 2).sum(-1))
    radii = d.max() * shrink ** -np.arange(1, M + 1)
    cot = np.linspace(1.0, 0.3, M)
    return sim, f0, w0, set1, set2, radii, cot


def compare(sim, f0, w0, set1, set2, radii, cot, model, par, dt, steps, mask, tau=0.05):
    Cg, gg = sim.adjoint(0, f0, mask, set1, set2, torch.from_numpy(radii), tau, torch.from_numpy(cot))
    Co, go = oracle.smooth_cil_grad(model, par, dt, steps, w0, mask, set1, set2, radii, tau, cot)
    Cg, gg = Cg.cpu().numpy(), gg.cpu().numpy()
    assert np.allclose(Cg, Co, rtol=1e-4, atol=5e-5)
    scale = np.abs(go).max()
    assert np.abs(gg - go).max() <= 2e-3 * scale, (gg, go)
    return gg, go


@pytest.mark.parametrize("model,par,dt,noise", [
    (W.FHN, (2.8e-4, 0.05, 10.0, 0.95), 2 ** -8, (-0.05, 0.05)),
    (W.GM, (2.5e-4, 0.01, 1.0, 0.5), 2 ** -8, (0.0, 0.01)),
    (W.BZ, W.BZ_THETA0, 2 ** -8, (0.0, 0.01)),
])
def test_adjoint_small_matches_oracle(p, model, par, dt, noise):
    steps = 300
    sim, f0, w0, s1, s2, radii, cot = problem(p, model, 32, 8, par, dt, steps, noise, 31, 3)
    compare(sim, f0, w0, s1, s2, radii, cot, model, par, dt, steps, 3)


def test_adjoint_u_only_mask_and_ragged_segments(p):
    # 97 steps: segments of 10 with a short last one
    par = (3e-4, 0.05, 10.0, 0.93)
    sim, f0, w0, s1, s2, radii, cot = problem(p, W.FHN, 64, 6, par, 2 ** -10, 97, (-0.05, 0.05), 4, 1)
    compare(sim, f0, w0, s1, s2, radii, cot, W.FHN, par, 2 ** -10, 97, 1)


def test_adjoint_c5_full_config(p):
    cfg = W.config("c5")
    g = cfg["groups"][0]
    sim, f0, w0, s1, s2, radii, cot = problem(p, g["model"], g["G"], g["n_real"], g["params"], g["dt"],
                                              g["n_steps"], g["noise"], g["seed"], g["species_mask"],
                                              M=cfg["M"], shrink=cfg["b"])
    cot = np.full(cfg["M"], 1.0 / cfg["M"])
    gg, go = compare(sim, f0, w0, s1, s2, radii, cot, g["model"], g["params"], g["dt"], g["n_steps"],
                     g["species_mask"], tau=cfg["tau_frac"])
    print("c5 gradient gpu", gg, "oracle", go)


def test_autograd_function(p):
    par = (2.8e-4, 0.05, 10.0, 0.95)
    sim, f0, w0, s1, s2, radii, cot = problem(p, W.FHN, 32, 6, par, 2 ** -8, 120, (-0.05, 0.05), 9, 3)
    theta = torch.tensor(par, dtype=torch.float64, requires_grad=True)
    C = p.SmoothCIL.apply(theta, sim, 0, f0, 3, s1, s2, torch.from_numpy(radii), 0.05)
    loss = (C * torch.from_numpy(cot).cuda()).sum()
    loss.backward()
    _, g = sim.adjoint(0, f0, 3, s1, s2, torch.from_numpy(radii), 0.05, torch.from_numpy(cot))
    assert torch.allclose(theta.grad.cuda(), g, rtol=1e-12, atol=0)
