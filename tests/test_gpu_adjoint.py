"""GPU adjoint (smoothed-CIL gradient) against the oracle's FP64 discrete
adjoint, which the CPU suite pins to central finite differences.

Tolerances.  The GPU runs the forward and reverse recursions in FP32 (FP64
only for the parameter accumulators), the oracle in FP64.
 * C: a distance error dd moves C_k by at most max(sigma')/tau_k * dd =
   dd / (4 tau_k) = 5 dd / R_k, so with field errors within the 1e-5 field
   tolerance and d <= R_0 the smoothed integral may differ by
   5e-5 * R_0 / R_M absolute at most; the test uses 5e-5 absolute plus 1e-4
   relative.
 * grad, per component p: g_p is a sum of terms dt lambda . dF/dtheta_p(w)
   over realisations, steps and cells.  FP32 perturbs every term relatively
   by about the relative error of the state (forward) and of lambda
   (reverse, the transposed linearisation of the same recursion, so the
   same order), so |g_gpu,p - g_p| <= K e_f A_p with e_f the field error
   this very run shows at its last step relative to the pattern's amplitude
   (measured in the test, GPU vs oracle) and A_p the oracle's sum of the
   terms' magnitudes (which
   is what cancellation inside g_p cannot shrink).  K = 32 covers the two
   relative errors, the Laplacian's differences inside dF/dDu and dF/dDv
   (which turn a relative state error into a larger relative error of the
   term) and margin; 1e-9 |g_p| covers the FP64 accumulation.
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


K_GRAD = 32.0


def field_error(sim, f0, w0, model, par, dt, steps):
    """Field error of the GPU's FP32 run against the oracle after `steps`,
    relative to the pattern's amplitude: per realisation and species
    max |a - b| / (max b - min b), then the largest.  (Relative to max |b|
    it would understate the error of patterns that are small deviations
    from a large equilibrium, as GM's are early on.)"""
    n = w0.shape[0]
    sim.fields.copy_(f0)
    sim.integrate(steps=steps, residual=False)
    wg = sim.group_fields(0).cpu().numpy().astype(np.float64).reshape(n, 2, -1)
    wo = oracle.step(model, par, dt, steps, w0).reshape(n, 2, -1)
    err = np.abs(wg - wo).max(-1) / (wo.max(-1) - wo.min(-1))
    sim.fields.copy_(f0)
    return float(err.max())


def compare(sim, f0, w0, set1, set2, radii, cot, model, par, dt, steps, mask, tau=0.05):
    Cg, gg = sim.adjoint(0, f0, mask, set1, set2, torch.from_numpy(radii), tau, torch.from_numpy(cot))
    Co, go, A = oracle.smooth_cil_grad(model, par, dt, steps, w0, mask, set1, set2, radii, tau, cot,
                                       with_abs=True)
    Cg, gg = Cg.cpu().numpy(), gg.cpu().numpy()
    assert np.allclose(Cg, Co, rtol=1e-4, atol=5e-5)
    e_f = field_error(sim, f0, w0, model, par, dt, steps)
    tol = 1e-9 * np.abs(go) + K_GRAD * max(e_f, 2.0 ** -24) * A
    print("grad gpu", gg, "oracle", go, "|diff|", np.abs(gg - go), "tol", tol, "A", A, "e_f", e_f)
    assert np.all(np.abs(gg - go) <= tol), (gg, go, tol)
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


@pytest.mark.parametrize("model,par,dt,noise,steps", [
    (W.FHN, (2.8e-4, 0.05, 10.0, 0.95), 2 ** -8, (-0.05, 0.05), 60),
    (W.GM, (2.5e-4, 0.01, 1.0, 0.5), 2 ** -8, (0.0, 0.5), 60),
    (W.BZ, W.BZ_THETA0, 2 ** -8, (0.0, 1.0), 60),
])
def test_adjoint_every_component_pinned(p, model, par, dt, noise, steps):
    """Cases in which the derived per-component bound pins every parameter's
    derivative (Du, Dv and the two reaction parameters) to within 10 % of
    its value, not only the largest one.  The bound scales with the FP32
    field error relative to the pattern's range; GM and BZ patterns that are
    0.01-deviations from an equilibrium of order 2-5 carry the equilibrium's
    rounding (e_f ~ 2e-5, and the reaction components sum terms far larger
    than their values), so here the initial perturbations are of order one
    and the horizon short."""
    sim, f0, w0, s1, s2, radii, cot = problem(p, model, 32, 8, par, dt, steps, noise, 57, 3)
    Cg, gg = sim.adjoint(0, f0, 3, s1, s2, torch.from_numpy(radii), 0.05, torch.from_numpy(cot))
    Co, go, A = oracle.smooth_cil_grad(model, par, dt, steps, w0, 3, s1, s2, radii, 0.05, cot, with_abs=True)
    gg = gg.cpu().numpy()
    e_f = field_error(sim, f0, w0, model, par, dt, steps)
    tol = 1e-9 * np.abs(go) + K_GRAD * max(e_f, 2.0 ** -24) * A
    print("pinned", model, "gpu", gg, "oracle", go, "tol/|g|", tol / np.abs(go), "e_f", e_f)
    assert np.all(np.abs(gg - go) <= tol), (gg, go, tol)
    assert np.all(tol <= 0.1 * np.abs(go)), tol / np.abs(go)


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


def test_smooth_cil_follows_theta(p):
    """SmoothCIL.apply evaluates C at the theta it is given (not at the
    handle's parameters), and its backward gives the gradient there: both
    match the oracle at theta_1 != theta_0, and C moves."""
    par0 = (2.8e-4, 0.05, 10.0, 0.95)
    par1 = (3.1e-4, 0.046, 10.6, 0.92)
    dt, steps = 2 ** -8, 150
    sim, f0, w0, s1, s2, radii, cot = problem(p, W.FHN, 32, 6, par0, dt, steps, (-0.05, 0.05), 9, 3)
    r = torch.from_numpy(radii)
    C0 = p.SmoothCIL.apply(torch.tensor(par0, dtype=torch.float64), sim, 0, f0, 3, s1, s2, r, 0.05)
    theta = torch.tensor(par1, dtype=torch.float64, requires_grad=True)
    C1 = p.SmoothCIL.apply(theta, sim, 0, f0, 3, s1, s2, r, 0.05)
    assert not torch.allclose(C0, C1, rtol=1e-3, atol=0)
    loss = (C1 * torch.from_numpy(cot).cuda()).sum()
    loss.backward()
    Co, go, A = oracle.smooth_cil_grad(W.FHN, par1, dt, steps, w0, 3, s1, s2, radii, 0.05, cot, with_abs=True)
    assert np.allclose(C1.detach().cpu().numpy(), Co, rtol=1e-4, atol=5e-5)
    e_f = field_error(sim, f0, w0, W.FHN, par1, dt, steps)
    tol = 1e-9 * np.abs(go) + K_GRAD * max(e_f, 2.0 ** -24) * A
    assert np.all(np.abs(theta.grad.numpy() - go) <= tol), (theta.grad, go, tol)


def test_smooth_cil_central_differences_on_gpu(p):
    """Directional central differences of the GPU's own smoothed integral
    through SmoothCIL.apply, relative step h_i = 1e-4 |theta_i| per
    component, against the GPU adjoint.  The FP32 forward runs at theta +- h
    round differently, which adds noise of order e_f |L| / h_i to the
    difference quotient; the bound is 2 % of |g_i| plus that noise (x 8)."""
    par = (2.8e-4, 0.05, 10.0, 0.95)
    dt, steps = 2 ** -8, 150
    sim, f0, w0, s1, s2, radii, cot = problem(p, W.FHN, 32, 6, par, dt, steps, (-0.05, 0.05), 19, 3)
    r = torch.from_numpy(radii)
    cot_t = torch.from_numpy(cot).cuda()
    theta = torch.tensor(par, dtype=torch.float64, requires_grad=True)
    L = (p.SmoothCIL.apply(theta, sim, 0, f0, 3, s1, s2, r, 0.05) * cot_t).sum()
    L.backward()
    g = theta.grad.numpy()
    e_f = field_error(sim, f0, w0, W.FHN, par, dt, steps)
    for i in range(4):
        h = 1e-4 * abs(par[i])
        tp, tm = list(par), list(par)
        tp[i] += h
        tm[i] -= h
        Lp = float((p.SmoothCIL.apply(torch.tensor(tp, dtype=torch.float64), sim, 0, f0, 3, s1, s2, r, 0.05)
                    * cot_t).sum())
        Lm = float((p.SmoothCIL.apply(torch.tensor(tm, dtype=torch.float64), sim, 0, f0, 3, s1, s2, r, 0.05)
                    * cot_t).sum())
        fd = (Lp - Lm) / (2 * h)
        noise = 8.0 * max(e_f, 2.0 ** -24) * abs(L.item()) / h
        print("param", i, "fd", fd, "adjoint", g[i], "noise bound", noise)
        assert abs(fd - g[i]) <= 0.02 * abs(g[i]) + noise, (i, fd, g[i], noise)


def test_autograd_function(p):
    par = (2.8e-4, 0.05, 10.0, 0.95)
    sim, f0, w0, s1, s2, radii, cot = problem(p, W.FHN, 32, 6, par, 2 ** -8, 120, (-0.05, 0.05), 9, 3)
    theta = torch.tensor(par, dtype=torch.float64, requires_grad=True)
    C = p.SmoothCIL.apply(theta, sim, 0, f0, 3, s1, s2, torch.from_numpy(radii), 0.05)
    loss = (C * torch.from_numpy(cot).cuda()).sum()
    loss.backward()
    _, g = sim.adjoint(0, f0, 3, s1, s2, torch.from_numpy(radii), 0.05, torch.from_numpy(cot))
    assert torch.allclose(theta.grad.cuda(), g, rtol=1e-12, atol=0)
