"""Pins of the oracle's reaction-diffusion part against facts the paper and
the mathematics fix (not against the oracle's own formulas).

Paper: arXiv 2203.14742 -- eq. (rdgen) and kinetics, Sec. 4.1; equilibria,
Sec. 4.1; 5-point Laplacian with mirrored Neumann ghosts, App. B.1.1;
initial noise, Sec. 4.1; explicit Euler, Sec. 5.1.
"""
import math

import numpy as np
import pytest

import oracle
import workloads as W

FHN, GM, DIFF, BZ = oracle.FHN, oracle.GM, oracle.DIFF, oracle.BZ


def dct_mode(G, k, l):
    xs = (np.arange(G) + 0.5) / G
    return np.outer(np.cos(math.pi * l * xs), np.cos(math.pi * k * xs))  # [y][x]


def sigma_kl(G, k, l):
    """Eigenvalue magnitude of the mirrored-ghost 5-point Laplacian on the
    DCT-II mode (k, l): 4 (G-1)^2 [sin^2(pi k/2G) + sin^2(pi l/2G)]."""
    return 4.0 * (G - 1) ** 2 * (math.sin(math.pi * k / (2 * G)) ** 2 +
                                 math.sin(math.pi * l / (2 * G)) ** 2)


# ---------------------------------------------------------------- generator

def test_splitmix64_published_outputs():
    # First outputs of SplitMix64 started from state 0 (Steele, Lea & Flood
    # 2014; the values printed by the reference implementation).
    assert oracle.sm64(0, 0) == 0xE220A8397B1DCDAF
    assert oracle.sm64(0, 1) == 0x6E789E6AA1B965F4
    assert oracle.sm64(0, 2) == 0x06C45D188009454F


def test_init_fields_range_moments_and_layout():
    p = W.FHN_THETA0
    f = oracle.init_fields(FHN, 64, 8, p, -0.05, 0.05, 12345)
    assert f.dtype == np.float32 and f.shape == (8, 2, 64, 64)
    assert f.min() >= -0.05 and f.max() <= 0.05
    n = f.size
    # U(-a, a): mean 0 (sd a/sqrt(3n)), variance a^2/3.
    assert abs(f.mean()) < 5 * 0.05 / math.sqrt(3 * n)
    assert abs(f.astype(np.float64).var() - 0.05 ** 2 / 3) < 0.05 * 0.05 ** 2 / 3
    # Counter layout: realisation r of a larger batch equals the smaller one.
    g = oracle.init_fields(FHN, 64, 3, p, -0.05, 0.05, 12345)
    assert np.array_equal(f[:3], g)
    # A different seed is a different stream.
    h = oracle.init_fields(FHN, 64, 3, p, -0.05, 0.05, 12346)
    assert not np.array_equal(g, h)


def test_init_gm_positive_noise_around_equilibrium():
    p = (2.5e-4, 0.01, 1.0, 0.5)
    f = oracle.init_fields(GM, 32, 4, p, 0.0, 0.01, 7)
    # Equilibrium (1/mu, 1/mu^2) = (2, 4) for mu = 0.5 (Sec. 4.1).
    assert f[:, 0].min() >= 2.0 and f[:, 0].max() <= 2.01
    assert f[:, 1].min() >= 4.0 and f[:, 1].max() <= 4.01


# ---------------------------------------------------------------- Laplacian

def test_constant_field_has_zero_laplacian():
    w = np.full((2, 16, 16), 0.37)
    F = oracle.rhs(DIFF, (1.0, 2.0), w)
    assert np.all(F == 0.0)


def test_mass_conservation_pure_diffusion():
    rng = np.random.default_rng(0)
    w0 = rng.uniform(-1, 1, size=(1, 2, 24, 24))
    w = oracle.step(DIFF, (0.3e-3, 1e-3), 1e-2 / 24 ** 2, 200, w0)
    for s in range(2):
        s0, s1 = w0[0, s].sum(), w[0, s].sum()
        assert abs(s1 - s0) < 1e-12 * np.abs(w0[0, s]).sum()
    # and diffusion actually happened
    assert np.abs(w - w0).max() > 1e-3


def test_laplacian_symmetric():
    rng = np.random.default_rng(1)
    G = 13
    x = rng.normal(size=(2, G, G))
    y = rng.normal(size=(2, G, G))
    Lx = oracle.rhs(DIFF, (1.0, 1.0), x)
    Ly = oracle.rhs(DIFF, (1.0, 1.0), y)
    a, b = np.vdot(Lx, y), np.vdot(x, Ly)
    assert abs(a - b) < 1e-10 * abs(a)


@pytest.mark.parametrize("G,k,l", [(16, 1, 0), (16, 2, 3), (32, 5, 1), (9, 4, 4)])
def test_dct_mode_decay_closed_form(G, k, l):
    Du, Dv = 2e-3, 5e-4
    dt = 0.2 / (G - 1) ** 2 / max(Du, Dv)
    n = 50
    m = dct_mode(G, k, l)
    w0 = np.stack([m, 0.5 * m])[None]
    w = oracle.step(DIFF, (Du, Dv), dt, n, w0)
    s = sigma_kl(G, k, l)
    fu = (1.0 - dt * Du * s) ** n
    fv = (1.0 - dt * Dv * s) ** n
    assert np.abs(w[0, 0] - fu * m).max() < 1e-12
    assert np.abs(w[0, 1] - fv * 0.5 * m).max() < 1e-12


def test_laplacian_orientation_non_square_mode():
    # A mode varying only in x must stay constant along y (rows identical).
    G = 12
    m = dct_mode(G, 3, 0)
    w = oracle.step(DIFF, (1e-3, 1e-3), 1e-3, 5, np.stack([m, m])[None])
    assert np.abs(w[0, 0] - w[0, 0][0:1, :]).max() == 0.0


# ---------------------------------------------------------------- equilibria

def test_fhn_equilibrium_is_exact_fixed_point():
    p = W.FHN_THETA0
    w0 = np.zeros((1, 2, 16, 16))
    F = oracle.rhs(FHN, p, w0[0])
    assert np.all(F == 0.0)
    w = oracle.step(FHN, p, 2 ** -10, 300, w0)
    assert np.array_equal(w, w0)


def test_gm_equilibrium_is_exact_fixed_point():
    p = (2.5e-4, 0.01, 1.0, 0.5)
    u0, v0 = oracle.equilibrium(GM, p)
    assert (u0, v0) == (2.0, 4.0)   # (mu_w/mu_v, mu_w/mu_v^2), Sec. 4.1
    w0 = np.stack([np.full((16, 16), u0), np.full((16, 16), v0)])[None]
    assert np.all(oracle.rhs(GM, p, w0[0]) == 0.0)
    w = oracle.step(GM, p, 2 ** -8, 300, w0)
    assert np.array_equal(w, w0)


def test_bz_equilibrium_is_exact_fixed_point():
    # A = 2, B = 3: the equilibrium (A, B/A) = (2, 1.5) is exact in FP64
    p = (1.6e-3, 1.32e-2, 2.0, 3.0)
    u0, v0 = oracle.equilibrium(BZ, p)
    assert (u0, v0) == (2.0, 1.5)   # (A, B/A), Sec. 4.1
    w0 = np.stack([np.full((16, 16), u0), np.full((16, 16), v0)])[None]
    assert np.all(oracle.rhs(BZ, p, w0[0]) == 0.0)
    w = oracle.step(BZ, p, 2 ** -8, 300, w0)
    assert np.array_equal(w, w0)


def test_bz_kinetics_at_a_worked_point():
    """F at u = 1, v = 2 with A = 4.5, B = 6.96 and no diffusion: by hand
    A - (B+1) u + u^2 v = 4.5 - 7.96 + 2 = -1.46 and B u - u^2 v = 4.96."""
    p = (0.0, 0.0, 4.5, 6.96)
    w = np.stack([np.ones((4, 4)), np.full((4, 4), 2.0)])
    F = oracle.rhs(BZ, p, w)
    assert np.allclose(F[0], -1.46, rtol=1e-15) and np.allclose(F[1], 4.96, rtol=1e-15)


def test_residual_zero_at_equilibrium_and_matches_one_step():
    p = W.FHN_THETA0
    assert np.all(oracle.residual(FHN, p, np.zeros((2, 2, 8, 8))) == 0.0)
    f = oracle.init_fields(FHN, 16, 2, p, -0.05, 0.05, 3).astype(np.float64)
    dt = 2 ** -10
    w1 = oracle.step(FHN, p, dt, 1, f)
    r = oracle.residual(FHN, p, f)
    dd = (w1 - f) / dt
    for i in range(2):
        assert r[i, 0] == pytest.approx(np.abs(dd[i]).max(), rel=1e-9)
        assert r[i, 1] == pytest.approx(math.sqrt((dd[i] ** 2).mean()), rel=1e-9)


# ---------------------------------------------------------------- dispersion

def jac(model, p):
    """Reaction Jacobian at the homogeneous equilibrium, from the kinetics of
    Sec. 4.1 (derived by hand)."""
    Du, Dv, a3, a4 = p
    if model == FHN:
        eps, a = a3, a4
        return np.array([[1.0, -1.0], [eps, -eps * a]])
    if model == GM:
        rho, mu = a3, a4
        return rho * np.array([[mu, -mu * mu], [2.0 / mu, -1.0]])
    # Brusselator at (A, B/A): d/du (A - (B+1) u + u^2 v) = -(B+1) + 2 u v = B - 1,
    # d/dv = u^2 = A^2; d/du (B u - u^2 v) = B - 2 u v = -B, d/dv = -A^2
    A, B = a3, a4
    return np.array([[B - 1.0, A * A], [-B, -A * A]])


@pytest.mark.parametrize("model,p,G,k,l,dt", [
    (FHN, W.FHN_THETA0, 32, 3, 2, 2 ** -9),
    (FHN, (2.6e-4, 0.052, 9.5, 0.93), 32, 5, 0, 2 ** -9),
    (GM, (2.5e-4, 0.01, 1.0, 0.5), 32, 4, 1, 2 ** -8),
    (GM, (2.5e-4, 0.01, 1.0, 0.53), 16, 2, 2, 2 ** -8),
    (BZ, W.BZ_THETA0, 32, 3, 1, 2 ** -8),
    (BZ, (1.6e-3, 1.32e-2, 4.4, 7.1), 16, 1, 1, 2 ** -8),
])
def test_linear_dispersion(model, p, G, k, l, dt):
    """A small perturbation along DCT mode (k,l) evolves by the matrix power
    (I + dt (J - sigma_kl D))^n of the linearised discrete system."""
    u0, v0 = oracle.equilibrium(model, p)
    m = dct_mode(G, k, l)
    amp = 1e-8
    c = np.array([1.0, -0.7])
    w0 = np.stack([u0 + amp * c[0] * m, v0 + amp * c[1] * m])[None]
    n = 200
    w = oracle.step(model, p, dt, n, w0)
    A = np.eye(2) + dt * (jac(model, p) - sigma_kl(G, k, l) * np.diag([p[0], p[1]]))
    cn = np.linalg.matrix_power(A, n) @ c
    got = np.array([(w[0, 0] - u0).ravel() @ m.ravel(), (w[0, 1] - v0).ravel() @ m.ravel()])
    got = got / (amp * (m.ravel() @ m.ravel()))
    scale = np.abs(cn).max()
    # O(amplitude) nonlinearity and FP64 rounding relative to u0 ~ 2.
    assert np.abs(got - cn).max() < 1e-5 * max(1.0, scale) + 1e-7 * scale


@pytest.mark.parametrize("cfg", ["c1", "c2", "c3", "c4", "c5", "c6"])
def test_drawn_parameters_are_turing_unstable(cfg):
    """Every drawn parameter vector has some non-constant discrete mode with
    Re lambda > 0 and a stable (or, at a = 1, marginal) constant mode: the
    diffusion-driven instability of Sec. 4.1."""
    c = W.config(cfg, steps_scale=1e-6)
    for g in c["groups"]:
        p, G, model = g["params"], g["G"], g["model"]
        J = jac(model, p)
        D = np.diag([p[0], p[1]])
        lam0 = np.linalg.eigvals(J).real.max()
        assert lam0 <= 1e-12
        best = -1e9
        for k in range(G):
            for l in range(G):
                if k == 0 and l == 0:
                    continue
                best = max(best, np.linalg.eigvals(J - sigma_kl(G, k, l) * D).real.max())
        assert best > 0.05, (cfg, p, best)


def test_explicit_time_step_below_diffusion_limit():
    for cfg in ("c1", "c2", "c3", "c4", "c5", "c6"):
        for g in W.config(cfg, steps_scale=1e-6)["groups"]:
            h2 = 1.0 / (g["G"] - 1) ** 2
            assert g["dt"] < h2 / (4 * max(g["params"][0], g["params"][1]))
            assert math.log2(g["dt"]) == int(math.log2(g["dt"]))
