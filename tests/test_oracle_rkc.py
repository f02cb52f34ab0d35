"""Pins of the oracle's stabilised second-order Runge-Kutta integrator
(App. B.2, Chebyshev coefficients) against facts fixed outside it:
closed forms of the Chebyshev polynomials, the exact amplification of
eigenmodes of the discrete Neumann Laplacian, convergence order against a
classical RK4 reference, the Gershgorin bound of a dense finite-difference
Jacobian, invariants (homogeneous steady state, mass under diffusion) and
the behaviour of the error control."""
import math

import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def cheb_closed(s, x):
    """T_s(x), T_s'(x), T_s''(x) for x > 1 from x = cosh(theta)."""
    th = math.acosh(x)
    sh, ch = math.sinh(th), math.cosh(th)
    T = math.cosh(s * th)
    T1 = s * math.sinh(s * th) / sh
    T2 = (s * s * math.cosh(s * th) * sh - s * math.sinh(s * th) * ch) / sh ** 3
    return T, T1, T2


def cheb_T(s, x):
    """T_s(x) for any real x (trigonometric / hyperbolic closed form)."""
    if abs(x) <= 1.0:
        return math.cos(s * math.acos(x))
    v = math.cosh(s * math.acosh(abs(x)))
    return v if x > 0 or s % 2 == 0 else -v


@pytest.mark.parametrize("s", [2, 3, 5, 17, 64, 200])
def test_coefficients_match_chebyshev_closed_form(s):
    c = oracle.rkc_coef(s)
    w0 = 1.0 + (2.0 / 13.0) / s ** 2
    T, T1, T2 = cheb_closed(s, w0)
    assert c["w0"] == pytest.approx(w0, rel=1e-15)
    assert c["w1"] == pytest.approx(T1 / T2, rel=1e-9)
    assert c["b_s"] == pytest.approx(T2 / T1 ** 2, rel=1e-9)
    assert c["a_s"] == pytest.approx(1.0 - (T2 / T1 ** 2) * T, rel=1e-9, abs=1e-12)
    assert c["beta"] == pytest.approx((1.0 + w0) * T2 / T1, rel=1e-9)
    assert oracle.rkc_beta(s) == pytest.approx(c["beta"], rel=1e-15)


def test_beta_grows_like_065_s_squared():
    # the damped (eps = 2/13) second-order Chebyshev interval: beta(s) / s^2
    # increases towards 0.653 (2/3 (1 - 2 eps / 15) at large s)
    r = [oracle.rkc_beta(s) / s ** 2 for s in (4, 16, 64, 256)]
    assert all(a < b for a, b in zip(r, r[1:]))
    assert r[-1] == pytest.approx(2.0 / 3.0 * (1.0 - 2.0 * (2.0 / 13.0) / 15.0), rel=2e-3)


def mode(G, k, l):
    x = np.arange(G)
    cx = np.cos(np.pi * k * (x + 0.5) / G)
    cy = np.cos(np.pi * l * (x + 0.5) / G)
    return np.outer(cy, cx)


def lam(G, D, k, l):
    # eigenvalue of D * Lap_h with mirrored ghosts (ghost = edge node) on
    # the DCT-II mode cos(pi k (x + 1/2) / G)
    g2 = (G - 1) ** 2
    return -4.0 * g2 * D * (math.sin(math.pi * k / (2 * G)) ** 2 + math.sin(math.pi * l / (2 * G)) ** 2)


@pytest.mark.parametrize("s", [2, 3, 7, 24])
def test_one_step_amplifies_eigenmodes_by_the_stability_polynomial(s):
    G = 16
    Du, Dv = 3e-3, 1.1e-2
    p = (Du, Dv, 0.0, 0.0)
    c = oracle.rkc_coef(s)
    rho = 8.0 * (G - 1) ** 2 * Dv
    h = 0.97 * c["beta"] / rho           # the stiffest mode near the interval's end
    for (k, l), (k2, l2) in [((1, 0), (0, 2)), ((3, 5), (15, 15)), ((15, 14), (7, 1))]:
        w = np.stack([mode(G, k, l), mode(G, k2, l2)])[None]
        out = oracle.rkc_fixed(oracle.DIFF, p, h, s, 1, w)[0]
        for sp, (kk, ll), D in ((0, (k, l), Du), (1, (k2, l2), Dv)):
            z = h * lam(G, D, kk, ll)
            R = c["a_s"] + c["b_s"] * cheb_T(s, c["w0"] + c["w1"] * z)
            assert abs(R) <= 1.0 + 1e-12
            np.testing.assert_allclose(out[sp], R * w[0, sp], rtol=0, atol=1e-12)


def test_stability_polynomial_is_second_order():
    # R_s(z) = 1 + z + z^2/2 + O(z^3): the cubic remainder shrinks by 8 per halving
    s = 9
    c = oracle.rkc_coef(s)
    rem = []
    for z in (-1e-2, -5e-3, -2.5e-3):
        R = c["a_s"] + c["b_s"] * cheb_T(s, c["w0"] + c["w1"] * z)
        rem.append(R - (1 + z + z * z / 2))
    assert rem[0] / rem[1] == pytest.approx(8.0, rel=0.02)
    assert rem[1] / rem[2] == pytest.approx(8.0, rel=0.02)


def rk4(model, p, w, T, n):
    h = T / n
    for _ in range(n):
        k1 = oracle.rhs(model, p, w)
        k2 = oracle.rhs(model, p, w + 0.5 * h * k1)
        k3 = oracle.rhs(model, p, w + 0.5 * h * k2)
        k4 = oracle.rhs(model, p, w + h * k3)
        w = w + (h / 6.0) * (k1 + 2 * k2 + 2 * k3 + k4)
    return w


@pytest.mark.parametrize("model", [oracle.FHN, oracle.GM, oracle.BZ])
def test_global_convergence_is_second_order(model):
    G = 12
    p = {oracle.FHN: W.FHN_THETA0, oracle.GM: W.GM_THETA0, oracle.BZ: W.BZ_THETA0}[model]
    lo, hi = (-0.05, 0.05) if model == oracle.FHN else (0.0, 0.01)
    w = oracle.init_fields(model, G, 1, p, lo, hi, 11).astype(np.float64)
    T = 0.5
    ref = rk4(model, p, w[0], T, 4000)
    errs = []
    rho = oracle.gershgorin(model, p, w[0])
    s = 2                                  # one stage count for all h (the
    while oracle.rkc_beta(s) < 1.2 * (T / 20) * rho:   # error constant depends on s)
        s += 1
    for n in (40, 80, 160):
        out = oracle.rkc_fixed(model, p, T / n, s, n, w)[0]
        errs.append(np.abs(out - ref).max())
    # a first-order method (a dropped or wrong coefficient) gives ratios near 2
    assert errs[0] / errs[1] == pytest.approx(4.0, rel=0.15)
    assert errs[1] / errs[2] == pytest.approx(4.0, rel=0.15)


@pytest.mark.parametrize("model", [oracle.FHN, oracle.GM, oracle.BZ])
@pytest.mark.parametrize("where", ["random", "corner", "edge"])
def test_gershgorin_equals_dense_jacobian_row_sums(model, where):
    # "corner" / "edge": a spike makes the largest row a node with 2 / 3
    # in-domain neighbours, so the boundary rows' exact weights are checked
    G = 4
    p = {oracle.FHN: W.FHN_THETA0, oracle.GM: W.GM_THETA0, oracle.BZ: W.BZ_THETA0}[model]
    rng = np.random.default_rng(5)
    u0, v0 = oracle.equilibrium(model, p)
    w = np.stack([u0 + 0.3 * rng.standard_normal((G, G)), v0 + 0.1 * rng.uniform(0.5, 1.0, (G, G))])
    if where != "random":
        w = np.stack([np.full((G, G), u0), np.full((G, G), v0 if v0 else 0.5)])
        y, x = (0, 0) if where == "corner" else (0, 2)
        w[0, y, x] = u0 + 3.0
    m = w.size
    J = np.zeros((m, m))
    for i in range(m):
        e = np.zeros(m)
        d = 1e-6 * max(1.0, abs(w.flat[i]))
        e[i] = d
        J[:, i] = (oracle.rhs(model, p, w + e.reshape(w.shape)) -
                   oracle.rhs(model, p, w - e.reshape(w.shape))).ravel() / (2 * d)
    bound = oracle.gershgorin(model, p, w)
    assert bound == pytest.approx(np.abs(J).sum(axis=1).max(), rel=1e-6)
    assert np.abs(np.linalg.eigvals(J)).max() <= bound * (1 + 1e-9)


def test_homogeneous_steady_state_stays_fixed():
    G = 16
    w = np.zeros((1, 2, G, G))
    out = oracle.rkc_fixed(oracle.FHN, W.FHN_THETA0, 0.3, 20, 5, w)
    assert np.all(out == 0.0)
    u0, v0 = oracle.equilibrium(oracle.GM, W.GM_THETA0)
    w = np.stack([np.full((G, G), u0), np.full((G, G), v0)])[None]
    out = oracle.rkc_fixed(oracle.GM, W.GM_THETA0, 0.3, 20, 5, w)
    # the stage weights (1 - mu - nu) + mu + nu sum to 1 up to rounding only
    np.testing.assert_allclose(out, w, rtol=1e-12)


def test_mass_is_conserved_under_diffusion():
    G = 20
    rng = np.random.default_rng(2)
    w = rng.uniform(0, 1, (1, 2, G, G))
    p = (2e-3, 7e-3)
    out = oracle.rkc_fixed(oracle.DIFF, p, 0.05, 12, 10, w)
    np.testing.assert_allclose(out.sum(axis=(2, 3)), w.sum(axis=(2, 3)), rtol=1e-13)
    assert np.abs(out - out.mean(axis=(2, 3), keepdims=True)).max() < np.abs(w - 0.5).max()


@pytest.mark.parametrize("model", [oracle.FHN, oracle.BZ])
def test_adaptive_accuracy_follows_the_tolerance(model):
    # Local-error control of a second-order method: each step's local error
    # ~ tol, steps ~ tol^(-1/3), so the global error ~ tol^(2/3) (a factor
    # 10^(2/3) = 4.6 per decade of tolerance).  An estimate that lost its
    # F terms (O(h) instead of O(h^3)) would give a factor 10; a controller
    # exponent that does not match the estimate oscillates and rejects.
    G = 12
    p = W.FHN_THETA0 if model == oracle.FHN else W.BZ_THETA0
    lo, hi = (-0.05, 0.05) if model == oracle.FHN else (0.0, 0.01)
    w = oracle.init_fields(model, G, 1, p, lo, hi, 3).astype(np.float64)
    T = 2.0
    ref = rk4(model, p, w[0], T, 20000)
    scale = np.abs(ref).max()
    err, steps = [], []
    for tol in (1e-5, 1e-6, 1e-7):
        wa, st, failed = oracle.rkc_adaptive(model, p, T, 1e-3, tol, tol, w)
        assert failed == 0
        acc, rej, nrhs, smax = st[0]
        assert rej <= 0.1 * acc + 2                    # the controller is stable
        assert 1 + 2 * (acc + rej) <= nrhs <= 1 + smax * (acc + rej)
        err.append(np.abs(wa[0] - ref).max() / scale)
        steps.append(acc)
    for a, b in zip(err, err[1:]):
        assert 3.0 < a / b < 7.0
    for a, b in zip(steps, steps[1:]):
        assert 1.6 < b / a < 2.8                       # 10^(1/3) = 2.15
    assert err[-1] < 1e-4


def test_adaptive_lands_on_t_end_and_counts_stages():
    G = 16
    w = oracle.init_fields(oracle.FHN, G, 2, W.FHN_THETA0, -0.05, 0.05, 9).astype(np.float64)
    wa, st, failed = oracle.rkc_adaptive(oracle.FHN, W.FHN_THETA0, 1.0, 0.01, 1e-4, 1e-4, w)
    assert failed == 0
    # integrating to 0.4 and then 0.6 more reaches (nearly) the same state
    wb, _, _ = oracle.rkc_adaptive(oracle.FHN, W.FHN_THETA0, 0.4, 0.01, 1e-4, 1e-4, w)
    wc, _, _ = oracle.rkc_adaptive(oracle.FHN, W.FHN_THETA0, 0.6, 0.01, 1e-4, 1e-4, wb)
    assert np.abs(wc - wa).max() < 1e-3 * np.abs(wa).max()
    # stage counts respect the stability rule at the first step
    rho = oracle.gershgorin(oracle.FHN, W.FHN_THETA0, w[0])
    assert st[0, 3] >= 2 and oracle.rkc_beta(int(st[0, 3])) >= 0.01 * rho


def test_stage_cap_cuts_the_step():
    G = 16
    w = oracle.init_fields(oracle.FHN, G, 1, W.FHN_THETA0, -0.05, 0.05, 4).astype(np.float64)
    wa, st, failed = oracle.rkc_adaptive(oracle.FHN, W.FHN_THETA0, 5.0, 1.0, 1e-2, 1e-2, w, s_max=4)
    assert failed == 0
    rho = oracle.gershgorin(oracle.FHN, W.FHN_THETA0, w[0])
    assert st[0, 3] == 4
    # every step is at most beta(4) / rho long (rho changes little here)
    assert st[0, 0] >= 5.0 * rho / oracle.rkc_beta(4) * 0.8
    assert np.isfinite(wa).all()
