"""Pins of the oracle's discrete adjoint (gradient of the sigmoid-smoothed
correlation integral with respect to the model parameters).

The paper itself is gradient-free (DE and adaptive MCMC, Sec. 2.1-2.2); the
smoothed surrogate C_tau,k = mean_ij sigma((R_k - d_ij)/tau_k) replaces the
indicator of eq. (eCDF).  Pinned by central finite differences of the FP64
forward oracle, a Taylor remainder test and a JVP/VJP dot-product test.
"""
import numpy as np
import pytest

import oracle
import workloads as W

FHN, GM, BZ = oracle.FHN, oracle.GM, oracle.BZ


def small_problem(model):
    G, n_real, steps = 12, 6, 120
    if model == FHN:
        p = np.array([2.8e-3, 0.05, 10.0, 0.95])
        dt, lo, hi = 2.0 ** -12, -0.05, 0.05
    elif model == GM:
        p = np.array([2.5e-3, 0.05, 1.0, 0.5])
        dt, lo, hi = 2.0 ** -10, 0.0, 0.01
    else:
        p = np.array([1.6e-3, 1.32e-2, 4.5, 6.96])
        dt, lo, hi = 2.0 ** -9, 0.0, 0.01
    w0 = oracle.init_fields(model, G, n_real, p, lo, hi, 4242).astype(np.float64)
    set1, set2 = np.arange(0, 3), np.arange(3, 6)
    wN = oracle.step(model, p, dt, steps, w0)
    X1 = oracle.patterns(wN[set1], 3)
    X2 = oracle.patterns(wN[set2], 3)
    d = np.sqrt(np.array([[((a - b) ** 2).sum() for b in X2] for a in X1]))
    M = 5
    radii = d.max() * 1.15 ** -np.arange(1, M + 1)
    cot = np.linspace(0.5, 1.5, M)
    return dict(model=model, p=p, dt=dt, steps=steps, w0=w0, set1=set1, set2=set2,
                radii=radii, cot=cot, mask=3)


@pytest.mark.parametrize("model", [FHN, GM, BZ])
def test_adjoint_matches_central_differences(model):
    P = small_problem(model)
    C, g = oracle.smooth_cil_grad(P["model"], P["p"], P["dt"], P["steps"], P["w0"], P["mask"],
                                  P["set1"], P["set2"], P["radii"], 0.05, P["cot"])
    assert np.all((C > 0) & (C < 1))
    for i in range(4):
        h = 1e-4 * abs(P["p"][i])
        pp, pm = P["p"].copy(), P["p"].copy()
        pp[i] += h
        pm[i] -= h
        Lp, _ = oracle.smooth_cil_loss(P["model"], pp, P["dt"], P["steps"], P["w0"], P["mask"],
                                       P["set1"], P["set2"], P["radii"], 0.05, P["cot"])
        Lm, _ = oracle.smooth_cil_loss(P["model"], pm, P["dt"], P["steps"], P["w0"], P["mask"],
                                       P["set1"], P["set2"], P["radii"], 0.05, P["cot"])
        fd = (Lp - Lm) / (2 * h)
        assert g[i] == pytest.approx(fd, rel=2e-5, abs=1e-9 * max(1.0, abs(fd))), i


def test_adjoint_taylor_remainder_is_second_order():
    P = small_problem(FHN)
    C, g = oracle.smooth_cil_grad(P["model"], P["p"], P["dt"], P["steps"], P["w0"], P["mask"],
                                  P["set1"], P["set2"], P["radii"], 0.05, P["cot"])
    L0, _ = oracle.smooth_cil_loss(P["model"], P["p"], P["dt"], P["steps"], P["w0"], P["mask"],
                                   P["set1"], P["set2"], P["radii"], 0.05, P["cot"])
    e = np.array([1.0, -0.5, 0.3, 0.8]) * P["p"]
    rem = []
    for eps in (1e-2, 5e-3, 2.5e-3):
        L, _ = oracle.smooth_cil_loss(P["model"], P["p"] + eps * e, P["dt"], P["steps"], P["w0"],
                                      P["mask"], P["set1"], P["set2"], P["radii"], 0.05, P["cot"])
        rem.append(abs(L - L0 - eps * g @ e))
    r1, r2 = rem[0] / rem[1], rem[1] / rem[2]
    assert 3.0 < r1 < 5.0 and 3.0 < r2 < 5.0, rem


@pytest.mark.parametrize("model", [FHN, GM, BZ])
def test_jvp_vjp_dot_product(model):
    rng = np.random.default_rng(3)
    G = 9
    if model == FHN:
        p = np.array([3e-3, 0.04, 9.0, 0.9])
        w = rng.normal(scale=0.5, size=(2, G, G))
    else:
        p = np.array([2e-3, 0.03, 1.2, 0.55])
        w = np.stack([2 + 0.1 * rng.normal(size=(G, G)), 4 + 0.1 * rng.normal(size=(G, G))])
    dw = rng.normal(size=(2, G, G))
    dth = rng.normal(size=4)
    lam = rng.normal(size=(2, G, G))
    jv = oracle.jvp(model, p, w, dw, dth)
    vw, vt = oracle.vjp(model, p, w, lam)
    a = np.vdot(lam, jv)
    b = np.vdot(vw, dw) + vt @ dth
    assert a == pytest.approx(b, rel=1e-12)
    # and the JVP is the derivative of F: central differences
    h = 1e-6
    Fp = oracle.rhs(model, p + h * dth, w + h * dw)
    Fm = oracle.rhs(model, p - h * dth, w - h * dw)
    assert np.allclose((Fp - Fm) / (2 * h), jv, rtol=1e-6, atol=1e-6 * np.abs(jv).max())


def test_smooth_cil_pattern_gradient_fd():
    rng = np.random.default_rng(5)
    X1 = rng.normal(size=(3, 20))
    X2 = rng.normal(size=(4, 20))
    radii = np.array([7.0, 6.0, 5.0])
    cot = np.array([1.0, -0.4, 2.0])
    C, g1, g2 = oracle.smooth_cil(X1, X2, radii, 0.05, cot)
    h = 1e-6
    for (X, g, first) in ((X1, g1, True), (X2, g2, False)):
        for idx in [(0, 0), (1, 7), (2, 19)]:
            Xp, Xm = X.copy(), X.copy()
            Xp[idx] += h
            Xm[idx] -= h
            Cp, _, _ = oracle.smooth_cil(Xp if first else X1, X2 if first else Xp, radii, 0.05, cot, grad=False)
            Cm, _, _ = oracle.smooth_cil(Xm if first else X1, X2 if first else Xm, radii, 0.05, cot, grad=False)
            fd = (cot @ Cp - cot @ Cm) / (2 * h)
            assert g[idx] == pytest.approx(fd, rel=1e-5, abs=1e-9)


def test_smooth_cil_tends_to_indicator():
    """As tau -> 0 the smoothed sum tends to the indicator count of eq. (eCDF)."""
    X1 = W.clustered_patterns(6, 10, 1).astype(np.float64)
    X2 = W.clustered_patterns(7, 10, 2).astype(np.float64)
    d2 = oracle.pair_d2(X1.astype(np.float32), X2.astype(np.float32))
    R0, radii = oracle.radii(d2, 1.1, 4)
    _, counts = oracle.bins_counts(d2, radii)
    C, _, _ = oracle.smooth_cil(X1.astype(np.float32).astype(np.float64),
                                X2.astype(np.float32).astype(np.float64),
                                radii, 1e-9, np.ones(4), grad=False)
    assert np.allclose(C * 42, counts, atol=1e-6)


@pytest.mark.parametrize("model", [FHN, GM, BZ])
def test_gradient_term_magnitudes(model):
    """A (the summed magnitudes of the gradient's terms, used to set the
    GPU comparison's per-component tolerance) bounds |grad|, is unchanged
    by flipping the cotangent's sign and scales with its magnitude, while
    the gradient itself is untouched by asking for it."""
    P = small_problem(model)
    args = (P["model"], P["p"], P["dt"], P["steps"], P["w0"], P["mask"], P["set1"], P["set2"], P["radii"], 0.05)
    C, g, A = oracle.smooth_cil_grad(*args, P["cot"], with_abs=True)
    C0, g0 = oracle.smooth_cil_grad(*args, P["cot"])
    assert np.array_equal(g, g0) and np.array_equal(C, C0)
    assert np.all(A >= np.abs(g)) and np.all(A > 0)
    _, gm, Am = oracle.smooth_cil_grad(*args, -P["cot"], with_abs=True)
    assert np.array_equal(gm, -g) and np.array_equal(Am, A)
    _, g2, A2 = oracle.smooth_cil_grad(*args, 2.0 * P["cot"], with_abs=True)
    assert np.allclose(A2, 2.0 * A, rtol=1e-12) and np.allclose(g2, 2.0 * g, rtol=1e-12)
