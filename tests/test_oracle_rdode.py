"""Pins of the oracle's 1-D reaction-diffusion-ODE model (Sec. 4.3, eq.
rdode; Table 1) against facts fixed outside it: the smoothing of the
initial noise as an exact DCT-II multiplier, closed-form right-hand sides
on homogeneous states and cosine modes, the Gershgorin bound of a dense
finite-difference Jacobian, the stabilised RK2 amplification of decaying
w-modes, second-order convergence against RK4, and the stationary relation
of the far-from-equilibrium pattern."""
import math

import numpy as np
import pytest

import oracle
import workloads as W

P0 = W.RDODE_THETA0


def dct_modes(N):
    x = np.arange(N)
    return np.array([np.cos(np.pi * k * (x + 0.5) / N) for k in range(N)])


@pytest.mark.parametrize("N,n_smooth", [(32, 0), (64, 10), (128, 3)])
def test_initial_smoothing_is_the_dct_multiplier(N, n_smooth):
    # one pass of ((u_{x-1} + u_x) + u_{x+1})/3 with ghost = edge node is
    # I + Lap/3 on the mirrored-ghost Laplacian: DCT-II mode k is scaled by
    # (1 + 2 cos(pi k / N)) / 3 per pass
    seed, lo, hi = 77, 0.0, 2.0
    noise = np.array([lo + (hi - lo) * ((oracle.sm64(seed, x) >> 11) * 2.0 ** -53) for x in range(N)])
    got = oracle.rdode_init(N, 1, lo, hi, seed, n_smooth)[0]
    C = dct_modes(N)
    coef = np.linalg.solve(C.T, noise)
    lam = (1.0 + 2.0 * np.cos(np.pi * np.arange(N) / N)) / 3.0
    ref = C.T @ (coef * lam ** n_smooth)
    np.testing.assert_allclose(got[0], ref, rtol=0, atol=2e-7)      # FP32 rounding
    assert np.all(got[1] == 0.0)
    assert abs(float(got[0].astype(np.float64).mean()) - noise.mean()) < 1e-6


def test_realisations_take_consecutive_streams():
    N = 64
    a = oracle.rdode_init(N, 3, 0.0, 2.0, 5, 10)
    for r in range(3):
        b = oracle.rdode_init(N, 1, 0.0, 2.0, 5, 10)   # realisation 0 of the same stream
        if r == 0:
            assert np.array_equal(a[0], b[0])
    assert not np.array_equal(a[0], a[1])


def test_rhs_on_homogeneous_states_and_modes():
    N = 64
    D, m1, m2, m3, k = P0[1:]
    for c in (0.0, 0.5, 3.0, 20.0):
        w = np.stack([np.full(N, c), np.zeros(N)])
        F = oracle.rdode_rhs(P0, w)
        q = c * c / (1 + k * c * c)
        np.testing.assert_allclose(F[0], -c + m1 * q, rtol=1e-14, atol=1e-15)
        np.testing.assert_allclose(F[1], m2 * q, rtol=1e-14, atol=1e-15)
    # u = 0, w = cosine mode: F_w = (-D lambda_k - m3) w with
    # lambda_k = 4 (N-1)^2 sin^2(pi k / (2N)), F_u = 0
    x = np.arange(N)
    for kk in (0, 1, 7, 63):
        wm = np.cos(np.pi * kk * (x + 0.5) / N)
        F = oracle.rdode_rhs(P0, np.stack([np.zeros(N), wm]))
        lam = 4 * (N - 1) ** 2 * math.sin(math.pi * kk / (2 * N)) ** 2
        np.testing.assert_allclose(F[1], (-D * lam - m3) * wm, rtol=0, atol=1e-9 * max(1.0, D * lam))
        assert np.all(F[0] == 0.0)


@pytest.mark.parametrize("where", ["random", "end"])
def test_gershgorin_equals_dense_jacobian_row_sums(where):
    N = 8
    rng = np.random.default_rng(3)
    w = np.stack([rng.uniform(0, 5, N), rng.uniform(0, 3, N)])
    if where == "end":
        w[0, 0] = 30.0          # the largest row at a node with one neighbour
    m = w.size
    J = np.zeros((m, m))
    for i in range(m):
        e = np.zeros(m)
        d = 1e-6 * max(1.0, abs(w.flat[i]))
        e[i] = d
        J[:, i] = (oracle.rdode_rhs(P0, w + e.reshape(w.shape)) -
                   oracle.rdode_rhs(P0, w - e.reshape(w.shape))).ravel() / (2 * d)
    bound = oracle.gershgorin(oracle.RDODE, P0, w)
    assert bound == pytest.approx(np.abs(J).sum(axis=1).max(), rel=1e-6)
    assert np.abs(np.linalg.eigvals(J)).max() <= bound * (1 + 1e-9)


def cheb_T(s, x):
    if abs(x) <= 1.0:
        return math.cos(s * math.acos(x))
    v = math.cosh(s * math.acosh(abs(x)))
    return v if x > 0 or s % 2 == 0 else -v


@pytest.mark.parametrize("s", [2, 5, 30])
def test_decaying_modes_follow_the_stability_polynomial(s):
    # u = 0 stays 0; w then obeys w_t = D w_xx - m3 w, linear: one step
    # multiplies mode k by R_s(h (-D lambda_k - m3))
    N = 64
    D, m3 = P0[1], P0[4]
    c = oracle.rkc_coef(s)
    lam_max = 4 * (N - 1) ** 2 * D + m3
    h = 0.9 * c["beta"] / (8 * (N - 1) ** 2 * D + m3)
    x = np.arange(N)
    for kk in (0, 3, 50):
        wm = np.cos(np.pi * kk * (x + 0.5) / N)
        out = oracle.rkc_fixed(oracle.RDODE, P0, h, s, 1, np.stack([np.zeros(N), wm])[None])[0]
        z = h * (-D * 4 * (N - 1) ** 2 * math.sin(math.pi * kk / (2 * N)) ** 2 - m3)
        R = c["a_s"] + c["b_s"] * cheb_T(s, c["w0"] + c["w1"] * z)
        np.testing.assert_allclose(out[1], R * wm, rtol=0, atol=1e-12)
        assert np.all(out[0] == 0.0)
    assert lam_max > 0


def rk4(p, w, T, n):
    h = T / n
    for _ in range(n):
        k1 = oracle.rdode_rhs(p, w)
        k2 = oracle.rdode_rhs(p, w + 0.5 * h * k1)
        k3 = oracle.rdode_rhs(p, w + 0.5 * h * k2)
        k4 = oracle.rdode_rhs(p, w + h * k3)
        w = w + (h / 6.0) * (k1 + 2 * k2 + 2 * k3 + k4)
    return w


def test_global_convergence_is_second_order():
    N = 32
    w = oracle.rdode_init(N, 1, 0.0, 2.0, 11, 10).astype(np.float64)
    T = 0.2
    ref = rk4(P0, w[0], T, 20000)
    rho = oracle.gershgorin(oracle.RDODE, P0, w[0])
    s = 2
    while oracle.rkc_beta(s) < 1.2 * (T / 40) * rho:
        s += 1
    errs = [np.abs(oracle.rkc_fixed(oracle.RDODE, P0, T / n, s, n, w)[0] - ref).max() for n in (40, 80, 160)]
    assert errs[0] / errs[1] == pytest.approx(4.0, rel=0.15)
    assert errs[1] / errs[2] == pytest.approx(4.0, rel=0.15)


def test_far_from_equilibrium_pattern():
    # Table 1: t in [0, 50].  The stationary pattern has u = 0 or u on the
    # branch 1 + w = m1 u / (1 + k u^2) (u_t = 0 with u != 0), with jumps
    # between the two, and a smooth w
    N = 64
    D, m1, m2, m3, k = P0[1:]
    w0 = oracle.rdode_init(N, 4, 0.0, 2.0, 123, 10)
    w, st, failed = oracle.rkc_adaptive(oracle.RDODE, P0, 50.0, 1e-3, 1e-6, 1e-6, w0)
    assert failed == 0
    for r in range(4):
        u, v = w[r]
        F = oracle.rdode_rhs(P0, w[r])
        assert np.abs(F).max() < 1e-3
        hi = u > 1.0
        assert hi.any() and (~hi).any()
        assert np.abs(u[~hi]).max() < 1e-3
        np.testing.assert_allclose(1 + v[hi], m1 * u[hi] / (1 + k * u[hi] ** 2), rtol=1e-3)
        assert (np.abs(np.diff(u)) > 1.0).sum() >= 1             # a jump
        assert np.abs(np.diff(v)).max() < 0.5                    # w stays smooth
