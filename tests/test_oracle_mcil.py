"""Pins of the oracle's multi-feature correlation integral (Sec. 3.1,
Alg. 2) and of min-max scaling (Sec. 4): a hand-worked fixture, exactness on
integer data, norm inequalities, symmetries, and consistency with the
single-norm CIL (itself pinned in test_oracle_cil.py)."""
import json
import math
import os

import numpy as np
import pytest

import oracle
import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden")
KEYS = ("L2_squared", "Linf", "W12_squared", "W12p", "W1inf", "W1infp")


def test_hand_worked_fixture():
    gd = json.load(open(os.path.join(GOLD, "hand_mcil.json")))
    G = gd["G"]
    zero = np.zeros((1, G * G), np.float32)
    for name, pat in gd["patterns"].items():
        X = np.array([pat], np.float32)
        V = oracle.mcil_values(X, zero, G, 1)[:, 0, 0]
        for f, key in enumerate(KEYS):
            assert V[f] == pytest.approx(gd["expected"][name][key], rel=1e-15, abs=0), (name, key)


def rand_int_patterns(n, G, nsp, seed, lo=-20, hi=20):
    rng = np.random.default_rng(seed)
    return rng.integers(lo, hi, size=(n, nsp * G * G)).astype(np.float32)


def test_integer_patterns_exact_brute_force():
    """Integer data: every difference and square is exact, so the values
    follow from integer arithmetic on the definitions."""
    G, nsp = 5, 2
    X1 = rand_int_patterns(3, G, nsp, 1)
    X2 = rand_int_patterns(4, G, nsp, 2)
    V = oracle.mcil_values(X1, X2, G, nsp)
    g = G - 1
    for i in range(3):
        for j in range(4):
            u = (X1[i].astype(np.int64) - X2[j].astype(np.int64)).reshape(nsp, G, G)
            dx = u[:, :, 1:] - u[:, :, :-1]
            dy = u[:, 1:, :] - u[:, :-1, :]
            q0, qx, qy = int((u * u).sum()), int((dx * dx).sum()), int((dy * dy).sum())
            m0, mx, my = int(abs(u).max()), int(abs(dx).max()), int(abs(dy).max())
            assert V[0, i, j] == q0 and V[1, i, j] == m0
            assert V[2, i, j] == pytest.approx(q0 / g ** 2 + qx + qy, rel=1e-15)
            assert V[3, i, j] == pytest.approx(math.sqrt(q0) / g + math.sqrt(qx) + math.sqrt(qy), rel=1e-15)
            assert V[4, i, j] == max(m0, g * mx, g * my)
            assert V[5, i, j] == m0 + g * mx + g * my


def test_norm_inequalities_and_symmetry():
    G, nsp = 16, 2
    X1 = W.cosine_patterns(6, G, nsp, 3)
    X2 = W.cosine_patterns(5, G, nsp, 4)
    V = oracle.mcil_values(X1, X2, G, nsp)
    Vt = oracle.mcil_values(X2, X1, G, nsp)
    assert np.array_equal(V, Vt.transpose(0, 2, 1))
    assert np.all(V[3] >= np.sqrt(V[2]) * (1 - 1e-12))        # sum of norms >= root of summed squares
    assert np.all(V[5] >= V[4]) and np.all(V[4] >= V[1])       # sum >= max >= its first term
    assert np.all(V[1] <= np.sqrt(V[0]) * (1 + 1e-12))         # max |u| <= ||u||_2


def test_constant_shift_has_no_derivative_part():
    G, nsp = 8, 1
    # values on a 2^-10 grid, so that the shift by 1/4 is exact
    X1 = (np.round(W.cosine_patterns(3, G, nsp, 5) * 1024.0) / 1024.0).astype(np.float32)
    X2 = X1 + np.float32(0.25)
    assert np.all((X2 - X1) == np.float32(0.25))
    V = oracle.mcil_values(X1, X2, G, nsp)
    h = 1.0 / (G - 1)
    d = np.diagonal(V, axis1=1, axis2=2)
    assert np.allclose(d[2], h * h * d[0], rtol=1e-15, atol=0)
    assert np.allclose(d[3], h * np.sqrt(d[0]), rtol=1e-15, atol=0)
    assert np.all(d[1] == 0.25) and np.all(d[4] == 0.25) and np.all(d[5] == 0.25)


def test_transposed_fields_give_the_same_features():
    """Swapping the x and y axes swaps the two derivative terms; with
    integer data the squared distances and maxima are exact, so L2, Linf and
    the W^{1,inf} features are unchanged exactly, and the W^{1,2} features,
    which add the two terms in a fixed order, to rounding."""
    G, nsp = 6, 1
    X1 = rand_int_patterns(3, G, nsp, 7)
    X2 = rand_int_patterns(3, G, nsp, 8)
    T1 = X1.reshape(-1, G, G).transpose(0, 2, 1).reshape(3, -1)
    T2 = X2.reshape(-1, G, G).transpose(0, 2, 1).reshape(3, -1)
    A, B = oracle.mcil_values(X1, X2, G, nsp), oracle.mcil_values(T1, T2, G, nsp)
    for f in (0, 1, 4, 5):
        assert np.array_equal(A[f], B[f]), f
    assert np.allclose(A[2:4], B[2:4], rtol=4e-16, atol=0)


def test_forward_differences_layout():
    G = 4
    X = np.arange(2 * G * G, dtype=np.float32).reshape(1, -1) ** 2   # two species
    Ax, Ay = oracle.fd(X, G, 2)
    f = X.reshape(2, G, G).astype(np.float64)
    assert np.array_equal(Ax.reshape(2, G, G - 1), (f[:, :, 1:] - f[:, :, :-1]).astype(np.float32))
    assert np.array_equal(Ay.reshape(2, G - 1, G), (f[:, 1:, :] - f[:, :-1, :]).astype(np.float32))


def test_minmax_scaling():
    G, nsp = 8, 2
    X = W.cosine_patterns(4, G, nsp, 9, amp=3.0, offset=1.5)
    S = oracle.minmax(X, G, nsp).reshape(4, nsp, -1)
    assert np.all(S.min(-1) == 0.0) and np.all(S.max(-1) == 1.0)
    # exact affine invariance for a power-of-two scale and a shift that
    # keeps every value exact (integer data)
    Xi = rand_int_patterns(3, G, nsp, 10, 0, 50)
    A = oracle.minmax(Xi, G, nsp)
    B = oracle.minmax(Xi * np.float32(4.0) + np.float32(-64.0), G, nsp)
    assert np.array_equal(A, B)
    # a constant species maps to zero
    Xc = Xi.copy().reshape(3, nsp, -1)
    Xc[:, 1, :] = 7.0
    C = oracle.minmax(Xc.reshape(3, -1), G, nsp).reshape(3, nsp, -1)
    assert np.all(C[:, 1] == 0.0) and np.all(C[:, 0].max(-1) == 1.0)


def test_l2_feature_equals_the_single_norm_cil():
    G, nsp = 16, 2
    X1 = W.clustered_patterns(20, nsp * G * G, 11)
    X2 = W.clustered_patterns(17, nsp * G * G, 12)
    m = oracle.mcil(X1, X2, G, nsp, b=1.2, M=10)
    c = oracle.cil(X1, X2, b=1.2, M=10)
    assert m["features"] == list(range(6))
    assert m["radii"][0, 0] == c["R0"] and np.array_equal(m["radii"][0, 1:], c["radii"])
    assert np.array_equal(m["bins"][0], c["bins"]) and np.array_equal(m["counts"][0], c["counts"])
    for a in range(6):                                     # counts non-increasing in k
        assert np.all(np.diff(m["counts"][a]) <= 0)
        assert m["counts"][a][0] <= 20 * 17


def test_value_feature_decisions_are_strict():
    """A value feature counts F < R_k: the pair that defines R0 is never in
    bin 1, and with b chosen so that R_1 equals another pair's value that
    pair is not counted."""
    G = 3
    X1 = np.array([[0, 0, 0, 0, 1, 0, 0, 0, 0], [0, 0, 0, 0, 2, 0, 0, 0, 0]], np.float32)
    X2 = np.zeros((1, 9), np.float32)
    m = oracle.mcil(X1, X2, G, 1, b=2.0, M=2, mask=0x02)   # Linf: values 1 and 2, R0 = 2, R1 = 1
    assert m["radii"][0].tolist() == [2.0, 1.0, 0.5]
    assert m["bins"][0].ravel().tolist() == [0, 0]
    assert m["counts"][0].tolist() == [0, 0]


def test_synlik_multi_shares_resamples():
    G, nsp = 8, 1
    X1 = W.clustered_patterns(12, G * G, 13)
    X2 = W.clustered_patterns(10, G * G, 14)
    m = oracle.mcil(X1, X2, G, nsp, b=1.3, M=6, mask=0x05)
    s = oracle.synlik_multi(m["bins"], 6, 40, 99)
    s0 = oracle.synlik(m["bins"][0], 6, 40, 99)
    s1 = oracle.synlik(m["bins"][1], 6, 40, 99)
    assert np.array_equal(s["Y"], np.concatenate([s0["Y"], s1["Y"]], axis=1))
    assert s["mu"].shape == (12,)


def test_one_dimensional_features_by_hand():
    # 1-D patterns (Gy = 1) of Gx = 3 nodes, h = 1/2, g = 2:  x = (0, 1, 3),
    # y = (1, 1, 1), u = x - y = (-1, 0, 2), Dx u = (1, 2):
    #   q0 = 1 + 0 + 4 = 5, qx = 1 + 4 = 5, m0 = 2, mx = 2, no y terms;
    #   L2^2 = 5, Linf = 2, W12^2 = h^2 q0 + qx = 6.25,
    #   W12' = h sqrt(q0) + sqrt(qx) = 1.5 sqrt(5), W1inf = max(2, 2*2) = 4,
    #   W1inf' = 2 + 2*2 = 6
    X1 = np.array([[0.0, 1.0, 3.0]], np.float32)
    X2 = np.array([[1.0, 1.0, 1.0]], np.float32)
    V = oracle.mcil_values(X1, X2, 3, 1, 63, Gy=1)[:, 0, 0]
    assert V[0] == 5.0 and V[1] == 2.0 and V[2] == 6.25
    assert V[3] == pytest.approx(1.5 * np.sqrt(5.0), rel=1e-15)
    assert V[4] == 4.0 and V[5] == 6.0
    Ax, Ay = oracle.fd(X1, 3, 1, Gy=1)
    assert Ax.tolist() == [[1.0, 2.0]] and Ay.shape == (1, 0)


def test_linear_law_by_hand():
    # patterns (v, 0) on a line: set 1 = {0, 1}, set 2 = {3, 5, 6}; the L2
    # and Linf features are both the distance |v - v'| (3, 5, 6 / 2, 4, 5):
    # R0 = 6, R_min = 2, M = 4, h = 1, radii 5, 4, 3, 2 (worked by hand),
    # counts 3, 2, 1, 0 for both
    X1 = np.array([[0.0, 0.0], [1.0, 0.0]], np.float32)
    X2 = np.array([[3.0, 0.0], [5.0, 0.0], [6.0, 0.0]], np.float32)
    o = oracle.mcil(X1, X2, 2, 1, None, 4, mask=0x03, Gy=1, law="linear")
    for a in range(2):
        assert o["radii"][a].tolist() == [6.0, 5.0, 4.0, 3.0, 2.0]
        assert o["counts"][a].tolist() == [3, 2, 1, 0]


def test_fitted_law_by_hand():
    # patterns (v, 0) on a line: set 1 = {0}, set 2 = {1, 2, 8}: L2 and Linf
    # are both |v - v'|: R0 = 8, R_min = 1, M = 3 -> b = 2, radii 4, 2, 1,
    # counts 2, 1, 0 (worked by hand)
    X1 = np.array([[0.0, 0.0]], np.float32)
    X2 = np.array([[1.0, 0.0], [2.0, 0.0], [8.0, 0.0]], np.float32)
    o = oracle.mcil(X1, X2, 2, 1, None, 3, mask=0x03, Gy=1, law="fitted")
    for a in range(2):
        assert o["radii"][a].tolist() == [8.0, 4.0, 2.0, 1.0]
        assert o["counts"][a].tolist() == [2, 1, 0]
