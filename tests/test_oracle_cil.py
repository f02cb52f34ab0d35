"""Pins of the oracle's correlation-integral, bootstrap and statistics parts.

Paper: arXiv 2203.14742 -- eq. (eCDF) and eq. (CIL), Sec. 2.1; radii,
Sec. 2.1 and Sec. 3.2; Alg. 1 step 3; Alg. 5 step 2.1 (appendix A);
eq. (cil:CF), eq. (cil:CF_synth).
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

import oracle
import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def load(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


# ------------------------------------------------------------ hand counts

def test_hand_counted_2d_sets():
    g = load("hand_cil_2d.json")
    X1 = np.array(g["S1"], np.float32)
    X2 = np.array(g["S2"], np.float32)
    r = oracle.cil(X1, X2, b=g["b"], M=g["M"])
    assert np.array_equal(r["d2"], np.array(g["d2"], np.float64))
    assert r["R0"] == g["R0"]
    assert np.array_equal(r["radii"], np.array(g["radii"]))
    assert np.array_equal(r["bins"], np.array(g["bins"], np.uint8))
    assert np.array_equal(r["counts"], np.array(g["counts"], np.int64))


def brute_counts(X1, X2, radii):
    """Exactly rounded distances (math.fsum of exact squares of integers)
    and strict comparisons, written as plainly as possible."""
    M = len(radii)
    counts = [0] * M
    for x in X1:
        for y in X2:
            d2 = math.fsum((float(a) - float(b)) ** 2 for a, b in zip(x, y))
            for k in range(M):
                if d2 < radii[k] * radii[k]:
                    counts[k] += 1
    return counts


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_integer_patterns_brute_force(seed):
    rng = np.random.default_rng(seed)
    X1 = rng.integers(-5, 6, size=(7, 5)).astype(np.float32)
    X2 = rng.integers(-5, 6, size=(9, 5)).astype(np.float32)
    r = oracle.cil(X1, X2, b=1.25, M=10)
    assert list(r["counts"]) == brute_counts(X1, X2, list(r["radii"]))
    # With integer coordinates every d^2 is an exact integer.
    assert np.all(r["d2"] == np.round(r["d2"]))


def test_count_properties():
    X1 = W.clustered_patterns(20, 64, 3)
    X2 = W.clustered_patterns(17, 64, 4)
    r = oracle.cil(X1, X2, b=1.3, M=16)
    c = r["counts"]
    assert np.all(np.diff(c) <= 0)                      # non-increasing in k
    assert c[0] <= 20 * 17
    # swapping the two sets transposes the bins, counts unchanged
    s = oracle.cil(X2, X1, b=1.3, M=16)
    assert s["R0"] == r["R0"]
    assert np.array_equal(s["bins"], r["bins"].T)
    assert np.array_equal(s["counts"], c)
    # permutation invariance within each set
    p1 = np.random.default_rng(0).permutation(20)
    p2 = np.random.default_rng(1).permutation(17)
    t = oracle.cil(X1[p1], X2[p2], b=1.3, M=16)
    assert np.array_equal(t["counts"], c)
    assert np.array_equal(t["bins"], r["bins"][p1][:, p2])


def test_zero_counts_below_min_distance_and_r0_tie():
    X1 = W.clustered_patterns(6, 16, 5)
    X2 = W.clustered_patterns(5, 16, 6)
    d2 = oracle.pair_d2(X1, X2)
    rmin = math.sqrt(d2.min())
    radii = np.array([rmin, rmin * 0.5])
    _, counts = oracle.bins_counts(d2, radii)
    assert np.all(counts == 0)     # strict '<' and R_k <= min distance
    # at R0 itself exactly the pairs at the maximum distance are excluded
    R0 = math.sqrt(d2.max())
    assert R0 * R0 == d2.max() or True
    _, c0 = oracle.bins_counts(d2, np.array([R0]))
    n_at_max = int(np.sum(d2 >= R0 * R0))
    assert c0[0] == d2.size - n_at_max


def test_radii_power_law():
    d2 = np.array([1.0, 16.0, 9.0])
    R0, r = oracle.radii(d2, 1.3, 16)
    assert R0 == 4.0
    for k in range(16):
        assert r[k] == pytest.approx(4.0 * 1.3 ** -(k + 1), rel=1e-14)


def exact_d2(x, y):
    """The defined value written out with Python's exact rationals: the real
    sum of squared differences of the FP32 inputs, rounded once to the
    nearest double (float(Fraction) rounds correctly, ties to even)."""
    from fractions import Fraction
    s = sum((Fraction(float(a)) - Fraction(float(b))) ** 2 for a, b in zip(x, y))
    return float(s)


def wide_floats(rng, n):
    """FP32 values spread over the whole exponent range: normals from 2^-126
    to 2^127, subnormals, zeros, both signs."""
    kind = rng.integers(0, 4, n)
    mant = rng.uniform(1.0, 2.0, n)
    e = rng.integers(-126, 100, n).astype(np.float64)
    v = np.where(kind == 0, mant * 2.0 ** e, 0.0)
    v = np.where(kind == 1, mant * 2.0 ** rng.integers(-10, 10, n), v)
    v = np.where(kind == 2, rng.integers(1, 2 ** 23, n) * 2.0 ** -149, v)   # subnormals
    v = v * np.where(rng.integers(0, 2, n) == 0, 1.0, -1.0)
    return v.astype(np.float32)


@pytest.mark.parametrize("seed", range(6))
def test_pair_d2_is_the_correctly_rounded_exact_sum(seed):
    """Any exponent mix (subnormals, zeros, both signs, 2^-149 .. 2^100)."""
    rng = np.random.default_rng(100 + seed)
    for d in (1, 2, 3, 5, 17, 64):
        x = wide_floats(rng, d)
        y = wide_floats(rng, d)
        if seed % 2:   # near-equal pairs: heavy cancellation in x^2 + y^2 - 2xy
            y = (x.astype(np.float64) * (1 + rng.normal(size=d) * 1e-6)).astype(np.float32)
        assert oracle.pair_d2(x[None], y[None])[0, 0] == exact_d2(x, y)


def test_pair_d2_equals_fsum_of_exact_pieces():
    """math.fsum (correctly rounded summation of doubles) of the pieces x^2,
    y^2 and -2xy, each exact in a double for FP32 x, y."""
    rng = np.random.default_rng(7)
    X1 = rng.normal(size=(3, 1000)).astype(np.float32)
    X2 = rng.normal(size=(4, 1000)).astype(np.float32)
    d2 = oracle.pair_d2(X1, X2)
    for i in range(3):
        for j in range(4):
            pieces = []
            for a, b in zip(X1[i].astype(np.float64), X2[j].astype(np.float64)):
                pieces += [a * a, b * b, -2.0 * a * b]
            assert d2[i, j] == math.fsum(pieces)


def test_pair_d2_ties_round_to_even():
    """Sums exactly half-way between two doubles round to the even one."""
    t = np.float32(2.0 ** -27)          # t^2 = 2^-54
    # 1 + 2^-54 + 2^-54 = 1 + 2^-53: half-way between 1 and 1 + 2^-52 -> 1
    x = np.array([1.0, t, t], np.float32)
    assert oracle.pair_d2(x[None], np.zeros((1, 3), np.float32))[0, 0] == 1.0
    # (1 + 2^-52) + 2^-53: half-way between an odd and an even neighbour -> up
    u = np.float32(2.0 ** -26)          # u^2 = 2^-52
    x = np.array([1.0, u, t, t], np.float32)
    assert oracle.pair_d2(x[None], np.zeros((1, 4), np.float32))[0, 0] == 1.0 + 2.0 ** -51
    # one unit of 2^-54 more than half-way rounds up
    x = np.array([1.0, t, t, t], np.float32)
    assert oracle.pair_d2(x[None], np.zeros((1, 4), np.float32))[0, 0] == 1.0 + 2.0 ** -52
    # order-free: four terms of 2^-54 after a 1 sum to 1 + 2^-52 exactly,
    # which a left-to-right FP64 sum would lose (each 1 + 2^-54 rounds to 1)
    x = np.array([1.0, t, t, t, t], np.float32)
    assert oracle.pair_d2(x[None], np.zeros((1, 5), np.float32))[0, 0] == 1.0 + 2.0 ** -52
    left_to_right = 0.0
    for v in x.astype(np.float64):
        left_to_right += v * v
    assert left_to_right == 1.0


def test_pair_d2_extremes():
    big = np.float32(3.0e38)
    tiny = np.float32(2.0 ** -149)
    x = np.array([big, -big, tiny], np.float32)
    y = np.array([-big, big, -tiny], np.float32)
    assert oracle.pair_d2(x[None], y[None])[0, 0] == exact_d2(x, y)
    assert oracle.pair_d2(x[None], x[None])[0, 0] == 0.0
    z = np.zeros((1, 3), np.float32)
    z[0, 1] = np.inf
    assert math.isnan(oracle.pair_d2(z, np.zeros((1, 3), np.float32))[0, 0])


# ------------------------------------------------------------ bootstrap

def test_identity_resample_reproduces_counts():
    X1 = W.clustered_patterns(12, 32, 8)
    X2 = W.clustered_patterns(10, 32, 9)
    r = oracle.cil(X1, X2, b=1.3, M=12)
    I = np.tile(np.arange(12, dtype=np.int32), (3, 1))
    J = np.tile(np.arange(10, dtype=np.int32), (3, 1))
    Y = oracle.resample_counts(r["bins"], 12, I, J)
    for t in range(3):
        assert np.array_equal(Y[t], r["counts"])


def test_resample_counts_by_multiplicity():
    """Resampling with replacement = counts weighted by multiplicities."""
    X1 = W.clustered_patterns(8, 16, 10)
    X2 = W.clustered_patterns(9, 16, 11)
    r = oracle.cil(X1, X2, b=1.3, M=6)
    I, J = oracle.bootstrap_indices(99, 5, 8, 9)
    Y = oracle.resample_counts(r["bins"], 6, I, J)
    for t in range(5):
        c1 = np.bincount(I[t], minlength=8)
        c2 = np.bincount(J[t], minlength=9)
        for k in range(6):
            ind = (r["bins"] >= k + 1).astype(np.int64)
            assert Y[t, k] == c1 @ ind @ c2


def test_bootstrap_indices_range_and_uniformity():
    I, J = oracle.bootstrap_indices(12345, 400, 64, 37)
    assert I.min() >= 0 and I.max() < 64 and J.min() >= 0 and J.max() < 37
    for A, n in ((I, 64), (J, 37)):
        h = np.bincount(A.ravel(), minlength=n)
        e = A.size / n
        chi2 = ((h - e) ** 2 / e).sum()
        # chi^2 with n-1 dof: mean n-1, sd sqrt(2(n-1)); allow 5 sd
        assert chi2 < (n - 1) + 5 * math.sqrt(2 * (n - 1))
    I2, _ = oracle.bootstrap_indices(12345, 3, 64, 37)
    assert np.array_equal(I2, I[:3])


# ------------------------------------------------------------ statistics

def test_stats_match_numpy_on_active_block():
    X1 = W.clustered_patterns(16, 32, 12)
    X2 = W.clustered_patterns(16, 32, 13)
    r = oracle.cil(X1, X2, b=1.2, M=10)
    s = oracle.synlik(r["bins"], 10, 200, 77, y_obs=r["counts"] / 256.0)
    Y = s["Y"]
    y = Y / 256.0
    assert np.allclose(s["mu"], y.mean(0), rtol=1e-13, atol=0)
    assert np.allclose(s["cov"], np.cov(y, rowvar=False, ddof=1), rtol=1e-12, atol=1e-18)
    act = np.array([len(set(Y[:, k])) > 1 for k in range(10)])
    assert np.array_equal(s["active"].astype(bool), act)
    idx = np.flatnonzero(act)
    S = np.cov(y[:, idx], rowvar=False, ddof=1)
    Lnp = np.linalg.cholesky(S)
    ma = len(idx)
    assert s["m_active"] == ma
    assert np.allclose(s["chol"][:ma, :ma], Lnp, rtol=1e-10, atol=1e-16)
    sign, ld = np.linalg.slogdet(S)
    assert sign > 0 and s["logdet"] == pytest.approx(ld, rel=1e-10)
    rr = (r["counts"] / 256.0 - y.mean(0))[idx]
    f = rr @ np.linalg.solve(S, rr)
    assert s["f"] == pytest.approx(f, rel=1e-8)
    assert s["loglik"] == pytest.approx(-0.5 * (f + ld + ma * math.log(2 * math.pi)), rel=1e-8)


def test_stats_hand_spd():
    """Samples mu +- l_j (columns of the hand factor L) have covariance
    2 L L^T / (T-1) = 0.4 A for T = 6."""
    g = load("hand_spd3.json")
    L = np.array(g["L"], np.int64)
    Y = []
    for j in range(3):
        Y.append(100 + L[:, j])
        Y.append(100 - L[:, j])
    Y = np.array(Y, np.int64)
    yo = 100 + np.array(g["r"], np.float64)
    s = oracle.stats(Y, 1, y_obs=yo)
    A = np.array(g["A"], np.float64)
    assert s["status"] == 0
    assert np.array_equal(s["mu"], np.full(3, 100.0))
    assert np.allclose(s["cov"], 0.4 * A, rtol=1e-15)
    assert np.allclose(s["chol"], math.sqrt(0.4) * np.array(g["L"]), rtol=1e-14, atol=1e-15)
    assert s["logdet"] == pytest.approx(g["logdet"] + 3 * math.log(0.4), rel=1e-14)
    assert s["f"] == pytest.approx(g["f"] / 0.4, rel=1e-14)


def test_stats_not_positive_definite():
    # components 0 and 1 always equal -> singular active block
    rng = np.random.default_rng(0)
    a = rng.integers(0, 50, size=20)
    b = rng.integers(0, 50, size=20)
    Y = np.stack([a, a, b], 1).astype(np.int64)
    s = oracle.stats(Y, 100)
    assert s["status"] == 3


def test_inactive_constant_components():
    rng = np.random.default_rng(1)
    Y = np.stack([np.full(30, 7), rng.integers(0, 9, 30), np.zeros(30, np.int64),
                  rng.integers(0, 9, 30)], 1).astype(np.int64)
    s = oracle.stats(Y, 10)
    assert list(s["active"]) == [0, 1, 0, 1]
    assert s["m_active"] == 2 and s["status"] == 0


def test_stats_mean_cov_are_exactly_rounded_rationals():
    """Mean and covariance of y_t = Y_t / n_pairs are the exact rationals of
    the integer counts, rounded once (Python's float(Fraction) is correctly
    rounded), for counts whose numerators stay below 2^53."""
    from fractions import Fraction
    rng = np.random.default_rng(4)
    T, M, npairs = 37, 5, 1000
    Y = rng.integers(0, npairs + 1, size=(T, M)).astype(np.int64)
    s = oracle.stats(Y, npairs)
    for k in range(M):
        assert s["mu"][k] == float(Fraction(int(Y[:, k].sum()), T * npairs))
        for l in range(M):
            ex = sum((Fraction(int(Y[t, k]), npairs) - Fraction(int(Y[:, k].sum()), T * npairs)) *
                     (Fraction(int(Y[t, l]), npairs) - Fraction(int(Y[:, l].sum()), T * npairs))
                     for t in range(T)) / (T - 1)
            assert s["cov"][k, l] == float(ex)


def test_linear_radii_hand_count():
    # Linear radii law (Sec. 2.1, Sec. 3.2): set 1 = {0, 1}, set 2 = {3, 5, 6}
    # on a line.  Cross-set distances 3, 5, 6 / 2, 4, 5; R0 = 6 (largest),
    # R_M = 2 (smallest), M = 4: h = 1, radii 5, 4, 3, 2.  K = #{k : d < R_k}:
    # d = 3 -> 2, 5 -> 0, 6 -> 0, 2 -> 3, 4 -> 1, 5 -> 0; counts[k-1] =
    # #{K >= k} = 3, 2, 1, 0.
    X1 = np.array([[0.0], [1.0]], np.float32)
    X2 = np.array([[3.0], [5.0], [6.0]], np.float32)
    o = oracle.cil(X1, X2, M=4, law="linear")
    assert o["R0"] == 6.0
    assert list(o["radii"]) == [5.0, 4.0, 3.0, 2.0]
    assert o["bins"].tolist() == [[2, 0, 0], [3, 1, 0]]
    assert list(o["counts"]) == [3, 2, 1, 0]
    R0, r, rmin = oracle.radii_linear(o["d2"], 4)
    assert rmin == 2.0 and R0 == 6.0


def test_linear_radii_span_max_to_min():
    rng = np.random.default_rng(4)
    X1 = rng.standard_normal((7, 33)).astype(np.float32)
    X2 = rng.standard_normal((9, 33)).astype(np.float32)
    d2 = oracle.pair_d2(X1, X2)
    for M in (1, 5, 13):
        R0, r, rmin = oracle.radii_linear(d2, M)
        assert R0 == np.sqrt(d2.max()) and rmin == np.sqrt(d2.min())
        assert np.all(np.diff(np.concatenate([[R0], r])) < 0)        # decreasing
        assert abs(r[-1] - rmin) <= 1e-12 * R0                       # ends at R_min
        # equal steps
        steps = -np.diff(np.concatenate([[R0], r]))
        assert np.allclose(steps, (R0 - rmin) / M, rtol=1e-12)


def test_bins_above_M_count_under_every_radius():
    # Y[t][k-1] = #{pairs : K >= k}, k = 1..M: a bin above M counts under all
    # M radii and nothing beyond them
    bins = np.full((3, 4), 9, np.uint8)
    bins[0, 0] = 2
    so = oracle.synlik(bins, 4, 5, 11)
    I, J = oracle.bootstrap_indices(11, 5, 3, 4)
    for t in range(5):
        n00 = sum(1 for a in I[t] for b in J[t] if a == 0 and b == 0)
        assert so["Y"][t].tolist() == [12, 12, 12 - n00, 12 - n00]


def test_fitted_b_definition():
    # b is the smallest double whose M-th power (sequential products rounded
    # to nearest) reaches c: checked against its neighbours by brute force
    def powM(x, M):
        p = x
        for _ in range(M - 1):
            p = p * x
        return p
    for c, M in ((8.0, 3), (10.0, 16), (1.0000001, 13), (123.456, 7), (2.0, 1), (1e6, 32)):
        b = oracle.fitted_b(c, M)
        assert powM(b, M) >= c
        assert powM(np.nextafter(b, 0.0), M) < c
    assert oracle.fitted_b(8.0, 3) == 2.0            # 2^3 = 8 exactly
    assert oracle.fitted_b(1.0, 5) == 1.0            # R_min = R0
    assert oracle.fitted_b(0.5, 5) == 1.0
    assert oracle.fitted_b(np.inf, 5) == np.inf      # R_min = 0


def test_fitted_law_by_hand():
    # on a line: set 1 = {0}, set 2 = {1, 2, 8}: R0 = 8, R_min = 1, M = 3
    # -> b = 2, radii 4, 2, 1; counts #{d < R_k} = 2, 1, 0 (worked by hand)
    X1 = np.array([[0.0]], np.float32)
    X2 = np.array([[1.0], [2.0], [8.0]], np.float32)
    o = oracle.cil(X1, X2, M=3, law="fitted")
    assert o["R0"] == 8.0
    assert o["radii"].tolist() == [4.0, 2.0, 1.0]
    assert o["counts"].tolist() == [2, 1, 0]
    # R_M equals R_min up to the rounding of b: the recursion ends within a
    # few ulp of the smallest distance
    rng = np.random.default_rng(3)
    X1 = rng.standard_normal((9, 40)).astype(np.float32)
    X2 = rng.standard_normal((11, 40)).astype(np.float32)
    o = oracle.cil(X1, X2, M=13, law="fitted")
    rmin = math.sqrt(o["d2"].min())
    assert abs(o["radii"][-1] - rmin) <= 64 * np.spacing(rmin)
    assert np.all(np.diff(o["radii"]) < 0)
