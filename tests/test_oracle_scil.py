"""Pins of the oracle's synthetic CIL with bootstrapping (Alg. 6, Sec. 3.3):
the composition of pinned oracle parts (multi-feature distances and radii,
bootstrap counts, statistics) checked against what the algorithm fixes."""
import numpy as np
import pytest

import oracle
import workloads as W


def synthetic(n, G, seed, offset=0.0):
    return W.cosine_patterns(n, G, 2, seed, amp=0.8, offset=offset)


def test_given_radii_reproduce_the_synthetic_bins():
    """Binning a pair set with the radii its own correlation integral chose
    (eq. eCDF with given R_k) gives that integral's bins and counts."""
    G = 8
    S = synthetic(30, G, 3)
    r = oracle.mcil(S[:10], S[10:], G, 2, 1.3, 6, mask=63, law="fitted")
    g = oracle.mcil_given(S[:10], S[10:], G, 2, r["radii"], mask=63)
    assert np.array_equal(g["bins"], r["bins"])
    assert np.array_equal(g["counts"], r["counts"])
    assert np.array_equal(g["C"], r["C"])


def test_data_vector_is_invariant_to_order_within_s2():
    G = 8
    S = synthetic(40, G, 5)
    data = synthetic(6, G, 6)
    a = oracle.scil(S, data, 8, G, 2, 5, 30, 11, mask=0x0B)
    perm = np.concatenate([np.arange(8), 8 + np.random.default_rng(0).permutation(32)])
    # permuting s^2 leaves the radii, the data vector and the bins' multiset unchanged
    b = oracle.scil(S[perm], data, 8, G, 2, 5, 30, 11, mask=0x0B)
    assert np.array_equal(a["radii"], b["radii"])
    assert np.array_equal(a["y_data"], b["y_data"])


@pytest.mark.parametrize("law", ["fitted", "power", "linear"])
def test_cost_is_the_mahalanobis_distance_of_the_data_vector(law):
    """f = (y~ - mu)^T Sigma^-1 (y~ - mu) on the active block, with mu and
    Sigma the sample mean and covariance (ddof = 1) of the resampled count
    vectors divided by n1 n2, evaluated here with numpy's solver."""
    G = 8
    S = synthetic(60, G, 9)
    data = synthetic(10, G, 10, offset=0.02)
    n_set = 10
    # two features (L2, Linf): identical count columns, which would make
    # Sigma singular, are unlikely between them
    r = oracle.scil(S, data, n_set, G, 2, 5, 400, 7, mask=0x03, law=law, b=1.3)
    st = r["stats"]
    y = r["Y"].astype(np.float64) / (n_set * (60 - n_set))
    act = y.std(0) > 0
    mu = y.mean(0)[act]
    cov = np.cov(y[:, act], rowvar=False, ddof=1)
    dv = r["y_data"][act] - mu
    f = float(dv @ np.linalg.solve(cov, dv))
    assert st["status"] == 0
    assert np.array_equal(st["active"].astype(bool), act)
    assert st["f"] == pytest.approx(f, rel=1e-8)
    # the data vector is the correlation integral of the data against s^2
    g = oracle.mcil_given(data, S[n_set:], G, 2, r["radii"], mask=0x03)
    assert np.array_equal(r["y_data"], g["C"])
