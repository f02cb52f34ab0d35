"""GPU parity of the bootstrap counts and synthetic-likelihood statistics.

Resampled counts are integers: bit-exact.  Mean and covariance are exact
rationals of the counts rounded once on both sides, and the Cholesky factor
is the same sequence of rounded operations: bit-exact.  log() is the only
library function involved (log-determinant, log-likelihood): relative 1e-13.
"""
import math

import numpy as np
import pytest
import torch

import oracle
import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture
def tc_all(p):
    """Every problem size through the tensor-core bootstrap counts."""
    p.lib().synlik_set_tc_min_pairs(0)
    yield
    p.lib().synlik_set_tc_min_pairs(-1)


@pytest.fixture(scope="module")
def p():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2203_14742_b300 as pk
    return pk


def oracle_bins(n1, n2, d, M, b, seed):
    X1 = W.clustered_patterns(n1, d, seed)
    X2 = W.clustered_patterns(n2, d, seed + 1)
    return oracle.cil(X1, X2, b=b, M=M)


@pytest.mark.parametrize("n1,n2,M,T", [(16, 16, 8, 50), (64, 64, 16, 200), (37, 90, 12, 33),
                                       (256, 256, 16, 200)])
@pytest.mark.parametrize("force_tc", [False, True])
def test_bootstrap_and_stats_match(p, n1, n2, M, T, force_tc):
    o = oracle_bins(n1, n2, 64, M, 1.08, n1 * 7 + n2)
    seed = 0x5EED + n1
    y_obs = o["counts"] / float(n1 * n2)
    so = oracle.synlik(o["bins"], M, T, seed, y_obs=y_obs)
    bins = torch.from_numpy(o["bins"]).cuda()
    p.lib().synlik_set_tc_min_pairs(0 if force_tc else -1)
    try:
        s = p.synlik(bins, M, T, seed, y_obs=torch.from_numpy(y_obs))
    finally:
        p.lib().synlik_set_tc_min_pairs(-1)
    assert np.array_equal(s["Y"].cpu().numpy(), so["Y"])
    assert np.array_equal(s["mu"].cpu().numpy(), so["mu"])
    assert np.array_equal(s["cov"].cpu().numpy(), so["cov"])
    assert np.array_equal(s["active"].cpu().numpy(), so["active"])
    assert int(s["status"]) == so["status"]
    if so["status"] == 0:
        assert np.array_equal(s["chol"].cpu().numpy(), so["chol"])
        for k in ("logdet", "f", "loglik"):
            assert float(s[k]) == pytest.approx(so[k], rel=1e-13, abs=1e-300)
    assert int(s["m_active"]) == so["m_active"]


def test_batched_problems(p):
    M, T = 16, 40
    bins, ys, refs = [], [], []
    for q in range(5):
        o = oracle_bins(20, 24, 32, M, 1.1, 300 + q)
        bins.append(o["bins"])
        y = o["counts"] / 480.0
        ys.append(y)
        refs.append(oracle.synlik(o["bins"], M, T, 77 + q, y_obs=y))
    s = p.synlik(torch.from_numpy(np.stack(bins)).cuda(), M, T, 77,
                 y_obs=torch.from_numpy(np.stack(ys)))
    for q in range(5):
        assert np.array_equal(s["Y"][q].cpu().numpy(), refs[q]["Y"])
        assert np.array_equal(s["cov"][q].cpu().numpy(), refs[q]["cov"])


def test_not_positive_definite_reported(p):
    # bins take only the values 0 and 2: counts of radius 1 and 2 coincide in
    # every resample, so the active block is singular
    rng = np.random.default_rng(0)
    bins = (2 * rng.integers(0, 2, size=(20, 20))).astype(np.uint8)
    so = oracle.synlik(bins, 4, 30, 5)
    s = p.synlik(torch.from_numpy(bins).cuda(), 4, 30, 5)
    assert so["status"] == 3 and int(s["status"]) == 3
    assert list(s["active"].cpu().numpy()) == [1, 1, 0, 0]


def test_identity_like_counts_are_resample_invariant_when_constant(p):
    # every pair in bin M: all components constant, nothing active, logdet 0
    bins = np.full((8, 9), 6, np.uint8)
    s = p.synlik(torch.from_numpy(bins).cuda(), 6, 10, 1, y_obs=torch.ones(6, dtype=torch.float64))
    assert int(s["status"]) == 0 and int(s["m_active"]) == 0
    assert float(s["logdet"]) == 0.0 and float(s["f"]) == 0.0
    assert torch.all(s["Y"] == 72)


@pytest.mark.parametrize("n1,n2,M,T", [(1000, 1000, 16, 40), (1, 300, 8, 20), (300, 1, 8, 20),
                                       (1024, 33, 13, 64), (5, 2049, 32, 9)])
@pytest.mark.parametrize("simt", [False, True])
def test_bootstrap_counts_large_and_ragged(p, tc_all, n1, n2, M, T, simt):
    # the paper's SCIL scale (N_syn = 1000 patterns, Sec. 4.2) and one-row /
    # one-column sets; bins drawn directly (every value 0..M), counts exact
    # on the tensor cores and with the SIMT kernel
    rng = np.random.default_rng(n1 * 31 + n2)
    bins = rng.integers(0, M + 1, (n1, n2)).astype(np.uint8)
    so = oracle.synlik(bins, M, T, 0xB00 + n1)
    s = p.synlik(torch.from_numpy(bins).cuda(), M, T, 0xB00 + n1, simt=simt)
    assert np.array_equal(s["Y"].cpu().numpy(), so["Y"])
    assert np.array_equal(s["mu"].cpu().numpy(), so["mu"])
    assert np.array_equal(s["cov"].cpu().numpy(), so["cov"])


@pytest.mark.parametrize("n1,n2,M,T,nf", [(50, 950, 13, 1000, 6), (129, 65, 16, 257, 1), (3, 7, 32, 2, 2),
                                          (200, 200, 5, 33, 3)])
def test_bootstrap_tensor_core_shapes(p, tc_all, n1, n2, M, T, nf):
    # Alg. 6 at the paper's SCIL setting (N_set = 50 against the other 950 of
    # N_syn = 1000, n_CIL = 1000 resamples, six features), more than one
    # 256-resample tile, tails of every tile dimension; values above M in
    # the bins count under every radius
    rng = np.random.default_rng(n1 + 7 * n2 + T)
    bins = rng.integers(0, M + 3, (nf, n1, n2)).astype(np.uint8)
    so = oracle.synlik_multi(bins, M, T, 0xC11 + T) if nf > 1 else oracle.synlik(bins[0], M, T, 0xC11 + T)
    tb = torch.from_numpy(bins).cuda()
    s = p.synlik(tb if nf > 1 else tb[0], M, T, 0xC11 + T, n_feat=nf)
    assert np.array_equal(s["Y"].cpu().numpy(), so["Y"])
    assert np.array_equal(s["cov"].cpu().numpy(), so["cov"])
    t = p.synlik(tb if nf > 1 else tb[0], M, T, 0xC11 + T, n_feat=nf, simt=True)
    assert torch.equal(t["Y"], s["Y"])


def test_bootstrap_tensor_core_batched_problems(p, tc_all):
    # several problems in one call (the c4 batch shape), against the SIMT path
    rng = np.random.default_rng(3)
    bins = torch.from_numpy(rng.integers(0, 17, (9, 64, 64)).astype(np.uint8)).cuda()
    s = p.synlik(bins, 16, 200, 12345)
    t = p.synlik(bins, 16, 200, 12345, simt=True)
    assert torch.equal(s["Y"], t["Y"])
    assert torch.equal(s["cov"], t["cov"])


@pytest.mark.parametrize("limit", [1, 2])
def test_bootstrap_multiplicity_fallback(p, tc_all, limit):
    # a multiplicity above the limit (256 in use: bf16's exact integers)
    # hands the counting to the SIMT kernel on the device; with a limit of
    # 1 or 2 every resample takes that path, and the counts stay exact
    rng = np.random.default_rng(77 + limit)
    bins = rng.integers(0, 14, (300, 200)).astype(np.uint8)
    so = oracle.synlik(bins, 13, 40, 0xFA11)
    p.lib().synlik_set_tc_mult_limit(limit)
    try:
        s = p.synlik(torch.from_numpy(bins).cuda(), 13, 40, 0xFA11)
    finally:
        p.lib().synlik_set_tc_mult_limit(-1)
    assert np.array_equal(s["Y"].cpu().numpy(), so["Y"])
    assert np.array_equal(s["cov"].cpu().numpy(), so["cov"])
