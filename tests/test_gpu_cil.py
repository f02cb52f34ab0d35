"""GPU parity of the correlation integral against the oracle: radii, bin
indices and counts must be bit-exact (integer results of an exact
definition), on shapes that span several tiles and ragged tails."""
import json
import math
import os

import numpy as np
import pytest
import torch

import oracle
import workloads as W

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def p():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2203_14742_b300 as pk
    return pk


def run_both(p, X1, X2, b=1.3, M=16, radii=None, exact=False):
    t1 = torch.from_numpy(np.ascontiguousarray(X1)).cuda()
    t2 = torch.from_numpy(np.ascontiguousarray(X2)).cuda()
    fn = p.cil_exact if exact else p.cil
    r = torch.from_numpy(np.asarray(radii, np.float64)) if radii is not None else None
    g = fn(t1, t2, b=b, M=M, radii=r)
    o = oracle.cil(X1, X2, b=b, M=M, radii_=radii)
    # -1 would mean a pair whose bound straddled a threshold the exact pass
    # did not foresee
    assert int(g["n_rechecked"]) >= 0
    return g, o


def assert_same(g, o, check_r0=True):
    if check_r0:
        assert float(g["R0"]) == o["R0"]
    assert np.array_equal(g["radii"].cpu().numpy(), o["radii"])
    assert np.array_equal(g["bins"].cpu().numpy(), o["bins"])
    assert np.array_equal(g["counts"].cpu().numpy(), o["counts"])


def test_hand_counted_fixture(p):
    gd = json.load(open(os.path.join(GOLD, "hand_cil_2d.json")))
    X1 = np.array(gd["S1"], np.float32)
    X2 = np.array(gd["S2"], np.float32)
    for exact in (False, True):
        g, o = run_both(p, X1, X2, b=gd["b"], M=gd["M"], exact=exact)
        assert_same(g, o)
        assert list(g["counts"].cpu().numpy()) == gd["counts"]
        assert np.array_equal(g["bins"].cpu().numpy(), np.array(gd["bins"], np.uint8))


@pytest.mark.parametrize("n1,n2,d", [(1, 1, 1), (3, 5, 7), (16, 16, 2048), (64, 64, 4096),
                                     (65, 130, 4100), (100, 37, 9000), (200, 200, 3000)])
def test_clustered_patterns_bit_exact(p, n1, n2, d):
    X1 = W.clustered_patterns(n1, d, 100 + n1)
    X2 = W.clustered_patterns(n2, d, 200 + n2)
    g, o = run_both(p, X1, X2, b=1.1, M=16)
    assert_same(g, o)
    ge, _ = run_both(p, X1, X2, b=1.1, M=16, exact=True)
    assert_same(ge, o)


@pytest.mark.parametrize("G,ns,n", [(32, 2, 16), (64, 1, 64), (128, 2, 40)])
def test_cosine_patterns_bit_exact(p, G, ns, n):
    X = W.cosine_patterns(2 * n, G, ns, 7 + G, amp=1.5, offset=2.0)
    g, o = run_both(p, X[:n], X[n:], b=1.05, M=32)
    assert_same(g, o)


def test_given_radii(p):
    X1 = W.clustered_patterns(40, 256, 1)
    X2 = W.clustered_patterns(33, 256, 2)
    d2 = oracle.pair_d2(X1, X2)
    # radii placed exactly on some realised distances: ties must not count
    qs = np.quantile(np.sqrt(d2).ravel(), [0.9, 0.7, 0.5, 0.3, 0.1])
    exact_r = np.sqrt(np.sort(d2.ravel())[[100, 500, 900]])
    radii = np.sort(np.concatenate([qs, exact_r]))[::-1].copy()
    g, o = run_both(p, X1, X2, radii=radii, M=len(radii))
    assert_same(g, o, check_r0=False)


def test_strided_sets_from_field_array(p):
    """Patterns read in place from [n][2][G][G] fields: u only and both."""
    G, n = 64, 24
    f = W.cosine_patterns(n, G, 2, 5, amp=1.0).reshape(n, 2, G, G)
    ft = torch.from_numpy(f).cuda().reshape(n, 2 * G * G)
    for mask in (1, 3):
        d = G * G * (2 if mask == 3 else 1)
        X1 = ft[:12, :d]
        X2 = ft[12:, :d]
        g = p.cil(X1, X2, b=1.2, M=16)
        Xo = oracle.patterns(f, mask)
        o = oracle.cil(Xo[:12], Xo[12:], b=1.2, M=16)
        assert_same(g, o)


def test_swapped_sets_transpose(p):
    X1 = W.clustered_patterns(30, 500, 3)
    X2 = W.clustered_patterns(45, 500, 4)
    a = p.cil(torch.from_numpy(X1).cuda(), torch.from_numpy(X2).cuda(), b=1.2, M=12)
    b = p.cil(torch.from_numpy(X2).cuda(), torch.from_numpy(X1).cuda(), b=1.2, M=12)
    assert torch.equal(a["bins"], b["bins"].T)
    assert torch.equal(a["counts"], b["counts"])


def test_full_size_c2_from_oracle_patterns(p):
    """c2 CIL at full size (2 x 64 patterns, d = 4096, M = 16): the patterns
    are the oracle's own FP64 FHN fields (rounded to FP32) after a short
    integration, so both sides see the same input."""
    cfg = W.config("c2", steps_scale=0.03)
    g = cfg["groups"][0]
    f0 = oracle.init_fields(g["model"], g["G"], g["n_real"], g["params"], g["noise"][0],
                            g["noise"][1], g["seed"]).astype(np.float64)
    f = oracle.step(g["model"], g["params"], g["dt"], g["n_steps"], f0).astype(np.float32)
    X = oracle.patterns(f, g["species_mask"])
    res, o = run_both(p, X[:64], X[64:], b=cfg["b"], M=cfg["M"])
    assert_same(res, o)
    assert int(res["n_rechecked"]) < 0.05 * 64 * 64


def test_full_size_c3_shape(p):
    """c3 shape: 2 x 256 patterns of d = 32768 (GM 128x128, both species),
    synthetic cosine fields around the GM equilibrium."""
    X = W.cosine_patterns(512, 128, 2, 33, amp=0.8, offset=2.0)
    res, o = run_both(p, X[:256], X[256:], b=1.3, M=16)
    assert_same(res, o)
    assert int(res["n_rechecked"]) < 0.05 * 256 * 256


def test_bound_holds_against_exact_path(p):
    """The fast path's classification equals the exact path's on every pair,
    including data far from the origin (centring matters)."""
    X1 = W.clustered_patterns(90, 2000, 9) + 50.0
    X2 = W.clustered_patterns(70, 2000, 10) + 50.0
    t1, t2 = torch.from_numpy(X1).cuda(), torch.from_numpy(X2).cuda()
    a = p.cil(t1, t2, b=1.02, M=32)
    e = p.cil_exact(t1, t2, b=1.02, M=32)
    assert float(a["R0"]) == float(e["R0"])
    assert torch.equal(a["bins"], e["bins"])
    assert torch.equal(a["counts"], e["counts"])


@pytest.mark.parametrize("n1,n2,d,off", [(64, 64, 4096, 0.0), (130, 70, 3000, 20.0), (256, 256, 32768, 2.0),
                                         (5, 300, 128, 0.0)])
def test_tensor_core_bound_holds_with_slack(p, n1, n2, d, off):
    """The rigorous error bound of the tensor-core approximation holds for
    every pair, with room to spare (the model is conservative): the
    approximation error stays below a quarter of the bound."""
    X1 = W.clustered_patterns(n1, d, 500 + n1) + off
    X2 = W.clustered_patterns(n2, d, 600 + n2) + off
    A, m = p.cil_approx(torch.from_numpy(X1).cuda(), torch.from_numpy(X2).cuda())
    ex = oracle.pair_d2(X1, X2)
    A, m = A.cpu().numpy(), m.cpu().numpy()
    err = np.abs(A - ex)
    assert np.all(err <= 0.25 * m), (err / m).max()
    # and the bound is tight enough to be useful: relative width < 1e-3
    assert np.all(m <= 1e-3 * ex + 1e-9)


def test_tensor_core_bound_at_paper_scale(p):
    """The tier-1 bound at the SCIL scale, 2 x 1024 patterns of d = 32768,
    where every K segment adds 64 chunk partials in an FP32 running sum:
    each pair's approximation error stays below a quarter of its bound.  The
    reference is a float64 Gram on the host, within (d + 2) 2^-53 (|x|^2 +
    |y|^2 + 2 |x| |y|) of every d2, far below the bound."""
    n = 1024
    X = W.cosine_patterns(2 * n, 128, 2, 78, amp=0.8, offset=2.0)
    X1, X2 = X[:n], X[n:]
    A, m = p.cil_approx(torch.from_numpy(X1).cuda(), torch.from_numpy(X2).cuda())
    A, m = A.cpu().numpy(), m.cpu().numpy()
    A1, A2 = X1.astype(np.float64), X2.astype(np.float64)
    n1s, n2s = (A1 * A1).sum(1), (A2 * A2).sum(1)
    D = n1s[:, None] + n2s[None, :] - 2.0 * (A1 @ A2.T)
    d = X.shape[1]
    eD = (d + 2) * 2.0 ** -53 * (n1s[:, None] + n2s[None, :] + 2.0 * np.sqrt(n1s[:, None] * n2s[None, :]))
    err = np.abs(A - D)
    assert np.all(err <= 0.25 * m + 2.0 * eD), (err / m).max()
    assert np.all(m <= 1e-3 * D + 1e-9)


def wide_floats(rng, n):
    """FP32 values over the whole exponent range: normals, subnormals,
    zeros, both signs."""
    kind = rng.integers(0, 4, n)
    mant = rng.uniform(1.0, 2.0, n)
    v = np.where(kind == 0, mant * 2.0 ** rng.integers(-126, 100, n).astype(np.float64), 0.0)
    v = np.where(kind == 1, mant * 2.0 ** rng.integers(-10, 10, n), v)
    v = np.where(kind == 2, rng.integers(1, 2 ** 23, n) * 2.0 ** -149, v)
    v = v * np.where(rng.integers(0, 2, n) == 0, 1.0, -1.0)
    return v.astype(np.float32)


@pytest.mark.parametrize("d", [1, 2, 3, 17, 64, 1000, 4099])
def test_exact_d2_bit_exact_over_the_exponent_range(p, d):
    """The exact kernel (the last tier of every correlation integral) equals
    the oracle's exactly rounded sum bit for bit, for inputs spanning
    subnormals to 2^100 and for near-equal pairs (heavy cancellation)."""
    rng = np.random.default_rng(d)
    n1, n2 = 9, 7
    X1 = np.stack([wide_floats(rng, d) for _ in range(n1)])
    X2 = np.stack([wide_floats(rng, d) for _ in range(n2)])
    X2[:3] = (X1[:3].astype(np.float64) * (1 + 1e-6 * rng.normal(size=(3, d)))).astype(np.float32)
    pairs = np.array([(i, j) for i in range(n1) for j in range(n2)], np.int64)
    g = p.exact_d2(torch.from_numpy(X1).cuda(), torch.from_numpy(X2).cuda(), torch.from_numpy(pairs))
    o = oracle.pair_d2(X1, X2).reshape(-1)
    assert np.array_equal(g.cpu().numpy(), o)


def test_exact_d2_ties_and_non_finite(p):
    t, u = np.float32(2.0 ** -27), np.float32(2.0 ** -26)
    X1 = np.zeros((5, 5), np.float32)
    X1[0, :3] = [1.0, t, t]              # 1 + 2^-53: tie, to even -> 1
    X1[1, :4] = [1.0, u, t, t]           # 1 + 2^-52 + 2^-53: tie -> 1 + 2^-51
    X1[2, :4] = [1.0, t, t, t]           # above half-way -> 1 + 2^-52
    X1[3, :] = [1.0, t, t, t, t]         # exactly 1 + 2^-52
    X1[4, 2] = np.inf
    X2 = np.zeros((1, 5), np.float32)
    pairs = np.array([(i, 0) for i in range(5)], np.int64)
    g = p.exact_d2(torch.from_numpy(X1).cuda(), torch.from_numpy(X2).cuda(), torch.from_numpy(pairs)).cpu().numpy()
    assert list(g[:4]) == [1.0, 1.0 + 2.0 ** -51, 1.0 + 2.0 ** -52, 1.0 + 2.0 ** -52]
    assert math.isnan(g[4])


def test_exact_d2_long_patterns(p):
    """d = 32768 (GM 128^2, both species): equal to the oracle on 64 pairs."""
    X = W.cosine_patterns(16, 128, 2, 41, amp=0.8, offset=2.0)
    rng = np.random.default_rng(3)
    pairs = rng.integers(0, 8, size=(64, 2)).astype(np.int64)
    g = p.exact_d2(torch.from_numpy(X[:8]).cuda(), torch.from_numpy(X[8:]).cuda(), torch.from_numpy(pairs))
    o = np.array([oracle.d2_exact(X[i], X[8 + j]) for i, j in pairs])
    assert np.array_equal(g.cpu().numpy(), o)


@pytest.mark.parametrize("products", [1, 3])
def test_paper_scale_every_pair(p, products):
    """2 x 1024 patterns of d = 32768 (the SCIL scale, as timed by bench.py
    --gram-large), every one of the 1.05e6 bins checked without the GPU's
    approximate stage: a float64 Gram on the host (numpy/BLAS) gives every
    d2 within the dot-product error bound (d + 2) 2^-53 (|x|^2 + |y|^2 +
    2 |x| |y|); pairs whose interval could hold the maximum or meets a
    threshold are evaluated by the oracle exactly, all others are decided
    by their interval.  Both forms of the tensor-core Gram (three products,
    the default, and one)."""
    n, G = 1024, 128
    X = W.cosine_patterns(2 * n, G, 2, 77, amp=0.8, offset=2.0)
    X1, X2 = X[:n], X[n:]
    t1, t2 = torch.from_numpy(X1).cuda(), torch.from_numpy(X2).cuda()
    assert p.gram_products(n, n, X.shape[1]) == 3
    try:
        p.set_gram_products(products)
        g = p.cil(t1, t2, b=1.3, M=16)
        torch.cuda.synchronize()
    finally:
        p.set_gram_products(0)
    assert int(g["n_rechecked"]) >= 0
    R0 = float(g["R0"])
    radii = g["radii"].cpu().numpy()
    bins = g["bins"].cpu().numpy()
    counts = g["counts"].cpu().numpy()
    for k in range(1, 17):
        assert counts[k - 1] == int((bins >= k).sum())
    # host float64 intervals of every d2 (the GPU plays no part)
    A1, A2 = X1.astype(np.float64), X2.astype(np.float64)
    n1s, n2s = (A1 * A1).sum(1), (A2 * A2).sum(1)
    D = n1s[:, None] + n2s[None, :] - 2.0 * (A1 @ A2.T)
    d = X.shape[1]
    err = (d + 2) * 2.0 ** -53 * (n1s[:, None] + n2s[None, :] + 2.0 * np.sqrt(n1s[:, None] * n2s[None, :]))
    err = 2.0 * err + 1e-300                    # slack for the rounding of D and err themselves
    lo, hi = D - err, D + err
    # the maximum: exact over every pair whose interval reaches the largest lower bound
    cand = np.argwhere(hi >= lo.max())
    best = max(oracle.d2_exact(X1[i], X2[j]) for i, j in cand)
    assert math.sqrt(best) == R0
    # bins: decided by the interval unless it meets a threshold
    T = radii * radii
    K = np.zeros((n, n), np.int64)
    open_ = np.zeros((n, n), bool)
    for t in T:
        K += hi < t
        open_ |= ~((hi < t) | (lo >= t))
    for i, j in np.argwhere(open_):
        d2 = oracle.d2_exact(X1[i], X2[j])
        K[i, j] = int(sum(d2 < t for t in T))
    assert np.array_equal(bins, K.astype(np.uint8))


# ---------------------------------------------------------------------------
# The one-product Gram (hi.hi alone, cross terms bounded by Cauchy-Schwarz),
# selected in place of the default three products: same bits, only the
# number of pairs re-evaluated beyond tier 1 moves.
# ---------------------------------------------------------------------------
@pytest.fixture
def one_product(p):
    p.set_gram_products(1)
    yield
    p.set_gram_products(0)


@pytest.mark.parametrize("n1,n2,d", [(1, 1, 1), (3, 5, 7), (64, 64, 4096), (65, 130, 4100), (200, 200, 3000)])
def test_one_product_clustered_bit_exact(p, one_product, n1, n2, d):
    assert p.gram_products(n1, n2, d) == 1
    X1 = W.clustered_patterns(n1, d, 100 + n1)
    X2 = W.clustered_patterns(n2, d, 200 + n2)
    g, o = run_both(p, X1, X2, b=1.1, M=16)
    assert_same(g, o)


def test_one_product_c3_shape_and_far_data(p, one_product):
    X = W.cosine_patterns(512, 128, 2, 33, amp=0.8, offset=2.0)
    res, o = run_both(p, X[:256], X[256:], b=1.3, M=16)
    assert_same(res, o)
    assert int(res["n_rechecked"]) < 0.05 * 256 * 256
    X1 = W.clustered_patterns(90, 2000, 9) + 50.0
    X2 = W.clustered_patterns(70, 2000, 10) + 50.0
    t1, t2 = torch.from_numpy(X1).cuda(), torch.from_numpy(X2).cuda()
    a = p.cil(t1, t2, b=1.02, M=32)
    e = p.cil_exact(t1, t2, b=1.02, M=32)
    assert float(a["R0"]) == float(e["R0"])
    assert torch.equal(a["bins"], e["bins"])


@pytest.mark.parametrize("n1,n2,d,off", [(64, 64, 4096, 0.0), (130, 70, 3000, 20.0), (256, 256, 32768, 2.0),
                                         (5, 300, 128, 0.0)])
def test_one_product_bound_holds(p, one_product, n1, n2, d, off):
    """The one-product interval holds every pair's exact d2 with room to
    spare (error below half the bound: the Cauchy-Schwarz terms assume the
    worst alignment of the dropped parts); its width stays within the
    predicted scale: 4 (|hi_i| |lo_j| + |lo_i| |hi_j|), about 2^-7 |x_i| |x_j|
    (bound 2^-5, since the library's centre is a sample mean)."""
    X1 = W.clustered_patterns(n1, d, 500 + n1) + off
    X2 = W.clustered_patterns(n2, d, 600 + n2) + off
    A, m = p.cil_approx(torch.from_numpy(X1).cuda(), torch.from_numpy(X2).cuda())
    ex = oracle.pair_d2(X1, X2)
    A, m = A.cpu().numpy(), m.cpu().numpy()
    assert np.all(np.abs(A - ex) <= 0.5 * m), (np.abs(A - ex) / m).max()
    c = np.concatenate([X1, X2]).astype(np.float64)
    c = c - c.mean(0)       # near the library's centre; the norms set the scale only
    nrm = np.sqrt((c * c).sum(1))
    scale = nrm[:n1, None] * nrm[None, n1:] + 1e-30
    assert np.all(m <= 2.0 ** -5 * scale + 1e-6 * ex + 1e-9)


def test_one_product_mcil_bit_exact(p, one_product):
    """The multi-feature correlation integral takes the same tier-1 stage."""
    X = W.cosine_patterns(37 + 90, 32, 2, 31 + 32 + 37, amp=1.2, offset=0.7)
    g = p.mcil(torch.from_numpy(X[:37]).cuda(), torch.from_numpy(X[37:]).cuda(), 32, 2, b=1.3, M=12)
    o = oracle.mcil(X[:37], X[37:], 32, 2, b=1.3, M=12, mask=63, scale=False)
    torch.cuda.synchronize()
    assert np.array_equal(g["bins"].cpu().numpy(), o["bins"])
    assert np.array_equal(g["counts"].cpu().numpy(), o["counts"])


def test_both_forms_at_paper_scale_agree(p):
    """The G-large shape under both forms: identical radii, bins and counts."""
    n = 1024
    X = W.cosine_patterns(2 * n, 128, 2, 78, amp=0.8, offset=2.0)
    t1, t2 = torch.from_numpy(X[:n]).cuda(), torch.from_numpy(X[n:]).cuda()
    out, ql = {}, {}
    try:
        for k in (1, 3):
            p.set_gram_products(k)
            out[k] = p.cil(t1, t2, b=1.3, M=16)
            ql[k] = p.cil_queue_lengths(n, n, X.shape[1])
    finally:
        p.set_gram_products(0)
    for key in ("radii", "bins", "counts"):
        assert torch.equal(out[1][key], out[3][key]), key
    # tier 3 is what n_rechecked reports; the wider interval leaves more to tier 2
    for k in (1, 3):
        assert ql[k][1] == int(out[k]["n_rechecked"]) >= 1      # the maximum at least
        assert ql[k][0] >= ql[k][1]
    assert ql[1][0] > ql[3][0]
