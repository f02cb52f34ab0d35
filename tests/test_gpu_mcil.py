"""GPU parity of the multi-feature correlation integral (Sec. 3.1, Alg. 2)
and min-max scaling (Sec. 4) against the oracle: radii, bins, counts and the
concatenated vector bit-exact (integer results of exact definitions), on
shapes that span several tiles, ragged tails and the degenerate cases."""
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


def run_both(p, X1, X2, G, nsp, b=1.3, M=12, features=63, scale=False):
    g = p.mcil(torch.from_numpy(np.ascontiguousarray(X1)).cuda(), torch.from_numpy(np.ascontiguousarray(X2)).cuda(),
               G, nsp, b=b, M=M, features=features, scale=scale)
    o = oracle.mcil(X1, X2, G, nsp, b=b, M=M, mask=features, scale=scale)
    torch.cuda.synchronize()
    assert int(g["n_exact"]) >= 0
    return g, o


def assert_same(g, o):
    assert np.array_equal(g["radii"].cpu().numpy(), o["radii"])
    assert np.array_equal(g["bins"].cpu().numpy(), o["bins"])
    assert np.array_equal(g["counts"].cpu().numpy(), o["counts"])
    assert np.array_equal(g["C"].cpu().numpy(), o["C"])


@pytest.mark.parametrize("n1,n2,G,nsp", [(1, 1, 8, 1), (3, 5, 4, 2), (16, 16, 16, 1), (20, 17, 32, 2),
                                         (37, 90, 32, 2), (64, 64, 64, 1), (130, 65, 16, 1)])
@pytest.mark.parametrize("scale", [False, True])
def test_cosine_patterns_bit_exact(p, n1, n2, G, nsp, scale):
    X = W.cosine_patterns(n1 + n2, G, nsp, 31 + G + n1, amp=1.2, offset=0.7)
    g, o = run_both(p, X[:n1], X[n1:], G, nsp, scale=scale)
    assert_same(g, o)


def test_hand_fixture_maxima(p):
    gd = json.load(open(os.path.join(GOLD, "hand_mcil.json")))
    G = gd["G"]
    X1 = np.array([gd["patterns"]["bump"], gd["patterns"]["ramp_x"]], np.float32)
    X2 = np.zeros((1, G * G), np.float32)
    g, o = run_both(p, X1, X2, G, 1, b=2.0, M=3)
    assert_same(g, o)
    R0 = g["radii"][:, 0].cpu().numpy()
    e = {k: max(gd["expected"][n][k] for n in ("bump", "ramp_x")) for k in gd["expected"]["bump"]}
    assert R0[0] == math.sqrt(e["L2_squared"]) and R0[1] == e["Linf"]
    assert R0[2] == pytest.approx(math.sqrt(e["W12_squared"]), rel=1e-15)
    assert R0[3] == pytest.approx(e["W12p"], rel=1e-15)
    assert R0[4] == e["W1inf"] and R0[5] == e["W1infp"]


def test_l2_feature_equals_cil_features(p):
    G, nsp = 32, 2
    X1 = W.clustered_patterns(40, nsp * G * G, 3)
    X2 = W.clustered_patterns(33, nsp * G * G, 4)
    t1, t2 = torch.from_numpy(X1).cuda(), torch.from_numpy(X2).cuda()
    m = p.mcil(t1, t2, G, nsp, b=1.2, M=16, features=63)
    c = p.cil(t1, t2, b=1.2, M=16)
    assert float(m["radii"][0, 0]) == float(c["R0"])
    assert torch.equal(m["radii"][0, 1:], c["radii"])
    assert torch.equal(m["bins"][0], c["bins"]) and torch.equal(m["counts"][0], c["counts"])


@pytest.mark.parametrize("features", [0x01, 0x02, 0x0C, 0x30, 0x2A, 0x15])
def test_feature_subsets(p, features):
    G, nsp = 16, 2
    X = W.cosine_patterns(50, G, nsp, 77 + features, amp=0.8)
    g, o = run_both(p, X[:23], X[23:], G, nsp, b=1.15, M=20, features=features)
    assert g["bins"].shape[0] == bin(features).count("1")
    assert_same(g, o)


def test_patterns_read_in_place_from_fields(p):
    """u only (species mask 1) and both species, strided rows of the field
    array [n][2][G][G]."""
    G, n = 32, 24
    f = W.cosine_patterns(n, G, 2, 5, amp=1.0)
    ft = torch.from_numpy(f).cuda().reshape(n, 2 * G * G)
    for nsp in (1, 2):
        d = nsp * G * G
        g = p.mcil(ft[:12, :d], ft[12:, :d], G, nsp, b=1.2, M=10)
        Xo = oracle.patterns(f.reshape(n, 2, G, G), 1 if nsp == 1 else 3)
        o = oracle.mcil(Xo[:12], Xo[12:], G, nsp, b=1.2, M=10)
        assert_same(g, o)


def test_multi_feature_bootstrap_statistics(p):
    G, nsp, M, T = 16, 1, 8, 60
    X = W.cosine_patterns(40, G, nsp, 19, amp=1.0)
    g, o = run_both(p, X[:20], X[20:], G, nsp, M=M, features=0x2B)
    s = p.synlik(g["bins"], M, T, 123, y_obs=g["C"], n_feat=4)
    so = oracle.synlik_multi(o["bins"], M, T, 123, y_obs=o["C"])
    assert np.array_equal(s["Y"].cpu().numpy(), so["Y"])
    assert np.array_equal(s["mu"].cpu().numpy(), so["mu"])
    assert np.array_equal(s["cov"].cpu().numpy(), so["cov"])
    assert np.array_equal(s["active"].cpu().numpy(), so["active"])
    assert int(s["status"]) == so["status"]
    if so["status"] == 0:
        assert np.array_equal(s["chol"].cpu().numpy(), so["chol"])
        for k in ("logdet", "f", "loglik"):
            assert float(s[k]) == pytest.approx(so[k], rel=1e-13, abs=1e-300)


def test_c2_shape_stepped_fields(p):
    """The FHN 64x64 workload's shape (2 x 64 patterns, u only) on the
    oracle's own stepped fields, all six features, raw and scaled."""
    cfg = W.config("c2", steps_scale=0.03)
    g0 = cfg["groups"][0]
    f0 = oracle.init_fields(g0["model"], g0["G"], g0["n_real"], g0["params"], g0["noise"][0], g0["noise"][1],
                            g0["seed"]).astype(np.float64)
    f = oracle.step(g0["model"], g0["params"], g0["dt"], g0["n_steps"], f0).astype(np.float32)
    X = oracle.patterns(f, 1)
    for scale in (False, True):
        g, o = run_both(p, X[:64], X[64:], 64, 1, b=cfg["b"], M=cfg["M"], scale=scale)
        assert_same(g, o)
        assert int(g["n_exact"]) < 0.25 * 64 * 64


def test_c3_shape(p):
    """GM 128x128 both species, 2 x 256 patterns (d = 32768): raw data."""
    X = W.cosine_patterns(512, 128, 2, 33, amp=0.8, offset=2.0)
    g, o = run_both(p, X[:256], X[256:], 128, 2, b=1.3, M=16)
    assert_same(g, o)


# ---------------------------------------------------------------------------
# Gy x Gx fields and the 1-D reaction-diffusion-ODE patterns (Sec. 5.2)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("n1,n2,Gy,Gx,nsp", [(7, 9, 1, 64, 2), (16, 16, 1, 128, 1), (33, 40, 8, 32, 2),
                                             (3, 4, 1, 3, 1)])
@pytest.mark.parametrize("scale", [False, True])
def test_rectangular_fields_bit_exact(p, n1, n2, Gy, Gx, nsp, scale):
    rng = np.random.default_rng(Gy * 100 + Gx + n1)
    X = (rng.standard_normal((n1 + n2, nsp * Gy * Gx)) * 0.7 + 1.3).astype(np.float32)
    t = torch.from_numpy(X).cuda()
    g = p.mcil(t[:n1], t[n1:], Gx, nsp, b=1.1, M=12, features=63, scale=scale, Gy=Gy)
    o = oracle.mcil(X[:n1], X[n1:], Gx, nsp, b=1.1, M=12, mask=63, scale=scale, Gy=Gy)
    torch.cuda.synchronize()
    assert int(g["n_exact"]) >= 0
    assert_same(g, o)


def test_rdode_patterns_mcil(p):
    # the RD-ODE workload's patterns at t = 50: L2 and Linf of both species,
    # the derivative-based norms of w alone, bit-exact with the oracle, and
    # the concatenated 6-feature bins through the bootstrap statistics
    cfg = W.config("c7")
    gd = dict(cfg["groups"][0])
    gd["n_real"] = 48
    sim = p.Simulation([p.Group.from_dict(gd)])
    sim.integrate_rkc(1e-3, rtol=cfg["rkc_tol"], atol=cfg["rkc_tol"])
    assert sim.sync_status() == 0
    F = sim.group_fields(0)
    a, c, bins = p.mcil_rdode(F, 24, b=1.1, M=cfg["M"])
    Fn = F.cpu().numpy()
    both = Fn.reshape(48, -1)
    w = np.ascontiguousarray(Fn[:, 1, :])
    oa = oracle.mcil(both[:24], both[24:], 64, 2, b=1.1, M=cfg["M"], mask=0x03, Gy=1)
    oc = oracle.mcil(w[:24], w[24:], 64, 1, b=1.1, M=cfg["M"], mask=0x3C, Gy=1)
    assert_same(a, oa)
    assert_same(c, oc)
    assert bins.shape == (6, 24, 24)
    s = p.synlik(bins, cfg["M"], 100, cfg["seed"], n_feat=6)
    so = oracle.synlik_multi(np.concatenate([oa["bins"], oc["bins"]]), cfg["M"], 100, cfg["seed"])
    assert np.array_equal(s["Y"].cpu().numpy(), so["Y"])


# ---------------------------------------------------------------------------
# the linear radii law per feature (Sec. 2.1 / Sec. 3.2)
# ---------------------------------------------------------------------------
def run_linear(p, X1, X2, Gx, nsp, M=13, features=63, scale=False, Gy=None):
    t1 = torch.from_numpy(np.ascontiguousarray(X1)).cuda()
    t2 = torch.from_numpy(np.ascontiguousarray(X2)).cuda()
    g = p.mcil(t1, t2, Gx, nsp, M=M, features=features, scale=scale, Gy=Gy, law="linear")
    o = oracle.mcil(X1, X2, Gx, nsp, None, M, mask=features, scale=scale, Gy=Gy, law="linear")
    torch.cuda.synchronize()
    assert int(g["n_exact"]) >= 0
    assert_same(g, o)
    return g, o


def test_linear_hand_example(p):
    # on a line: set 1 = {0, 1}, set 2 = {3, 5, 6} -> R0 = 6, R_min = 2,
    # M = 4: radii 5, 4, 3, 2 and counts 3, 2, 1, 0 for L2 and Linf (by hand)
    X1 = np.array([[0.0, 0.0], [1.0, 0.0]], np.float32)
    X2 = np.array([[3.0, 0.0], [5.0, 0.0], [6.0, 0.0]], np.float32)
    g, _ = run_linear(p, X1, X2, 2, 1, M=4, features=0x03, Gy=1)
    for a in range(2):
        assert g["radii"][a].cpu().numpy().tolist() == [6.0, 5.0, 4.0, 3.0, 2.0]
        assert g["counts"][a].cpu().numpy().tolist() == [3, 2, 1, 0]


@pytest.mark.parametrize("n1,n2,Gy,Gx,nsp", [(3, 5, 4, 4, 2), (20, 17, 32, 32, 2), (64, 64, 64, 64, 1),
                                             (7, 9, 1, 64, 2), (33, 40, 8, 32, 2), (130, 65, 16, 16, 1)])
@pytest.mark.parametrize("scale", [False, True])
def test_linear_law_bit_exact(p, n1, n2, Gy, Gx, nsp, scale):
    X = W.cosine_patterns(n1 + n2, Gx, nsp, 71 + Gx + n1, amp=1.2, offset=0.7)
    X = np.ascontiguousarray(X.reshape(n1 + n2, nsp, Gx, Gx)[:, :, :Gy, :].reshape(n1 + n2, -1))
    run_linear(p, X[:n1], X[n1:], Gx, nsp, M=13, scale=scale, Gy=Gy)


def test_linear_near_duplicates(p):
    # set 2 holds slightly perturbed copies of set 1: the smallest values
    # are tiny differences, where the tensor-core interval is widest, so the
    # minimum goes through the re-bounding and the exact evaluation
    rng = np.random.default_rng(42)
    G, n = 32, 40
    X1 = (rng.standard_normal((n, G * G)) * 0.5 + 1.0).astype(np.float32)
    X2 = X1 + (rng.standard_normal((n, G * G)) * 1e-4).astype(np.float32)
    g, o = run_linear(p, X1, X2, G, 1, M=16)
    assert o["radii"][0, -1] < 0.1 * o["radii"][0, 0]
    assert int(g["n_exact"]) >= 1


def test_linear_degenerate_cases(p):
    rng = np.random.default_rng(9)
    G = 8
    # a single pair: R0 = R_min, every radius R0, nothing below it
    X1 = rng.standard_normal((1, G * G)).astype(np.float32)
    X2 = rng.standard_normal((1, G * G)).astype(np.float32)
    g, _ = run_linear(p, X1, X2, G, 1, M=5)
    assert (g["counts"].cpu().numpy() == 0).all()
    # a pattern in both sets: every feature's minimum is 0
    X1 = rng.standard_normal((6, G * G)).astype(np.float32)
    X2 = np.concatenate([rng.standard_normal((5, G * G)).astype(np.float32), X1[2:3]])
    g, o = run_linear(p, X1, X2, G, 1, M=13)
    # ties at the minimum: two pairs at the same smallest values
    X1 = np.zeros((2, G * G), np.float32)
    X1[1] += 10.0
    X2 = np.stack([X1[0] + 1.0, X1[1] + 1.0, X1[0] + 5.0]).astype(np.float32)
    run_linear(p, X1, X2, G, 1, M=7)


def test_linear_rdode_patterns(p):
    # Table 1's pairing: the RD-ODE patterns at t = 50 with the linear law,
    # L2/Linf of both species and the W norms of w, bit-exact
    cfg = W.config("c7")
    gd = dict(cfg["groups"][0])
    gd["n_real"] = 48
    sim = p.Simulation([p.Group.from_dict(gd)])
    sim.integrate_rkc(1e-3, rtol=cfg["rkc_tol"], atol=cfg["rkc_tol"])
    assert sim.sync_status() == 0
    F = sim.group_fields(0)
    a, c, bins = p.mcil_rdode(F, 24, M=cfg["M"], law="linear")
    Fn = F.cpu().numpy()
    both = Fn.reshape(48, -1)
    w = np.ascontiguousarray(Fn[:, 1, :])
    oa = oracle.mcil(both[:24], both[24:], 64, 2, None, cfg["M"], mask=0x03, Gy=1, law="linear")
    oc = oracle.mcil(w[:24], w[24:], 64, 1, None, cfg["M"], mask=0x3C, Gy=1, law="linear")
    assert_same(a, oa)
    assert_same(c, oc)
    assert bins.shape == (6, 24, 24)


# ---------------------------------------------------------------------------
# the power law fitted to each feature's range (Sec. 2.1 / Sec. 3.2)
# ---------------------------------------------------------------------------
def run_fitted(p, X1, X2, Gx, nsp, M=13, features=63, scale=False, Gy=None):
    t1 = torch.from_numpy(np.ascontiguousarray(X1)).cuda()
    t2 = torch.from_numpy(np.ascontiguousarray(X2)).cuda()
    g = p.mcil(t1, t2, Gx, nsp, M=M, features=features, scale=scale, Gy=Gy, law="fitted")
    o = oracle.mcil(X1, X2, Gx, nsp, None, M, mask=features, scale=scale, Gy=Gy, law="fitted")
    torch.cuda.synchronize()
    assert int(g["n_exact"]) >= 0
    assert_same(g, o)
    return g, o


def test_fitted_hand_example(p):
    X1 = np.array([[0.0, 0.0]], np.float32)
    X2 = np.array([[1.0, 0.0], [2.0, 0.0], [8.0, 0.0]], np.float32)
    g, _ = run_fitted(p, X1, X2, 2, 1, M=3, features=0x03, Gy=1)
    for a in range(2):
        assert g["radii"][a].cpu().numpy().tolist() == [8.0, 4.0, 2.0, 1.0]
        assert g["counts"][a].cpu().numpy().tolist() == [2, 1, 0]


@pytest.mark.parametrize("n1,n2,Gy,Gx,nsp", [(3, 5, 4, 4, 2), (20, 17, 32, 32, 2), (64, 64, 64, 64, 1),
                                             (7, 9, 1, 64, 2), (33, 40, 8, 32, 2)])
@pytest.mark.parametrize("scale", [False, True])
def test_fitted_law_bit_exact(p, n1, n2, Gy, Gx, nsp, scale):
    X = W.cosine_patterns(n1 + n2, Gx, nsp, 171 + Gx + n1, amp=1.2, offset=0.7)
    X = np.ascontiguousarray(X.reshape(n1 + n2, nsp, Gx, Gx)[:, :, :Gy, :].reshape(n1 + n2, -1))
    run_fitted(p, X[:n1], X[n1:], Gx, nsp, M=13, scale=scale, Gy=Gy)


def test_fitted_degenerate(p):
    rng = np.random.default_rng(12)
    G = 8
    X1 = rng.standard_normal((6, G * G)).astype(np.float32)
    X2 = np.concatenate([rng.standard_normal((5, G * G)).astype(np.float32), X1[2:3]])
    g, _ = run_fitted(p, X1, X2, G, 1, M=13)   # R_min = 0 for every feature: b = +inf
    assert (g["radii"][:, 1:].cpu().numpy() == 0.0).all()
    X1 = rng.standard_normal((1, G * G)).astype(np.float32)
    X2 = rng.standard_normal((1, G * G)).astype(np.float32)
    run_fitted(p, X1, X2, G, 1, M=5)           # one pair: b = 1
