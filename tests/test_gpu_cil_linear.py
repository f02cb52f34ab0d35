"""GPU parity of the correlation integral with the linear radii law of Sec.
2.1 / Sec. 3.2 (R_k = R0 - k (R0 - R_min) / M; Table 1's law for the MC and
RD-ODE models): R0, R_min, every radius, the bins and the counts bit-exact
against the oracle, including the degenerate cases (a single pair, a
pattern repeated across the sets, ties at the minimum)."""
import numpy as np
import pytest
import torch

import oracle
import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def p():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2203_14742_b300 as pk
    return pk


def run_both(p, X1, X2, M):
    g = p.cil_linear(torch.from_numpy(np.ascontiguousarray(X1)).cuda(),
                     torch.from_numpy(np.ascontiguousarray(X2)).cuda(), M=M)
    o = oracle.cil(X1, X2, M=M, law="linear")
    assert int(g["n_rechecked"]) >= 0
    assert float(g["R0"]) == o["R0"]
    assert np.array_equal(g["radii"].cpu().numpy(), o["radii"])
    assert np.array_equal(g["bins"].cpu().numpy(), o["bins"])
    assert np.array_equal(g["counts"].cpu().numpy(), o["counts"])
    return g, o


def test_hand_example(p):
    # on a line: set 1 = {0, 1}, set 2 = {3, 5, 6}: R0 = 6, R_min = 2, M = 4
    # -> radii 5, 4, 3, 2, counts 3, 2, 1, 0 (worked by hand)
    X1 = np.array([[0.0], [1.0]], np.float32)
    X2 = np.array([[3.0], [5.0], [6.0]], np.float32)
    g, o = run_both(p, X1, X2, 4)
    assert list(g["counts"].cpu().numpy()) == [3, 2, 1, 0]
    assert g["radii"].cpu().numpy().tolist() == [5.0, 4.0, 3.0, 2.0]


@pytest.mark.parametrize("n1,n2,d,M", [(3, 5, 7, 13), (16, 16, 2048, 13), (64, 64, 4096, 16),
                                       (65, 130, 4100, 13), (100, 37, 9000, 32), (200, 200, 3000, 13)])
def test_clustered_patterns_bit_exact(p, n1, n2, d, M):
    X1 = W.clustered_patterns(n1, d, 300 + n1)
    X2 = W.clustered_patterns(n2, d, 400 + n2)
    run_both(p, X1, X2, M)


@pytest.mark.parametrize("G,ns,n", [(32, 2, 16), (64, 1, 64)])
def test_cosine_patterns_bit_exact(p, G, ns, n):
    X = W.cosine_patterns(2 * n, G, ns, 17 + G, amp=1.5, offset=2.0)
    run_both(p, X[:n], X[n:], 13)


def test_rdode_patterns(p):
    # the RD-ODE workload's patterns (both species, d = 128) at t = 50, the
    # setting Table 1 pairs with the linear law (M = 13)
    cfg = W.config("c7")
    gd = dict(cfg["groups"][0])
    gd["n_real"] = 40
    sim = p.Simulation([p.Group.from_dict(gd)])
    sim.integrate_rkc(1e-3, rtol=cfg["rkc_tol"], atol=cfg["rkc_tol"])
    assert sim.sync_status() == 0
    X = sim.group_fields(0).reshape(40, -1).cpu().numpy()
    g, o = run_both(p, X[:20], X[20:], cfg["M"])
    assert o["counts"][0] > 0


def test_degenerate_cases(p):
    rng = np.random.default_rng(8)
    # a single pair: R0 = R_min, h = 0, every radius R0, nothing below it
    X1 = rng.standard_normal((1, 50)).astype(np.float32)
    X2 = rng.standard_normal((1, 50)).astype(np.float32)
    g, _ = run_both(p, X1, X2, 5)
    assert g["counts"].cpu().numpy().tolist() == [0] * 5
    # a pattern in both sets: R_min = 0 and R_M = 0
    X1 = rng.standard_normal((6, 300)).astype(np.float32)
    X2 = np.concatenate([rng.standard_normal((5, 300)).astype(np.float32), X1[2:3]])
    g, o = run_both(p, X1, X2, 13)
    assert float(g["radii"][-1]) == 0.0
    # ties at the minimum: two pairs at the same smallest distance
    X1 = np.array([[0.0, 0.0], [10.0, 0.0]], np.float32)
    X2 = np.array([[1.0, 0.0], [11.0, 0.0], [5.0, 3.0]], np.float32)
    run_both(p, X1, X2, 7)
