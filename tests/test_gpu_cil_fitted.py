"""GPU parity of the correlation integral with the power law fitted to the
distance range (Sec. 2.1 / Sec. 3.2; Table 1's law for the FHN, GM and BZ
models): R0, every radius (through the fitted b), the bins and the counts
bit-exact against the oracle, including the degenerate cases."""
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
    g = p.cil_fitted(torch.from_numpy(np.ascontiguousarray(X1)).cuda(),
                     torch.from_numpy(np.ascontiguousarray(X2)).cuda(), M=M)
    o = oracle.cil(X1, X2, M=M, law="fitted")
    assert int(g["n_rechecked"]) >= 0
    assert float(g["R0"]) == o["R0"]
    assert np.array_equal(g["radii"].cpu().numpy(), o["radii"])
    assert np.array_equal(g["bins"].cpu().numpy(), o["bins"])
    assert np.array_equal(g["counts"].cpu().numpy(), o["counts"])
    return g, o


def test_hand_example(p):
    # set 1 = {0}, set 2 = {1, 2, 8} on a line: R0 = 8, R_min = 1, M = 3
    # -> b = 2, radii 4, 2, 1, counts 2, 1, 0 (worked by hand)
    X1 = np.array([[0.0]], np.float32)
    X2 = np.array([[1.0], [2.0], [8.0]], np.float32)
    g, _ = run_both(p, X1, X2, 3)
    assert g["radii"].cpu().numpy().tolist() == [4.0, 2.0, 1.0]
    assert g["counts"].cpu().numpy().tolist() == [2, 1, 0]


@pytest.mark.parametrize("n1,n2,d,M", [(3, 5, 7, 13), (16, 16, 2048, 16), (64, 64, 4096, 16),
                                       (65, 130, 4100, 13), (100, 37, 9000, 32), (200, 200, 3000, 8)])
def test_clustered_patterns_bit_exact(p, n1, n2, d, M):
    X1 = W.clustered_patterns(n1, d, 500 + n1)
    X2 = W.clustered_patterns(n2, d, 600 + n2)
    run_both(p, X1, X2, M)


@pytest.mark.parametrize("G,ns,n", [(64, 1, 64), (128, 2, 48)])
def test_rd_field_patterns(p, G, ns, n):
    # RD-like cosine-mode fields (the FHN / GM shapes of Table 1)
    X = W.cosine_patterns(2 * n, G, ns, 31 + G, amp=1.2, offset=0.5)
    run_both(p, X[:n], X[n:], 16)


def test_degenerate_cases(p):
    rng = np.random.default_rng(21)
    # a single pair: R_min = R0, b = 1, every radius R0, nothing below it
    X1 = rng.standard_normal((1, 50)).astype(np.float32)
    X2 = rng.standard_normal((1, 50)).astype(np.float32)
    g, _ = run_both(p, X1, X2, 5)
    assert g["counts"].cpu().numpy().tolist() == [0] * 5
    # a pattern in both sets: R_min = 0, b = +inf, every R_k = 0
    X1 = rng.standard_normal((6, 300)).astype(np.float32)
    X2 = np.concatenate([rng.standard_normal((5, 300)).astype(np.float32), X1[2:3]])
    g, _ = run_both(p, X1, X2, 13)
    assert (g["radii"].cpu().numpy() == 0.0).all()


def test_pipeline_fitted_law(p):
    # the whole pass with the fitted law: counts against the oracle on the
    # fields the pass produced
    g = p.Group(W.FHN, 32, 32, W.FHN_THETA0, 2 ** -8, 200, (-0.05, 0.05), 7)
    pipe = p.Pipeline([g], [(16, 16, 1)], M=8, b=None, T=30, seed=5, law="fitted")
    pipe.run()
    torch.cuda.synchronize()
    F = pipe.sim.group_fields(0).reshape(32, -1).cpu().numpy()
    o = oracle.cil(F[:16, :1024], F[16:, :1024], M=8, law="fitted")
    assert np.array_equal(pipe.bins[0].cpu().numpy(), o["bins"])
