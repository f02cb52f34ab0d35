"""Pins of the oracle's semi-implicit (IMEX) Euler step (Sec. 5.1 and
App. B.2: implicit diffusion through a linear solve; Sec. 4.1 kinetics;
App. B.1.1 discretisation), checked against facts fixed by the mathematics
rather than against the oracle itself."""
import numpy as np
import pytest

import oracle as O
from oracle import imex as I


def _mode(G, p, q):
    x = (np.arange(G) + 0.5) * np.pi / G
    return np.outer(np.cos(q * x), np.cos(p * x))   # [y][x]: p along x, q along y


@pytest.mark.parametrize("G", [8, 12, 128])
def test_cosine_modes_decay_by_the_closed_form_factor(G):
    """Pure diffusion: the cosine modes cos(pi p (x+1/2)/G) cos(pi q (y+1/2)/G)
    are the eigenvectors of the mirrored-ghost Laplacian with eigenvalue
    -(G-1)^2 (4 sin^2(pi p/2G) + 4 sin^2(pi q/2G)), so one implicit step
    divides each by 1 + dt D (G-1)^2 (...).  Fixes the ghost rule, the
    (G-1)^2 scaling and the sign of the implicit term; G = 128 runs the
    sparse factorisation."""
    D = (0.003, 0.02)
    dt = 0.01
    for (p, q) in ((0, 0), (1, 0), (0, 3), (2, 5), (G - 1, G - 1)):
        m = _mode(G, p, q)
        w0 = np.stack([m, 2.0 * m])[None]
        w1 = I.imex_run(O.DIFF, (D[0], D[1], 0, 0), dt, 1, w0)
        lam = (G - 1) ** 2 * (4 * np.sin(np.pi * p / (2 * G)) ** 2 + 4 * np.sin(np.pi * q / (2 * G)) ** 2)
        for s in range(2):
            want = w0[0, s] / (1.0 + dt * D[s] * lam)
            np.testing.assert_allclose(w1[0, s], want, rtol=0, atol=1e-13 * (1 + abs(w0[0, s]).max()))


def test_pure_diffusion_conserves_mass():
    G = 10
    rng = np.random.default_rng(3)
    w0 = rng.uniform(-1, 1, (2, 2, G, G))
    w = I.imex_run(O.DIFF, (0.01, 0.05, 0, 0), 0.05, 6, w0)
    np.testing.assert_allclose(w.sum(axis=(2, 3)), w0.sum(axis=(2, 3)), rtol=0, atol=1e-11)


@pytest.mark.parametrize("model,p", [
    (O.FHN, (2.8e-4, 0.05, 10.0, 0.95)),
    (O.GM, (2.5e-4, 0.01, 1.0, 0.47)),
    (O.BZ, (0.002, 0.02, 1.5, 2.3)),
])
def test_homogeneous_equilibrium_stays_fixed(model, p):
    G = 8
    u0, v0 = O.equilibrium(model, p)
    w0 = np.stack([np.full((G, G), u0), np.full((G, G), v0)])[None]
    w = I.imex_run(model, p, 0.05, 5, w0)
    np.testing.assert_allclose(w, w0, rtol=0, atol=1e-13)


@pytest.mark.parametrize("model,p", [
    (O.FHN, (2.8e-4, 0.05, 10.0, 0.95)),
    (O.GM, (2.5e-4, 0.01, 1.0, 0.47)),
])
def test_step_solves_the_implicit_equation_of_the_explicit_laplacian(model, p):
    """A step satisfies w1 - dt D Lap(w1) = w0 + dt R(w0), with the left side
    formed by the C oracle's explicit Euler step of pure diffusion taken with
    step -dt (whose Laplacian is pinned separately) and the right side by its
    explicit step with the diffusion switched off."""
    G, dt = 9, 0.02
    w0 = O.init_fields(model, G, 2, p, -0.05, 0.05, 17).astype(np.float64)
    if model == O.GM:
        w0 = O.init_fields(model, G, 2, p, 0.0, 0.01, 17).astype(np.float64)
    w1 = I.imex_run(model, p, dt, 1, w0)
    lhs = O.step(O.DIFF, (p[0], p[1], 0, 0), -dt, 1, w1)
    rhs = O.step(model, (0.0, 0.0) + tuple(p[2:]), dt, 1, w0)
    np.testing.assert_allclose(lhs, rhs, rtol=0, atol=1e-12 * abs(rhs).max())


def test_first_order_agreement_with_explicit_euler():
    """One IMEX step and one explicit Euler step differ by
    dt^2 D L (D L w + R): halving dt divides the gap by 4."""
    G = 8
    p = (0.002, 0.01, 10.0, 0.95)
    w0 = O.init_fields(O.FHN, G, 1, p, -0.05, 0.05, 5).astype(np.float64)
    gaps = []
    for dt in (1e-3, 5e-4, 2.5e-4):
        a = I.imex_run(O.FHN, p, dt, 1, w0)
        b = O.step(O.FHN, p, dt, 1, w0)
        gaps.append(abs(a - b).max())
    for g0, g1 in zip(gaps, gaps[1:]):
        assert 3.6 < g0 / g1 < 4.4, gaps


@pytest.mark.parametrize("G", [5, 9])
def test_sparse_and_dense_operators_are_the_same_matrix(G):
    """The sparse assembly holds exactly the dense matrix's entries, each row
    sums to zero (Neumann: constants are in the kernel) and the matrix is
    symmetric."""
    dense = I.laplacian_matrix(G)
    sparse = I.laplacian_sparse(G).toarray()
    np.testing.assert_array_equal(sparse, dense)
    np.testing.assert_array_equal(dense.sum(axis=1), np.zeros(G * G))
    np.testing.assert_array_equal(dense, dense.T)
    # interior row: the 5-point stencil scaled by (G-1)^2
    k = 2 * G + 2
    g2 = (G - 1) ** 2
    assert dense[k, k] == -4 * g2
    assert sorted(dense[k][dense[k] > 0].tolist()) == [g2] * 4


def test_sparse_and_dense_solves_agree():
    """The two factorisations of the same step give the same fields to FP64
    rounding."""
    G = 12
    p = (2.8e-4, 0.05, 10.0, 0.95)
    w0 = O.init_fields(O.FHN, G, 2, p, -0.05, 0.05, 41).astype(np.float64)
    a = I.imex_run(O.FHN, p, 0.02, 5, w0, sparse=False)
    b = I.imex_run(O.FHN, p, 0.02, 5, w0, sparse=True)
    np.testing.assert_allclose(a, b, rtol=0, atol=1e-13)
