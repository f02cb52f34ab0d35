"""ORACLE — test infrastructure only.

Semi-implicit (IMEX) Euler for the 2-D reaction-diffusion systems of
Sec. 4.1, in plain FP64: the diffusion term is taken implicitly and the
pointwise reaction explicitly, so a step is the linear solve

    (I - dt D_s L_h) w_s^{n+1} = w_s^n + dt R_s(u^n, v^n)     (s = u, v)

with L_h the 5-point Laplacian with mirrored Neumann ghosts of App. B.1.1
(ghost = adjacent edge node, scaled by (G-1)^2).  Sec. 5.1 and App. B.2
contrast explicit stepping with implicit stepping that needs linear solves;
this is the cheapest member of the implicit family, the diffusion solve
alone.

Written as the definition: L_h is assembled node by node from the stencil,
the matrix of each species is factored once with an LU (a library
primitive: dense up to 4096 nodes, sparse beyond, where the dense matrix of
a 128 x 128 grid would take 2 GB) and every step is one forward/back
substitution.  The reaction
R is the C oracle's right-hand side with the diffusion coefficients set to
zero (then F = 0 * Lap + R = R exactly).  No cosine transform appears here;
the GPU path's transform is checked against this solve.

Only ``tests/``, the smoke check and the benchmark's CPU legs may import it.
"""
import numpy as np
import scipy.linalg as sla
import scipy.sparse as sps
import scipy.sparse.linalg as spla

from . import rhs as _rhs


def laplacian_entries(G):
    """The entries of L_h over nodes k = y*G + x as (row, column, value)
    lists: each node takes +1 per neighbour and -4 for itself; a missing
    neighbour is the node's own mirrored ghost, so it adds +1 back on the
    diagonal.  Values are scaled by (G-1)^2; repeated (row, column) pairs
    add up."""
    rows, cols, vals = [], [], []
    g2 = float(G - 1) * float(G - 1)
    for y in range(G):
        for x in range(G):
            k = y * G + x
            rows.append(k)
            cols.append(k)
            vals.append(-4.0 * g2)
            for (yy, xx) in ((y, x + 1), (y, x - 1), (y + 1, x), (y - 1, x)):
                rows.append(k)
                if 0 <= yy < G and 0 <= xx < G:
                    cols.append(yy * G + xx)
                else:
                    cols.append(k)
                vals.append(g2)
    return rows, cols, vals


def laplacian_matrix(G):
    """L_h as a dense (G*G) x (G*G) FP64 matrix."""
    n = G * G
    L = np.zeros((n, n), np.float64)
    for r, c, v in zip(*laplacian_entries(G)):
        L[r, c] += v
    return L


def laplacian_sparse(G):
    """L_h as a sparse (CSC) FP64 matrix, the same entries."""
    n = G * G
    r, c, v = laplacian_entries(G)
    return sps.coo_matrix((v, (r, c)), shape=(n, n)).tocsc()


DENSE_MAX_NODES = 4096


class _SparseFactor:
    """Sparse LU of one species' matrix, solved like a dense factor."""

    def __init__(self, A):
        self.lu = spla.splu(A.tocsc())

    def solve(self, b):
        return self.lu.solve(b)


def imex_matrices(G, D, dt, sparse=None):
    """LU factors of I - dt*D*L_h for the diffusion coefficients D[0], D[1]
    (sparse when the grid has more than DENSE_MAX_NODES nodes, or when
    asked)."""
    if sparse is None:
        sparse = G * G > DENSE_MAX_NODES
    if sparse:
        L = laplacian_sparse(G)
        eye = sps.identity(G * G, format="csc")
        return [_SparseFactor(eye - (dt * d) * L) for d in (D[0], D[1])]
    L = laplacian_matrix(G)
    eye = np.eye(G * G)
    return [sla.lu_factor(eye - (dt * d) * L) for d in (D[0], D[1])]


def _solve(factor, b):
    if isinstance(factor, _SparseFactor):
        return factor.solve(b)
    return sla.lu_solve(factor, b)


def reaction_step(model, p, dt, w):
    """w + dt*R(w) for one realisation w[2, G, G] (FP64): R from the C
    oracle's right-hand side with Du = Dv = 0."""
    p0 = np.zeros(6, np.float64)
    p0[:len(p)] = p
    p0[0] = 0.0
    p0[1] = 0.0
    R = _rhs(model, p0, w)
    return w + dt * R


def imex_run(model, p, dt, n_steps, w0, factors=None, sparse=None):
    """n_steps IMEX Euler steps of every realisation w0[n_real, 2, G, G];
    returns the FP64 state."""
    w = np.array(w0, dtype=np.float64, copy=True)
    G = w.shape[-1]
    if factors is None:
        factors = imex_matrices(G, (p[0], p[1]), dt, sparse)
    n = w.shape[0]
    for _ in range(int(n_steps)):
        b = np.stack([reaction_step(model, p, dt, w[r]) for r in range(n)])
        for s in range(2):
            # all realisations as the columns of one right-hand side
            x = _solve(factors[s], b[:, s].reshape(n, G * G).T)
            w[:, s] = x.T.reshape(n, G, G)
    return w
