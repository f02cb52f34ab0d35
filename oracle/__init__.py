"""ORACLE — test infrastructure only.

Plain FP64 CPU reference of the CIL hot path (arXiv 2203.14742), written
from the paper.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline / reference leg may import it; the product package
never does, and it shares no code with the CUDA path.

Thin ctypes wrappers over ``oracle/liboracle.so`` (plain C, built by
``oracle/build.py``).  Every function takes and returns numpy arrays.
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

FHN, GM, DIFF, BZ, RDODE = 0, 1, 2, 3, 4

_lib = None


def threads():
    """OpenMP threads the oracle's parallel loops use."""
    return int(lib().orc_threads())


def set_threads(n):
    """Use n OpenMP threads in the oracle's parallel loops."""
    lib().orc_set_threads(int(n))


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        dp, fp, i64p, i32p, u8p = (C.POINTER(C.c_double), C.POINTER(C.c_float),
                                   C.POINTER(C.c_int64), C.POINTER(C.c_int32),
                                   C.POINTER(C.c_uint8))
        L.orc_threads.restype = C.c_int
        L.orc_set_threads.argtypes = [C.c_int]
        L.orc_rdode_init.argtypes = [C.c_int, C.c_int, C.c_double, C.c_double, C.c_uint64, C.c_int, fp]
        L.orc_rdode_rhs.argtypes = [C.c_int, dp, dp, dp]
        L.orc_rdode_gershgorin.argtypes = [C.c_int, dp, dp]
        L.orc_rdode_gershgorin.restype = C.c_double
        L.orc_radii_linear.argtypes = [dp, C.c_int64, C.c_int, dp, dp]
        L.orc_radii_linear.restype = C.c_double
        L.orc_fitted_b.argtypes = [C.c_double, C.c_int]
        L.orc_fitted_b.restype = C.c_double
        L.orc_radii_fitted.argtypes = [dp, C.c_int64, C.c_int, dp, dp]
        L.orc_radii_fitted.restype = C.c_double
        L.orc_rkc_coef.argtypes = [C.c_int, dp, dp, dp, dp, dp]
        L.orc_rkc_beta.argtypes = [C.c_int]
        L.orc_rkc_beta.restype = C.c_double
        L.orc_gershgorin.argtypes = [C.c_int, C.c_int, dp, dp]
        L.orc_gershgorin.restype = C.c_double
        L.orc_rkc_fixed.argtypes = [C.c_int, C.c_int, C.c_int, dp, C.c_double, C.c_int, C.c_int64, dp]
        L.orc_rkc_adaptive.argtypes = [C.c_int, C.c_int, C.c_int, dp, C.c_double, C.c_double,
                                       C.c_double, C.c_double, C.c_int, C.c_int64, dp, i64p]
        L.orc_rkc_adaptive.restype = C.c_int
        L.orc_minmax.argtypes = [fp, C.c_int64, C.c_int64, C.c_int, fp]
        L.orc_fd.argtypes = [fp, C.c_int64, C.c_int, C.c_int, C.c_int, fp, fp]
        L.orc_maxabs.argtypes = [fp, fp, C.c_int64]
        L.orc_maxabs.restype = C.c_double
        L.orc_d2_exact.argtypes = [fp, fp, C.c_int64]
        L.orc_d2_exact.restype = C.c_double
        L.orc_mcil_values.argtypes = [fp, fp, fp, C.c_int64, fp, fp, fp, C.c_int64, C.c_int, C.c_int, C.c_int,
                                      C.c_int, dp]
        L.orc_mcil_bins.argtypes = [dp, C.c_int64, C.c_int, C.c_int, C.c_double, C.c_int, dp, u8p, i64p]
        L.orc_mcil_squared.argtypes = [C.c_int]
        L.orc_mcil_squared.restype = C.c_int
        L.orc_sm64.argtypes = [C.c_uint64, C.c_uint64]
        L.orc_sm64.restype = C.c_uint64
        L.orc_equilibrium.argtypes = [C.c_int, dp, dp, dp]
        L.orc_init_fields.argtypes = [C.c_int, C.c_int, C.c_int, dp, C.c_double,
                                      C.c_double, C.c_uint64, fp]
        L.orc_rhs.argtypes = [C.c_int, C.c_int, dp, dp, dp]
        L.orc_step.argtypes = [C.c_int, C.c_int, C.c_int, dp, C.c_double, C.c_int64, dp]
        L.orc_residual.argtypes = [C.c_int, C.c_int, C.c_int, dp, dp, dp]
        L.orc_jvp.argtypes = [C.c_int, C.c_int, dp, dp, dp, dp, dp]
        L.orc_vjp.argtypes = [C.c_int, C.c_int, dp, dp, dp, dp, dp]
        L.orc_pair_d2.argtypes = [fp, C.c_int64, fp, C.c_int64, C.c_int64, dp]
        L.orc_radii.argtypes = [dp, C.c_int64, C.c_double, C.c_int, dp]
        L.orc_radii.restype = C.c_double
        L.orc_bins_counts.argtypes = [dp, C.c_int64, dp, C.c_int, u8p, i64p]
        L.orc_bootstrap_indices.argtypes = [C.c_uint64, C.c_int, C.c_int64, C.c_int64, i32p, i32p]
        L.orc_resample_counts.argtypes = [u8p, C.c_int64, C.c_int64, C.c_int, C.c_int,
                                          i32p, i32p, i64p]
        L.orc_stats.argtypes = [i64p, C.c_int, C.c_int, C.c_int64, dp, dp, dp, dp, dp, dp,
                                dp, u8p, C.POINTER(C.c_int)]
        L.orc_stats.restype = C.c_int
        L.orc_smooth_cil.argtypes = [dp, C.c_int64, dp, C.c_int64, C.c_int64, dp, C.c_int,
                                     C.c_double, dp, dp, dp, dp]
        L.orc_smooth_cil_grad.argtypes = [C.c_int, C.c_int, C.c_int, dp, C.c_double, C.c_int64,
                                          dp, C.c_int, i32p, C.c_int64, i32p, C.c_int64, dp,
                                          C.c_int, C.c_double, dp, dp, dp, dp]
        L.orc_smooth_cil_grad.restype = C.c_int
        L.orc_smooth_cil_loss.argtypes = [C.c_int, C.c_int, C.c_int, dp, C.c_double, C.c_int64,
                                          dp, C.c_int, i32p, C.c_int64, i32p, C.c_int64, dp,
                                          C.c_int, C.c_double, dp, dp]
        L.orc_smooth_cil_loss.restype = C.c_double
        _lib = L
    return _lib


def _p(a, ct):
    return a.ctypes.data_as(C.POINTER(ct))


def _d(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a


def _params(p):
    p = np.zeros(6, np.float64) if p is None else np.asarray(p, np.float64)
    out = np.zeros(6, np.float64)
    out[:len(p)] = p
    return out


def sm64(seed, i):
    """SplitMix64 output number i of stream `seed`."""
    return lib().orc_sm64(seed & 0xFFFFFFFFFFFFFFFF, i)


def equilibrium(model, p):
    p = _params(p)
    u0, v0 = C.c_double(), C.c_double()
    lib().orc_equilibrium(model, _p(p, C.c_double), C.byref(u0), C.byref(v0))
    return u0.value, v0.value


def init_fields(model, G, n_real, p, lo, hi, seed):
    """Initial state [n_real, 2, G, G] float32 (equilibrium + U(lo, hi))."""
    p = _params(p)
    out = np.empty((n_real, 2, G, G), np.float32)
    lib().orc_init_fields(model, G, n_real, _p(p, C.c_double), lo, hi,
                          C.c_uint64(seed & 0xFFFFFFFFFFFFFFFF), _p(out, C.c_float))
    return out


def rhs(model, p, w):
    """F(w) for one realisation w[2, G, G] (float64)."""
    p = _params(p)
    w = _d(w)
    G = w.shape[-1]
    F = np.empty_like(w)
    lib().orc_rhs(model, G, _p(p, C.c_double), _p(w, C.c_double), _p(F, C.c_double))
    return F


def step(model, p, dt, n_steps, w):
    """Forward Euler on w[n_real, 2, G, G] (float64 copy returned)."""
    p = _params(p)
    w = np.array(w, dtype=np.float64, order="C", copy=True)
    n_real, G = w.shape[0], w.shape[-1]
    lib().orc_step(model, G, n_real, _p(p, C.c_double), float(dt), int(n_steps),
                   _p(w, C.c_double))
    return w


def residual(model, p, w):
    """[n_real, 2]: max |F| and RMS of F for each realisation."""
    p = _params(p)
    w = _d(w)
    n_real, G = w.shape[0], w.shape[-1]
    out = np.empty((n_real, 2), np.float64)
    lib().orc_residual(model, G, n_real, _p(p, C.c_double), _p(w, C.c_double),
                       _p(out, C.c_double))
    return out


def jvp(model, p, w, dw, dtheta):
    p = _params(p)
    w, dw = _d(w), _d(dw)
    dtheta = _d(dtheta)
    out = np.empty_like(w)
    lib().orc_jvp(model, w.shape[-1], _p(p, C.c_double), _p(w, C.c_double),
                  _p(dw, C.c_double), _p(dtheta, C.c_double), _p(out, C.c_double))
    return out


def vjp(model, p, w, lam):
    p = _params(p)
    w, lam = _d(w), _d(lam)
    ow = np.empty_like(w)
    ot = np.empty(4, np.float64)
    lib().orc_vjp(model, w.shape[-1], _p(p, C.c_double), _p(w, C.c_double),
                  _p(lam, C.c_double), _p(ow, C.c_double), _p(ot, C.c_double))
    return ow, ot


def patterns(fields, species_mask):
    """Pattern vectors from fields[n, 2, G, G]: selected species, flattened."""
    sel = [s for s in (0, 1) if species_mask & (1 << s)]
    f = np.asarray(fields)
    return np.ascontiguousarray(f[:, sel].reshape(f.shape[0], -1))


def pair_d2(X1, X2):
    """Canonical squared distances [n1, n2] of float32 patterns."""
    X1 = np.ascontiguousarray(X1, np.float32)
    X2 = np.ascontiguousarray(X2, np.float32)
    n1, d = X1.shape
    n2 = X2.shape[0]
    out = np.empty((n1, n2), np.float64)
    lib().orc_pair_d2(_p(X1, C.c_float), n1, _p(X2, C.c_float), n2, d, _p(out, C.c_double))
    return out


def radii(d2, b, M):
    """(R0, radii[M]) with R0 = sqrt(max d2), R_k = R_{k-1}/b."""
    d2 = _d(d2)
    out = np.empty(M, np.float64)
    R0 = lib().orc_radii(_p(d2, C.c_double), d2.size, float(b), M, _p(out, C.c_double))
    return R0, out


def bins_counts(d2, radii_):
    d2 = _d(d2)
    r = _d(radii_)
    M = r.size
    bins = np.empty(d2.shape, np.uint8)
    counts = np.empty(M, np.int64)
    lib().orc_bins_counts(_p(d2, C.c_double), d2.size, _p(r, C.c_double), M,
                          _p(bins, C.c_uint8), _p(counts, C.c_int64))
    return bins, counts


def radii_linear(d2, M):
    """(R0, radii[M], R_min): the linear law R_k = R0 - k (R0 - R_min) / M
    with R0 / R_min the largest / smallest distance."""
    d2 = _d(d2)
    out = np.empty(M, np.float64)
    rmin = C.c_double()
    R0 = lib().orc_radii_linear(_p(d2, C.c_double), d2.size, M, _p(out, C.c_double), C.byref(rmin))
    return R0, out, rmin.value


def fitted_b(c, M):
    """The fitted power-law decay: smallest double b with fl(b^M) >= c (see
    cil.c)."""
    return float(lib().orc_fitted_b(float(c), int(M)))


def radii_fitted(d2, M):
    """(R0, radii[M], b): the power law R_k = R0 b^-k with b fitted so that
    R_M = R_min, the smallest distance."""
    d2 = _d(d2)
    out = np.empty(M, np.float64)
    b = C.c_double()
    R0 = lib().orc_radii_fitted(_p(d2, C.c_double), d2.size, M, _p(out, C.c_double), C.byref(b))
    return R0, out, b.value


def cil(X1, X2, b=None, M=None, radii_=None, law="power"):
    """Full CIL of two FP32 pattern sets (law "power": R_k = R0 b^-k;
    "linear": R_k = R0 - k (R0 - R_min) / M; "fitted": the power law with b
    fitted so that R_M = R_min).  Returns dict with d2, R0, radii, bins,
    counts."""
    d2 = pair_d2(X1, X2)
    if radii_ is None and law == "linear":
        R0, r, _ = radii_linear(d2, M)
    elif radii_ is None and law == "fitted":
        R0, r, _ = radii_fitted(d2, M)
    elif radii_ is None:
        R0, r = radii(d2, b, M)
    else:
        r = _d(radii_)
        R0 = float("nan")
    bins, counts = bins_counts(d2, r)
    return {"d2": d2, "R0": R0, "radii": r, "bins": bins, "counts": counts}


def bootstrap_indices(seed, T, n1, n2):
    I = np.empty((T, n1), np.int32)
    J = np.empty((T, n2), np.int32)
    lib().orc_bootstrap_indices(C.c_uint64(seed & 0xFFFFFFFFFFFFFFFF), T, n1, n2,
                                _p(I, C.c_int32), _p(J, C.c_int32))
    return I, J


def resample_counts(bins, M, I, J):
    bins = np.ascontiguousarray(bins, np.uint8)
    I = np.ascontiguousarray(I, np.int32)
    J = np.ascontiguousarray(J, np.int32)
    n1, n2 = bins.shape
    T = I.shape[0]
    Y = np.empty((T, M), np.int64)
    lib().orc_resample_counts(_p(bins, C.c_uint8), n1, n2, M, T, _p(I, C.c_int32),
                              _p(J, C.c_int32), _p(Y, C.c_int64))
    return Y


def stats(Y, n_pairs, y_obs=None):
    Y = np.ascontiguousarray(Y, np.int64)
    T, M = Y.shape
    mu = np.empty(M)
    cov = np.empty((M, M))
    chol = np.empty((M, M))
    logdet, f, ll = C.c_double(), C.c_double(), C.c_double()
    active = np.empty(M, np.uint8)
    ma = C.c_int()
    yo = None if y_obs is None else _d(y_obs)
    st = lib().orc_stats(_p(Y, C.c_int64), T, M, int(n_pairs),
                         None if yo is None else _p(yo, C.c_double),
                         _p(mu, C.c_double), _p(cov, C.c_double), _p(chol, C.c_double),
                         C.byref(logdet), C.byref(f), C.byref(ll), _p(active, C.c_uint8),
                         C.byref(ma))
    return {"status": st, "mu": mu, "cov": cov, "chol": chol, "logdet": logdet.value,
            "f": f.value, "loglik": ll.value, "active": active, "m_active": ma.value}


def synlik(bins, M, T, seed, y_obs=None):
    """Bootstrap counts + statistics (Alg. 5 steps 2-3)."""
    n1, n2 = bins.shape
    I, J = bootstrap_indices(seed, T, n1, n2)
    Y = resample_counts(bins, M, I, J)
    out = stats(Y, n1 * n2, y_obs)
    out["Y"] = Y
    return out


def smooth_cil(X1, X2, radii_, tau_frac, cot, grad=True):
    X1, X2 = _d(X1), _d(X2)
    n1, d = X1.shape
    n2 = X2.shape[0]
    r = _d(radii_)
    c = _d(cot)
    M = r.size
    Cv = np.empty(M)
    g1 = np.empty_like(X1) if grad else None
    g2 = np.empty_like(X2) if grad else None
    lib().orc_smooth_cil(_p(X1, C.c_double), n1, _p(X2, C.c_double), n2, d, _p(r, C.c_double),
                         M, float(tau_frac), _p(c, C.c_double), _p(Cv, C.c_double),
                         None if g1 is None else _p(g1, C.c_double),
                         None if g2 is None else _p(g2, C.c_double))
    return Cv, g1, g2


def smooth_cil_grad(model, p, dt, n_steps, w0, species_mask, set1, set2, radii_,
                    tau_frac, cot, with_abs=False):
    """(C[M], grad[4]) of loss = cot . C_tau by the FP64 discrete adjoint;
    with_abs: also A[4], the sum over realisations, steps and cells of the
    magnitudes of the terms whose sum is grad (A_i >= |grad_i|; a large
    A_i / |grad_i| means cancellation, so relative errors of the terms
    reach grad_i amplified by that ratio)."""
    p = _params(p)
    w0 = _d(w0)
    n_real, G = w0.shape[0], w0.shape[-1]
    s1 = np.ascontiguousarray(set1, np.int32)
    s2 = np.ascontiguousarray(set2, np.int32)
    r = _d(radii_)
    c = _d(cot)
    M = r.size
    Cv = np.empty(M)
    g = np.empty(4)
    A = np.empty(4)
    rc = lib().orc_smooth_cil_grad(model, G, n_real, _p(p, C.c_double), float(dt), int(n_steps),
                                   _p(w0, C.c_double), int(species_mask), _p(s1, C.c_int32),
                                   s1.size, _p(s2, C.c_int32), s2.size, _p(r, C.c_double), M,
                                   float(tau_frac), _p(c, C.c_double), _p(Cv, C.c_double),
                                   _p(g, C.c_double), _p(A, C.c_double))
    if rc:
        raise MemoryError("oracle adjoint: allocation failed")
    return (Cv, g, A) if with_abs else (Cv, g)


def smooth_cil_loss(model, p, dt, n_steps, w0, species_mask, set1, set2, radii_,
                    tau_frac, cot):
    p = _params(p)
    w0 = _d(w0)
    n_real, G = w0.shape[0], w0.shape[-1]
    s1 = np.ascontiguousarray(set1, np.int32)
    s2 = np.ascontiguousarray(set2, np.int32)
    r = _d(radii_)
    c = _d(cot)
    M = r.size
    Cv = np.empty(M)
    L = lib().orc_smooth_cil_loss(model, G, n_real, _p(p, C.c_double), float(dt), int(n_steps),
                                  _p(w0, C.c_double), int(species_mask), _p(s1, C.c_int32),
                                  s1.size, _p(s2, C.c_int32), s2.size, _p(r, C.c_double), M,
                                  float(tau_frac), _p(c, C.c_double), _p(Cv, C.c_double))
    return L, Cv


# ---------------------------------------------------------------------------
# multi-feature correlation integral (Sec. 3.1, Alg. 2; min-max scaling,
# Sec. 4) -- see mcil.c for the definitions and readings
# ---------------------------------------------------------------------------
FEATURES = ("L2", "Linf", "W12", "W12p", "W1inf", "W1infp")


def _f32(a):
    return np.ascontiguousarray(a, np.float32)


def minmax(X, G, nsp, Gy=None):
    """Min-max scaled copy of patterns X [n, nsp*Gy*G] (per species; Gy = G
    by default, 1 for 1-D patterns)."""
    Gy = G if Gy is None else Gy
    X = _f32(X)
    out = np.empty_like(X)
    lib().orc_minmax(_p(X, C.c_float), X.shape[0], Gy * G, nsp, _p(out, C.c_float))
    return out


def fd(X, G, nsp, Gy=None):
    """Forward-difference patterns (Ax [n, nsp*Gy*(G-1)], Ay [n,
    nsp*(Gy-1)*G]) float32 of Gy x G fields (Gy = G by default)."""
    Gy = G if Gy is None else Gy
    X = _f32(X)
    n = X.shape[0]
    Ax = np.empty((n, nsp * Gy * (G - 1)), np.float32)
    Ay = np.empty((n, max(nsp * (Gy - 1) * G, 1)), np.float32)
    lib().orc_fd(_p(X, C.c_float), n, Gy, G, nsp, _p(Ax, C.c_float), _p(Ay, C.c_float))
    return Ax, Ay[:, :nsp * (Gy - 1) * G]


def maxabs(x, y):
    x, y = _f32(x), _f32(y)
    return lib().orc_maxabs(_p(x, C.c_float), _p(y, C.c_float), x.size)


def d2_exact(x, y):
    x, y = _f32(x), _f32(y)
    return lib().orc_d2_exact(_p(x, C.c_float), _p(y, C.c_float), x.size)


def mcil_values(X1, X2, G, nsp, mask=63, Gy=None):
    """Feature values V[6, n1, n2] of every cross-set pair (NaN where the
    feature is not in mask): squared for L2 and W12, plain otherwise.
    Fields Gy x G (Gy = G by default, 1 for 1-D patterns)."""
    Gy = G if Gy is None else Gy
    X1, X2 = _f32(X1), _f32(X2)
    Ax1, Ay1 = fd(X1, G, nsp, Gy)
    Ax2, Ay2 = fd(X2, G, nsp, Gy)
    Ay1 = Ay1 if Ay1.size else np.zeros((X1.shape[0], 1), np.float32)
    Ay2 = Ay2 if Ay2.size else np.zeros((X2.shape[0], 1), np.float32)
    n1, n2 = X1.shape[0], X2.shape[0]
    V = np.full((6, n1, n2), np.nan)
    lib().orc_mcil_values(_p(X1, C.c_float), _p(Ax1, C.c_float), _p(Ay1, C.c_float), n1,
                          _p(X2, C.c_float), _p(Ax2, C.c_float), _p(Ay2, C.c_float), n2,
                          Gy, G, nsp, int(mask), _p(V, C.c_double))
    return V


def mcil(X1, X2, G, nsp, b, M, mask=63, scale=False, Gy=None, law="power"):
    """Multi-feature correlation integral (Alg. 2 step 2.2): per feature in
    mask (ascending), radii [K, M+1] (R0 first), bins [K, n1, n2], counts
    [K, M]; C = the concatenated vector (K*M) of eq. (CIL).  Fields Gy x G
    (Gy = G by default, 1 for 1-D patterns); law "power" (R0 b^-k),
    "linear" (R0 - k (R0 - R_min) / M, b unused) or "fitted" (R0 b^-k with b
    fitted so that R_M = R_min, b unused)."""
    if scale:
        X1, X2 = minmax(X1, G, nsp, Gy), minmax(X2, G, nsp, Gy)
    V = mcil_values(X1, X2, G, nsp, mask, Gy)
    feats = [f for f in range(6) if mask & (1 << f)]
    n1, n2 = V.shape[1], V.shape[2]
    K = len(feats)
    radii = np.empty((K, M + 1))
    bins = np.empty((K, n1, n2), np.uint8)
    counts = np.empty((K, M), np.int64)
    for a, f in enumerate(feats):
        v = np.ascontiguousarray(V[f])
        lib().orc_mcil_bins(_p(v, C.c_double), n1 * n2, lib().orc_mcil_squared(f),
                            {"power": 0, "linear": 1, "fitted": 2}[law],
                            float(b or 0.0), M,
                            _p(radii[a], C.c_double), _p(bins[a], C.c_uint8), _p(counts[a], C.c_int64))
    return {"features": feats, "values": V, "radii": radii, "bins": bins, "counts": counts,
            "C": counts.reshape(-1) / float(n1 * n2)}


def mcil_given(X1, X2, G, nsp, radii, mask=63, scale=False, Gy=None):
    """Multi-feature correlation integral with given radii [K, M+1] (R0
    first, unused): per feature K_ij = #{k : V_ij < T_k}, T_k = R_k * R_k
    for the squared features (L2, W12) and R_k for the others (eq. eCDF);
    the data vector of Alg. 6 step 5 (eq. CIL_synth)."""
    if scale:
        X1, X2 = minmax(X1, G, nsp, Gy), minmax(X2, G, nsp, Gy)
    V = mcil_values(X1, X2, G, nsp, mask, Gy)
    feats = [f for f in range(6) if mask & (1 << f)]
    radii = np.asarray(radii, np.float64)
    K, M = len(feats), radii.shape[1] - 1
    n1, n2 = V.shape[1], V.shape[2]
    bins = np.zeros((K, n1, n2), np.uint8)
    counts = np.zeros((K, M), np.int64)
    for a, f in enumerate(feats):
        for k in range(1, M + 1):
            T = radii[a, k] * radii[a, k] if lib().orc_mcil_squared(f) else radii[a, k]
            inside = V[f] < T
            bins[a] += inside.astype(np.uint8)
            counts[a, k - 1] = int(inside.sum())
    return {"features": feats, "values": V, "radii": radii, "bins": bins, "counts": counts,
            "C": counts.reshape(-1) / float(n1 * n2)}


def scil(S, data, n_set, G, nsp, M, T, seed, mask=63, scale=False, law="fitted", b=None, Gy=None):
    """Synthetic CIL with bootstrapping (Alg. 6) on given synthetic patterns
    S (N_syn rows, simulated at theta) and data patterns (rows), in the
    algorithm's order:
      step 2 (reading: one fixed partition): s^1 = S[:n_set], s^2 = the
        other N_syn - n_set rows; the radii and bins of the multi-feature
        correlation integral of s^1 against s^2 (Alg. 2 step 2.2);
      steps 2.1-3: T resamples (each part with replacement at its own
        size), the concatenated count vectors, their mean and covariance;
      steps 4-5: y~ = C(R, s_data, s^2) with those radii (eq. CIL_synth)
        and the cost f = (y~ - mu)^T Sigma^-1 (y~ - mu) (eq. cil:CF_synth)."""
    S = _f32(S)
    S1, S2 = S[:n_set], S[n_set:]
    syn = mcil(S1, S2, G, nsp, b, M, mask=mask, scale=scale, Gy=Gy, law=law)
    dat = mcil_given(data, S2, G, nsp, syn["radii"], mask=mask, scale=scale, Gy=Gy)
    st = synlik_multi(syn["bins"], M, T, seed, y_obs=dat["C"])
    return {"radii": syn["radii"], "bins": syn["bins"], "y_data": dat["C"], "data_bins": dat["bins"],
            "Y": st["Y"], "stats": st}


def synlik_multi(bins, M, T, seed, y_obs=None):
    """Bootstrap statistics of a concatenated feature vector (Alg. 5 with
    the multi-feature vector of Alg. 2): every resample draws one pair of
    index sets and counts it under every feature; Y[t] = (Y_feature0[t],
    Y_feature1[t], ...)."""
    bins = np.asarray(bins, np.uint8)
    K, n1, n2 = bins.shape
    I, J = bootstrap_indices(seed, T, n1, n2)
    Y = np.concatenate([resample_counts(bins[a], M, I, J) for a in range(K)], axis=1)
    out = stats(Y, n1 * n2, y_obs)
    out["Y"] = Y
    return out


# ---------------------------------------------------------------------------
# Stabilised explicit second-order Runge-Kutta (App. B.2; Chebyshev
# coefficients, see rkc.c for the readings).

def rkc_coef(s):
    """Coefficients of the s-stage method: dict of arrays mu, nu, mt, gt
    (index = stage j) and scalars w0, w1, b_s, a_s, beta."""
    mu, nu, mt, gt = (np.zeros(s + 1) for _ in range(4))
    ex = np.zeros(5)
    lib().orc_rkc_coef(int(s), _p(mu, C.c_double), _p(nu, C.c_double), _p(mt, C.c_double),
                       _p(gt, C.c_double), _p(ex, C.c_double))
    return dict(mu=mu, nu=nu, mt=mt, gt=gt, w0=ex[0], w1=ex[1], b_s=ex[2], a_s=ex[3], beta=ex[4])


def rkc_beta(s):
    """Length of the real stability interval of the s-stage method."""
    return float(lib().orc_rkc_beta(int(s)))


def gershgorin(model, p, w):
    """Gershgorin bound of the spectral radius of dF/dw at w[2, G, G]
    (w[2, N] for RDODE)."""
    p = _params(p)
    w = _d(w)
    return float(lib().orc_gershgorin(model, w.shape[-1], _p(p, C.c_double), _p(w, C.c_double)))


# ---------------------------------------------------------------------------
# Reaction-diffusion-ODE model (Sec. 4.3, eq. rdode), 1-D, [2][N] per
# realisation, p = (unused, D, m1, m2, m3, k).

def rdode_init(N, n_real, lo, hi, seed, n_smooth):
    """[n_real, 2, N] float32: u = smoothed U(lo, hi) noise, w = 0."""
    out = np.empty((n_real, 2, N), np.float32)
    lib().orc_rdode_init(int(N), int(n_real), float(lo), float(hi),
                         C.c_uint64(seed & 0xFFFFFFFFFFFFFFFF), int(n_smooth), _p(out, C.c_float))
    return out


def rdode_rhs(p, w):
    """F(w) of one realisation w[2, N] (float64)."""
    p = _params(p)
    w = _d(w)
    F = np.empty_like(w)
    lib().orc_rdode_rhs(w.shape[-1], _p(p, C.c_double), _p(w, C.c_double), _p(F, C.c_double))
    return F


def rkc_fixed(model, p, h, s, n_steps, w):
    """n_steps steps of size h with s stages on w[n_real, 2, G, G] (float64 copy)."""
    p = _params(p)
    w = np.array(w, dtype=np.float64, order="C", copy=True)
    n_real, G = w.shape[0], w.shape[-1]
    lib().orc_rkc_fixed(model, G, n_real, _p(p, C.c_double), float(h), int(s), int(n_steps),
                        _p(w, C.c_double))
    return w


def rkc_adaptive(model, p, t_end, h0, rtol, atol, w, s_max=256, max_attempts=100000):
    """Adaptive integration of w[n_real, 2, G, G] from 0 to t_end.
    Returns (w float64, stats int64 [n_real, 4] = accepted, rejected, RHS
    evaluations, largest s; number of failed realisations)."""
    p = _params(p)
    w = np.array(w, dtype=np.float64, order="C", copy=True)
    n_real, G = w.shape[0], w.shape[-1]
    stats = np.zeros((n_real, 4), np.int64)
    failed = lib().orc_rkc_adaptive(model, G, n_real, _p(p, C.c_double), float(t_end), float(h0),
                                    float(rtol), float(atol), int(s_max), int(max_attempts),
                                    _p(w, C.c_double), _p(stats, C.c_int64))
    return w, stats, int(failed)
