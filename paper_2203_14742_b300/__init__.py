"""B300-native hot path of the Correlation Integral Likelihood (arXiv 2203.14742).

Thin Python binding over the C ABI in ``include/rdcil.h`` (librdcil.so, built
in-tree by ``paper_2203_14742_b300/build.py``).  This module only marshals
arguments: every step of the path runs in the library's CUDA kernels.  It
takes torch CUDA tensors for device memory and the current torch stream.
There is no CPU fallback: importing fails loudly when the library is missing.

    sim  = Simulation(groups)                  # rd_init: fields + initial noise
    res  = sim.integrate()                     # rd_integrate_batch (+ FP64 residual)
    out  = cil(X1, X2, b=1.3, M=16)            # cil_features: radii, bins, counts
    st   = synlik(out["bins"], M=16, T=200, seed=...)   # synlik_stats
    C, g = sim.adjoint(...)                    # rd_adjoint (smoothed-CIL gradient)
"""
import ctypes as C
import math
import os

import torch

__all__ = ["FHN", "GM", "DIFF", "BZ", "RDODE", "Group", "Simulation", "cil", "cil_exact", "exact_d2", "synlik",
           "mcil", "mcil_given", "Scil",
           "SmoothCIL", "lib", "status_str"]

FHN, GM, DIFF, BZ, RDODE = 0, 1, 2, 3, 4
GROUP_ADJOINT = 1
GROUP_STREAM = 2
_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "librdcil.so")


class RdGroup(C.Structure):
    _fields_ = [("model", C.c_int32), ("G", C.c_int32), ("n_real", C.c_int32), ("flags", C.c_int32),
                ("n_steps", C.c_int64), ("field_offset", C.c_int64), ("dt", C.c_double),
                ("params", C.c_double * 6), ("noise_lo", C.c_double), ("noise_hi", C.c_double),
                ("seed", C.c_uint64)]


class RdRkcOpts(C.Structure):
    _fields_ = [("t_end", C.c_double), ("h0", C.c_double), ("rtol", C.c_double), ("atol", C.c_double),
                ("s_max", C.c_int32), ("s_fixed", C.c_int32), ("n_fixed", C.c_int64),
                ("max_attempts", C.c_int64)]


class ScilSpec(C.Structure):
    _fields_ = [("group", C.c_int32), ("integrator", C.c_int32), ("rkc", RdRkcOpts), ("n_set", C.c_int64),
                ("n_species", C.c_int32), ("features", C.c_int32), ("scale", C.c_int32), ("law", C.c_int32),
                ("b", C.c_double), ("M", C.c_int32), ("T", C.c_int32), ("seed", C.c_uint64),
                ("reinit", C.c_int32), ("pad", C.c_int32)]


RKC_S_MAX = 256

_vp, _i64, _i32, _dbl, _u64, _sz = C.c_void_p, C.c_int64, C.c_int32, C.c_double, C.c_uint64, C.c_size_t

_SIGS = {
    "rd_init": (_i32, [C.POINTER(RdGroup), _i32, _vp, _vp, C.POINTER(_vp)]),
    "rd_reinit": (_i32, [_vp, _vp, _vp]),
    "rd_set_params": (_i32, [_vp, _i32, C.POINTER(_dbl), _vp]),
    "rd_set_seed": (_i32, [_vp, _i32, _u64]),
    "scil_workspace_size": (_i32, [_vp, C.POINTER(ScilSpec), _i64, C.POINTER(_sz)]),
    "scil_evaluate": (_i32, [_vp, _vp, C.POINTER(ScilSpec), _vp, _i64, _i64, _vp, _vp, _vp, _vp, _vp, _vp, _vp,
                             _vp, _vp, _vp, _vp, _sz, _vp]),
    "mcil_features_given_rect": (_i32, [_vp, _i64, _i64, _vp, _i64, _i64, _i32, _i32, _i32, _i32, _i32, _i32,
                                        _vp, _vp, _vp, _vp, _vp, _vp, _vp, _sz, _vp]),
    "rd_tables_size": (_i32, [C.POINTER(RdGroup), _i32, C.POINTER(_sz)]),
    "rd_handle_table_bytes": (_sz, [_vp]),
    "rd_integrate_batch": (_i32, [_vp, _vp, _i64, _vp, _vp]),
    "rd_integrate_reference": (_i32, [_vp, _vp, _vp, _i64, _vp]),
    "rd_integrate_plain": (_i32, [_vp, _vp, _vp, _i64, _vp]),
    "rd_integrate_f64": (_i32, [_vp, _vp, _vp, _i64, _vp]),
    "rd_integrate_rkc": (_i32, [_vp, _vp, C.POINTER(RdRkcOpts), _vp, _vp, _vp]),
    "rd_integrate_imex": (_i32, [_vp, _vp, _vp, _vp]),
    "rd_imex_n_variants": (_i32, []),
    "rd_imex_set_variant": (_i32, [_i32, _i32]),
    "rd_imex_get_variant": (_i32, [_i32]),
    "rd_rkc_n_variants": (_i32, []),
    "rd_rkc_set_variant": (_i32, [_i32, _i32]),
    "rd_rkc_get_variant": (_i32, [_i32]),
    "rd_sync_status": (_i32, [_vp, _vp]),
    "rd_n_real_total": (_i64, [_vp]),
    "rd_free": (None, [_vp]),
    "rd_status_str": (C.c_char_p, [_i32]),
    "cil_workspace_size": (_i32, [_i64, _i64, _i64, C.POINTER(_sz)]),
    "cil_features": (_i32, [_vp, _i64, _i64, _vp, _i64, _i64, _i64, _vp, _dbl, _i32, _vp, _vp, _vp,
                            _vp, _vp, _vp, _sz, _vp]),
    "cil_features_linear": (_i32, [_vp, _i64, _i64, _vp, _i64, _i64, _i64, _i32, _vp, _vp, _vp, _vp, _vp,
                                   _vp, _sz, _vp]),
    "cil_features_fitted": (_i32, [_vp, _i64, _i64, _vp, _i64, _i64, _i64, _i32, _vp, _vp, _vp, _vp, _vp,
                                   _vp, _sz, _vp]),
    "cil_features_exact": (_i32, [_vp, _i64, _i64, _vp, _i64, _i64, _i64, _vp, _dbl, _i32, _vp, _vp,
                                  _vp, _vp, _vp, _sz, _vp]),
    "cil_exact_d2": (_i32, [_vp, _i64, _vp, _i64, _i64, _vp, _i64, _vp, _vp]),
    "cil_gram_only": (_i32, [_i64, _i64, _i64, _vp, _sz, C.POINTER(_dbl), _vp]),
    "cil_set_gram_products": (_i32, [_i32]),
    "cil_gram_products": (_i32, [_i64, _i64, _i64]),
    "cil_queue_lengths": (_i32, [_i64, _i64, _i64, _vp, _sz, _vp, _vp]),
    "cil_debug_approx": (_i32, [_vp, _i64, _i64, _vp, _i64, _i64, _i64, _vp, _vp, _vp, _sz, _vp]),
    "synlik_stats": (_i32, [_vp, _i64, _i64, _i32, _i32, _u64, _i32, _vp, _vp, _vp, _vp, _vp, _vp,
                            _vp, _vp, _vp]),
    "synlik_stats_multi": (_i32, [_vp, _i32, _i64, _i64, _i32, _i32, _u64, _i32, _vp, _vp, _vp, _vp, _vp,
                                  _vp, _vp, _vp, _vp]),
    "synlik_workspace_size": (_i32, [_i64, _i64, _i32, _i32, _i32, _i32, C.POINTER(_sz)]),
    "synlik_set_tc_min_pairs": (None, [_i64]),
    "synlik_set_tc_mult_limit": (None, [_i32]),
    "synlik_stats_ws": (_i32, [_vp, _i32, _i64, _i64, _i32, _i32, _u64, _i32, _vp, _vp, _vp, _vp, _vp, _vp,
                               _vp, _vp, _vp, _sz, _vp]),
    "mcil_workspace_size": (_i32, [_i64, _i64, _i32, _i32, _i32, _i32, _i32, C.POINTER(_sz)]),
    "mcil_features": (_i32, [_vp, _i64, _i64, _vp, _i64, _i64, _i32, _i32, _i32, _i32, _dbl, _i32, _vp, _vp,
                             _vp, _vp, _vp, _vp, _sz, _vp]),
    "mcil_workspace_size_rect": (_i32, [_i64, _i64, _i32, _i32, _i32, _i32, _i32, _i32, C.POINTER(_sz)]),
    "mcil_features_rect": (_i32, [_vp, _i64, _i64, _vp, _i64, _i64, _i32, _i32, _i32, _i32, _i32, _dbl, _i32,
                                  _vp, _vp, _vp, _vp, _vp, _vp, _sz, _vp]),
    "mcil_features_linear_rect": (_i32, [_vp, _i64, _i64, _vp, _i64, _i64, _i32, _i32, _i32, _i32, _i32, _i32,
                                         _vp, _vp, _vp, _vp, _vp, _vp, _sz, _vp]),
    "mcil_features_fitted_rect": (_i32, [_vp, _i64, _i64, _vp, _i64, _i64, _i32, _i32, _i32, _i32, _i32, _i32,
                                         _vp, _vp, _vp, _vp, _vp, _vp, _sz, _vp]),
    "rd_kernel_launches": (_u64, []),
    "rd_set_spin_limit": (None, [C.c_uint32]),
    "rd_n_variants": (_i32, []),
    "rd_set_schedule": (_i32, [_vp, _i32]),
    "rd_set_stream_depth": (_i32, [_vp, _i32]),
    "rd_get_stream_depth": (_i32, [_vp]),
    "rd_set_variant": (_i32, [_i32, _i32, _i32]),
    "rd_get_variant": (_i32, [_i32, _i32]),
    "rd_variant_shape": (_i32, [_i32, _i32, C.POINTER(_i32)]),
    "rd_autotune": (_i32, [_vp, _vp, _i64, _vp, C.POINTER(_i32)]),
    "rd_adjoint": (_i32, [_vp, _i32, _vp, _i32, C.POINTER(_i32), _i64, C.POINTER(_i32), _i64, _vp,
                          _i32, _dbl, _vp, _vp, _vp, _vp]),
}

_lib = None


def lib():
    """The loaded librdcil.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("librdcil.so is not built (run `python -m paper_2203_14742_b300.build`)")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def status_str(st):
    return lib().rd_status_str(int(st)).decode()


class RdError(RuntimeError):
    def __init__(self, fn, st):
        super().__init__("%s failed: %s (%d)" % (fn, status_str(st), st))
        self.status = st


def _check(fn, st):
    if st != 0:
        raise RdError(fn, st)


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    return C.c_void_p(t.data_ptr())


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


class Group:
    """One parameter group (a theta): n_real realisations of `model` on a
    G x G grid.  params: FHN (Du, Dv, eps, a); GM (Du, Dv, rho, mu); BZ (Du,
    Dv, A, B).  stream=True runs it on the streaming stepper even where the
    resident one fits."""

    def __init__(self, model, G, n_real, params, dt, n_steps, noise=(-0.05, 0.05), seed=0,
                 adjoint=False, stream=False):
        self.model, self.G, self.n_real = int(model), int(G), int(n_real)
        self.params = tuple(float(p) for p in params) + (0.0,) * (6 - len(params))
        self.dt, self.n_steps = float(dt), int(n_steps)
        self.noise = (float(noise[0]), float(noise[1]))
        self.seed = int(seed) & 0xFFFFFFFFFFFFFFFF
        self.adjoint = bool(adjoint)
        self.stream = bool(stream)

    @property
    def cells(self):
        """Nodes per species: G x G, or G for the 1-D RDODE model."""
        return self.G if self.model == RDODE else self.G * self.G

    @property
    def shape(self):
        return (self.n_real, 2, self.G) if self.model == RDODE else (self.n_real, 2, self.G, self.G)

    @property
    def floats(self):
        return self.n_real * 2 * self.cells

    @classmethod
    def from_dict(cls, d, adjoint=False, stream=False):
        return cls(d["model"], d["G"], d["n_real"], d["params"], d["dt"], d["n_steps"],
                   d["noise"], d["seed"], adjoint=adjoint, stream=stream)


class Simulation:
    """A batch of groups sharing one field tensor (rd_init / rd_integrate_batch)."""

    def __init__(self, groups, device=None, fields=None):
        self.groups = list(groups)
        self.device = torch.device(device or "cuda")
        offs, off = [], 0
        for g in self.groups:
            offs.append(off)
            off += g.floats
        self.offsets = offs
        self.total_floats = off
        if fields is None:
            fields = torch.empty(off, dtype=torch.float32, device=self.device)
        if fields.numel() < off or fields.dtype != torch.float32 or not fields.is_contiguous():
            raise ValueError("fields: contiguous float32 tensor of >= %d elements" % off)
        self.fields = fields
        arr = (RdGroup * len(self.groups))()
        for i, g in enumerate(self.groups):
            a = arr[i]
            a.model, a.G, a.n_real = g.model, g.G, g.n_real
            a.flags = (GROUP_ADJOINT if g.adjoint else 0) | (GROUP_STREAM if g.stream else 0)
            a.n_steps, a.field_offset, a.dt = g.n_steps, offs[i], g.dt
            for k in range(6):
                a.params[k] = g.params[k]
            a.noise_lo, a.noise_hi, a.seed = g.noise[0], g.noise[1], g.seed
        self._arr = arr
        h = C.c_void_p()
        with torch.cuda.device(self.device):
            _check("rd_init", lib().rd_init(arr, len(self.groups), _ptr(self.fields), _stream(),
                                            C.byref(h)))
        self.handle = h
        self.n_real_total = sum(g.n_real for g in self.groups)

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value and _lib is not None:
            _lib.rd_free(h)
            self.handle = None

    # -- views -------------------------------------------------------------
    def group_fields(self, i, fields=None):
        g = self.groups[i]
        f = self.fields if fields is None else fields
        o = self.offsets[i]
        return f[o:o + g.floats].view(*g.shape)

    # -- calls -------------------------------------------------------------
    def reinit(self):
        _check("rd_reinit", lib().rd_reinit(self.handle, _ptr(self.fields), _stream()))

    def integrate(self, steps=-1, residual=True):
        res = None
        if residual:
            res = torch.empty((self.n_real_total, 2), dtype=torch.float64, device=self.device)
        _check("rd_integrate_batch", lib().rd_integrate_batch(self.handle, _ptr(self.fields), int(steps),
                                                              _ptr(res), _stream()))
        return res

    def integrate_reference(self, steps=-1, tmp=None):
        if tmp is None:
            tmp = torch.empty(max(2 * g.G * g.G for g in self.groups), dtype=torch.float32,
                              device=self.device)
        _check("rd_integrate_reference", lib().rd_integrate_reference(
            self.handle, _ptr(self.fields), _ptr(tmp), int(steps), _stream()))

    def integrate_plain(self, steps=-1, tmp=None):
        """The plain step with every realisation of a group in one launch."""
        if tmp is None:
            tmp = torch.empty(max(2 * g.G * g.G * g.n_real for g in self.groups), dtype=torch.float32,
                              device=self.device)
        _check("rd_integrate_plain", lib().rd_integrate_plain(
            self.handle, _ptr(self.fields), _ptr(tmp), int(steps), _stream()))

    def integrate_f64(self, fields64, steps=-1):
        tmp = torch.empty_like(fields64)
        _check("rd_integrate_f64", lib().rd_integrate_f64(self.handle, _ptr(fields64), _ptr(tmp),
                                                          int(steps), _stream()))
        return fields64

    def integrate_rkc(self, h0, t_end=0.0, rtol=1e-5, atol=1e-5, s_max=RKC_S_MAX, max_attempts=100000,
                      s_fixed=0, n_fixed=0, stats=True, residual=False):
        """Stabilised second-order Runge-Kutta (App. B.2, Chebyshev
        coefficients) in place.  Adaptive by default: every realisation from
        0 to t_end (<= 0: each group's dt * n_steps) with its own step
        control; s_fixed >= 2: n_fixed steps of size h0 with s_fixed stages.
        Returns (stats int64 [n_real, 4] = accepted, rejected, RHS
        evaluations, largest s; residual or None)."""
        o = RdRkcOpts(float(t_end), float(h0), float(rtol), float(atol), int(s_max), int(s_fixed),
                      int(n_fixed), int(max_attempts))
        st = torch.empty((self.n_real_total, 4), dtype=torch.int64, device=self.device) if stats else None
        res = (torch.empty((self.n_real_total, 2), dtype=torch.float64, device=self.device)
               if residual else None)
        _check("rd_integrate_rkc", lib().rd_integrate_rkc(self.handle, _ptr(self.fields), C.byref(o),
                                                          _ptr(st), _ptr(res), _stream()))
        return st, res

    def integrate_imex(self, residual=False):
        """Semi-implicit Euler in place: each group's n_steps steps of its dt,
        diffusion implicit (solved in the cosine basis), reaction explicit.
        Returns the residual [n_real, 2] or None."""
        res = (torch.empty((self.n_real_total, 2), dtype=torch.float64, device=self.device)
               if residual else None)
        _check("rd_integrate_imex", lib().rd_integrate_imex(self.handle, _ptr(self.fields), _ptr(res),
                                                            _stream()))
        return res

    def set_stream_depth(self, depth):
        """Euler steps fused per launch of the streaming stepper (1, 2, 4, 8)."""
        _check("rd_set_stream_depth", lib().rd_set_stream_depth(self.handle, int(depth)))

    def set_schedule(self, mode):
        """0 automatic, 1 one launch per group, 2 one persistent launch."""
        _check("rd_set_schedule", lib().rd_set_schedule(self.handle, int(mode)))

    def autotune(self, steps=200):
        """Pick the fastest tile shape per (model, G); re-initialises the fields."""
        chosen = (C.c_int32 * 12)(*([-1] * 12))
        _check("rd_autotune", lib().rd_autotune(self.handle, _ptr(self.fields), int(steps), _stream(),
                                                chosen))
        return list(chosen)

    def sync_status(self):
        return lib().rd_sync_status(self.handle, _stream())

    def table_bytes(self):
        """Device bytes of the step tables the handle formed in rd_init."""
        return int(lib().rd_handle_table_bytes(self.handle))

    def set_params(self, group, params):
        """Replace group `group`'s parameter vector (rd_set_params) for every
        later call; params: up to 6 floats (the group's layout)."""
        vals = [float(x) for x in params] + [0.0] * (6 - len(params))
        arr = (C.c_double * 6)(*vals)
        _check("rd_set_params", lib().rd_set_params(self.handle, int(group), arr, _stream()))
        g = self.groups[group]
        g.params = tuple(vals)
        self._arr[group].params[:] = vals

    def adjoint(self, group, fields0, species_mask, set1, set2, radii, tau_frac, cotangent):
        """(C[M], grad[4]) float64 tensors: smoothed CIL and its gradient.
        cotangent=None: forward only (C, no reverse sweep; grad is None)."""
        s1 = (C.c_int32 * len(set1))(*[int(x) for x in set1])
        s2 = (C.c_int32 * len(set2))(*[int(x) for x in set2])
        radii = radii.to(device=self.device, dtype=torch.float64).contiguous()
        M = radii.numel()
        Cv = torch.empty(M, dtype=torch.float64, device=self.device)
        if cotangent is None:
            cot, g = None, None
        else:
            cot = cotangent.to(device=self.device, dtype=torch.float64).contiguous()
            g = torch.empty(4, dtype=torch.float64, device=self.device)
        _check("rd_adjoint", lib().rd_adjoint(self.handle, int(group), _ptr(fields0), int(species_mask),
                                              s1, len(set1), s2, len(set2), _ptr(radii), M,
                                              float(tau_frac), _ptr(cot), _ptr(Cv), _ptr(g), _stream()))
        return Cv, g


# ---------------------------------------------------------------------------
# correlation integral
# ---------------------------------------------------------------------------
_work_cache = {}


def rkc_set_variant(G, variant):
    """Tile shape of the adaptive RK2 kernel for grid side G (32 or 64)."""
    _check("rd_rkc_set_variant", lib().rd_rkc_set_variant(int(G), int(variant)))


def rkc_get_variant(G):
    return int(lib().rd_rkc_get_variant(int(G)))


def imex_set_variant(G, variant):
    """Product variant of the semi-implicit stepper for grid side G (32 or
    64): output tiles 0 = 4x4, 1 = 8x4, 2 = 4x8, 3 = 8x8; 4 = the even/odd
    split (half the FMAs; the default)."""
    _check("rd_imex_set_variant", lib().rd_imex_set_variant(int(G), int(variant)))


def imex_get_variant(G):
    return int(lib().rd_imex_get_variant(int(G)))


def variant_shape(G, variant):
    """(packed, TY, TX) of stepper tile variant `variant` at grid side G."""
    sh = (_i32 * 3)()
    _check("rd_variant_shape", lib().rd_variant_shape(int(G), int(variant), sh))
    return int(sh[0]), int(sh[1]), int(sh[2])


def _workspace(n1, n2, d, device):
    device = torch.device(device)
    if device.type == "cuda" and device.index is None:
        device = torch.device("cuda", torch.cuda.current_device())
    sz = C.c_size_t()
    _check("cil_workspace_size", lib().cil_workspace_size(n1, n2, d, C.byref(sz)))
    key = (device, )
    w = _work_cache.get(key)
    if w is None or w.numel() < sz.value:
        w = torch.empty(max(sz.value, 1 << 20), dtype=torch.uint8, device=device)
        _work_cache[key] = w
    return w, sz.value


def _as_rows(X):
    """(tensor, ld, n, d) for a 2-D float32 CUDA tensor with unit column stride."""
    if X.dtype != torch.float32 or X.dim() != 2 or X.stride(1) != 1:
        raise ValueError("patterns: 2-D float32 tensor with contiguous rows")
    return X, X.stride(0), X.shape[0], X.shape[1]


def _cil_call(fn, X1, X2, b, M, radii, work=None, out=None):
    X1, ld1, n1, d = _as_rows(X1)
    X2, ld2, n2, d2 = _as_rows(X2)
    if d != d2:
        raise ValueError("pattern length mismatch")
    dev = X1.device
    if radii is not None:
        radii = radii.to(device=dev, dtype=torch.float64).contiguous()
        M = radii.numel()
    if out is not None:
        radii_out, bins, counts, Cvec, nre = out["radii"], out["bins"], out["counts"], out["C"], out["n_rechecked"]
    else:
        radii_out = torch.empty(M + 1, dtype=torch.float64, device=dev)
        bins = torch.empty((n1, n2), dtype=torch.uint8, device=dev)
        counts = torch.empty(M, dtype=torch.int64, device=dev)
        Cvec = torch.empty(M, dtype=torch.float64, device=dev)
        nre = torch.zeros(1, dtype=torch.int64, device=dev)
    if work is None:
        w, wb = _workspace(n1, n2, d, dev)
    else:
        w, wb = work, work.numel()
    if fn in ("cil_features_linear", "cil_features_fitted"):
        args = [_ptr(X1), ld1, n1, _ptr(X2), ld2, n2, d, int(M)]
    else:
        args = [_ptr(X1), ld1, n1, _ptr(X2), ld2, n2, d, _ptr(radii), float(b or 0.0), int(M)]
    args += [_ptr(radii_out), _ptr(bins), _ptr(counts), _ptr(Cvec)]
    if fn in ("cil_features", "cil_features_linear", "cil_features_fitted"):
        args.append(_ptr(nre))
    args += [_ptr(w), wb, _stream()]
    _check(fn, getattr(lib(), fn)(*args))
    return {"R0": radii_out[0], "radii": radii_out[1:], "bins": bins, "counts": counts, "C": Cvec,
            "n_rechecked": nre}


def cil_approx(X1, X2):
    """(A, m): approximate squared distances and their error bounds (checking)."""
    X1, ld1, n1, d = _as_rows(X1)
    X2, ld2, n2, _ = _as_rows(X2)
    A = torch.empty((n1, n2), dtype=torch.float64, device=X1.device)
    m = torch.empty_like(A)
    w, wb = _workspace(n1, n2, d, X1.device)
    _check("cil_debug_approx", lib().cil_debug_approx(_ptr(X1), ld1, n1, _ptr(X2), ld2, n2, d, _ptr(A),
                                                      _ptr(m), _ptr(w), wb, _stream()))
    return A, m


def gram_only(n1, n2, d, device=None):
    """Re-run the tensor-core Gram stage on the cached workspace (benchmarking);
    returns the FLOPs of the launch."""
    w, wb = _workspace(n1, n2, d, torch.device(device or "cuda"))
    fl = C.c_double()
    _check("cil_gram_only", lib().cil_gram_only(n1, n2, d, _ptr(w), wb, C.byref(fl), _stream()))
    return fl.value


def set_gram_products(mode):
    """The tensor-core Gram's form for every later correlation integral,
    process-wide: 3 (hi.hi + hi.lo + lo.hi, the default; 0 restores it) or
    1 (hi.hi alone, a wider rigorous interval).  Results are identical; only
    the time changes."""
    _check("cil_set_gram_products", lib().cil_set_gram_products(int(mode)))


def cil_queue_lengths(n1, n2, d, device=None):
    """(tier-2 pairs, tier-3 pairs) of the last correlation integral of this
    size on the cached workspace (checking and benchmarking)."""
    dev = torch.device(device or "cuda")
    w, wb = _workspace(n1, n2, d, dev)
    out = torch.zeros(2, dtype=torch.int64, device=dev)
    _check("cil_queue_lengths", lib().cil_queue_lengths(int(n1), int(n2), int(d), _ptr(w), wb, _ptr(out),
                                                        _stream()))
    return tuple(int(v) for v in out.cpu())


def gram_products(n1, n2, d):
    """The product count (1 or 3) a correlation integral of this size uses."""
    return int(lib().cil_gram_products(int(n1), int(n2), int(d)))


def cil(X1, X2, b=1.3, M=16, radii=None, work=None, out=None):
    """Correlation integral of two pattern sets (rows of X1, X2).  `out`
    (optional) supplies the output tensors: radii [M+1], bins [n1, n2] uint8,
    counts [M] int64, C [M] float64, n_rechecked [1] int64."""
    return _cil_call("cil_features", X1, X2, b, M, radii, work, out)


def cil_linear(X1, X2, M=13, work=None, out=None):
    """Correlation integral with the linear radii law R_k = R0 - k (R0 - R_min)/M
    (Sec. 2.1; Table 1's law for the MC and RD-ODE models)."""
    return _cil_call("cil_features_linear", X1, X2, None, M, None, work, out)


def cil_fitted(X1, X2, M=16, work=None, out=None):
    """Correlation integral with the power law fitted to the distance range:
    R_k = R0 b^-k, b > 1 with R_M = R_min (Sec. 2.1; Table 1's law for the
    FHN, GM and BZ models)."""
    return _cil_call("cil_features_fitted", X1, X2, None, M, None, work, out)


def cil_exact(X1, X2, b=1.3, M=16, radii=None, work=None):
    """Same outputs, every pair evaluated exactly (checking)."""
    return _cil_call("cil_features_exact", X1, X2, b, M, radii, work)


def exact_d2(X1, X2, pairs):
    """d2 of the listed pairs (int64 [n, 2] of row indices into X1, X2): the
    exact real sum of squared differences rounded once (checking)."""
    X1, ld1, n1, d = _as_rows(X1)
    X2, ld2, n2, d2_ = _as_rows(X2)
    if d2_ != d:
        raise ValueError("pattern lengths differ")
    pairs = torch.as_tensor(pairs, dtype=torch.int64).to(X1.device).contiguous()
    if pairs.numel() and (int(pairs[:, 0].min()) < 0 or int(pairs[:, 0].max()) >= n1 or
                          int(pairs[:, 1].min()) < 0 or int(pairs[:, 1].max()) >= n2):
        raise IndexError("pair index outside the sets")
    out = torch.empty(pairs.shape[0], dtype=torch.float64, device=X1.device)
    _check("cil_exact_d2", lib().cil_exact_d2(_ptr(X1), ld1, _ptr(X2), ld2, d, _ptr(pairs), pairs.shape[0],
                                              _ptr(out), _stream()))
    return out


# ---------------------------------------------------------------------------
# synthetic likelihood
# ---------------------------------------------------------------------------
def synlik_outputs(P, M, T, device):
    dev = torch.device(device)
    return {"Y": torch.empty((P, T, M), dtype=torch.int64, device=dev),
            "mu": torch.empty((P, M), dtype=torch.float64, device=dev),
            "cov": torch.empty((P, M, M), dtype=torch.float64, device=dev),
            "chol": torch.empty((P, M, M), dtype=torch.float64, device=dev),
            "scalars": torch.empty((P, 4), dtype=torch.float64, device=dev),
            "active": torch.empty((P, M), dtype=torch.uint8, device=dev),
            "status": torch.empty(P, dtype=torch.int32, device=dev)}


def synlik_workspace(n1, n2, M, T, n_feat=1, n_problems=1, device="cuda"):
    """Workspace of synlik_stats_ws (tensor-core bootstrap counts)."""
    sz = _sz(0)
    _check("synlik_workspace_size", lib().synlik_workspace_size(int(n1), int(n2), int(M), int(T), int(n_feat),
                                                                int(n_problems), C.byref(sz)))
    return torch.empty(max(int(sz.value), 256), dtype=torch.uint8, device=device)


def synlik(bins, M, T, seed, y_obs=None, out=None, n_feat=1, work=None, simt=False):
    """Bootstrap statistics of bins [P, n1, n2] (or [n1, n2]) uint8; with
    n_feat > 1, bins [P, n_feat, n1, n2] (or [n_feat, n1, n2]) of a
    concatenated feature vector (n_feat * M components).  The counts run on
    the tensor cores (synlik_stats_ws, workspace `work` or a fresh one);
    simt=True takes the SIMT kernel (synlik_stats_multi) instead."""
    squeeze = bins.dim() == (2 if n_feat == 1 else 3)
    if squeeze:
        bins = bins.unsqueeze(0)
    if not bins.is_contiguous():
        raise ValueError("bins must be contiguous")
    P, n1, n2 = bins.shape[0], bins.shape[-2], bins.shape[-1]
    Mt = n_feat * M
    dev = bins.device
    o = out if out is not None else synlik_outputs(P, Mt, T, dev)
    Y, mu, cov, chol, sc, act, st = (o["Y"], o["mu"], o["cov"], o["chol"], o["scalars"], o["active"],
                                     o["status"])
    yo = None
    if y_obs is not None:
        yo = y_obs
        if yo.dtype != torch.float64 or yo.device != dev or not yo.is_contiguous():
            yo = yo.to(device=dev, dtype=torch.float64).contiguous()   # marshalling only
        if yo.numel() != P * Mt:
            raise ValueError("y_obs must hold P x n_feat*M values")
    if simt:
        _check("synlik_stats_multi", lib().synlik_stats_multi(_ptr(bins), int(n_feat), n1, n2, int(M), int(T),
                                                              int(seed) & 0xFFFFFFFFFFFFFFFF, P, _ptr(yo),
                                                              _ptr(Y), _ptr(mu), _ptr(cov), _ptr(chol), _ptr(sc),
                                                              _ptr(act), _ptr(st), _stream()))
    else:
        if work is None:
            work = synlik_workspace(n1, n2, M, T, n_feat, P, dev)
        _check("synlik_stats_ws", lib().synlik_stats_ws(_ptr(bins), int(n_feat), n1, n2, int(M), int(T),
                                                        int(seed) & 0xFFFFFFFFFFFFFFFF, P, _ptr(yo), _ptr(Y),
                                                        _ptr(mu), _ptr(cov), _ptr(chol), _ptr(sc), _ptr(act),
                                                        _ptr(st), _ptr(work), work.numel(), _stream()))
    out = {"Y": Y, "mu": mu, "cov": cov, "chol": chol, "scalars": sc, "logdet": sc[:, 0], "f": sc[:, 1],
           "loglik": sc[:, 2], "m_active": sc[:, 3], "active": act, "status": st}
    if squeeze:
        out = {k: v[0] for k, v in out.items()}
    return out


# ---------------------------------------------------------------------------
# multi-feature correlation integral
# ---------------------------------------------------------------------------
FEATURES = ("L2", "Linf", "W12", "W12p", "W1inf", "W1infp")


def mcil_workspace(n1, n2, G, n_species, features=63, scale=False, M=16, device=None, Gy=None):
    """A device workspace for mcil() with these sizes (reusable across calls)."""
    Gy = G if Gy is None else Gy
    sz = _sz()
    _check("mcil_workspace_size_rect", lib().mcil_workspace_size_rect(
        int(n1), int(n2), int(Gy), int(G), int(n_species), int(features), 1 if scale else 0, int(M), C.byref(sz)))
    return torch.empty(sz.value, dtype=torch.uint8, device=device)


def mcil(X1, X2, G, n_species, b=1.3, M=16, features=63, scale=False, work=None, Gy=None, law="power"):
    """Multi-feature correlation integral of two pattern sets (rows of n_species
    Gy x G fields, read in place; Gy = G by default, 1 for 1-D patterns).
    law "power" (R0 b^-k), "linear" (R0 - k (R0 - R_min) / M, b unused) or
    "fitted" (R0 b^-k with b fitted so that R_M = R_min, b unused).
    Returns radii [K, M+1], bins [K, n1, n2], counts [K, M], C [K*M] and
    n_exact for the K selected features."""
    if law not in ("power", "linear", "fitted"):
        raise ValueError("law must be 'power', 'linear' or 'fitted'")
    Gy = G if Gy is None else Gy
    X1, ld1, n1, d = _as_rows(X1)
    X2, ld2, n2, d2 = _as_rows(X2)
    if d != d2 or d != n_species * Gy * G:
        raise ValueError("pattern length must be n_species * Gy * G")
    dev = X1.device
    K = bin(int(features)).count("1")
    if work is None:
        work = mcil_workspace(n1, n2, G, n_species, features, scale, M, dev, Gy=Gy)
    radii = torch.empty((K, M + 1), dtype=torch.float64, device=dev)
    bins = torch.empty((K, n1, n2), dtype=torch.uint8, device=dev)
    counts = torch.empty((K, M), dtype=torch.int64, device=dev)
    Cv = torch.empty(K * M, dtype=torch.float64, device=dev)
    nex = torch.zeros(1, dtype=torch.int64, device=dev)
    if law in ("linear", "fitted"):
        fn = "mcil_features_%s_rect" % law
        _check(fn, getattr(lib(), fn)(
            _ptr(X1), ld1, n1, _ptr(X2), ld2, n2, int(Gy), int(G), int(n_species), int(features),
            1 if scale else 0, int(M), _ptr(radii), _ptr(bins), _ptr(counts), _ptr(Cv), _ptr(nex), _ptr(work),
            work.numel(), _stream()))
    else:
        _check("mcil_features_rect", lib().mcil_features_rect(
            _ptr(X1), ld1, n1, _ptr(X2), ld2, n2, int(Gy), int(G), int(n_species), int(features),
            1 if scale else 0, float(b), int(M), _ptr(radii), _ptr(bins), _ptr(counts), _ptr(Cv), _ptr(nex),
            _ptr(work), work.numel(), _stream()))
    return {"radii": radii, "bins": bins, "counts": counts, "C": Cv, "n_exact": nex}


def mcil_given(X1, X2, G, n_species, radii, features=63, scale=False, work=None, Gy=None):
    """Multi-feature correlation integral with given radii [K, M+1] (R0
    first, not used): the data vector of Alg. 6 step 5 (eq. CIL_synth).
    Returns bins [K, n1, n2], counts [K, M], C [K*M], n_exact."""
    Gy = G if Gy is None else Gy
    X1, ld1, n1, d = _as_rows(X1)
    X2, ld2, n2, d2 = _as_rows(X2)
    if d != d2 or d != n_species * Gy * G:
        raise ValueError("pattern length must be n_species * Gy * G")
    dev = X1.device
    K = bin(int(features)).count("1")
    radii = radii.to(device=dev, dtype=torch.float64).contiguous()
    if radii.dim() != 2 or radii.shape[0] != K:
        raise ValueError("radii: [K, M+1]")
    M = radii.shape[1] - 1
    if work is None:
        work = mcil_workspace(n1, n2, G, n_species, features, scale, M, dev, Gy=Gy)
    rout = torch.empty_like(radii)
    bins = torch.empty((K, n1, n2), dtype=torch.uint8, device=dev)
    counts = torch.empty((K, M), dtype=torch.int64, device=dev)
    Cv = torch.empty(K * M, dtype=torch.float64, device=dev)
    nex = torch.zeros(1, dtype=torch.int64, device=dev)
    _check("mcil_features_given_rect", lib().mcil_features_given_rect(
        _ptr(X1), ld1, n1, _ptr(X2), ld2, n2, int(Gy), int(G), int(n_species), int(features), 1 if scale else 0,
        int(M), _ptr(radii), _ptr(rout), _ptr(bins), _ptr(counts), _ptr(Cv), _ptr(nex), _ptr(work), work.numel(),
        _stream()))
    return {"radii": rout, "bins": bins, "counts": counts, "C": Cv, "n_exact": nex}


class Scil:
    """One evaluation of the synthetic-likelihood cost f(theta) with
    bootstrapping (Alg. 6) per call of run(): scil_evaluate on group `group`
    of `sim` (its n_real = N_syn patterns at its parameters) against the
    data patterns `data` (rows, n_species * G * G floats).  Outputs and the
    workspace are allocated once here, so run() can be captured in a CUDA
    graph.  law "power" (b), "linear" or "fitted"; integrator "euler" or
    "rkc" (rkc = dict of h0, rtol, atol, s_max, max_attempts, t_end)."""

    def __init__(self, sim, group, data, n_set, n_species=2, features=63, scale=False, law="fitted", b=1.3,
                 M=13, T=1000, seed=0, reinit=True, integrator="euler", rkc=None):
        self.sim, self.group = sim, int(group)
        self.data, self.ld_data, self.n_data, d = _as_rows(data)
        g = sim.groups[group]
        if d != n_species * g.G * g.G:
            raise ValueError("data rows must hold n_species * G * G floats")
        r = dict(h0=1e-3, rtol=1e-5, atol=1e-5, s_max=RKC_S_MAX, max_attempts=100000, t_end=0.0)
        r.update(rkc or {})
        o = RdRkcOpts(float(r["t_end"]), float(r["h0"]), float(r["rtol"]), float(r["atol"]), int(r["s_max"]), 0, 0,
                      int(r["max_attempts"]))
        self.spec = ScilSpec(self.group, {"euler": 0, "rkc": 1}[integrator], o, int(n_set), int(n_species),
                             int(features), 1 if scale else 0, {"power": 0, "linear": 1, "fitted": 2}[law],
                             float(b), int(M), int(T), int(seed) & 0xFFFFFFFFFFFFFFFF, 1 if reinit else 0, 0)
        sz = _sz(0)
        _check("scil_workspace_size", lib().scil_workspace_size(sim.handle, C.byref(self.spec), self.n_data,
                                                                C.byref(sz)))
        dev = sim.device
        self.work = torch.empty(sz.value, dtype=torch.uint8, device=dev)
        K = bin(int(features)).count("1")
        Mt = K * M
        self.K, self.M, self.T = K, M, T
        self.out = {"radii": torch.empty((K, M + 1), dtype=torch.float64, device=dev),
                    "y_data": torch.empty(Mt, dtype=torch.float64, device=dev),
                    "Y": torch.empty((T, Mt), dtype=torch.int64, device=dev),
                    "mu": torch.empty(Mt, dtype=torch.float64, device=dev),
                    "cov": torch.empty((Mt, Mt), dtype=torch.float64, device=dev),
                    "chol": torch.empty((Mt, Mt), dtype=torch.float64, device=dev),
                    "scalars": torch.empty(4, dtype=torch.float64, device=dev),
                    "active": torch.empty(Mt, dtype=torch.uint8, device=dev),
                    "status": torch.empty(1, dtype=torch.int32, device=dev),
                    "n_exact": torch.zeros(2, dtype=torch.int64, device=dev)}

    def run(self):
        o = self.out
        _check("scil_evaluate", lib().scil_evaluate(
            self.sim.handle, _ptr(self.sim.fields), C.byref(self.spec), _ptr(self.data), self.ld_data, self.n_data,
            _ptr(o["radii"]), _ptr(o["y_data"]), _ptr(o["Y"]), _ptr(o["mu"]), _ptr(o["cov"]), _ptr(o["chol"]),
            _ptr(o["scalars"]), _ptr(o["active"]), _ptr(o["status"]), _ptr(o["n_exact"]), _ptr(self.work),
            self.work.numel(), _stream()))
        return o


def mcil_rdode(fields, n1, b=1.3, M=13, scale=False, law="power"):
    """Multi-feature correlation integral of 1-D reaction-diffusion-ODE
    patterns (Sec. 5.2): fields [n, 2, N] (u, w); set 1 = rows 0..n1-1, set 2
    the rest.  L2 and Linf of both species, the derivative-based norms
    (W12, W12', W1inf, W1inf') of w alone (u is discontinuous).  Returns the
    two mcil() results and the bins [6, n1, n2] concatenated in feature
    order for synlik(..., n_feat=6)."""
    n, _, N = fields.shape
    both = fields.reshape(n, 2 * N)
    w = fields[:, 1, :]
    a = mcil(both[:n1], both[n1:], N, 2, b=b, M=M, features=0x03, scale=scale, Gy=1, law=law)
    c = mcil(w[:n1], w[n1:], N, 1, b=b, M=M, features=0x3C, scale=scale, Gy=1, law=law)
    return a, c, torch.cat([a["bins"], c["bins"]], dim=0)


# ---------------------------------------------------------------------------
# one pass of the whole hot path
# ---------------------------------------------------------------------------
class Pipeline:
    """initial state -> integration (+ residual) -> per-group correlation
    integral of two pattern sets -> bootstrap statistics of every group, with
    every output buffer allocated once, so that a pass can be captured in a
    CUDA graph and replayed.  sets[i] = (n1, n2, species_mask) of group i:
    set 1 = realisations 0..n1-1, set 2 = n1..n1+n2-1.  The cost is
    evaluated at each group's own correlation vector (y_obs = C).
    integrator: "euler" (rd_integrate_batch, each group's n_steps), "rkc"
    (rd_integrate_rkc to each group's dt * n_steps; `rkc` = dict of h0,
    rtol, atol, s_max, max_attempts) or "imex" (rd_integrate_imex, each
    group's n_steps of its dt, diffusion implicit); law: "power" (R0 b^-k), "linear"
    (R0 - k (R0 - R_min) / M, b unused) or "fitted" (R0 b^-k with b fitted
    so that R_M = R_min, b unused).  RDODE groups need "rkc".  cil_streams:
    the groups' correlation integrals (independent problems of a few small
    launches each) run on that many side streams at once, each with its own
    workspace, forked from and joined back into the calling stream (1: all
    on the calling stream)."""

    def __init__(self, groups, sets, M, b, T, seed, device=None, integrator="euler", rkc=None, law="power",
                 cil_streams=8):
        if integrator not in ("euler", "rkc", "imex") or law not in ("power", "linear", "fitted"):
            raise ValueError("integrator / law")
        self.sim = Simulation(groups, device=device)
        self.dev = self.sim.device
        self.M, self.b, self.T, self.seed = M, b, T, seed
        self.integrator, self.law = integrator, law
        r = dict(h0=1e-3, rtol=1e-5, atol=1e-5, s_max=RKC_S_MAX, max_attempts=100000)
        r.update(rkc or {})
        self.rkc_opts = RdRkcOpts(0.0, float(r["h0"]), float(r["rtol"]), float(r["atol"]), int(r["s_max"]), 0, 0,
                                  int(r["max_attempts"]))
        self.rkc_stats = torch.empty((self.sim.n_real_total, 4), dtype=torch.int64, device=self.dev)
        self.views = []
        n1s = set(s[0] for s in sets)
        n2s = set(s[1] for s in sets)
        if len(n1s) != 1 or len(n2s) != 1:
            raise ValueError("all groups need the same set sizes (batched statistics)")
        self.n1, self.n2 = n1s.pop(), n2s.pop()
        P = len(groups)
        for i, (g, (n1, n2, mask)) in enumerate(zip(groups, sets)):
            cells = g.cells
            fv = self.sim.group_fields(i).reshape(g.n_real, 2 * cells)
            off = 0 if mask in (1, 3) else cells
            d = cells * (2 if mask == 3 else 1)
            self.views.append((fv[:n1, off:off + d], fv[n1:n1 + n2, off:off + d]))
        self.bins = torch.empty((P, self.n1, self.n2), dtype=torch.uint8, device=self.dev)
        self.C = torch.empty((P, M), dtype=torch.float64, device=self.dev)
        self.cil_out = [{"radii": torch.empty(M + 1, dtype=torch.float64, device=self.dev),
                         "bins": self.bins[i], "counts": torch.empty(M, dtype=torch.int64, device=self.dev),
                         "C": self.C[i], "n_rechecked": torch.zeros(1, dtype=torch.int64, device=self.dev)}
                        for i in range(P)]
        self.stats = synlik_outputs(P, M, T, self.dev)
        self.syn_work = synlik_workspace(self.n1, self.n2, M, T, 1, P, self.dev)
        self.residual = torch.empty((self.sim.n_real_total, 2), dtype=torch.float64, device=self.dev)
        dmax = max(x.shape[1] for x, _ in self.views)
        self.work, self.work_bytes = _workspace(self.n1, self.n2, dmax, self.dev)
        ns = max(1, min(int(cil_streams), P))
        self.side = [torch.cuda.Stream(device=self.dev) for _ in range(ns)] if ns > 1 else []
        self.side_work = [torch.empty(self.work_bytes, dtype=torch.uint8, device=self.dev) for _ in self.side]
        self.graph = None

    def run_cils(self):
        """Every group's correlation integral (radii, bins, counts, C), in
        stream order after the calling stream's prior work and before its
        later work."""
        fn = {"linear": "cil_features_linear", "fitted": "cil_features_fitted"}.get(self.law, "cil_features")
        if not self.side:
            for (X1, X2), out in zip(self.views, self.cil_out):
                _cil_call(fn, X1, X2, self.b, self.M, None, self.work, out)
            return
        main = torch.cuda.current_stream(self.dev)
        fork = torch.cuda.Event()
        fork.record(main)
        for st in self.side:
            st.wait_event(fork)
        for i, ((X1, X2), out) in enumerate(zip(self.views, self.cil_out)):
            k = i % len(self.side)
            with torch.cuda.stream(self.side[k]):
                _cil_call(fn, X1, X2, self.b, self.M, None, self.side_work[k], out)
        for st in self.side:
            join = torch.cuda.Event()
            join.record(st)
            main.wait_event(join)

    def run(self, reinit=True):
        if reinit:
            self.sim.reinit()
        if self.integrator == "euler":
            _check("rd_integrate_batch", lib().rd_integrate_batch(
                self.sim.handle, _ptr(self.sim.fields), -1, _ptr(self.residual), _stream()))
        elif self.integrator == "imex":
            _check("rd_integrate_imex", lib().rd_integrate_imex(
                self.sim.handle, _ptr(self.sim.fields), _ptr(self.residual), _stream()))
        else:
            _check("rd_integrate_rkc", lib().rd_integrate_rkc(
                self.sim.handle, _ptr(self.sim.fields), C.byref(self.rkc_opts), _ptr(self.rkc_stats),
                _ptr(self.residual), _stream()))
        self.run_cils()
        synlik(self.bins, self.M, self.T, self.seed, y_obs=self.C, out=self.stats, work=self.syn_work)

    def capture(self):
        """Record one pass (from the initial state) as a CUDA graph."""
        torch.cuda.synchronize()
        s = torch.cuda.Stream(device=self.dev)
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            self.run()            # warm every lazy set-up outside the capture
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self.run()
        return self.graph

    def replay(self):
        self.graph.replay()


# ---------------------------------------------------------------------------
# autograd
# ---------------------------------------------------------------------------
class SmoothCIL(torch.autograd.Function):
    """C_tau(theta): the sigmoid-smoothed correlation integral of one group
    after its n_steps, as a differentiable function of theta (the group's
    first four parameters: FHN (Du, Dv, eps, a), GM (Du, Dv, rho, mu), BZ
    (Du, Dv, A, B)).

    forward(theta, sim, group, fields0, species_mask, set1, set2, radii,
            tau_frac) -> C[M]: writes theta into the group (rd_set_params,
    keeping its other parameter slots) and evaluates C by one forward
    integration (no reverse sweep).  backward calls rd_adjoint with the
    incoming gradient as cotangent, at the theta of the forward pass."""

    @staticmethod
    def forward(ctx, theta, sim, group, fields0, species_mask, set1, set2, radii, tau_frac):
        th = [float(x) for x in theta.detach().cpu().tolist()]
        if len(th) != 4:
            raise ValueError("theta: 4 parameters")
        full = list(th) + list(sim.groups[group].params[4:])
        sim.set_params(group, full)
        Cv, _ = sim.adjoint(group, fields0, species_mask, set1, set2, radii, tau_frac, None)
        ctx.args = (sim, group, fields0, species_mask, set1, set2, radii, tau_frac)
        ctx.full = full
        ctx.theta_device = theta.device
        return Cv

    @staticmethod
    def backward(ctx, gC):
        sim, group, fields0, species_mask, set1, set2, radii, tau_frac = ctx.args
        if list(sim.groups[group].params) != ctx.full:   # another call moved theta since
            sim.set_params(group, ctx.full)
        _, g = sim.adjoint(group, fields0, species_mask, set1, set2, radii, tau_frac,
                           gC.detach().to(torch.float64))
        return (g.to(ctx.theta_device), None, None, None, None, None, None, None, None)
