"""The C-ABI library builds, loads without a GPU and exports every symbol the
header declares; the binding's struct matches the C layout."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rdcil.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:[A-Za-z_][\w\s\*]*?)\b([a-z_][a-z0-9_]*)\s*\(", src, flags=re.M)
    return sorted(set(n for n in names if n not in ("if", "while", "sizeof")))


@pytest.fixture(scope="module")
def libpath():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2203_14742_b300 import LIB_PATH
    return LIB_PATH


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("rd_init", "rd_integrate_batch", "cil_features", "synlik_stats", "rd_adjoint"):
        assert n in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True,
                         check=True).stdout
    exported = set(l.split()[-1] for l in out.splitlines() if l.strip())
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing


def test_library_loads_without_gpu(libpath):
    import paper_2203_14742_b300 as p
    L = p.lib()
    assert L.rd_status_str(0) == b"ok"
    assert L.rd_status_str(3) == b"covariance not positive definite"
    sz = ctypes.c_size_t()
    assert L.cil_workspace_size(64, 64, 4096, ctypes.byref(sz)) == 0 and sz.value > 0
    assert L.cil_workspace_size(0, 64, 4096, ctypes.byref(sz)) == 1


def test_rd_group_layout_matches_header(libpath):
    import paper_2203_14742_b300 as p
    # offsets written out from the C struct (natural alignment)
    expect = {"model": 0, "G": 4, "n_real": 8, "flags": 12, "n_steps": 16, "field_offset": 24,
              "dt": 32, "params": 40, "noise_lo": 88, "noise_hi": 96, "seed": 104}
    for name, off in expect.items():
        assert getattr(p.RdGroup, name).offset == off
    assert ctypes.sizeof(p.RdGroup) == 112


def test_argument_errors_before_any_launch(libpath):
    import paper_2203_14742_b300 as p
    L = p.lib()
    h = ctypes.c_void_p()
    g = (p.RdGroup * 1)()
    g[0].model, g[0].n_real, g[0].dt = 0, 1, 1e-3
    for G in (50, 4, 8192):                                           # unsupported G
        g[0].G = G
        assert L.rd_init(g, 1, ctypes.c_void_p(256), None, ctypes.byref(h)) == 1
    g[0].G, g[0].flags = 48, 4                                        # unknown flag
    assert L.rd_init(g, 1, ctypes.c_void_p(256), None, ctypes.byref(h)) == 1
    g[0].flags = 1                                                    # adjoint needs a resident grid
    assert L.rd_init(g, 1, ctypes.c_void_p(256), None, ctypes.byref(h)) == 6
    g[0].flags = 0
    g[0].G = 64
    g[0].field_offset = 2                                             # misaligned
    assert L.rd_init(g, 1, ctypes.c_void_p(256), None, ctypes.byref(h)) == 1
    g[0].field_offset = 0
    g[0].dt = -1.0
    assert L.rd_init(g, 1, ctypes.c_void_p(256), None, ctypes.byref(h)) == 1
    assert L.rd_init(g, 1, None, None, ctypes.byref(h)) == 1
    # cil: M out of range, b <= 1
    w = ctypes.c_void_p(256)
    assert L.cil_features(w, 8, 4, w, 8, 4, 8, None, 1.3, 33, w, w, w, None, None, w, 1 << 20, None) == 1
    assert L.cil_features(w, 8, 4, w, 8, 4, 8, None, 1.0, 8, w, w, w, None, None, w, 1 << 20, None) == 1
    # synlik: T < 2
    assert L.synlik_stats(w, 4, 4, 8, 1, 0, 1, None, w, w, w, w, w, w, w, None) == 1


def test_variant_shapes_are_valid_tilings(libpath):
    """Every stepper tile variant tiles its grid with whole warps, and keeps
    a tile row inside one warp (the east/west shuffles assume it)."""
    import paper_2203_14742_b300 as p
    for G in (32, 64, 128):
        for v in range(p.lib().rd_n_variants()):
            packed, TY, TX = p.variant_shape(G, v)
            assert packed in (0, 1) and G % TY == 0 and G % TX == 0
            NX, NY = G // TX, G // TY
            assert NX <= 32 and NX & (NX - 1) == 0 and NX % 2 == 0
            assert (NX * NY) % 32 == 0 and NX * NY <= 1024
            # the double-buffered halo ring of the variant fits one CTA
            ring = {0: 2 * 2 * 2 * NY * G * 4, 1: 2 * 2 * NY * G * 8}[packed]
            assert ring <= 227 * 1024, (G, v, ring)
        assert p.variant_shape(G, 0)[0] == 0
    sh = (ctypes.c_int32 * 3)()
    assert p.lib().rd_variant_shape(48, 0, sh) == 1
    assert p.lib().rd_variant_shape(64, p.lib().rd_n_variants(), sh) == 1


def test_stream_depth_argument_checks(libpath):
    import paper_2203_14742_b300 as p
    L = p.lib()
    assert L.rd_set_stream_depth(None, 4) == 1
    assert L.rd_get_stream_depth(None) == -1


def test_rkc_argument_checks_without_gpu(libpath):
    # null handle / options, and the tile-shape setters, need no device
    import paper_2203_14742_b300 as p
    L = p.lib()
    o = p.RdRkcOpts(0.0, 1e-3, 1e-5, 1e-5, 256, 0, 0, 1000)
    assert L.rd_integrate_rkc(None, ctypes.c_void_p(256), ctypes.byref(o), None, None, None) == 1
    assert ctypes.sizeof(p.RdRkcOpts) == 56
    assert L.rd_rkc_n_variants() == 3
    assert L.rd_rkc_get_variant(64) == 1 and L.rd_rkc_get_variant(32) == 0
    assert L.rd_rkc_get_variant(128) == -1
    assert L.rd_rkc_set_variant(128, 0) == 1 and L.rd_rkc_set_variant(64, 3) == 1
    assert L.rd_rkc_set_variant(64, 0) == 0 and L.rd_rkc_get_variant(64) == 0
    assert L.rd_rkc_set_variant(64, 1) == 0
    assert L.rd_status_str(8) == b"adaptive step control gave up"


def test_imex_argument_checks_without_gpu(libpath):
    # a null handle or field pointer is refused before any device work
    import paper_2203_14742_b300 as p
    L = p.lib()
    assert L.rd_integrate_imex(None, ctypes.c_void_p(256), None, None) == 1
    assert L.rd_integrate_imex(ctypes.c_void_p(256), None, None, None) == 1
    assert L.rd_imex_n_variants() == 5
    assert L.rd_imex_get_variant(128) == -1
    assert L.rd_imex_set_variant(128, 0) == 1 and L.rd_imex_set_variant(64, 5) == 1
