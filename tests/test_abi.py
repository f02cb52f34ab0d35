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
            assert packed in (0, 1, 2, 3) and G % TY == 0 and G % TX == 0
            NX, NY = G // TX, G // TY
            assert NX <= 32 and NX & (NX - 1) == 0 and NX % 2 == 0
            assert (NX * NY) % 32 == 0 and NX * NY <= 1024
            # the double-buffered halo ring of the variant fits one CTA
            ring = {0: 2 * 2 * 2 * NY * G * 4, 1: 2 * 2 * NY * G * 8, 2: 2 * 2 * 2 * NY * G * 4,
                    3: 2 * 2 * NY * G * 8}[packed]
            assert ring <= 227 * 1024, (G, v, ring)
        assert p.variant_shape(G, 0)[0] in (0, 2, 3)   # the default: a plain or rotating tile
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


def test_step_table_sizes_without_gpu(libpath):
    """rd_tables_size (host only): the stabilised RK2 tables ((S+1)^2 float4
    coefficients + (S+1) doubles, S = 256) when a group can run the RK2
    integrator, plus the semi-implicit cosine-basis tables (2 G^2 + G and
    G^2 + G floats) per grid side 32 / 64 present and the even/odd table
    alone (G^2 + G floats) at 128, each rounded up to 256 bytes; none for
    groups no table-using integrator runs (G = 256)."""
    import paper_2203_14742_b300 as p

    def up(b):
        return (b + 255) // 256 * 256

    rkc = up(257 * 257 * 16 + 257 * 8)

    def imex(G):
        return up(4 * (2 * G * G + G)) + up(4 * (G * G + G))

    def size(spec):
        arr = (p.RdGroup * len(spec))()
        off = 0
        for i, (model, G) in enumerate(spec):
            a = arr[i]
            a.model, a.G, a.n_real, a.n_steps, a.dt, a.field_offset = model, G, 2, 10, 1e-4, off
            a.params[0], a.params[1], a.params[2], a.params[3] = 1e-4, 1e-2, 1.0, 0.5
            a.noise_hi = 0.01
            off += 2 * 2 * G * (1 if model == p.RDODE else G)
        sz = ctypes.c_size_t()
        assert p.lib().rd_tables_size(arr, len(spec), ctypes.byref(sz)) == 0
        return sz.value

    assert size([(p.FHN, 64)]) == rkc + imex(64)
    assert size([(p.GM, 128)]) == rkc + up(4 * (128 * 128 + 128))
    assert size([(p.FHN, 32), (p.GM, 64), (p.FHN, 64)]) == rkc + imex(32) + imex(64)
    assert size([(p.FHN, 256)]) == 0
    assert size([(p.RDODE, 256)]) == rkc
    sz = ctypes.c_size_t()
    assert p.lib().rd_tables_size(None, 1, ctypes.byref(sz)) == 1


def test_structs_match_the_header_layout(tmp_path, libpath):
    """The binding's ctypes structs have the C compiler's layout of the
    header's structs (offsets from offsetof in a compiled probe)."""
    import paper_2203_14742_b300 as p
    src = tmp_path / "probe.c"
    fields = {"rd_group": ("RdGroup", ["model", "G", "n_real", "flags", "n_steps", "field_offset", "dt", "params",
                                       "noise_lo", "noise_hi", "seed"]),
              "rd_rkc_opts": ("RdRkcOpts", ["t_end", "h0", "rtol", "atol", "s_max", "s_fixed", "n_fixed",
                                            "max_attempts"]),
              "scil_spec": ("ScilSpec", ["group", "integrator", "rkc", "n_set", "n_species", "features", "scale",
                                         "law", "b", "M", "T", "seed", "reinit", "pad"])}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "rdcil.h"', 'int main(void) {']
    for cs, (_, names) in fields.items():
        lines.append('printf("%s sizeof %%zu\\n", sizeof(%s));' % (cs, cs))
        for n in names:
            lines.append('printf("%s %s %%zu\\n", offsetof(%s, %s));' % (cs, n, cs, n))
    lines += ['return 0;', '}']
    src.write_text("\n".join(lines))
    exe = tmp_path / "probe"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = {}
    for line in out:
        if line:
            cs, n, v = line.split()
            got[(cs, n)] = int(v)
    for cs, (py, names) in fields.items():
        cls = getattr(p, py)
        assert ctypes.sizeof(cls) == got[(cs, "sizeof")], cs
        for n in names:
            assert getattr(cls, n).offset == got[(cs, n)], (cs, n)


def test_gram_product_count_choice_without_gpu(libpath):
    """cil_gram_products (host only): three products by default at every
    size; cil_set_gram_products selects one or three, 0 restores the
    default, anything else is rejected."""
    L = ctypes.CDLL(libpath)
    L.cil_gram_products.restype = ctypes.c_int32
    L.cil_gram_products.argtypes = [ctypes.c_int64] * 3
    L.cil_set_gram_products.restype = ctypes.c_int32
    L.cil_set_gram_products.argtypes = [ctypes.c_int32]
    try:
        assert L.cil_gram_products(1024, 1024, 32768) == 3
        assert L.cil_gram_products(64, 64, 4096) == 3
        assert L.cil_gram_products(0, 64, 4096) == -1
        assert L.cil_set_gram_products(1) == 0
        assert L.cil_gram_products(1024, 1024, 32768) == 1
        assert L.cil_gram_products(64, 64, 4096) == 1
        assert L.cil_set_gram_products(0) == 0
        assert L.cil_gram_products(64, 64, 4096) == 3
        assert L.cil_set_gram_products(2) == 1                 # RD_ERR_INVALID_ARG
    finally:
        L.cil_set_gram_products(0)
