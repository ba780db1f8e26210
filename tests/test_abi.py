"""The C ABI library builds, loads without a GPU and exports every entry point
declared in include/gpmg.h; the binding declares the same set.  No compute
call is made here."""
import ctypes
import os
import re

from paper_1911_00994_gb300 import build, gpmg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "gpmg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^[A-Za-z_][\w \*]*?\b([a-z_][a-z0-9_]*)\s*\(", src, flags=re.M)
    return sorted(set(n for n in names if n not in ("if", "while")))


def test_library_exports_every_declared_symbol():
    path = build.build()
    lib = ctypes.CDLL(path)
    names = declared_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_the_header():
    bound = {n for n, _, _ in gpmg.SIGNATURES}
    assert bound == set(declared_functions())


def test_layout_helpers():
    assert gpmg.pitch(30) == 32 and gpmg.pitch(31) == 64
    assert gpmg.vec_len(16) == 3 * 18 * 32 + 32
    m = gpmg.flat_to_vec(8)
    assert len(m) == 2 * 9 * 10 + 64 + 1
    assert len(set(m.tolist())) == len(m)


def test_parameter_checks_on_the_host():
    # gp_params_default and gp_workspace_size make no CUDA call: defaults,
    # a workspace size, and GP_INVALID for an inner-cycle count out of range
    L = gpmg.lib()
    p = gpmg.gp_params()
    assert L.gp_params_default(ctypes.byref(p), 64, -1.0, -1.0, 2.0) == 0
    assert p.inner == 0 and p.precision == gpmg.GP_FP64 and p.nu1 == 2 and p.nu2 == 1
    nb = ctypes.c_size_t(0)
    assert L.gp_workspace_size(ctypes.byref(p), ctypes.byref(nb)) == 0 and nb.value > 0
    for bad in (-1, 9):
        p.inner = bad
        assert L.gp_workspace_size(ctypes.byref(p), ctypes.byref(nb)) == 1
    p.inner = 8
    assert L.gp_workspace_size(ctypes.byref(p), ctypes.byref(nb)) == 0


def test_invalid_sizes_are_rejected_on_the_host():
    # bad N or levels: GP_INVALID from gp_workspace_size and gp_create, before
    # any CUDA call (the context is not created)
    L = gpmg.lib()
    p = gpmg.gp_params()
    assert L.gp_params_default(ctypes.byref(p), 64, -1.0, -1.0, 2.0) == 0
    nb = ctypes.c_size_t(0)
    ctx = ctypes.c_void_p(1)
    for N, levels in ((64, 0), (64, 17), (2, 1), (60, 4), (256, 2), (64, 6)):
        q = gpmg.gp_params.from_buffer_copy(p)
        q.N, q.levels = N, levels
        assert L.gp_workspace_size(ctypes.byref(q), ctypes.byref(nb)) == gpmg.GP_INVALID, (N, levels)
        assert L.gp_create(ctypes.byref(ctx), ctypes.byref(q), None, 0, None) == gpmg.GP_INVALID, (N, levels)
        assert ctx.value is None
    assert L.gp_params_default(ctypes.byref(p), 3, -1.0, -1.0, 2.0) == gpmg.GP_INVALID
    assert L.gp_last_error(None) == b"null context"
    # a non-power-of-two grid whose coarsening stays integral is accepted
    q = gpmg.gp_params.from_buffer_copy(p)
    q.N, q.levels = 60, 3
    assert L.gp_workspace_size(ctypes.byref(q), ctypes.byref(nb)) == 0


def declared_3d():
    src = open(os.path.join(ROOT, "include", "gpmg3d.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^[A-Za-z_][\w \*]*?\b([a-z_][a-z0-9_]*)\s*\(", src, flags=re.M)
    return sorted(set(n for n in names if n not in ("if", "while")))


def test_3d_library_exports_and_binding_cover_gpmg3d_h():
    from paper_1911_00994_gb300 import mac3d
    lib = ctypes.CDLL(build.build())
    names = declared_3d()
    assert len(names) >= 12
    for n in names:
        assert hasattr(lib, n), n
    assert {n for n, _, _ in mac3d.SIGNATURES} == set(names)


def test_3d_sizes_are_checked_on_the_host():
    # gp3_workspace_size makes no CUDA call: a size for valid hierarchies,
    # GP_INVALID for N not divisible down the levels, a coarsest grid below
    # 2, a coarsest dense matrix above 1024 unknowns or N above 1024 (frames
    # of 2^31 slots or more)
    from paper_1911_00994_gb300 import mac3d
    L = mac3d.lib()
    nb = ctypes.c_size_t(0)
    assert L.gp3_workspace_size(64, 5, 0, ctypes.byref(nb)) == 0 and nb.value > 0
    n64 = nb.value
    assert L.gp3_workspace_size(64, 5, 1, ctypes.byref(nb)) == 0 and nb.value > n64
    assert L.gp3_workspace_size(64, 5, 2, ctypes.byref(nb)) == 1
    assert L.gp3_vec_len(64) == 4 * 66 ** 3 + 32
    assert L.gp3_workspace_size(1024, 9, 0, ctypes.byref(nb)) == 0
    for N, lev in ((64, 7), (48, 6), (64, 3), (0, 1), (64, 0), (2048, 10)):
        assert L.gp3_workspace_size(N, lev, 0, ctypes.byref(nb)) == 1, (N, lev)
