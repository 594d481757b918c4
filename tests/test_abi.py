"""Host-side checks of the C-ABI library (no GPU needed): it builds for
sm_103a, loads, exports every symbol include/mgauss.h declares, and the
host-only entry points behave (sizes, options, argument errors)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "mgauss.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mg_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2603_00145_b300 import build, _lib
    build.build()
    return _lib.lib()


def test_exports_every_declared_symbol(lib):
    from paper_2603_00145_b300 import build, _lib
    names = _declared()
    assert "mg_render_fwd" in names and "mg_render_bwd" in names and "mg_sample_volume" in names
    out = subprocess.check_output(["nm", "-D", "--defined-only", build.LIB]).decode()
    exported = set(re.findall(r"\sT\s(\w+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    assert set(names) == set(_lib.SIGNATURES), set(names) ^ set(_lib.SIGNATURES)
    for n in names:
        getattr(lib, n)


def test_library_is_sm_103a(lib):
    from paper_2603_00145_b300 import build
    out = subprocess.check_output(["cuobjdump", "--list-elf", build.LIB]).decode()
    assert "sm_103a" in out


def test_host_entry_points(lib):
    from paper_2603_00145_b300 import _lib as L
    o = lib.mg_default_opts()
    assert o.cutoff_k == 3.0 and o.f64_ratio == 16.0
    g = L.MgGaussians(1000, None, None, None, None)
    st = (L.MgStack * 2)(L.MgStack(10, 40, 33, 1.0, 1.0, 3.0, None), L.MgStack(5, 17, 64, 0.5, 0.5, 0.0, None))
    n1 = lib.mg_render_workspace_size(ctypes.byref(g), st, 2, ctypes.byref(o))
    assert n1 > 0 and n1 % 256 == 0
    o2 = L.MgOpts(3.0, 100.0, 5000, 40000)
    n2 = lib.mg_render_workspace_size(ctypes.byref(g), st, 2, ctypes.byref(o2))
    lay = L.MgWsLayout()
    assert lib.mg_render_ws_layout(ctypes.byref(g), st, 2, ctypes.byref(o2), ctypes.byref(lay)) == 0
    assert lay.total_bytes == n2
    assert lay.tile_off % 256 == 0 and lay.entries % 256 == 0 and lay.entries + 4 * 40000 <= n2
    # invalid arguments: nothing launched, errors returned
    bad = (L.MgStack * 1)(L.MgStack(0, 40, 33, 1.0, 1.0, 3.0, None))
    assert lib.mg_render_workspace_size(ctypes.byref(g), bad, 1, ctypes.byref(o)) == 0
    out = ctypes.c_void_p(0)
    s = lib.mg_render_fwd(ctypes.byref(g), st, 2, ctypes.byref(o), None, None, 0, None)
    assert s == L.MG_ERR_INVALID_ARG and b"NULL" in lib.mg_last_error()
    assert lib.mg_render_bwd(ctypes.byref(g), st, 2, ctypes.byref(o), None, None, None, None, None, None, 0,
                             None) == L.MG_ERR_INVALID_ARG
    assert lib.mg_sample_workspace_size(1000, 64, ctypes.byref(o)) > 0
    assert lib.mg_sample_workspace_size(1000, 0, ctypes.byref(o)) == 0
    assert lib.mg_reduce_workspace_size(12345) >= 16
    assert lib.mg_loss_recon_workspace_size(st, 2) >= 16 * (10 * 2 * 2 + 5 * 1 * 2)
    assert lib.mg_loss_recon_workspace_size(bad, 1) == 0
    grp = L.MgAdamGroup(None, None, None, None, 10, 0.1, 1.0, 0.0)
    assert lib.mg_adam_step(ctypes.byref(grp), 1, 0.9, 0.999, 1e-8, None, None, 0, None) == L.MG_ERR_INVALID_ARG
    assert lib.mg_status_string(L.MG_ERR_CAPACITY) == b"workspace capacity exceeded"
    assert lib.mg_version().startswith(b"mgauss")


def test_tile_edge_agrees_with_the_header():
    """The binding's and the oracle's tile edge are the header's MG_TILE_EDGE
    (the tile size is part of the definition of the local set)."""
    import re

    import oracle
    from paper_2603_00145_b300 import _lib

    hdr = open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include",
                            "mgauss.h")).read()
    edge = int(re.search(r"#define MG_TILE_EDGE (\d+)", hdr).group(1))
    assert edge == _lib.MG_TILE_EDGE == oracle.TILE
