"""The C-ABI library loads without a GPU and exports every function that
include/*.h declares (no compute calls here)."""
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w \*]*?\b(velo_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


def test_header_declares_entry_points():
    names = _declared_functions()
    for n in ("velo_create", "velo_reconstruct", "velo_destroy", "velo_sync_status", "velo_reconstruct_host"):
        assert n in names


def test_library_exports_every_declared_symbol():
    import paper_1912_09161_gb300 as V
    lib = V.load_library()
    missing = [n for n in sorted(_declared_functions()) if not hasattr(lib, n)]
    assert not missing, missing
    assert set(V.velo.EXPORTED) == _declared_functions()
    assert "sm_103a" in V.velo.velo_version()


def test_errors_without_gpu_are_reported():
    """Argument validation happens before any device work."""
    import ctypes
    import paper_1912_09161_gb300 as V
    lib = V.load_library()
    h = ctypes.c_void_p()
    rc = lib.velo_create(None, None, None, ctypes.byref(h))
    assert rc == V.velo.VELO_ERR_INPUT
    assert b"geometry" in lib.velo_last_error()
