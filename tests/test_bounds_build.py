"""The bounds-checking debug build (-DCOLA_BOUNDS), without a GPU.

The default library says it has no checks (COLA_ERR_UNSUPPORTED); the debug
build compiles for sm_103a into its own folder, exports every entry point the
header declares, and its cola_debug_bounds is live: it validates its
arguments and reaches the CUDA runtime (which, on a machine without a GPU,
fails with COLA_ERR_CUDA rather than reporting no support).
"""
import ctypes
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_default_build_has_no_bounds_checks():
    import paper_2302_00850_gb300 as cola
    from paper_2302_00850_gb300 import _lib, build

    build.build()
    lib = _lib.load()
    c, line = ctypes.c_ulonglong(5), ctypes.c_int(5)
    assert lib.cola_debug_bounds(None, None, 0) == -1
    assert lib.cola_debug_bounds(ctypes.byref(c), ctypes.byref(line), 0) == -7
    assert b"COLA_BOUNDS" in lib.cola_last_error()
    assert c.value == 0 and line.value == 0
    with pytest.raises(cola.ColaError, match="UNSUPPORTED"):
        cola.debug_bounds()


def test_bounds_build_compiles_and_is_live():
    from paper_2302_00850_gb300 import build
    from test_library_abi import declared_functions

    path = build.build_bounds()
    assert path.endswith(os.path.join("_build_bounds", "libcola.so")) and os.path.exists(path)
    # in a child process: the debug library next to nothing else
    code = (
        "import ctypes, sys\n"
        f"lib = ctypes.CDLL({path!r})\n"
        f"missing = [n for n in {declared_functions()!r} if not hasattr(lib, n)]\n"
        "c, l = ctypes.c_ulonglong(5), ctypes.c_int(5)\n"
        "f = lib.cola_debug_bounds\n"
        "f.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]\n"
        "print(missing, f(None, None, 0), f(ctypes.byref(c), ctypes.byref(l), 0))\n"
    )
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    missing, st_null, st = r.stdout.split("]")[0] + "]", *r.stdout.split("]")[1].split()
    assert missing == "[]", r.stdout
    assert int(st_null) == -1
    # no device here: the runtime call fails (COLA_ERR_CUDA); with one, the count is read (COLA_OK)
    assert int(st) in (0, -2), r.stdout
