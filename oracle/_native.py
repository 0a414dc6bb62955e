"""Oracle: builds and loads the plain-C COCG solver (``cocg.c``).

TEST INFRASTRUCTURE ONLY.  The shared object is compiled with the host C
compiler into ``oracle/_build/`` (git-ignored) on first use or by
``build()``; nothing else links it.
"""
import ctypes
import os
import subprocess
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cocg.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_OUT_DIR, "liboracle_cocg.so")
_lock = threading.Lock()
_handle = None


def build(force: bool = False) -> str:
    """Compile the oracle's plain C COCG (gcc, OpenMP) into oracle/_build
    if it is missing or older than its source; returns the library path.
    Test infrastructure: nothing on the product path calls it."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    stale = (not os.path.exists(_LIB)) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC)
    if force or stale:
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def load_cocg():
    """The compiled oracle COCG (built on first use), loaded once per
    process."""
    global _handle
    with _lock:
        if _handle is None:
            lib = ctypes.CDLL(build())
            lib.oracle_cocg_batch.restype = ctypes.c_int
            _handle = lib
    return _handle
