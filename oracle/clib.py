"""Build and load ``tdeig_oracle.c`` (plain C, gcc) through ctypes.

Test infrastructure only (see the package docstring).
"""
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tdeig_oracle.c")
_SO = os.path.join(_HERE, "_liboracle.so")
_lock = threading.Lock()
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


def build_oracle(force=False):
    """Compile the oracle's C routines into ``oracle/_liboracle.so``."""
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC):
        return _SO
    tmp = _SO + ".tmp%d" % os.getpid()
    # -ffp-contract=off: every operation rounded once as written, on x86 and Arm alike
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC,
           "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build_oracle()
            L = ctypes.CDLL(_SO)
            L.orc_leaf_qr.argtypes = [ctypes.c_int, _dp, _dp, _dp, _dp]
            L.orc_leaf_qr.restype = ctypes.c_int
            L.orc_deflate.argtypes = [ctypes.c_int, _dp, _dp, ctypes.c_double, _dp, ctypes.c_int,
                                      ctypes.c_int, _ip, _ip, _ip, _dp, _dp, _ip]
            L.orc_deflate.restype = ctypes.c_int
            L.orc_secular_root.argtypes = [ctypes.c_int, _dp, _dp, ctypes.c_double, ctypes.c_int,
                                           _dp, _dp, _dp, _dp]
            L.orc_secular_root.restype = ctypes.c_int
            L.orc_secular_all.argtypes = [ctypes.c_int, _dp, _dp, ctypes.c_double, _dp, _dp, _dp,
                                          _ip, _dp, ctypes.c_int]
            L.orc_secular_all.restype = ctypes.c_int
            L.orc_lowner.argtypes = [ctypes.c_int, _dp, _dp, _dp, ctypes.c_double, _dp, _dp]
            L.orc_lowner.restype = None
            L.orc_cauchy.argtypes = [ctypes.c_int, _dp, _dp, _dp, _dp, _dp, _dp]
            L.orc_cauchy.restype = None
            L.orc_cauchy_entries.argtypes = [ctypes.c_int, _ip, ctypes.c_int, _ip, _dp, _dp, _dp,
                                             _dp, _dp, _dp]
            L.orc_cauchy_entries.restype = None
            L.orc_dminus_entries.argtypes = [ctypes.c_int, _ip, ctypes.c_int, _ip, _dp, _dp, _dp,
                                             _dp]
            L.orc_dminus_entries.restype = None
            _lib = L
    return _lib


def dptr(a):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"] or a.flags["F_CONTIGUOUS"]
    return a.ctypes.data_as(_dp)


def iptr(a):
    assert a.dtype == np.int32
    return a.ctypes.data_as(_ip)
