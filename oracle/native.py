"""Build and load the C part of the oracle (``tgba_oracle.c``) with gcc.

Test infrastructure only (see the package docstring).
"""
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tgba_oracle.c")
_SO = os.path.join(_HERE, "_liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force=False):
    """Compile the oracle's C file into ``oracle/_liboracle.so``."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + ".tmp.%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            L.oracle_wick_batch.restype = ctypes.c_int
            L.oracle_wick_batch.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                            ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]
            L.oracle_reduced_table.restype = ctypes.c_int
            L.oracle_reduced_table.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                               ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
            L.oracle_reduced_batch.restype = ctypes.c_int
            L.oracle_reduced_batch.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double,
                                               ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                               ctypes.c_int]
            L.oracle_pfaffian_batch.restype = None
            L.oracle_pfaffian_batch.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
            _lib = L
    return _lib


def pfaffian(a):
    """Pfaffian of one dense complex skew matrix (Parlett-Reid with pivoting, in C)."""
    a = np.array(a, dtype=np.complex128, order="C", copy=True)
    n = a.shape[0]
    out = np.zeros(1, dtype=np.complex128)
    lib().oracle_pfaffian_batch(n, 1, a.ctypes.data, out.ctypes.data)
    return out[0]


def wick_batch(N, strings, n_threads=0):
    """<0|O_1...O_m|0>_c for each operator string.

    ``strings`` is a list of lists of (kind, k, theta) triples.  Returns (values, threads used).
    """
    lens = np.array([len(s) for s in strings], dtype=np.int64)
    offsets = np.zeros(len(strings) + 1, dtype=np.int64)
    np.cumsum(lens, out=offsets[1:])
    flat = [op for s in strings for op in s]
    kinds = np.array([o[0] for o in flat], dtype=np.int32)
    ks = np.array([o[1] for o in flat], dtype=np.float64)
    th = np.array([o[2] for o in flat], dtype=np.float64)
    if len(flat) == 0:
        kinds = np.zeros(1, np.int32); ks = np.zeros(1); th = np.zeros(1)
    out = np.zeros(len(strings), dtype=np.complex128)
    used = lib().oracle_wick_batch(int(N), len(strings), offsets.ctypes.data, kinds.ctypes.data,
                                   ks.ctypes.data, th.ctypes.data, out.ctypes.data, int(n_threads))
    return out, used


def reduced_table(N, string, is_f):
    """(S, Pf(A_FF)) of the reduced form over one operator string: S is the Schur complement
    onto the operators with is_f = 0, in string order."""
    m = len(string)
    kinds = np.array([o[0] for o in string], dtype=np.int32)
    ks = np.array([o[1] for o in string], dtype=np.float64)
    th = np.array([o[2] for o in string], dtype=np.float64)
    f = np.ascontiguousarray(np.asarray(is_f, dtype=np.int32))
    nE = int(m - f.sum())
    S = np.zeros((nE, nE), dtype=np.complex128)
    pf = np.zeros(1, dtype=np.complex128)
    if lib().oracle_reduced_table(int(N), m, kinds.ctypes.data, ks.ctypes.data, th.ctypes.data, f.ctypes.data,
                                  S.ctypes.data, pf.ctypes.data):
        raise ZeroDivisionError("the F block of the contraction matrix is singular")
    return S, pf[0]


def reduced_batch(S, pf, scale, sels, n_threads=0):
    """scale Pf(A_FF) Pf(S[sel, sel]) for each index list in sels.  Returns (values, threads)."""
    S = np.ascontiguousarray(S, dtype=np.complex128)
    lens = np.array([len(x) for x in sels], dtype=np.int64)
    off = np.zeros(len(sels) + 1, dtype=np.int64)
    np.cumsum(lens, out=off[1:])
    idx = np.ascontiguousarray(np.concatenate([np.asarray(x, np.int32) for x in sels]) if len(sels) and off[-1]
                               else np.zeros(1, np.int32), dtype=np.int32)
    pfa = np.array([pf.real, pf.imag], dtype=np.float64)
    out = np.zeros(len(sels), dtype=np.complex128)
    used = lib().oracle_reduced_batch(S.shape[0], S.ctypes.data, pfa.ctypes.data, float(scale), len(sels),
                                      off.ctypes.data, idx.ctypes.data, out.ctypes.data, int(n_threads))
    return out, used


OP_C, OP_CDAG, OP_D, OP_DDAG, OP_SIGMA1, OP_MAJ_A, OP_MAJ_B = 0, 1, 2, 3, 4, 5, 6
