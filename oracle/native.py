"""ctypes loader for the oracle's plain C per-row code (test infrastructure only)."""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "og_rows.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_OUT_DIR, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile og_rows.c with gcc (plain IEEE FP64: no fast-math, no contraction)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
               "-ffp-contract=off", "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        dp = ctypes.POINTER(ctypes.c_double)
        up = ctypes.POINTER(ctypes.c_uint64)
        ip = ctypes.POINTER(ctypes.c_int)
        L.oracle_connections.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, dp,
                                         ctypes.c_uint64, ctypes.c_int, up, dp, ip]
        L.oracle_connections.restype = ctypes.c_int
        L.oracle_rows.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                  dp, dp, dp, up, ctypes.c_int64, dp, dp, dp, dp]
        L.oracle_rows.restype = ctypes.c_int
        L.oracle_rows_abs.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                      dp, dp, dp, up, ctypes.c_int64, dp, dp, dp, ctypes.c_int]
        L.oracle_rows_abs.restype = ctypes.c_int
        _lib = L
    return _lib


def _p(a, t):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(t))


def connections(n_orb, n_alpha, n_beta, h, eri, det):
    """(dets, H elements, signs) of every determinant connected to ``det`` (diagonal first)."""
    h = np.ascontiguousarray(h, dtype=np.float64)
    eri = np.ascontiguousarray(eri, dtype=np.float64)
    cap = 1 << 16
    od = np.zeros(cap, dtype=np.uint64)
    oh = np.zeros(cap)
    osg = np.zeros(cap, dtype=np.int32)
    n = lib().oracle_connections(n_orb, n_alpha, n_beta, _p(h, ctypes.c_double),
                                 _p(eri, ctypes.c_double), int(det), cap,
                                 _p(od, ctypes.c_uint64), _p(oh, ctypes.c_double),
                                 _p(osg, ctypes.c_int))
    if n < 0:
        raise RuntimeError("oracle_connections failed")
    return od[:n].copy(), oh[:n].copy(), osg[:n].copy()


def rows(n_orb, n_alpha, n_beta, n_hidden, h, eri, theta, dets, want_o=True, want_g=True):
    """Per-row ln psi, O, E_loc, G (O and G: n_rows x (Nh+1)(M+1), or None)."""
    h = np.ascontiguousarray(h, dtype=np.float64)
    eri = np.ascontiguousarray(eri, dtype=np.float64)
    theta = np.ascontiguousarray(theta, dtype=np.float64)
    dets = np.ascontiguousarray(dets, dtype=np.uint64)
    nr = dets.shape[0]
    p1 = (n_hidden + 1) * (2 * n_orb + 1)
    lnpsi = np.zeros(nr)
    eloc = np.zeros(nr)
    O = np.zeros((nr, p1)) if want_o else None
    G = np.zeros((nr, p1)) if want_g else None
    rc = lib().oracle_rows(n_orb, n_alpha, n_beta, n_hidden, _p(h, ctypes.c_double),
                           _p(eri, ctypes.c_double), _p(theta, ctypes.c_double),
                           _p(dets, ctypes.c_uint64), nr, _p(lnpsi, ctypes.c_double),
                           _p(O, ctypes.c_double), _p(eloc, ctypes.c_double),
                           _p(G, ctypes.c_double))
    if rc != 0:
        raise RuntimeError(f"oracle_rows failed ({rc})")
    return lnpsi, O, eloc, G


def rows_abs(n_orb, n_alpha, n_beta, n_hidden, h, eri, theta, dets, union_occ=False):
    """Condition scales of the per-row quantities: (sum_x' |c_x'|, sum_x' |c_x'| Oa(x'), Oa(x))
    with c_x' = H_xx' psi(x')/psi(x) and Oa the first-order rounding scale of the O row
    (|tanh z| + (1 - tanh^2 z) (|b| + sum |W x|) on hidden rows, |O| elsewhere).
    union_occ: in the G scale, Oa(x') takes its visible factors from x' | x."""
    h = np.ascontiguousarray(h, dtype=np.float64)
    eri = np.ascontiguousarray(eri, dtype=np.float64)
    theta = np.ascontiguousarray(theta, dtype=np.float64)
    dets = np.ascontiguousarray(dets, dtype=np.uint64)
    nr = dets.shape[0]
    p1 = (n_hidden + 1) * (2 * n_orb + 1)
    ea = np.zeros(nr)
    ga = np.zeros((nr, p1))
    oa = np.zeros((nr, p1))
    rc = lib().oracle_rows_abs(n_orb, n_alpha, n_beta, n_hidden, _p(h, ctypes.c_double),
                               _p(eri, ctypes.c_double), _p(theta, ctypes.c_double),
                               _p(dets, ctypes.c_uint64), nr, _p(ea, ctypes.c_double),
                               _p(ga, ctypes.c_double), _p(oa, ctypes.c_double),
                               int(bool(union_occ)))
    if rc != 0:
        raise RuntimeError(f"oracle_rows_abs failed ({rc})")
    return ea, ga, oa
