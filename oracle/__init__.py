"""CPU oracle for arc-consistency enforcement (TEST INFRASTRUCTURE ONLY).

Only tests/, the package's smoke() check and the benchmark's CPU-baseline leg
may import this.  It shares no code with the CUDA library.

  rac(...)         Eq. 1 swept synchronously (Sec. 3), optional Proposition 2
                   restriction; returns (dom, iterations, status[, trace]).
  ac3(...)         AC-3 propagation queue (Mackworth 1977), returns D_ac.
  bruteforce(...)  union of all arc-consistent subsets of D (Sec. 3), |D|<=22.

Status codes mirror the library's: 0 ok, 1 wipe-out, -4 sweep cap reached.
"""
import ctypes
import os

import numpy as np

from .build import build as _build

OK, WIPEOUT, EINVAL, ENOMEM, ETIMEOUT = 0, 1, -1, -2, -4

_libs = {}


def _setup(L):
    vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    L.oracle_rac.restype = ctypes.c_int
    L.oracle_rac.argtypes = [i32, i32, i64, vp, vp, vp, vp, i32, i32, i32, i32, vp, vp, vp, i32, vp]
    L.oracle_ac3.restype = ctypes.c_int
    L.oracle_ac3.argtypes = [i32, i32, i64, vp, vp, vp, vp, vp, vp]
    L.oracle_bruteforce.restype = ctypes.c_int
    L.oracle_bruteforce.argtypes = [i32, i32, i64, vp, vp, vp, vp, vp]
    return L


def load(path=None):
    """Load the oracle library (built on demand); `path` selects another build
    of the same source (the mutation tests load planted-mistake copies)."""
    key = path or "default"
    if key not in _libs:
        _libs[key] = _setup(ctypes.CDLL(path or _build()))
    return _libs[key]


def _prep(scope, rel, dom):
    scope = np.ascontiguousarray(scope, dtype=np.int32).reshape(-1, 2)
    rel = np.ascontiguousarray(rel, dtype=np.uint32)
    dom = np.ascontiguousarray(dom, dtype=np.uint32)
    return scope, rel, dom


def rac(n, d, scope, rel, dom, stop_on_wipeout=False, incremental=False, max_sweeps=0,
        threads=1, trace=False, trace_cap=None, lib=None):
    """Eq. 1 to its fixpoint.  Returns (dom_out, iterations, status) and, with
    trace=True, also (per-sweep domains (K, n), per-sweep removal counts (K,))."""
    L = lib or load()
    scope, rel, dom = _prep(scope, rel, dom)
    m = scope.shape[0]
    out = np.empty(n, dtype=np.uint32)
    it = ctypes.c_int32()
    st = ctypes.c_int32()
    cap = 0
    tr = rem = None
    if trace:
        cap = trace_cap or (n * d + 2)
        tr = np.zeros((cap, n), dtype=np.uint32)
        rem = np.zeros(cap, dtype=np.int64)
    rc = L.oracle_rac(n, d, m, scope.ctypes.data, rel.ctypes.data, dom.ctypes.data,
                      out.ctypes.data, int(bool(stop_on_wipeout)), int(bool(incremental)),
                      int(max_sweeps), int(threads), ctypes.addressof(it), ctypes.addressof(st),
                      tr.ctypes.data if trace else None, cap,
                      rem.ctypes.data if trace else None)
    if rc != 0:
        raise ValueError("oracle_rac rejected its input: %d" % rc)
    if trace:
        k = min(it.value, cap)
        return out, it.value, st.value, tr[:k].copy(), rem[:k].copy()
    return out, it.value, st.value


def ac3(n, d, scope, rel, dom, lib=None):
    """AC-3.  Returns (dom_out, revisions, status)."""
    L = lib or load()
    scope, rel, dom = _prep(scope, rel, dom)
    out = np.empty(n, dtype=np.uint32)
    revs = ctypes.c_int64()
    st = ctypes.c_int32()
    rc = L.oracle_ac3(n, d, scope.shape[0], scope.ctypes.data, rel.ctypes.data, dom.ctypes.data,
                      out.ctypes.data, ctypes.addressof(revs), ctypes.addressof(st))
    if rc != 0:
        raise ValueError("oracle_ac3 rejected its input: %d" % rc)
    return out, revs.value, st.value


def bruteforce(n, d, scope, rel, dom, lib=None):
    """Union of every arc-consistent subset of D.  Returns (dom_out, status)."""
    L = lib or load()
    scope, rel, dom = _prep(scope, rel, dom)
    out = np.empty(n, dtype=np.uint32)
    st = ctypes.c_int32()
    rc = L.oracle_bruteforce(n, d, scope.shape[0], scope.ctypes.data, rel.ctypes.data,
                             dom.ctypes.data, out.ctypes.data, ctypes.addressof(st))
    if rc != 0:
        raise ValueError("oracle_bruteforce rejected its input: %d" % rc)
    return out, st.value
