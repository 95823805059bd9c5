"""Seeded synthetic binary-CSP inputs (networks and domain states).

Holds no arc-consistency arithmetic: it only draws random networks in the
format the library boundary takes (scope pairs plus one relation word per
row, bit b of word a = R_xy[a][b]) and domain words (bit a = value a).
The hashing rule is documented in gen.c.
"""
import ctypes
import os
from dataclasses import dataclass

import numpy as np

from .build import build as _build

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build()
        L = ctypes.CDLL(path)
        L.racgen_splitmix64.restype = ctypes.c_uint64
        L.racgen_splitmix64.argtypes = [ctypes.c_uint64]
        L.racgen_key.restype = ctypes.c_uint64
        L.racgen_key.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int,
                                 ctypes.POINTER(ctypes.c_uint64)]
        L.racgen_count_constraints.restype = ctypes.c_int64
        L.racgen_count_constraints.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int32,
                                               ctypes.c_double]
        L.racgen_fill_network.restype = ctypes.c_int
        L.racgen_fill_network.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int32,
                                          ctypes.c_int32, ctypes.c_double, ctypes.c_double,
                                          ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p]
        L.racgen_batch_params.restype = None
        L.racgen_batch_params.argtypes = [ctypes.c_uint64, ctypes.c_uint64,
                                          ctypes.POINTER(ctypes.c_int32),
                                          ctypes.POINTER(ctypes.c_int32),
                                          ctypes.POINTER(ctypes.c_double),
                                          ctypes.POINTER(ctypes.c_double)]
        L.racgen_assignment_state.restype = ctypes.c_int32
        L.racgen_assignment_state.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64,
                                              ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p]
        _lib = L
    return _lib


@dataclass
class Network:
    """A binary CSP: n variables with domain {0..d-1}, m constraints.

    scope: (m, 2) int32, rel: (m, d) uint32 with bit b of rel[c, a] = R[a][b]
    for scope (x, y) = scope[c]."""
    n: int
    d: int
    scope: np.ndarray
    rel: np.ndarray

    @property
    def m(self) -> int:
        return int(self.scope.shape[0])


def splitmix64(z: int) -> int:
    return int(lib().racgen_splitmix64(z & 0xFFFFFFFFFFFFFFFF))


def key(seed: int, tag: int, *fields: int) -> int:
    arr = (ctypes.c_uint64 * max(1, len(fields)))(*[f & 0xFFFFFFFFFFFFFFFF for f in fields])
    return int(lib().racgen_key(seed, tag, len(fields), arr))


def full_word(d: int) -> int:
    return 0xFFFFFFFF if d >= 32 else (1 << d) - 1


def full_domain(n: int, d: int) -> np.ndarray:
    return np.full(n, full_word(d), dtype=np.uint32)


def random_network(seed: int, inst: int, n: int, d: int, density: float, tightness: float) -> Network:
    L = lib()
    m = int(L.racgen_count_constraints(seed, inst, n, float(density)))
    scope = np.empty((m, 2), dtype=np.int32)
    rel = np.empty((m, d), dtype=np.uint32)
    rc = L.racgen_fill_network(seed, inst, n, d, float(density), float(tightness), m,
                               scope.ctypes.data, rel.ctypes.data)
    if rc != 0:
        raise RuntimeError("racgen_fill_network failed: %d" % rc)
    return Network(n, d, scope, rel)


def batch_params(seed: int, inst: int):
    n = ctypes.c_int32()
    d = ctypes.c_int32()
    p = ctypes.c_double()
    t = ctypes.c_double()
    lib().racgen_batch_params(seed, inst, ctypes.byref(n), ctypes.byref(d), ctypes.byref(p),
                              ctypes.byref(t))
    return n.value, d.value, p.value, t.value


def assignment_state(seed: int, inst: int, s: int, n: int, d: int) -> np.ndarray:
    dom = np.empty(n, dtype=np.uint32)
    lib().racgen_assignment_state(seed, inst, s, n, d, dom.ctypes.data)
    return dom
