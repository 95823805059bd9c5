"""Arc-consistency enforcement on binary CSPs for B300 (sm_103a).

A thin ctypes binding over librac.so, whose C ABI is declared in
include/rac.h.  It only marshals arguments: every step of the enforcement
runs in the library's CUDA kernels.  Device buffers are passed as torch
tensors (their data_ptr()) or as raw integer addresses; `stream` is a
torch.cuda.Stream, a raw cudaStream_t integer, or None for torch's current
stream.

Recurrent arc consistency (Eq. 1, Sec. 3 of the paper): each sweep removes
every value (x,a) that has lost all its supports on some constraint c_xy,
reading only the previous sweep's domains, until a sweep removes nothing.
"""
import ctypes
import os

import numpy as np

from .build import LIB as _LIB_PATH

OK, WIPEOUT = 0, 1
EINVAL, ENOMEM, ECUDA, ETIMEOUT, EBARRIER, ENOTSUP = -1, -2, -3, -4, -5, -6
LAYOUT_BITS = 0x1
STOP_ON_WIPEOUT = 0x1
INCREMENTAL = 0x2
KERNEL_TENSOR = 0x10  # tcgen05 tensor-core kernel (see include/rac.h)
TEST_WITHHOLD_ARRIVAL = 0x80000000  # failure-detection test hook (see include/rac.h)

STATUS_NAMES = {OK: "ok", WIPEOUT: "wipeout", EINVAL: "einval", ENOMEM: "enomem",
                ECUDA: "ecuda", ETIMEOUT: "etimeout", EBARRIER: "ebarrier", ENOTSUP: "enotsup"}

ABI_FUNCTIONS = ("rac_create_network", "rac_destroy", "rac_enforce", "rac_enforce_batch",
                 "rac_enforce_host", "rac_enforce_noalloc", "rac_network_info", "rac_last_error",
                 "rac_plan_create", "rac_plan_enforce", "rac_plan_destroy", "rac_assign_enforce")
NOALLOC_MAX_VARS = 65536


class RacError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%s)" % (msg, STATUS_NAMES.get(code, code)))
        self.code = code


_lib = None


def lib():
    """Load librac.so.  There is no fallback: a missing library is an error."""
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB_PATH):
            raise RacError(ENOTSUP, "librac.so is not built (python -m paper_2407_11388_b300.build)")
        L = ctypes.CDLL(_LIB_PATH)
        vp, i32, i64, u32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32
        L.rac_create_network.restype = i32
        L.rac_create_network.argtypes = [i32, i32, i64, vp, vp, u32, ctypes.POINTER(vp)]
        L.rac_destroy.restype = None
        L.rac_destroy.argtypes = [vp]
        L.rac_enforce.restype = i32
        L.rac_enforce.argtypes = [vp, vp, vp, vp, vp, i32, u32, vp]
        L.rac_enforce_batch.restype = i32
        L.rac_enforce_batch.argtypes = [vp, i32, i32, vp, vp, vp, vp, vp, vp, i32, u32, vp]
        L.rac_enforce_host.restype = i32
        L.rac_enforce_host.argtypes = [vp, i32, vp, vp, vp, vp, i32, u32, vp]
        L.rac_enforce_noalloc.restype = i32
        L.rac_enforce_noalloc.argtypes = [vp, vp, vp, vp, vp, i32, u32, vp]
        L.rac_plan_create.restype = i32
        L.rac_plan_create.argtypes = [vp, i32, i32, vp, vp, ctypes.POINTER(vp)]
        L.rac_plan_enforce.restype = i32
        L.rac_plan_enforce.argtypes = [vp, vp, vp, vp, vp, i32, u32, vp]
        L.rac_plan_destroy.restype = None
        L.rac_plan_destroy.argtypes = [vp]
        L.rac_assign_enforce.restype = i32
        L.rac_assign_enforce.argtypes = [vp, vp, vp, i32, i32, vp, vp, i32, u32, vp]
        L.rac_network_info.restype = i32
        L.rac_network_info.argtypes = [vp, ctypes.POINTER(i64), i32]
        L.rac_last_error.restype = ctypes.c_char_p
        L.rac_last_error.argtypes = []
        _lib = L
    return _lib


def last_error():
    return lib().rac_last_error().decode()


def _check(code, what):
    if code < 0:
        raise RacError(code, "%s failed: %s" % (what, last_error()))
    return code


def _ptr(x):
    """Device address of a torch tensor (or an int address)."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        if not x.is_cuda:
            raise RacError(EINVAL, "expected a CUDA tensor")
        if not x.is_contiguous():
            raise RacError(EINVAL, "expected a contiguous tensor")
        return x.data_ptr()
    raise TypeError("cannot take a device address of %r" % type(x))


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


class Network:
    """A constraint network resident on the current CUDA device.

    scope: (m, 2) int32 host array; rel: (m, d) uint32 host array, bit b of
    rel[c, a] = R_xy[a][b] for (x, y) = scope[c]."""

    def __init__(self, n, d, scope, rel, layout=LAYOUT_BITS):
        scope = np.ascontiguousarray(scope, dtype=np.int32).reshape(-1, 2)
        rel = np.ascontiguousarray(rel, dtype=np.uint32).reshape(-1, d)
        if rel.shape[0] != scope.shape[0]:
            raise RacError(EINVAL, "scope and rel disagree on the number of constraints")
        h = ctypes.c_void_p()
        _check(lib().rac_create_network(int(n), int(d), scope.shape[0], scope.ctypes.data,
                                        rel.ctypes.data, int(layout), ctypes.byref(h)),
               "rac_create_network")
        self.handle = h.value
        self.n, self.d, self.m = int(n), int(d), int(scope.shape[0])

    def info(self):
        buf = (ctypes.c_int64 * 7)()
        k = lib().rac_network_info(self.handle, buf, 7)
        keys = ("n", "d", "m", "rel_bytes", "n_slabs", "rows_per_slab", "words_per_relation")
        return dict(zip(keys[:k], list(buf)[:k]))

    def close(self):
        if getattr(self, "handle", None):
            lib().rac_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def create_network(n, d, scope, rel, layout=LAYOUT_BITS):
    return Network(n, d, scope, rel, layout)


def enforce(net, dom_in, dom_out, iterations, status, max_sweeps=0, flags=0, stream=None):
    """One domain state on the device: rac_enforce (asynchronous on `stream`)."""
    _check(lib().rac_enforce(net.handle, _ptr(dom_in), _ptr(dom_out), _ptr(iterations),
                             _ptr(status), int(max_sweeps), int(flags), _stream(stream)),
           "rac_enforce")


def assign_enforce(net, dom_in, dom_out, var, value, iterations, status, max_sweeps=0, flags=0,
                   stream=None):
    """One backtrack-search step (Algorithm 2): dom(var) := {value}, then
    enforcement whose first sweep examines only the constraints on var.
    dom_in must be arc consistent (rac_assign_enforce in include/rac.h)."""
    _check(lib().rac_assign_enforce(net.handle, _ptr(dom_in), _ptr(dom_out), int(var), int(value),
                                    _ptr(iterations), _ptr(status), int(max_sweeps), int(flags),
                                    _stream(stream)),
           "rac_assign_enforce")


def enforce_noalloc(net, dom_in, dom_out, iterations, status, max_sweeps=0, flags=0,
                    stream=None):
    """rac_enforce_noalloc: like enforce(), with the library's static scratch
    array instead of an allocated workspace, for callers that cannot allocate
    device memory at call time (for example while a CUDA graph is being
    captured).  At most NOALLOC_MAX_VARS variables; calls must not overlap on
    the GPU; the first call on a device should precede any stream capture."""
    _check(lib().rac_enforce_noalloc(net.handle, _ptr(dom_in), _ptr(dom_out), _ptr(iterations),
                                     _ptr(status), int(max_sweeps), int(flags), _stream(stream)),
           "rac_enforce_noalloc")


def enforce_batch(nets, item_net, item_dom_off, dom_in, dom_out, iterations, status,
                  max_sweeps=0, flags=0, stream=None):
    """Many (network, state) items: rac_enforce_batch (asynchronous on `stream`)."""
    handles = (ctypes.c_void_p * max(1, len(nets)))(*[n.handle for n in nets])
    item_net = np.ascontiguousarray(item_net, dtype=np.int32)
    item_dom_off = np.ascontiguousarray(item_dom_off, dtype=np.int64)
    _check(lib().rac_enforce_batch(handles, len(nets), item_net.shape[0], item_net.ctypes.data,
                                   item_dom_off.ctypes.data, _ptr(dom_in), _ptr(dom_out),
                                   _ptr(iterations), _ptr(status), int(max_sweeps), int(flags),
                                   _stream(stream)),
           "rac_enforce_batch")


class Plan:
    """A fixed batch of (network, state) items enforced in one persistent
    launch (rac_plan_*).  The networks must outlive the plan."""

    def __init__(self, nets, item_net, item_dom_off):
        handles = (ctypes.c_void_p * max(1, len(nets)))(*[n.handle for n in nets])
        item_net = np.ascontiguousarray(item_net, dtype=np.int32)
        item_dom_off = np.ascontiguousarray(item_dom_off, dtype=np.int64)
        h = ctypes.c_void_p()
        _check(lib().rac_plan_create(handles, len(nets), item_net.shape[0], item_net.ctypes.data,
                                     item_dom_off.ctypes.data, ctypes.byref(h)),
               "rac_plan_create")
        self.handle = h.value
        self.nets = list(nets)  # keep the networks alive
        self.n_items = int(item_net.shape[0])

    def enforce(self, dom_in, dom_out, iterations, status, max_sweeps=0, flags=0, stream=None):
        _check(lib().rac_plan_enforce(self.handle, _ptr(dom_in), _ptr(dom_out), _ptr(iterations),
                                      _ptr(status), int(max_sweeps), int(flags), _stream(stream)),
               "rac_plan_enforce")

    def close(self):
        if getattr(self, "handle", None):
            lib().rac_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def enforce_host(net, dom_in, max_sweeps=0, flags=0, stream=None):
    """Host arrays in and out: rac_enforce_host (blocks until done).

    dom_in: (n,) or (B, n) uint32.  Returns (dom_out, iterations, status)."""
    dom_in = np.ascontiguousarray(dom_in, dtype=np.uint32)
    single = dom_in.ndim == 1
    states = dom_in.reshape(-1, net.n)
    out = np.empty_like(states)
    it = np.empty(states.shape[0], dtype=np.int32)
    st = np.empty(states.shape[0], dtype=np.int32)
    _check(lib().rac_enforce_host(net.handle, states.shape[0], states.ctypes.data,
                                  out.ctypes.data, it.ctypes.data, st.ctypes.data,
                                  int(max_sweeps), int(flags), _stream(stream)),
           "rac_enforce_host")
    if single:
        return out[0], int(it[0]), int(st[0])
    return out, it, st
