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
LAYOUT_FP8 = 0x2  # the tensor-core kernel's operand store, built at creation
LAYOUT_PACKED = 0x4  # relation rows packed back to back (d <= 28: fewer bytes per sweep)


def LAYOUT_ROWS(log2_rows):
    """layout flag: relation tiles of 2**log2_rows rows (RAC_LAYOUT_ROWS)."""
    return (int(log2_rows) + 1) << 8


def LAYOUT_MAX_CTAS(ctas):
    """layout flag: at most `ctas` CTAs per launch (RAC_LAYOUT_MAX_CTAS)."""
    return int(ctas) << 16
STOP_ON_WIPEOUT = 0x1
INCREMENTAL = 0x2
VERIFY_FULL = 0x4  # rac_enforce_learned: literal full verification sweep (see include/rac.h)
KERNEL_TENSOR = 0x10  # tcgen05 tensor-core kernel (see include/rac.h)
TEST_WITHHOLD_ARRIVAL = 0x80000000  # failure-detection test hook (see include/rac.h)

STATUS_NAMES = {OK: "ok", WIPEOUT: "wipeout", EINVAL: "einval", ENOMEM: "enomem",
                ECUDA: "ecuda", ETIMEOUT: "etimeout", EBARRIER: "ebarrier", ENOTSUP: "enotsup"}

ABI_FUNCTIONS = ("rac_create_network", "rac_create_network_u8", "rac_destroy", "rac_enforce", "rac_enforce_batch",
                 "rac_enforce_host", "rac_enforce_noalloc", "rac_network_info", "rac_last_error",
                 "rac_plan_create", "rac_plan_enforce", "rac_plan_destroy", "rac_assign_enforce",
                 "rac_predictor_num_params", "rac_predictor_create", "rac_predictor_destroy",
                 "rac_predictor_set_weights", "rac_predictor_get_weights",
                 "rac_predictor_gradient", "rac_predictor_train", "rac_predictor_predict",
                 "rac_enforce_learned", "rac_combine_partials", "rac_search")
NOALLOC_MAX_VARS = 65536
PREDICTOR_FEATURES = 8
PREDICTOR_PARAMS = 4801


class RacTrace(ctypes.Structure):
    """struct rac_trace of include/rac.h (device pointers)."""
    _fields_ = [("features", ctypes.c_void_p), ("label", ctypes.c_void_p),
                ("logit", ctypes.c_void_p), ("where", ctypes.c_void_p),
                ("capacity", ctypes.c_int64), ("count", ctypes.c_void_p),
                ("evaluated", ctypes.c_void_p)]


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
        L.rac_create_network_u8.restype = i32
        L.rac_create_network_u8.argtypes = [i32, i32, i64, vp, vp, u32, ctypes.POINTER(vp)]
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
        L.rac_search.restype = i32
        L.rac_search.argtypes = [vp, vp, i64, u32, vp, vp, vp, vp, vp, vp, vp, i64]
        L.rac_combine_partials.restype = i32
        L.rac_combine_partials.argtypes = [i32, i32, vp, vp, vp, vp, vp]
        L.rac_network_info.restype = i32
        L.rac_network_info.argtypes = [vp, ctypes.POINTER(i64), i32]
        L.rac_last_error.restype = ctypes.c_char_p
        L.rac_last_error.argtypes = []
        f32, u64 = ctypes.c_float, ctypes.c_uint64
        L.rac_predictor_num_params.restype = i32
        L.rac_predictor_num_params.argtypes = []
        L.rac_predictor_create.restype = i32
        L.rac_predictor_create.argtypes = [u64, ctypes.POINTER(vp)]
        L.rac_predictor_destroy.restype = None
        L.rac_predictor_destroy.argtypes = [vp]
        L.rac_predictor_set_weights.restype = i32
        L.rac_predictor_set_weights.argtypes = [vp, vp]
        L.rac_predictor_get_weights.restype = i32
        L.rac_predictor_get_weights.argtypes = [vp, vp, i32]
        L.rac_predictor_gradient.restype = i32
        L.rac_predictor_gradient.argtypes = [vp, vp, vp, i64, f32, vp, vp]
        L.rac_predictor_train.restype = i32
        L.rac_predictor_train.argtypes = [vp, vp, vp, i64, i32, i32, f32, f32, u64, vp]
        L.rac_predictor_predict.restype = i32
        L.rac_predictor_predict.argtypes = [vp, vp, i64, vp, i32]
        L.rac_enforce_learned.restype = i32
        L.rac_enforce_learned.argtypes = [vp, i32, vp, vp, vp, vp, i32, u32, vp, f32, i32,
                                          ctypes.POINTER(RacTrace), vp]
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

    scope: (m, 2) int32 host array; rel: either (m, d) uint32 host array, bit
    b of rel[c, a] = R_xy[a][b] for (x, y) = scope[c], or the 0/1 matrices
    themselves, an (m, d, d) uint8 or bool array with rel[c, a, b] =
    R_xy[a][b] (packed by the library: rac_create_network_u8)."""

    def __init__(self, n, d, scope, rel, layout=LAYOUT_BITS, rows=None, max_ctas=None,
                 states=None, plan=False, packed=None):
        """rows: tile rows (a power of two); max_ctas: grid cap of the
        network's launches; packed: relation rows packed back to back
        (LAYOUT_PACKED) or a word each.  None takes the autotuned table's
        choice for this (d, density, states per launch) if one is installed
        (tile_table.json), else the library default (a word per row unless
        `layout` has LAYOUT_PACKED); `states` is the number of domain states
        the caller expects to enforce per launch (1 if not given), `plan`
        whether the network is to be enforced with others in multi-network
        plans."""
        scope = np.ascontiguousarray(scope, dtype=np.int32).reshape(-1, 2)
        rel = np.asarray(rel)
        if rel.ndim == 3:
            if rel.dtype not in (np.uint8, np.bool_):
                raise RacError(EINVAL, "0/1 relation matrices must be uint8 or bool")
            rel = np.ascontiguousarray(rel.view(np.uint8) if rel.dtype == np.bool_ else rel)
            create = lib().rac_create_network_u8
            if rel.shape[1:] != (d, d):
                raise RacError(EINVAL, "relation matrices must be d x d")
        else:
            rel = np.ascontiguousarray(rel, dtype=np.uint32).reshape(-1, d)
            create = lib().rac_create_network
        if rel.shape[0] != scope.shape[0]:
            raise RacError(EINVAL, "scope and rel disagree on the number of constraints")
        m = scope.shape[0]
        if packed is None and not (int(layout) & LAYOUT_PACKED):
            from .autotune import table_packed
            packed = table_packed(int(d), m / max(1.0, n * (n - 1) / 2.0), int(states or 1),
                                  kind="plan" if plan else "single", m=m)
        if packed:
            layout = int(layout) | LAYOUT_PACKED
        if (rows is None and not (int(layout) & 0xF00)) or \
                (max_ctas is None and not (int(layout) & 0xFFFF0000)):
            from .autotune import table_choice
            t_rows, t_ctas = table_choice(int(d), m / max(1.0, n * (n - 1) / 2.0),
                                          int(states or 1), kind="plan" if plan else "single",
                                          packed=bool(int(layout) & LAYOUT_PACKED), m=m)
            if rows is None and not (int(layout) & 0xF00):
                rows = t_rows
            if max_ctas is None and not (int(layout) & 0xFFFF0000):
                max_ctas = t_ctas
        if max_ctas is not None:
            max_ctas = int(max_ctas)
            if not 1 <= max_ctas <= 65535:
                raise RacError(EINVAL, "max_ctas must be in [1, 65535]")
            layout = int(layout) | LAYOUT_MAX_CTAS(max_ctas)
        if rows is not None:
            rows = int(rows)
            if rows < 2 or rows > 32 or rows & (rows - 1):
                raise RacError(EINVAL, "tile rows must be a power of two in [2, 32]")
            layout = int(layout) | LAYOUT_ROWS(rows.bit_length() - 1)
        h = ctypes.c_void_p()
        _check(create(int(n), int(d), scope.shape[0], scope.ctypes.data, rel.ctypes.data,
                      int(layout), ctypes.byref(h)),
               create.__name__)
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
    device memory at call time (a process whose device memory another
    allocator has reserved, a loop that cannot take the synchronisation
    cudaMalloc may imply).  At most NOALLOC_MAX_VARS variables; calls must not
    overlap on the GPU; the first call on a device should precede any stream
    capture."""
    _check(lib().rac_enforce_noalloc(net.handle, _ptr(dom_in), _ptr(dom_out), _ptr(iterations),
                                     _ptr(status), int(max_sweeps), int(flags), _stream(stream)),
           "rac_enforce_noalloc")


def run_search(net, dom0, max_nodes=10_000, flags=0, stream=None):
    """rac_search: Algorithm 2's backtrack search with the loop inside the
    library.  dom0: host uint32 words (n).  Returns a dict: solution (uint32
    words or None), found, exhausted, nodes, root (sweeps, status) and steps
    (nodes x 5 int32: level, variable, value, sweep count, status)."""
    dom0 = np.ascontiguousarray(dom0, dtype=np.uint32).reshape(-1)
    if dom0.size != net.n:
        raise RacError(EINVAL, "search: dom0 must have n words")
    sol = np.zeros(net.n, np.uint32)
    found, exhausted = ctypes.c_int32(), ctypes.c_int32()
    nodes = ctypes.c_int64()
    root = np.zeros(2, np.int32)
    steps = np.zeros((max(int(max_nodes), 1), 5), np.int32)
    _check(lib().rac_search(net.handle, dom0.ctypes.data, int(max_nodes), int(flags),
                            _stream(stream), sol.ctypes.data, ctypes.byref(found),
                            ctypes.byref(exhausted), ctypes.byref(nodes), root.ctypes.data,
                            steps.ctypes.data, int(max_nodes)),
           "rac_search")
    return {"solution": sol if found.value else None, "found": bool(found.value),
            "exhausted": bool(exhausted.value), "nodes": int(nodes.value),
            "root": (int(root[0]), int(root[1])), "steps": steps[:nodes.value].copy()}


def combine_partials(partials, dom_prev, dom_next, flags, stream=None):
    """rac_combine_partials: dom_next = dom_prev AND every row of partials
    (n_parts, n_vars); flags[0] = some domain changed, flags[1] = some domain
    empty (asynchronous on `stream`)."""
    n_parts, n_vars = (int(v) for v in partials.shape)
    if dom_prev.numel() != n_vars or dom_next.numel() != n_vars or flags.numel() < 2:
        raise RacError(EINVAL, "combine_partials: sizes disagree")
    _check(lib().rac_combine_partials(n_parts, n_vars, _ptr(partials), _ptr(dom_prev),
                                      _ptr(dom_next), _ptr(flags), _stream(stream)),
           "rac_combine_partials")


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


class Predictor:
    """The active-block predictor (rac_predictor_*): an MLP 8 -> 64 -> 64 -> 1
    with BF16 weights, trained and evaluated by the library's kernels."""

    def __init__(self, seed=0):
        h = ctypes.c_void_p()
        _check(lib().rac_predictor_create(int(seed), ctypes.byref(h)), "rac_predictor_create")
        self.handle = h.value

    @staticmethod
    def num_params():
        return int(lib().rac_predictor_num_params())

    def set_weights(self, params):
        params = np.ascontiguousarray(params, dtype=np.float32).reshape(-1)
        if params.shape[0] != PREDICTOR_PARAMS:
            raise RacError(EINVAL, "expected %d parameters" % PREDICTOR_PARAMS)
        _check(lib().rac_predictor_set_weights(self.handle, params.ctypes.data),
               "rac_predictor_set_weights")

    def get_weights(self, bf16=False):
        out = np.empty(PREDICTOR_PARAMS, dtype=np.float32)
        _check(lib().rac_predictor_get_weights(self.handle, out.ctypes.data, int(bool(bf16))),
               "rac_predictor_get_weights")
        return out

    def gradient(self, x, y, pos_weight=1.0):
        """Mean loss and gradient over the samples (x: (N, 8) float32 CUDA
        tensor, y: (N,) float32 CUDA tensor).  Returns (grad, loss)."""
        grad = np.empty(PREDICTOR_PARAMS, dtype=np.float32)
        loss = ctypes.c_float()
        _check(lib().rac_predictor_gradient(self.handle, _ptr(x), _ptr(y), int(y.numel()),
                                            float(pos_weight), grad.ctypes.data,
                                            ctypes.addressof(loss)),
               "rac_predictor_gradient")
        return grad, float(loss.value)

    def train(self, x, y, steps, batch=4096, lr=1e-3, pos_weight=1.0, seed=0):
        """Adam steps on minibatches drawn from (x, y); returns the last
        minibatch loss."""
        loss = ctypes.c_float()
        _check(lib().rac_predictor_train(self.handle, _ptr(x), _ptr(y), int(y.numel()), int(steps),
                                         int(batch), float(lr), float(pos_weight), int(seed),
                                         ctypes.addressof(loss)),
               "rac_predictor_train")
        return float(loss.value)

    def predict(self, x, logits, tensor_cores=True):
        _check(lib().rac_predictor_predict(self.handle, _ptr(x), int(x.shape[0]), _ptr(logits),
                                           int(bool(tensor_cores))),
               "rac_predictor_predict")

    def close(self):
        if getattr(self, "handle", None):
            lib().rac_predictor_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Trace:
    """Device buffers for the records of rac_enforce_learned (struct
    rac_trace), held as torch tensors on the current device."""

    def __init__(self, capacity):
        import torch
        dev = torch.device("cuda", torch.cuda.current_device())
        self.capacity = int(capacity)
        c = max(1, self.capacity)
        self.features = torch.zeros((c, PREDICTOR_FEATURES), dtype=torch.float32, device=dev)
        self.label = torch.zeros(c, dtype=torch.float32, device=dev)
        self.logit = torch.zeros(c, dtype=torch.float32, device=dev)
        self.where = torch.zeros((c, 4), dtype=torch.int32, device=dev)
        self.counters = torch.zeros(2, dtype=torch.int64, device=dev)  # count, evaluated

    def struct(self):
        return RacTrace(self.features.data_ptr(), self.label.data_ptr(), self.logit.data_ptr(),
                        self.where.data_ptr(), self.capacity, self.counters.data_ptr(),
                        self.counters.data_ptr() + 8)

    def count(self):
        return int(self.counters[0].item())

    def evaluated(self):
        return int(self.counters[1].item())

    def records(self):
        """Host copies of the stored records: dict of numpy arrays."""
        k = min(self.count(), self.capacity)
        return {"features": self.features[:k].cpu().numpy(), "label": self.label[:k].cpu().numpy(),
                "logit": self.logit[:k].cpu().numpy(), "where": self.where[:k].cpu().numpy()}


def enforce_learned(net, dom_in, dom_out, sweeps, status, predictor=None, threshold=0.0,
                    trace=None, max_sweeps=0, flags=0, n_states=None, stream=None,
                    min_scored=0):
    """rac_enforce_learned: states s at word s * n of dom_in / dom_out, with
    learned gating (predictor) or, with predictor=None, Proposition-2 sweeps
    (the mode that records training traces).  min_scored: a 32-state group
    of a slab with fewer gated candidates is evaluated unscored.
    Asynchronous on `stream`."""
    if n_states is None:
        n_states = dom_in.numel() // net.n
    tr = trace.struct() if trace is not None else None
    _check(lib().rac_enforce_learned(net.handle, int(n_states), _ptr(dom_in), _ptr(dom_out),
                                     _ptr(sweeps), _ptr(status), int(max_sweeps), int(flags),
                                     predictor.handle if predictor is not None else None,
                                     float(threshold), int(min_scored),
                                     ctypes.byref(tr) if tr is not None else None,
                                     _stream(stream)),
           "rac_enforce_learned")
