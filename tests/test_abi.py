"""The C-ABI library loads, exports every symbol include/rac.h declares, and
rejects bad arguments before touching the device (no GPU needed)."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_2407_11388_b300 as rac
from paper_2407_11388_b300.build import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    build()
    return rac.lib()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "rac.h")).read()
    return re.findall(r"^RAC_API\s+[\w\s\*]+?\b(rac_\w+)\s*\(", src, flags=re.M)


def test_every_declared_symbol_is_exported(L):
    names = declared_functions()
    assert set(names) >= set(rac.ABI_FUNCTIONS)
    for name in names:
        assert hasattr(L, name), name
    # and nothing internal leaks out of the library
    out = os.popen("nm -D --defined-only %s" % rac.build.LIB).read()
    exported = set(re.findall(r"\b(rac_\w+)\b", out))
    assert exported == set(names)


def _create(L, n, d, scope, rel, flags=1):
    h = ctypes.c_void_p()
    scope = np.ascontiguousarray(scope, np.int32)
    rel = np.ascontiguousarray(rel, np.uint32)
    rc = L.rac_create_network(n, d, scope.shape[0], scope.ctypes.data, rel.ctypes.data, flags,
                              ctypes.byref(h))
    return rc, h


@pytest.mark.parametrize("case", ["d0", "d33", "n0", "self_loop", "out_of_range", "dup_pair",
                                  "dup_pair_reversed", "bit_above_d", "bad_layout",
                                  "bad_rows_code"])
def test_create_rejects(L, case):
    n, d = 4, 3
    scope = np.array([[0, 1], [1, 2]], np.int32)
    rel = np.full((2, 3), 7, np.uint32)
    flags = 1
    if case == "d0":
        d = 0
    elif case == "d33":
        d = 33
    elif case == "n0":
        n = 0
    elif case == "self_loop":
        scope[1] = (2, 2)
    elif case == "out_of_range":
        scope[1] = (1, 4)
    elif case == "dup_pair":
        scope[1] = (0, 1)
    elif case == "dup_pair_reversed":
        scope[1] = (1, 0)
    elif case == "bit_above_d":
        rel[1, 2] = 8
    elif case == "bad_layout":
        flags = 0x1000
    elif case == "bad_rows_code":
        flags = 1 | (7 << 8)  # RAC_LAYOUT_ROWS takes l <= 5
    rc, h = _create(L, n, d, scope, rel.reshape(2, -1) if d == 3 else np.zeros((2, max(d, 1)), np.uint32), flags)
    assert rc == rac.EINVAL
    assert h.value is None
    assert L.rac_last_error().decode() != ""


def test_null_and_flag_checks(L):
    assert L.rac_enforce(None, None, None, None, None, 0, 0, None) == rac.EINVAL
    assert L.rac_enforce_batch(None, 0, 0, None, None, None, None, None, None, 0, 0, None) == rac.OK
    assert L.rac_enforce_batch(None, 1, 1, None, None, None, None, None, None, 0, 0, None) == rac.EINVAL
    assert L.rac_enforce_host(None, 1, None, None, None, None, 0, 0, None) == rac.EINVAL
    L.rac_destroy(None)  # NULL-safe
    assert L.rac_network_info(None, None, 0) == 0


def test_python_binding_wraps_errors(L):
    with pytest.raises(rac.RacError) as e:
        rac.Network(3, 40, np.zeros((0, 2), np.int32), np.zeros((0, 40), np.uint32))
    assert e.value.code == rac.EINVAL


def test_predictor_entry_points_check_arguments(L):
    assert L.rac_predictor_num_params() == rac.PREDICTOR_PARAMS
    assert L.rac_predictor_create(0, None) == rac.EINVAL
    L.rac_predictor_destroy(None)  # NULL-safe
    assert L.rac_predictor_set_weights(None, None) == rac.EINVAL
    assert L.rac_predictor_get_weights(None, None, 0) == rac.EINVAL
    assert L.rac_predictor_gradient(None, None, None, 0, 1.0, None, None) == rac.EINVAL
    assert L.rac_predictor_train(None, None, None, 0, 1, 1, 1e-3, 1.0, 0, None) == rac.EINVAL
    assert L.rac_predictor_predict(None, None, 1, None, 1) == rac.EINVAL
    assert L.rac_enforce_learned(None, 1, None, None, None, None, 0, 0, None, 0.0, 0, None,
                                 None) == rac.EINVAL
    assert L.rac_last_error().decode() != ""


def test_trace_struct_matches_header():
    """struct rac_trace: four pointers, an int64, two pointers (no padding
    on LP64)."""
    assert ctypes.sizeof(rac.RacTrace) == 7 * 8
    src = open(os.path.join(ROOT, "include", "rac.h")).read()
    body = src[src.index("typedef struct rac_trace {"):src.index("} rac_trace;")]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = re.findall(r"\*?\s*(\w+);", body)
    assert fields == [f[0] for f in rac.RacTrace._fields_]


def test_tile_rows_too_large_rejected(L):
    # 16 rows x 32 columns x 32 words x 4 bytes = 64 KiB > the 32 KiB staging buffer
    rc, h = _create(L, 4, 32, np.array([[0, 1]], np.int32), np.zeros((1, 32), np.uint32),
                    flags=1 | (5 << 8))
    assert rc == rac.EINVAL and h.value is None
    assert "staging buffer" in L.rac_last_error().decode()
    # one row would leave the tile header (2 x rows words) unaligned
    rc, h = _create(L, 4, 8, np.array([[0, 1]], np.int32), np.zeros((1, 8), np.uint32),
                    flags=1 | (1 << 8))
    assert rc == rac.EINVAL and h.value is None
    for rows in (1, 3, 64):
        with pytest.raises(rac.RacError):
            rac.Network(4, 8, np.array([[0, 1]], np.int32), np.zeros((1, 8), np.uint32), rows=rows)


def _create_u8(L, n, d, scope, mats, flags=1):
    h = ctypes.c_void_p()
    scope = np.ascontiguousarray(scope, np.int32)
    mats = np.ascontiguousarray(mats, np.uint8)
    rc = L.rac_create_network_u8(n, d, scope.shape[0], scope.ctypes.data, mats.ctypes.data, flags,
                                 ctypes.byref(h))
    return rc, h


@pytest.mark.parametrize("case", ["entry_2", "entry_255", "d0", "d33", "null_rel", "null_out"])
def test_create_u8_rejects(L, case):
    """Entries other than 0/1 and bad shapes are refused on the host, before
    any device allocation (so this runs without a GPU)."""
    n, d = 4, 3
    scope = np.array([[0, 1], [1, 2]], np.int32)
    mats = np.ones((2, 3, 3), np.uint8)
    if case == "entry_2":
        mats[1, 2, 0] = 2
    elif case == "entry_255":
        mats[0, 0, 2] = 255
    elif case == "d0":
        d = 0
    elif case == "d33":
        d = 33
    if case == "null_rel":
        h = ctypes.c_void_p()
        rc = L.rac_create_network_u8(n, d, 2, scope.ctypes.data, None, 1, ctypes.byref(h))
    elif case == "null_out":
        rc = L.rac_create_network_u8(n, d, 2, scope.ctypes.data, mats.ctypes.data, 1, None)
        h = ctypes.c_void_p()
    else:
        rc, h = _create_u8(L, n, d, scope, mats)
    assert rc == rac.EINVAL
    assert h.value is None
    msg = L.rac_last_error().decode()
    assert msg != ""
    if case.startswith("entry"):
        assert "constraint %d" % (1 if case == "entry_2" else 0) in msg


def test_python_binding_u8_checks(L):
    scope = np.array([[0, 1]], np.int32)
    with pytest.raises(rac.RacError):  # not d x d
        rac.Network(3, 3, scope, np.ones((1, 3, 2), np.uint8))
    with pytest.raises(rac.RacError):  # not 0/1 bytes or bools
        rac.Network(3, 3, scope, np.ones((1, 3, 3), np.float32))
    with pytest.raises(rac.RacError) as e:
        rac.Network(3, 3, scope, np.full((1, 3, 3), 3, np.uint8))
    assert e.value.code == rac.EINVAL


def test_more_constraints_than_pairs_rejected(L):
    """Each unordered pair takes at most one constraint, so n_cons above
    n(n-1)/2 is refused before anything is read or allocated; the same holds
    for sizes no host could hold (no C++ exception crosses the ABI)."""
    scope = np.zeros((1, 2), np.int32)
    rel = np.zeros((1, 3), np.uint32)
    mats = np.zeros((1, 3, 3), np.uint8)
    for n_cons in (7, 1 << 40, (1 << 62) + 5):
        h = ctypes.c_void_p()
        assert L.rac_create_network(4, 3, n_cons, scope.ctypes.data, rel.ctypes.data, 1,
                                    ctypes.byref(h)) == rac.EINVAL
        assert h.value is None and "pairs" in L.rac_last_error().decode()
        assert L.rac_create_network_u8(4, 3, n_cons, scope.ctypes.data, mats.ctypes.data, 1,
                                       ctypes.byref(h)) == rac.EINVAL
        assert h.value is None


def test_binding_constants_match_the_header():
    """Every flag and status constant of the binding has the value rac.h
    defines for it."""
    src = open(os.path.join(ROOT, "include", "rac.h")).read()
    defs = {k: int(v, 0) for k, v in
            re.findall(r"^#define RAC_(\w+)\s+\(?(-?(?:0x[0-9A-Fa-f]+|\d+))u?\)?", src, flags=re.M)}
    checked = 0
    for name, value in defs.items():
        if hasattr(rac, name) and isinstance(getattr(rac, name), int):
            assert getattr(rac, name) == value, name
            checked += 1
    assert checked >= 12
    assert rac.LAYOUT_PACKED == defs["LAYOUT_PACKED"]


def test_packed_rows_change_the_tile_size_rule(L):
    """A tile's size counts the words of its relations: 16 rows of d = 20
    take 40 KiB with a word per row (rejected before anything is allocated)
    but 26 KiB packed (accepted by the size rule; without a GPU the call then
    fails on the device, not on the size)."""
    scope, rel = np.array([[0, 1]], np.int32), np.zeros((1, 20), np.uint32)
    rc, h = _create(L, 4, 20, scope, rel, flags=1 | (5 << 8))
    assert rc == rac.EINVAL and "staging buffer" in L.rac_last_error().decode()
    rc, h = _create(L, 4, 20, scope, rel, flags=1 | rac.LAYOUT_PACKED | (5 << 8))
    assert "staging buffer" not in L.rac_last_error().decode()
    if rc == rac.OK:
        L.rac_destroy(h)
    # 32 rows of d = 20 do not fit even packed (53 KiB)
    rc, h = _create(L, 4, 20, scope, rel, flags=1 | rac.LAYOUT_PACKED | (6 << 8))
    assert rc == rac.EINVAL and "staging buffer" in L.rac_last_error().decode()
