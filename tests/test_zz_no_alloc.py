"""rac_enforce_noalloc, the entry point for callers that cannot allocate
device memory while they enforce (a process whose device memory another
allocator has reserved, or a loop that cannot take the synchronisation
cudaMalloc may imply): it must give exactly what rac_enforce gives, call
after call, although every call reuses the same static scratch array (GPU).

This file is collected last so that a run stopping at the first failure has
already run every other test."""
import time

import numpy as np
import pytest

import racgen
import paper_2407_11388_b300 as rac
from gpu_helpers import from_dev, oracle_enforce, to_dev, torch

pytestmark = pytest.mark.gpu


def _via(entry, net, dom, flags):
    T = torch()
    din = to_dev(dom)
    dout = T.empty_like(din)
    it = T.full((1,), -7, dtype=T.int32, device="cuda:0")
    st = T.full((1,), -7, dtype=T.int32, device="cuda:0")
    entry(net, din, dout, it, st, flags=flags)
    T.cuda.synchronize()
    return from_dev(dout), int(it.item()), int(st.item())


def test_noalloc_matches_enforce_on_consecutive_calls():
    from paper_2407_11388_b300.build import build
    build()
    n, d = 400, 16
    net_np = racgen.random_network(12, 0, n, d, 0.6, 0.55)
    states = [racgen.assignment_state(12, 0, s, n, d) for s in range(4)]
    states.append(racgen.full_domain(n, d))
    with rac.Network(n, d, net_np.scope, net_np.rel) as net:
        for flags in (0, rac.INCREMENTAL, rac.STOP_ON_WIPEOUT):
            # two calls in a row on the same input, then different inputs in a
            # row: leftovers of one call in the shared array must not leak
            for dom in [states[0], states[0]] + states[1:]:
                want = _via(rac.enforce, net, dom, flags)
                got = _via(rac.enforce_noalloc, net, dom, flags)
                assert np.array_equal(got[0], want[0]), flags
                assert got[1:] == want[1:], (flags, got[1:], want[1:])
        assert max(_via(rac.enforce, net, s, 0)[1] for s in states) >= 3


def test_noalloc_on_a_packed_network():
    """The same with the network's relation rows packed (d = 20)."""
    n, d = 300, 20
    net_np = racgen.random_network(13, 0, n, d, 0.6, 0.45)
    states = [racgen.full_domain(n, d)] + [racgen.assignment_state(13, 0, s, n, d)
                                            for s in range(3)]
    with rac.Network(n, d, net_np.scope, net_np.rel,
                     layout=rac.LAYOUT_BITS | rac.LAYOUT_PACKED) as net:
        for flags in (0, rac.INCREMENTAL):
            for dom in states:
                want = oracle_enforce(n, d, net_np.scope, net_np.rel, dom, flags)
                got = _via(rac.enforce_noalloc, net, dom, flags)
                assert np.array_equal(got[0], want[0][0]), flags
                assert got[1:] == (want[1][0], want[2][0]), (flags, got[1:])


def test_noalloc_rejects_networks_above_its_limit():
    n = rac.NOALLOC_MAX_VARS + 1
    scope = np.array([[0, n - 1]], np.int32)
    rel = np.array([[1, 2]], np.uint32)
    T = torch()
    with rac.Network(n, 2, scope, rel) as net:
        buf = to_dev(racgen.full_domain(n, 2))
        it = T.empty(1, dtype=T.int32, device="cuda:0")
        L = rac.lib()
        rc = L.rac_enforce_noalloc(net.handle, buf.data_ptr(), buf.data_ptr(), it.data_ptr(),
                                   it.data_ptr(), 0, 0, None)
        assert rc == rac.EINVAL
        assert "65536" in rac.last_error()


def test_noalloc_refuses_the_tensor_kernel():
    n, d = 40, 8
    net_np = racgen.random_network(3, 0, n, d, 0.5, 0.3)
    T = torch()
    with rac.Network(n, d, net_np.scope, net_np.rel) as net:
        buf = to_dev(racgen.full_domain(n, d))
        it = T.empty(1, dtype=T.int32, device="cuda:0")
        rc = rac.lib().rac_enforce_noalloc(net.handle, buf.data_ptr(), buf.data_ptr(),
                                           it.data_ptr(), it.data_ptr(), 0,
                                           rac.KERNEL_TENSOR, None)
        assert rc == rac.ENOTSUP
        assert "bit-packed" in rac.last_error()


def test_noalloc_wait_that_runs_out_does_not_poison_the_next_call():
    """A bounded device wait made to run out (one CTA withholds its barrier
    arrival under the test hook, 50 ms limit) gives RAC_EBARRIER; the next
    call resets the shared array, error word included, and matches the
    oracle."""
    T = torch()
    n, d = 300, 12
    net_np = racgen.random_network(8, 0, n, d, 0.5, 0.5)
    dom = racgen.assignment_state(8, 0, 1, n, d)
    want = oracle_enforce(n, d, net_np.scope, net_np.rel, dom)
    with rac.Network(n, d, net_np.scope, net_np.rel) as net:
        t0 = time.perf_counter()
        got = _via(rac.enforce_noalloc, net, dom, rac.TEST_WITHHOLD_ARRIVAL)
        assert got[2] == rac.EBARRIER
        assert time.perf_counter() - t0 < 1.5, "the wait limit under the test hook is 50 ms"
        for _ in range(2):
            out, it, st = _via(rac.enforce_noalloc, net, dom, 0)
            assert np.array_equal(out, want[0][0])
            assert it == want[1][0] and st == want[2][0]
