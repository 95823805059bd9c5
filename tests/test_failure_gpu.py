"""Failure detection without a GPU fault: a device-side wait that runs out
(one CTA withholds its grid-barrier arrival, a flag nobody else sets) must
end the launch with RAC_EBARRIER within its short limit, poison only that
workspace, and leave the CUDA context usable (GPU)."""
import time

import numpy as np
import pytest

import racgen
import paper_2407_11388_b300 as rac
from gpu_helpers import from_dev, oracle_enforce, to_dev, torch

pytestmark = pytest.mark.gpu


def test_bounded_wait_runs_out_and_reports():
    T = torch()
    n, d = 300, 12
    net_np = racgen.random_network(8, 0, n, d, 0.5, 0.5)
    dom = racgen.assignment_state(8, 0, 1, n, d)
    want = oracle_enforce(n, d, net_np.scope, net_np.rel, dom)
    with rac.Network(n, d, net_np.scope, net_np.rel) as net:
        bad_stream = T.cuda.Stream()
        din = to_dev(dom)
        dout = T.empty_like(din)
        it = T.full((1,), -7, dtype=T.int32, device="cuda:0")
        st = T.full((1,), -7, dtype=T.int32, device="cuda:0")
        t0 = time.perf_counter()
        rac.enforce(net, din, dout, it, st, flags=rac.TEST_WITHHOLD_ARRIVAL, stream=bad_stream)
        bad_stream.synchronize()
        elapsed = time.perf_counter() - t0
        assert int(st.item()) == rac.EBARRIER
        assert elapsed < 1.5, "the wait limit under the test hook is 50 ms"
        # the workspace of that stream is poisoned: later calls report at once
        st.fill_(-7)
        rac.enforce(net, din, dout, it, st, stream=bad_stream)
        bad_stream.synchronize()
        assert int(st.item()) == rac.EBARRIER
        # the context and other workspaces still work
        good = T.cuda.Stream()
        st.fill_(-7)
        rac.enforce(net, din, dout, it, st, stream=good)
        good.synchronize()
        assert np.array_equal(from_dev(dout), want[0][0])
        assert int(it.item()) == want[1][0] and int(st.item()) == want[2][0]


def test_bounded_wait_reported_through_the_host_entry_point():
    """The host entry point returns the status the kernel writes into pinned
    memory: a wait that runs out gives RAC_EBARRIER (also on the poisoned
    workspace's next call), and another stream still gets the oracle's
    result."""
    T = torch()
    n, d = 300, 12
    net_np = racgen.random_network(9, 0, n, d, 0.5, 0.5)
    doms = np.array([racgen.assignment_state(9, 0, s, n, d) for s in range(3)])
    want = oracle_enforce(n, d, net_np.scope, net_np.rel, doms)
    with rac.Network(n, d, net_np.scope, net_np.rel) as net:
        bad_stream = T.cuda.Stream()
        _, _, st = rac.enforce_host(net, doms, flags=rac.TEST_WITHHOLD_ARRIVAL, stream=bad_stream)
        assert list(st) == [rac.EBARRIER] * 3
        _, _, st = rac.enforce_host(net, doms, stream=bad_stream)
        assert list(st) == [rac.EBARRIER] * 3
        out, it, st = rac.enforce_host(net, doms, stream=T.cuda.Stream())
        assert np.array_equal(out, want[0]) and list(it) == list(want[1])
        assert list(st) == list(want[2])


def test_bounded_wait_runs_out_in_the_tensor_core_kernel():
    """The tensor-core kernel's grid barrier takes the same hook: a wait that
    runs out gives RAC_EBARRIER within the short limit, the workspace stays
    poisoned, and another stream's workspace still enforces correctly."""
    T = torch()
    n, d = 200, 16
    net_np = racgen.random_network(10, 0, n, d, 0.5, 0.5)
    doms = np.array([racgen.assignment_state(10, 0, s, n, d) for s in range(5)])
    want = oracle_enforce(n, d, net_np.scope, net_np.rel, doms)
    TC = rac.KERNEL_TENSOR
    with rac.Network(n, d, net_np.scope, net_np.rel) as net:
        din = to_dev(doms.reshape(-1))
        dout = T.empty_like(din)
        it = T.full((5,), -7, dtype=T.int32, device="cuda:0")
        st = T.full((5,), -7, dtype=T.int32, device="cuda:0")
        items, offs = np.zeros(5, np.int32), np.arange(5, dtype=np.int64) * n
        bad = T.cuda.Stream()
        t0 = time.perf_counter()
        rac.enforce_batch([net], items, offs, din, dout, it, st,
                          flags=TC | rac.TEST_WITHHOLD_ARRIVAL, stream=bad)
        bad.synchronize()
        assert time.perf_counter() - t0 < 1.5, "the wait limit under the test hook is 50 ms"
        assert list(st.cpu().numpy()) == [rac.EBARRIER] * 5
        good = T.cuda.Stream()
        rac.enforce_batch([net], items, offs, din, dout, it, st, flags=TC, stream=good)
        good.synchronize()
        assert np.array_equal(from_dev(dout).reshape(5, n), want[0])
        assert list(it.cpu().numpy()) == list(want[1]) and list(st.cpu().numpy()) == list(want[2])
