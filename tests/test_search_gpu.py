"""The search driver (Algorithm 2) on the device against the same search
run with the CPU oracle: the same assignments, the same sweep counts per
assignment (the seeded first sweep must not change them), the same outcome
(GPU)."""
import numpy as np
import pytest

import oracle
import racgen
from oracle.search import dfs as oracle_dfs
import paper_2407_11388_b300 as rac
from paper_2407_11388_b300.search import dfs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("seed,n,d,p,t", [(1, 40, 8, 0.3, 0.35), (2, 60, 10, 0.5, 0.3),
                                          (3, 90, 6, 0.2, 0.25), (4, 150, 12, 0.8, 0.2)])
def test_search_matches_oracle(seed, n, d, p, t):
    net_np = racgen.random_network(seed, 0, n, d, p, t)
    dom0 = racgen.full_domain(n, d)
    want = oracle_dfs(n, d, net_np.scope, net_np.rel, dom0, max_nodes=200)
    with rac.Network(n, d, net_np.scope, net_np.rel) as net:
        for flags in (0, rac.INCREMENTAL):
            got = dfs(net, dom0, max_nodes=200, flags=flags)
            assert (got.root_iterations, got.root_status) == want["root"]
            assert got.steps == want["steps"]
            assert got.exhausted == want["exhausted"]
            if want["solution"] is None:
                assert got.solution is None
            else:
                assert np.array_equal(got.solution, want["solution"])
    assert len(want["steps"]) >= 5


def test_assign_enforce_equals_full_enforcement():
    """From arc-consistent states: the seeded enforcement gives the plain
    recurrence's result and sweep count for every single assignment."""
    T = __import__("torch")
    n, d = 200, 16
    net_np = racgen.random_network(11, 0, n, d, 0.6, 0.45)
    base, _, st = oracle.rac(n, d, net_np.scope, net_np.rel, racgen.full_domain(n, d))
    assert st == oracle.OK
    rng = np.random.default_rng(11)
    with rac.Network(n, d, net_np.scope, net_np.rel) as net:
        din = T.from_numpy(base.view(np.int32)).to("cuda:0")
        dout = T.empty_like(din)
        it = T.empty(1, dtype=T.int32, device="cuda:0")
        stt = T.empty(1, dtype=T.int32, device="cuda:0")
        for _ in range(25):
            var = int(rng.integers(0, n))
            value = int(rng.integers(0, d))  # possibly outside the domain: a wipe-out
            assigned = base.copy()
            assigned[var] = base[var] & np.uint32(1 << value)
            ro, ri, rs = oracle.rac(n, d, net_np.scope, net_np.rel, assigned)
            for flags in (0, rac.INCREMENTAL, rac.STOP_ON_WIPEOUT):
                rac.assign_enforce(net, din, dout, var, value, it, stt, flags=flags)
                T.cuda.synchronize()
                if flags & rac.STOP_ON_WIPEOUT:
                    so, si, ss = oracle.rac(n, d, net_np.scope, net_np.rel, assigned,
                                            stop_on_wipeout=True)
                    want = (so, si, ss)
                else:
                    want = (ro, ri, rs)
                assert np.array_equal(dout.cpu().numpy().view(np.uint32), want[0])
                assert int(it.item()) == want[1] and int(stt.item()) == want[2]


@pytest.mark.parametrize("seed,n,d,p,t", [(1, 40, 8, 0.3, 0.35), (2, 60, 10, 0.5, 0.3),
                                          (3, 90, 6, 0.2, 0.25), (4, 150, 12, 0.8, 0.2)])
def test_library_search_matches_oracle(seed, n, d, p, t):
    """rac_search, the same search with its loop inside the library: the same
    root, assignments, sweep counts, statuses and outcome as the oracle's."""
    net_np = racgen.random_network(seed, 0, n, d, p, t)
    dom0 = racgen.full_domain(n, d)
    for budget in (200, 7):
        want = oracle_dfs(n, d, net_np.scope, net_np.rel, dom0, max_nodes=budget)
        with rac.Network(n, d, net_np.scope, net_np.rel) as net:
            for flags in (0, rac.INCREMENTAL):
                got = rac.run_search(net, dom0, max_nodes=budget, flags=flags)
                assert got["root"] == tuple(want["root"])
                assert [tuple(int(v) for v in r) for r in got["steps"]] == \
                    [tuple(int(v) for v in r) for r in want["steps"]]
                assert got["exhausted"] == want["exhausted"]
                if want["solution"] is None:
                    assert got["solution"] is None
                else:
                    assert np.array_equal(got["solution"], want["solution"])


def test_library_search_solves_and_reports_a_wiped_root():
    """A chain on enough values has a solution the search finds without
    backtracking; a network whose root enforcement wipes out stops there."""
    from cases import chain, full_word
    n, d = 12, 16
    scope, rel = chain(n, d)
    dom0 = np.full(n, full_word(d), np.uint32)
    with rac.Network(n, d, scope, rel) as net:
        got = rac.run_search(net, dom0, max_nodes=100)
        want = oracle_dfs(n, d, scope, rel, dom0, max_nodes=100)
        assert got["found"] and np.array_equal(got["solution"], want["solution"])
        assert got["nodes"] == len(want["steps"])
    scope, rel = chain(20, 8)  # d < n: the root wipes out
    with rac.Network(20, 8, scope, rel) as net:
        got = rac.run_search(net, np.full(20, 0xFF, np.uint32), max_nodes=100)
        assert got["root"][1] == rac.WIPEOUT and got["nodes"] == 0 and not got["found"]
