"""The CPU oracle against what the paper and the mathematics fix (no GPU)."""
import numpy as np
import pytest

import oracle
import pins
from cases import chain, full_word


@pytest.mark.parametrize("pin", pins.ALL_PINS, ids=lambda p: p.__name__)
def test_pin(pin):
    fails = pin(oracle.load())
    assert not fails, "\n".join(fails[:10])


def test_threads_do_not_change_the_result():
    import racgen
    net = racgen.random_network(3, 0, 120, 8, 0.4, 0.55)
    dom = racgen.full_domain(120, 8)
    a = oracle.rac(net.n, net.d, net.scope, net.rel, dom, threads=1, trace=True)
    b = oracle.rac(net.n, net.d, net.scope, net.rel, dom, threads=4, trace=True)
    assert a[1] == b[1] and np.array_equal(a[0], b[0]) and np.array_equal(a[3], b[3])
    assert a[1] >= 2  # the case exercises more than one sweep


def test_oracle_rejects_bad_input():
    scope, rel = chain(3, 3)
    dom = np.full(3, full_word(3), np.uint32)
    with pytest.raises(ValueError):
        oracle.rac(3, 33, scope, np.zeros((2, 33), np.uint32), dom)
    bad = scope.copy()
    bad[0, 1] = bad[0, 0]
    with pytest.raises(ValueError):
        oracle.rac(3, 3, bad, rel, dom)
    with pytest.raises(ValueError):
        oracle.bruteforce(30, 1, np.zeros((0, 2), np.int32), np.zeros((0, 1), np.uint32),
                          np.ones(30, np.uint32))


def test_oracle_search_on_a_chain():
    """Algorithm 2 on the chain x_0 < x_1 < x_2 with 3 values: the root is
    already the unique solution's singletons, so the search assigns nothing
    and returns it."""
    from oracle.search import dfs
    n, d = 3, 3
    scope = np.array([[0, 1], [1, 2]], np.int32)
    lt = np.array([sum(1 << b for b in range(d) if a < b) for a in range(d)], np.uint32)
    rel = np.array([lt, lt], np.uint32)
    out = dfs(n, d, scope, rel, np.full(n, (1 << d) - 1, np.uint32), max_nodes=10)
    assert out["root"] == (3, oracle.OK) and out["nodes"] == 0
    assert list(out["solution"]) == [1, 2, 4]


def test_oracle_search_backtracks_to_a_solution():
    """x, y, z pairwise different: on 2 values both assignments of x wipe
    out and there is no solution; on 3 values x=0 succeeds, then y=1 (y=0 is
    gone by propagation after x=0, so it is never a node), leaving z=2."""
    from oracle.search import dfs
    ne2 = np.array([0b10, 0b01], np.uint32)
    scope = np.array([[0, 1], [1, 2], [0, 2]], np.int32)
    out2 = dfs(3, 2, scope, np.array([ne2] * 3, np.uint32), np.full(3, 3, np.uint32), 50)
    assert out2["solution"] is None and not out2["exhausted"]
    assert all(st == oracle.WIPEOUT for *_, st in out2["steps"]) and out2["nodes"] == 2
    ne3 = np.array([0b110, 0b101, 0b011], np.uint32)
    out3 = dfs(3, 3, scope, np.array([ne3] * 3, np.uint32), np.full(3, 7, np.uint32), 50)
    assert list(out3["solution"]) == [1, 2, 4]
    assert [(lv, var, val) for lv, var, val, _, _ in out3["steps"]] == [(0, 0, 0), (1, 1, 1)]
