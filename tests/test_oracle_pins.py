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
