"""Kernel (b), the tcgen05 tensor-core path (RAC_KERNEL_TENSOR), against the
CPU oracle and against kernel (a), bit for bit (GPU)."""
import numpy as np
import pytest

import racgen
import paper_2407_11388_b300 as rac
from cases import chain, chain_closed_form, full_word, golden_names, load_golden, width_cases
from gpu_helpers import assert_same, gpu_enforce, oracle_enforce

pytestmark = pytest.mark.gpu
TC = rac.KERNEL_TENSOR


@pytest.mark.parametrize("name", golden_names())
def test_golden_tensor(name):
    g = load_golden(name)
    flags = TC | (rac.STOP_ON_WIPEOUT if g["stop"] else 0)
    out, it, st = gpu_enforce(g["n"], g["d"], g["scope"], g["rel"], g["dom"], flags)
    assert np.array_equal(out[0], g["expected"]) and it[0] == g["iterations"] and st[0] == g["status"]


@pytest.mark.parametrize("d", [1, 2, 5, 8, 12, 16, 20, 24, 27, 32])
def test_tensor_every_width(d):
    for n, scope, rel, doms in width_cases(d):
        for flags in (0, rac.INCREMENTAL | rac.STOP_ON_WIPEOUT):
            ref = oracle_enforce(n, d, scope, rel, doms, flags)
            assert_same(gpu_enforce(n, d, scope, rel, doms, flags | TC, shuffle_seed=d), ref,
                        "tensor d=%d n=%d" % (d, n))
            assert_same(gpu_enforce(n, d, scope, rel, doms[:1], flags | TC),
                        (ref[0][:1], ref[1][:1], ref[2][:1]), "tensor single d=%d" % d)


def test_tensor_chain():
    n = 200
    perm = np.random.default_rng(7).permutation(n)[:12]
    s, r = chain(12, 16)
    scope = perm[s]
    dom = np.full(n, full_word(16), np.uint32)
    assert_same(gpu_enforce(n, 16, scope, r, dom, TC), oracle_enforce(n, 16, scope, r, dom), "chain")


@pytest.mark.parametrize("B", [2, 31, 64, 128, 150])
def test_tensor_many_states_vs_oracle(B):
    """Up to 128 states per launch (150 is split into two launches)."""
    n, d = 180, 20
    net = racgen.random_network(40 + B, 0, n, d, 0.7, 0.45)
    doms = np.array([racgen.assignment_state(40 + B, 0, s, n, d) for s in range(B)])
    ref = oracle_enforce(n, d, net.scope, net.rel, doms)
    assert_same(gpu_enforce(n, d, net.scope, net.rel, doms, TC, shuffle_seed=B), ref, "B=%d" % B)
    assert ref[1].max() >= 3


@pytest.mark.parametrize("seed", range(5))
def test_tensor_learned_shape_config(seed):
    """n=1000, d=24, density 0.8, tightness 0.3, 32 assignment states, seeds
    0-4: the tensor path equals kernel (a) bit for bit, and a sample equals
    the oracle."""
    n, d = 1000, 24
    net = racgen.random_network(seed, 0, n, d, 0.8, 0.3)
    doms = np.array([racgen.assignment_state(seed, 0, s, n, d) for s in range(32)])
    a = gpu_enforce(n, d, net.scope, net.rel, doms, 0, shuffle_seed=1)
    b = gpu_enforce(n, d, net.scope, net.rel, doms, TC, shuffle_seed=2)
    assert_same(b, a, "tensor vs bit-packed")
    ref = oracle_enforce(n, d, net.scope, net.rel, doms[:4], threads=16)
    assert_same((b[0][:4], b[1][:4], b[2][:4]), ref, "tensor vs oracle")


def test_tensor_dense_500():
    net = racgen.random_network(0, 0, 500, 20, 1.0, 0.35)
    doms = np.array([racgen.full_domain(500, 20)] + [racgen.assignment_state(0, 0, s, 500, 20)
                                                    for s in range(7)])
    assert_same(gpu_enforce(500, 20, net.scope, net.rel, doms, TC, shuffle_seed=5),
                oracle_enforce(500, 20, net.scope, net.rel, doms), "dense500 tensor")


def test_fp8_store_built_at_creation():
    """RAC_LAYOUT_FP8 builds the tensor-core operand store when the network is
    created; the tensor-core kernel then reads it (the other tests build it
    on their first tensor-core call)."""
    n, d = 300, 24
    net_np = racgen.random_network(5, 0, n, d, 0.7, 0.55)
    doms = np.array([racgen.assignment_state(5, 0, s, n, d) for s in range(40)])
    ref = oracle_enforce(n, d, net_np.scope, net_np.rel, doms)
    with rac.Network(n, d, net_np.scope, net_np.rel,
                     layout=rac.LAYOUT_BITS | rac.LAYOUT_FP8) as net:
        for flags in (TC, TC | rac.INCREMENTAL, TC | rac.STOP_ON_WIPEOUT):
            want = ref if flags == TC or flags == TC | rac.INCREMENTAL else \
                oracle_enforce(n, d, net_np.scope, net_np.rel, doms, rac.STOP_ON_WIPEOUT)
            assert_same(gpu_enforce(n, d, net_np.scope, net_np.rel, doms, flags, net=net), want,
                        "flags %d" % flags)
    assert ref[1].max() >= 3
