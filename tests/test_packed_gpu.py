"""Packed relation rows (RAC_LAYOUT_PACKED) against the CPU oracle, bit for
bit (domains, sweep counts, statuses), through every entry point and kernel
that reads the relation store: one- and many-state launches, the host entry
point, the search, the multi-network plan, the tensor-core kernel and the
learned gating (GPU)."""
import numpy as np
import pytest

import racgen
from oracle.search import dfs as oracle_dfs
import paper_2407_11388_b300 as rac
from cases import random_tiny, tuned_tightness, width_cases
from gpu_helpers import assert_same, from_dev, gpu_enforce, oracle_enforce, to_dev, torch

pytestmark = pytest.mark.gpu

PK = rac.LAYOUT_BITS | rac.LAYOUT_PACKED
FLAG_SETS = [0, rac.INCREMENTAL, rac.STOP_ON_WIPEOUT, rac.STOP_ON_WIPEOUT | rac.INCREMENTAL]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2407_11388_b300.build import build
    build()


def words_per_relation(d):
    """4q rows of 4q bits, q = ceil(d / 4), in whole words; d > 28 keeps one
    word per row."""
    q = (d + 3) // 4
    return (16 * q * q + 31) // 32 if q < 8 else 4 * q


@pytest.mark.parametrize("d", list(range(1, 33)))
def test_packed_every_width(d):
    """Every width (every packed instance, and the unchanged store at d > 28),
    ragged n, dense and sparse graphs, three kinds of input domain, one state
    and several, all flag combinations."""
    from paper_2407_11388_b300.autotune import admissible_rows
    rows = max(admissible_rows(d))  # the whole-word default, which packed rows also fit
    for n, scope, rel, doms in width_cases(d):
        with rac.Network(n, d, scope, rel, layout=PK, rows=rows) as net, \
                rac.Network(n, d, scope, rel, packed=False, rows=rows) as plain:
            info, pinfo = net.info(), plain.info()
            assert info["words_per_relation"] == words_per_relation(d)
            assert pinfo["words_per_relation"] == (d + 3) // 4 * 4
            assert info["n_slabs"] == pinfo["n_slabs"]
            if d > 28:
                assert info["rel_bytes"] == pinfo["rel_bytes"]
            else:
                assert info["rel_bytes"] <= pinfo["rel_bytes"]
                if scope.shape[0] >= 64:
                    assert info["rel_bytes"] < pinfo["rel_bytes"]
            for flags in FLAG_SETS:
                ref = oracle_enforce(n, d, scope, rel, doms, flags)
                assert_same(gpu_enforce(n, d, scope, rel, doms[:1], flags, net=net),
                            (ref[0][:1], ref[1][:1], ref[2][:1]), "d=%d n=%d single" % (d, n))
                assert_same(gpu_enforce(n, d, scope, rel, doms, flags, net=net, shuffle_seed=d),
                            ref, "d=%d n=%d batch" % (d, n))


@pytest.mark.parametrize("d,rows", [(20, 16), (12, 32), (24, 8), (6, 32), (17, 2), (28, 4)])
def test_packed_tile_rows(d, rows):
    """Tiles of every height the packed store allows, including heights the
    whole-word store cannot hold in one stage (d = 20 with 16 rows, d = 12
    with 32)."""
    rng = np.random.default_rng(d * 64 + rows)
    n = 300
    scope, rel, _ = random_tiny(rng, n, d, 0.4, tuned_tightness(n, d, 0.4, 0.6))
    doms = np.array([random_tiny(rng, n, d, 0.0, 0.0, restrict=r)[2] for r in (0.0, 0.2, 0.35)])
    with rac.Network(n, d, scope, rel, layout=PK, rows=rows) as net:
        assert net.info()["rows_per_slab"] == rows
        for flags in (0, rac.INCREMENTAL | rac.STOP_ON_WIPEOUT):
            ref = oracle_enforce(n, d, scope, rel, doms, flags)
            assert_same(gpu_enforce(n, d, scope, rel, doms, flags, net=net, shuffle_seed=rows),
                        ref, "d=%d rows=%d" % (d, rows))
            assert_same(gpu_enforce(n, d, scope, rel, doms[1:2], flags, net=net),
                        (ref[0][1:2], ref[1][1:2], ref[2][1:2]), "d=%d rows=%d single" % (d, rows))


@pytest.mark.parametrize("seed", range(3))
def test_packed_dense_500(seed):
    """n=500, d=20, complete graph, tightness 0.35 (13 words per relation
    instead of 20): full domains and assignment states."""
    net_np = racgen.random_network(seed, 0, 500, 20, 1.0, 0.35)
    full = racgen.full_domain(500, 20)
    doms = np.array([racgen.assignment_state(seed, 0, s, 500, 20) for s in range(6)])
    with rac.Network(500, 20, net_np.scope, net_np.rel, layout=PK) as net:
        assert_same(gpu_enforce(500, 20, net_np.scope, net_np.rel, full, net=net),
                    oracle_enforce(500, 20, net_np.scope, net_np.rel, full), "full")
        assert_same(gpu_enforce(500, 20, net_np.scope, net_np.rel, doms, rac.INCREMENTAL,
                                net=net, shuffle_seed=1),
                    oracle_enforce(500, 20, net_np.scope, net_np.rel, doms), "states")


def test_packed_dense_2000_d20():
    """n=2000, d=20, density 0.9, tightness 0.3: a 94 MB packed store (144 MB
    with whole-word rows), full domains and two assignment states."""
    net_np = racgen.random_network(0, 0, 2000, 20, 0.9, 0.3)
    full = racgen.full_domain(2000, 20)
    doms = np.array([racgen.assignment_state(0, 0, s, 2000, 20) for s in range(2)])
    with rac.Network(2000, 20, net_np.scope, net_np.rel, layout=PK) as net:
        assert net.info()["rel_bytes"] < 0.68 * 144e6
        assert_same(gpu_enforce(2000, 20, net_np.scope, net_np.rel, full, net=net),
                    oracle_enforce(2000, 20, net_np.scope, net_np.rel, full, threads=32), "full")
        assert_same(gpu_enforce(2000, 20, net_np.scope, net_np.rel, doms, net=net,
                                shuffle_seed=3),
                    oracle_enforce(2000, 20, net_np.scope, net_np.rel, doms, threads=32),
                    "states")


@pytest.mark.parametrize("B", [32, 128])
def test_packed_n1000_d24_many_states(B):
    """n=1000, d=24, density 0.8, tightness 0.3 (18 words per relation instead
    of 24) with 32 or 128 assignment states in one launch: every state, plain
    and with Proposition 2."""
    net_np = racgen.random_network(0, 0, 1000, 24, 0.8, 0.3)
    doms = np.array([racgen.assignment_state(0, 0, s, 1000, 24) for s in range(B)])
    ref = oracle_enforce(1000, 24, net_np.scope, net_np.rel, doms, threads=32)
    with rac.Network(1000, 24, net_np.scope, net_np.rel, layout=PK) as net:
        for flags in (0, rac.INCREMENTAL):
            assert_same(gpu_enforce(1000, 24, net_np.scope, net_np.rel, doms, flags, net=net),
                        ref, "B=%d flags %d" % (B, flags))


def test_packed_host_entry_point():
    """rac_enforce_host on a packed network: one, two and five states."""
    n, d = 220, 14
    net_np = racgen.random_network(11, 0, n, d, 0.5, 0.3)
    doms = np.array([racgen.full_domain(n, d)] +
                    [racgen.assignment_state(11, 0, s, n, d) for s in range(4)])
    with rac.Network(n, d, net_np.scope, net_np.rel, layout=PK) as net:
        for B in (1, 2, 5):
            ref = oracle_enforce(n, d, net_np.scope, net_np.rel, doms[:B])
            assert_same(rac.enforce_host(net, doms[:B]), ref, "host B=%d" % B)


@pytest.mark.parametrize("seed,n,d,p,t", [(2, 60, 10, 0.5, 0.3), (4, 150, 12, 0.8, 0.2),
                                          (5, 80, 19, 0.4, 0.3)])
def test_packed_search(seed, n, d, p, t):
    """rac_search on a packed network: the oracle's root, assignments, sweep
    counts, statuses and outcome."""
    net_np = racgen.random_network(seed, 0, n, d, p, t)
    dom0 = racgen.full_domain(n, d)
    want = oracle_dfs(n, d, net_np.scope, net_np.rel, dom0, max_nodes=200)
    with rac.Network(n, d, net_np.scope, net_np.rel, layout=PK) as net:
        for flags in (0, rac.INCREMENTAL):
            got = rac.run_search(net, dom0, max_nodes=200, flags=flags)
            assert got["root"] == tuple(want["root"])
            assert [tuple(int(v) for v in r) for r in got["steps"]] == \
                [tuple(int(v) for v in r) for r in want["steps"]]
            assert got["exhausted"] == want["exhausted"]
            if want["solution"] is not None:
                assert np.array_equal(got["solution"], want["solution"])


def test_packed_and_whole_word_networks_in_one_plan():
    """The multi-network launch with packed and whole-word networks of
    several widths side by side: every item against the oracle."""
    T = torch()
    shapes = [(90, 5), (130, 12), (70, 20), (160, 24), (60, 28), (110, 32), (50, 3), (120, 17)]
    nets_np, nets, items, offs, doms = [], [], [], [], []
    pos = 1
    for i, (n, d) in enumerate(shapes):
        x = racgen.random_network(21, i, n, d, 0.6, 0.3)
        nets_np.append(x)
        nets.append(rac.Network(n, d, x.scope, x.rel, packed=i % 2 == 0))
        for s in range(4):
            items.append(i)
            offs.append(pos)
            doms.append(racgen.assignment_state(21, i, s, n, d))
            pos += n
    flat = np.zeros(pos, np.uint32)
    for o, dm in zip(offs, doms):
        flat[o:o + dm.size] = dm
    items, offs = np.array(items, np.int32), np.array(offs, np.int64)
    try:
        with rac.Plan(nets, items, offs) as plan:
            for flags in (0, rac.INCREMENTAL | rac.STOP_ON_WIPEOUT):
                din = to_dev(flat)
                dout = T.zeros_like(din)
                it = T.full((len(items),), -7, dtype=T.int32, device="cuda:0")
                st = T.full((len(items),), -7, dtype=T.int32, device="cuda:0")
                plan.enforce(din, dout, it, st, flags=flags)
                T.cuda.synchronize()
                out, its, sts = from_dev(dout), it.cpu().numpy(), st.cpu().numpy()
                for j in range(len(items)):
                    x = nets_np[items[j]]
                    ro, ri, rs = oracle_enforce(x.n, x.d, x.scope, x.rel, doms[j], flags)
                    o = offs[j]
                    assert np.array_equal(out[o:o + x.n], ro[0]), (j, flags)
                    assert its[j] == ri[0] and sts[j] == rs[0], (j, flags, its[j], ri, sts[j], rs)
    finally:
        for net in nets:
            net.close()


@pytest.mark.parametrize("d", [3, 12, 20, 24])
def test_packed_tensor_core_kernel(d):
    """The tensor-core kernel's operand store built from packed rows."""
    T = torch()
    n = 180
    net_np = racgen.random_network(30 + d, 0, n, d, 0.6, 0.3)
    doms = np.array([racgen.full_domain(n, d)] +
                    [racgen.assignment_state(30 + d, 0, s, n, d) for s in range(6)])
    ref = oracle_enforce(n, d, net_np.scope, net_np.rel, doms)
    with rac.Network(n, d, net_np.scope, net_np.rel, layout=PK) as net:
        B = doms.shape[0]
        din = to_dev(doms.reshape(-1))
        dout = T.empty_like(din)
        it = T.full((B,), -7, dtype=T.int32, device="cuda:0")
        st = T.full((B,), -7, dtype=T.int32, device="cuda:0")
        rac.enforce_batch([net], np.zeros(B, np.int32), np.arange(B, dtype=np.int64) * n, din,
                          dout, it, st, flags=rac.KERNEL_TENSOR)
        T.cuda.synchronize()
        assert_same((from_dev(dout).reshape(B, n), it.cpu().numpy(), st.cpu().numpy()), ref,
                    "tensor d=%d" % d)


def test_packed_learned_gating_is_exact():
    """rac_enforce_learned on a packed network: with every pair evaluated
    (threshold -inf) and with every gated pair skipped (+inf, exact through
    the verification sweeps) the oracle's domains and statuses."""
    T = torch()
    n, d = 140, 20
    net_np = racgen.random_network(41, 0, n, d, 0.6, 0.3)
    doms = np.array([racgen.assignment_state(41, 0, s, n, d) for s in range(8)])
    ref = oracle_enforce(n, d, net_np.scope, net_np.rel, doms)
    pred = rac.Predictor(seed=3)
    with rac.Network(n, d, net_np.scope, net_np.rel, layout=PK) as net:
        for thr in (-np.inf, np.inf):
            B = doms.shape[0]
            din = to_dev(doms.reshape(-1))
            dout = T.empty_like(din)
            sw = T.full((B,), -7, dtype=T.int32, device="cuda:0")
            st = T.full((B,), -7, dtype=T.int32, device="cuda:0")
            rac.enforce_learned(net, din, dout, sw, st, predictor=pred, threshold=thr)
            T.cuda.synchronize()
            out = from_dev(dout).reshape(B, n)
            assert np.array_equal(out, ref[0]), thr
            assert np.array_equal(st.cpu().numpy(), ref[2]), thr
            if thr == -np.inf:
                assert np.array_equal(sw.cpu().numpy(), ref[1])
