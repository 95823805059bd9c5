"""CUDA path versus the CPU oracle, bit for bit: domains, sweep counts and
status (GPU).  Every case goes through the C ABI."""
import numpy as np
import pytest

import oracle
import racgen
import paper_2407_11388_b300 as rac
from cases import (chain, chain_closed_form, full_word, golden_names, load_golden, mixed_states,
                   random_tiny, width_cases)
from gpu_helpers import assert_same, from_dev, gpu_enforce, oracle_enforce, to_dev, torch

pytestmark = pytest.mark.gpu

FLAG_SETS = [0, rac.INCREMENTAL, rac.STOP_ON_WIPEOUT, rac.STOP_ON_WIPEOUT | rac.INCREMENTAL]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2407_11388_b300.build import build
    build()


@pytest.mark.parametrize("name", golden_names())
def test_golden(name):
    g = load_golden(name)
    flags = rac.STOP_ON_WIPEOUT if g["stop"] else 0
    for extra in (0, rac.INCREMENTAL):
        out, it, st = gpu_enforce(g["n"], g["d"], g["scope"], g["rel"], g["dom"], flags | extra)
        assert np.array_equal(out[0], g["expected"]), (name, out[0], g["expected"])
        assert it[0] == g["iterations"] and st[0] == g["status"], (name, it, st)


@pytest.mark.parametrize("n_chain,d", [(2, 2), (5, 9), (17, 20), (32, 32), (9, 8)])
def test_chain_spread_over_tiles(n_chain, d):
    """The chain closed form with the chain's variables scattered over 300
    variables, so every link crosses tiles; d < n_chain wipes out."""
    n = 300
    perm = np.random.default_rng(n_chain * 100 + d).permutation(n)[:n_chain]
    s, r = chain(n_chain, d)
    scope = perm[s]
    dom = np.full(n, full_word(d), np.uint32)
    ref = oracle_enforce(n, d, scope, r, dom)
    if d >= n_chain:
        want = np.full(n, full_word(d), np.uint32)
        want[perm] = chain_closed_form(n_chain, d)
        assert np.array_equal(ref[0][0], want) and ref[1][0] == n_chain
    for flags in FLAG_SETS:
        assert_same(gpu_enforce(n, d, scope, r, dom, flags), oracle_enforce(n, d, scope, r, dom, flags),
                    "chain %d/%d flags %d" % (n_chain, d, flags))


@pytest.mark.parametrize("d", list(range(1, 33)))
def test_random_every_width(d):
    """Every relation width (all kernel instantiations), ragged n, dense and
    sparse graphs, tightness near the cascade point, three kinds of input
    domain; single-state and batched launches, all flag combinations."""
    for n, scope, rel, doms in width_cases(d):
        for flags in FLAG_SETS:
            ref = oracle_enforce(n, d, scope, rel, doms, flags)
            assert_same(gpu_enforce(n, d, scope, rel, doms[:1], flags),
                        (ref[0][:1], ref[1][:1], ref[2][:1]), "d=%d n=%d single" % (d, n))
            assert_same(gpu_enforce(n, d, scope, rel, doms, flags, shuffle_seed=d), ref,
                        "d=%d n=%d batch" % (d, n))


@pytest.mark.parametrize("B", [2, 3, 5, 8, 40, 64, 96])
def test_state_groupings(B):
    """Warp-to-state mappings for different state counts in one launch (with
    more than 32 states a slab's states come in several 32-state chunks, each
    split over the group's warps its own way)."""
    rng = np.random.default_rng(B)
    n, d = 150, 12
    scope, rel, _ = random_tiny(rng, n, d, 0.3, 0.62)
    doms = np.array([random_tiny(rng, n, d, 0.0, 0.0, restrict=0.25)[2] for _ in range(B)])
    for flags in (0, rac.INCREMENTAL | rac.STOP_ON_WIPEOUT):
        assert_same(gpu_enforce(n, d, scope, rel, doms, flags, shuffle_seed=B),
                    oracle_enforce(n, d, scope, rel, doms, flags), "B=%d" % B)


@pytest.mark.parametrize("seed", range(10))
def test_small_random_csp_config(seed):
    """n=50, d=10, density 0.5, tightness 0.3: full domains and assignment
    states (1-5 variables reduced to one value), seeds 0-9."""
    net = racgen.random_network(seed, 0, 50, 10, 0.5, 0.3)
    doms = np.array([racgen.full_domain(50, 10)] +
                    [racgen.assignment_state(seed, 0, s, 50, 10) for s in range(16)])
    for flags in (0, rac.INCREMENTAL):
        assert_same(gpu_enforce(50, 10, net.scope, net.rel, doms, flags, shuffle_seed=seed),
                    oracle_enforce(50, 10, net.scope, net.rel, doms, flags), "seed %d" % seed)
        assert_same(gpu_enforce(50, 10, net.scope, net.rel, doms[:1], flags),
                    oracle_enforce(50, 10, net.scope, net.rel, doms[:1], flags), "seed %d" % seed)


@pytest.mark.parametrize("seed", range(10))
def test_dense_500_config(seed):
    """n=500, d=20, complete graph, tightness 0.35, full domains (the
    single-state launch the benchmark times) plus assignment states, seeds
    0-9."""
    net = racgen.random_network(seed, 0, 500, 20, 1.0, 0.35)
    full = racgen.full_domain(500, 20)
    assert_same(gpu_enforce(500, 20, net.scope, net.rel, full),
                oracle_enforce(500, 20, net.scope, net.rel, full), "dense500 full")
    doms = np.array([racgen.assignment_state(seed, 0, s, 500, 20) for s in range(6)])
    assert_same(gpu_enforce(500, 20, net.scope, net.rel, doms, rac.INCREMENTAL, shuffle_seed=1),
                oracle_enforce(500, 20, net.scope, net.rel, doms), "dense500 states")


@pytest.mark.parametrize("seed", range(10))
def test_dense_2000_config(seed):
    """n=2000, d=32, density 0.9, tightness 0.3 (a 230 MB relation store),
    full domains and two assignment states, seeds 0-9."""
    net = racgen.random_network(seed, 0, 2000, 32, 0.9, 0.3)
    full = racgen.full_domain(2000, 32)
    assert_same(gpu_enforce(2000, 32, net.scope, net.rel, full),
                oracle_enforce(2000, 32, net.scope, net.rel, full, threads=32), "dense2000 full")
    doms = np.array([racgen.assignment_state(seed, 0, s, 2000, 32) for s in range(2)])
    assert_same(gpu_enforce(2000, 32, net.scope, net.rel, doms, shuffle_seed=3),
                oracle_enforce(2000, 32, net.scope, net.rel, doms, threads=32), "dense2000 states")


@pytest.mark.parametrize("B,seed", [(32, s) for s in range(10)] + [(128, 0)])
def test_n1000_d24_many_states_config(B, seed):
    """n=1000, d=24, density 0.8, tightness 0.3 with 32 assignment states
    (seeds 0-9) or 128 (seed 0) in one launch (the benchmark's many-state
    launches): every state against the oracle, plain and with Proposition 2."""
    net_np = racgen.random_network(seed, 0, 1000, 24, 0.8, 0.3)
    doms = np.array([racgen.assignment_state(seed, 0, s, 1000, 24) for s in range(B)])
    ref = oracle_enforce(1000, 24, net_np.scope, net_np.rel, doms, threads=32)
    with rac.Network(1000, 24, net_np.scope, net_np.rel) as net:
        for flags in (0, rac.INCREMENTAL):
            got = gpu_enforce(1000, 24, net_np.scope, net_np.rel, doms, flags, net=net)
            assert_same(got, ref, "B=%d seed %d flags %d" % (B, seed, flags))


def test_search_path_states():
    """States built the way backtrack search builds them (Algorithm 2):
    enforce, assign one more variable, enforce again -- the multi-sweep regime
    of Table 1.  The states come from the oracle."""
    n, d = 120, 10
    net = racgen.random_network(4, 0, n, d, 0.5, 0.3)
    rng = np.random.default_rng(4)
    dom, _, _ = oracle.rac(n, d, net.scope, net.rel, racgen.full_domain(n, d))
    states = []
    for _ in range(12):
        free = [x for x in range(n) if bin(int(dom[x])).count("1") > 1]
        if not free:
            break
        x = int(rng.choice(free))
        vals = [a for a in range(d) if (int(dom[x]) >> a) & 1]
        nxt = dom.copy()
        nxt[x] = 1 << int(rng.choice(vals))
        states.append(nxt)
        out, it, st = oracle.rac(n, d, net.scope, net.rel, nxt)
        if st == oracle.OK:
            dom = out
    doms = np.array(states)
    ref = oracle_enforce(n, d, net.scope, net.rel, doms)
    assert ref[1].max() >= 3
    for flags in FLAG_SETS:
        assert_same(gpu_enforce(n, d, net.scope, net.rel, doms, flags, shuffle_seed=2),
                    oracle_enforce(n, d, net.scope, net.rel, doms, flags), "search path")


def test_sweep_cap():
    scope, rel = chain(12, 16)
    dom = np.full(12, full_word(16), np.uint32)
    for cap in (1, 2, 5, 11, 12, 13):
        for flags in (0, rac.INCREMENTAL):
            assert_same(gpu_enforce(12, 16, scope, rel, dom, flags, max_sweeps=cap),
                        oracle_enforce(12, 16, scope, rel, dom, flags, max_sweeps=cap), "cap %d" % cap)


def test_in_place_and_repeat():
    """dom_out == dom_in, and repeated launches on one workspace."""
    T = torch()
    net_np = racgen.random_network(9, 0, 90, 7, 0.4, 0.55)
    dom = racgen.assignment_state(9, 0, 0, 90, 7)
    ref = oracle_enforce(90, 7, net_np.scope, net_np.rel, dom)
    with rac.Network(90, 7, net_np.scope, net_np.rel) as net:
        it = T.empty(1, dtype=T.int32, device="cuda:0")
        st = T.empty(1, dtype=T.int32, device="cuda:0")
        for _ in range(5):
            buf = to_dev(dom)
            rac.enforce(net, buf, buf, it, st)
            T.cuda.synchronize()
            assert_same((from_dev(buf)[None], it.cpu().numpy(), st.cpu().numpy()), ref, "in place")


def test_batch_of_different_networks():
    """rac_enforce_batch over networks of different n and d, items
    interleaved and stored at scattered offsets."""
    T = torch()
    rng = np.random.default_rng(21)
    specs = [(64, 8, 0.6, 0.5), (200, 16, 0.3, 0.6), (33, 32, 1.0, 0.45), (5, 3, 1.0, 0.5)]
    nps = [racgen.random_network(21, i, n, d, p, t) for i, (n, d, p, t) in enumerate(specs)]
    nets = [rac.Network(x.n, x.d, x.scope, x.rel) for x in nps]
    items, offs, doms = [], [], []
    pos = 7
    for i in range(23):
        k = int(rng.integers(0, len(specs)))
        dom = racgen.assignment_state(21, k, i, nps[k].n, nps[k].d)
        items.append(k)
        offs.append(pos)
        doms.append(dom)
        pos += nps[k].n + int(rng.integers(0, 5))
    flat = np.zeros(pos + 3, np.uint32)
    for o, dmn in zip(offs, doms):
        flat[o:o + dmn.size] = dmn
    din = to_dev(flat)
    dout = T.zeros_like(din)
    it = T.empty(len(items), dtype=T.int32, device="cuda:0")
    st = T.empty(len(items), dtype=T.int32, device="cuda:0")
    rac.enforce_batch(nets, items, offs, din, dout, it, st, flags=rac.INCREMENTAL)
    T.cuda.synchronize()
    got = from_dev(dout)
    its, sts = it.cpu().numpy(), st.cpu().numpy()
    for j, (k, o, dmn) in enumerate(zip(items, offs, doms)):
        x = nps[k]
        ro, ri, rs = oracle.rac(x.n, x.d, x.scope, x.rel, dmn)
        assert np.array_equal(got[o:o + x.n], ro) and its[j] == ri and sts[j] == rs, j
    for n in nets:
        n.close()


def test_host_entry_point():
    net_np = racgen.random_network(2, 0, 300, 24, 0.7, 0.33)
    doms = np.array([racgen.assignment_state(2, 0, s, 300, 24) for s in range(5)])
    with rac.Network(300, 24, net_np.scope, net_np.rel) as net:
        out, it, st = rac.enforce_host(net, doms, flags=rac.INCREMENTAL)
    assert_same((out, it, st), oracle_enforce(300, 24, net_np.scope, net_np.rel, doms), "host")


def test_host_entry_point_replayed():
    """Repeated host calls replay a recorded graph: new inputs each call, a
    change of state count, flags or sweep cap records a new one, and every
    result matches the oracle."""
    n, d = 260, 16
    net_np = racgen.random_network(12, 0, n, d, 0.6, 0.35)
    all_doms = np.array([racgen.assignment_state(12, 0, s, n, d) for s in range(12)])
    calls = [(slice(0, 4), 0, 0), (slice(4, 8), 0, 0), (slice(8, 12), 0, 0),   # replays
             (slice(0, 6), 0, 0), (slice(6, 12), 0, 0),                         # new count
             (slice(0, 6), rac.INCREMENTAL, 0), (slice(6, 12), rac.INCREMENTAL, 0),
             (slice(0, 6), rac.STOP_ON_WIPEOUT, 2), (slice(6, 12), rac.STOP_ON_WIPEOUT, 2),
             (slice(0, 5), rac.KERNEL_TENSOR, 0), (slice(5, 10), rac.KERNEL_TENSOR, 0),
             (slice(0, 4), 0, 0)]
    with rac.Network(n, d, net_np.scope, net_np.rel) as net:
        for sl, flags, cap in calls:
            doms = all_doms[sl]
            got = rac.enforce_host(net, doms, max_sweeps=cap, flags=flags)
            ref = oracle_enforce(n, d, net_np.scope, net_np.rel, doms,
                                 flags & ~rac.KERNEL_TENSOR, max_sweeps=cap)
            assert_same(got, ref, "host replay %s flags %d cap %d" % (sl, flags, cap))


def test_more_states_than_one_launch():
    """1,100 states of one network: two launches of 1,024 and 76 states on the
    same workspace, through the device and the host entry points."""
    n, d = 40, 8
    net_np = racgen.random_network(21, 0, n, d, 0.6, 0.33)
    doms = np.array([racgen.assignment_state(21, 0, s, n, d) for s in range(1100)])
    ref = oracle_enforce(n, d, net_np.scope, net_np.rel, doms, rac.INCREMENTAL)
    with rac.Network(n, d, net_np.scope, net_np.rel) as net:
        assert_same(gpu_enforce(n, d, net_np.scope, net_np.rel, doms, rac.INCREMENTAL, net=net,
                                shuffle_seed=3), ref, "1100 states")
        assert_same(rac.enforce_host(net, doms, flags=rac.INCREMENTAL), ref, "1100 states, host")


def test_two_streams():
    """Each stream gets its own workspace; concurrent calls do not interfere."""
    T = torch()
    net_np = racgen.random_network(6, 0, 256, 16, 0.5, 0.5)
    doms = [racgen.assignment_state(6, 0, s, 256, 16) for s in range(2)]
    ref = [oracle_enforce(256, 16, net_np.scope, net_np.rel, d_) for d_ in doms]
    with rac.Network(256, 16, net_np.scope, net_np.rel) as net:
        streams = [T.cuda.Stream(), T.cuda.Stream()]
        bufs = [to_dev(d_) for d_ in doms]
        outs = [T.empty_like(b) for b in bufs]
        its = [T.empty(1, dtype=T.int32, device="cuda:0") for _ in range(2)]
        sts = [T.empty(1, dtype=T.int32, device="cuda:0") for _ in range(2)]
        T.cuda.synchronize()
        for rep in range(3):
            for i in range(2):
                rac.enforce(net, bufs[i], outs[i], its[i], sts[i], stream=streams[i])
        T.cuda.synchronize()
        for i in range(2):
            assert_same((from_dev(outs[i])[None], its[i].cpu().numpy(), sts[i].cpu().numpy()),
                        ref[i], "stream %d" % i)


def test_no_constraints_and_single_variable():
    for n, d in [(1, 1), (1, 32), (40, 5)]:
        dom = np.random.default_rng(n).integers(0, 1 << min(d, 31), n).astype(np.uint32)
        dom &= np.uint32(full_word(d))
        scope = np.zeros((0, 2), np.int32)
        rel = np.zeros((0, d), np.uint32)
        for flags in FLAG_SETS:
            assert_same(gpu_enforce(n, d, scope, rel, dom, flags),
                        oracle_enforce(n, d, scope, rel, dom, flags), "empty net")


def test_many_launches_on_one_workspace():
    """Back-to-back launches on the same (network, stream) workspace with
    different state counts and flags: the scratch state each launch leaves
    behind (rotating barrier slots, all-ones scratch domains) must be what
    the next one expects, and no launch may give up a wait."""
    T = torch()
    n, d = 700, 24
    net_np = racgen.random_network(31, 0, n, d, 0.9, 0.33)
    states = np.array([racgen.assignment_state(31, 0, s, n, d) for s in range(9)] +
                      [racgen.full_domain(n, d)])
    refs = oracle_enforce(n, d, net_np.scope, net_np.rel, states)
    flush = T.empty(256 << 20, dtype=T.uint8, device="cuda:0")
    with rac.Network(n, d, net_np.scope, net_np.rel) as net:
        plan = [(1, 0), (7, rac.INCREMENTAL), (1, rac.STOP_ON_WIPEOUT), (3, 0), (10, 0),
                (1, rac.INCREMENTAL), (2, rac.STOP_ON_WIPEOUT | rac.INCREMENTAL)] * 4
        for rep, (B, flags) in enumerate(plan):
            pick = [(rep + j) % states.shape[0] for j in range(B)]
            flush.zero_()
            got = gpu_enforce(n, d, net_np.scope, net_np.rel, states[pick], flags, net=net,
                              shuffle_seed=rep if B > 1 else None)
            want = oracle_enforce(n, d, net_np.scope, net_np.rel, states[pick], flags)
            assert not np.any(got[2] == rac.EBARRIER), "launch %d gave up a wait" % rep
            assert_same(got, want, "launch %d (B=%d flags=%d)" % (rep, B, flags))
    assert refs[1].max() >= 3


def _split_wipe_network():
    """Variable 0 is emptied by the AND of two removals from different slabs,
    neither of which empties it alone: (0, 40) keeps {0, 1} and (0, 65) keeps
    {2, 3} while variables 40 and 65 hold the value 0.  By Eq. 1 the first
    sweep empties variable 0, the second empties 40 and 65 (their only value
    lost its support), the third removes nothing: 3 sweeps, wiped out; with
    stop-on-wipeout the run ends after sweep 1."""
    n, d = 70, 4
    scope = np.array([[0, 40], [0, 65], [3, 50], [33, 66]], np.int32)
    rel = np.array([[1, 1, 0, 0], [0, 0, 1, 1], [15, 15, 15, 15], [15, 15, 15, 15]], np.uint32)
    dom = np.full(n, 15, np.uint32)
    dom[40] = dom[65] = 1
    return n, d, scope, rel, dom


@pytest.mark.parametrize("B", [1, 5])
def test_wipe_split_over_slabs(B):
    n, d, scope, rel, dom = _split_wipe_network()
    doms = np.tile(dom, (B, 1))
    doms[1:, 7] = 3  # the other states differ elsewhere
    for flags in FLAG_SETS:
        ref = oracle_enforce(n, d, scope, rel, doms, flags)
        stop = bool(flags & rac.STOP_ON_WIPEOUT)
        assert list(ref[1]) == [1 if stop else 3] * B and list(ref[2]) == [rac.WIPEOUT] * B
        assert_same(gpu_enforce(n, d, scope, rel, doms, flags), ref, "split wipe-out")


@pytest.mark.parametrize("n,d,density,c,as_bool", [(40, 1, 0.5, 0.3, False), (70, 7, 0.6, 0.3, True),
                                                   (300, 20, 0.3, 0.2, False),
                                                   (90, 32, 0.8, 0.05, False)])
def test_network_from_u8_matrices(n, d, density, c, as_bool):
    """A network given as the relation tensor's 0/1 matrices
    (rac_create_network_u8) gets the layout of the same network given as
    packed rows, and the oracle's domains, sweep counts and status."""
    rng = np.random.default_rng(7000 + d)
    tight = min(0.95, (c / max(1.0, n * density)) ** (1.0 / d))
    pairs = [(x, y) for x in range(n) for y in range(x + 1, n) if rng.random() < density]
    # scopes in both orientations, as a caller may give them
    scope = np.array([(y, x) if rng.random() < 0.5 else (x, y) for x, y in pairs],
                     np.int32).reshape(-1, 2)
    mats = (rng.random((len(pairs), d, d)) >= tight).astype(np.uint8)
    rel = np.zeros((len(pairs), d), np.uint32)
    for b in range(d):  # packed rows for the oracle: bit b of row a = R[a][b]
        rel |= mats[:, :, b].astype(np.uint32) << np.uint32(b)
    doms = mixed_states(rng, n, d)
    net_u8 = rac.Network(n, d, scope, mats.astype(bool) if as_bool else mats)
    net_w = rac.Network(n, d, scope, rel)
    try:
        assert net_u8.info() == net_w.info()
        for flags in (0, rac.INCREMENTAL):
            got = gpu_enforce(n, d, scope, rel, doms, flags, net=net_u8)
            assert_same(got, oracle_enforce(n, d, scope, rel, doms, flags), "u8 %d %d" % (n, d))
    finally:
        net_u8.close()
        net_w.close()


_MAX_N_CASE = {}


def _max_n_case():
    """n_vars = 2,000,000, the largest network the library takes, with d = 8:
    the chain x_0 < ... < x_7 on eight variables scattered over the whole
    range (one value each at the fixpoint, after 8 sweeps), 50,000 random
    loose constraints between far-apart blocks, and 2,000 more that touch the
    chain's variables, so the removals spread from the chain over further
    sweeps (9 in all, about 1,300 domains reduced).  The domains do not fit
    in shared memory here, so the sweep reads them from global memory."""
    if not _MAX_N_CASE:
        n, d = 2_000_000, 8
        rng = np.random.default_rng(77)
        perm = rng.choice(n, size=8, replace=False)
        s, r = chain(8, d)
        cs = perm[s]
        pairs = set((min(a, b), max(a, b)) for a, b in cs.tolist())
        extra = []
        while len(extra) < 50_000:
            a, b = (int(v) for v in rng.integers(0, n, 2))
            if a != b and (min(a, b), max(a, b)) not in pairs:
                pairs.add((min(a, b), max(a, b)))
                extra.append((a, b))
        for i in range(2000):
            a, b = int(perm[i % 8]), int(rng.integers(0, n))
            if a != b and (min(a, b), max(a, b)) not in pairs:
                pairs.add((min(a, b), max(a, b)))
                extra.append((a, b))
        bits = rng.random((len(extra), d, d)) >= 0.12
        er = (bits * (1 << np.arange(d))[None, None, :]).sum(axis=2).astype(np.uint32)
        scope = np.concatenate([cs.astype(np.int32), np.array(extra, np.int32)])
        rel = np.concatenate([r, er])
        dom = np.full(n, full_word(d), np.uint32)
        ref = oracle_enforce(n, d, scope, rel, dom)
        assert ref[1][0] >= 5 and np.count_nonzero(ref[0][0] != full_word(d)) > 100
        _MAX_N_CASE.update(n=n, d=d, scope=scope, rel=rel, dom=dom, ref=ref)
    return _MAX_N_CASE


@pytest.mark.parametrize("flags", [0, rac.INCREMENTAL])
def test_maximum_variable_count(flags):
    c = _max_n_case()
    got = gpu_enforce(c["n"], c["d"], c["scope"], c["rel"], c["dom"], flags)
    assert_same(got, c["ref"], "n = 2,000,000, flags %d" % flags)


@pytest.mark.parametrize("ctas", [1, 2, 7, 37, 65535])
def test_grid_cap_does_not_change_results(ctas):
    """RAC_LAYOUT_MAX_CTAS: a CTA then owns many tiles (one CTA: all of them)
    and the grid barrier joins fewer CTAs; domains, sweep counts and statuses
    stay the oracle's, one state and many, plain and with Proposition 2 and
    stop-on-wipeout, and through the no-allocation and host entry points."""
    n, d = 400, 16
    net_np = racgen.random_network(31, 0, n, d, 0.3, 0.58)
    doms = np.array([racgen.assignment_state(31, 0, s, n, d) for s in range(9)])
    with rac.Network(n, d, net_np.scope, net_np.rel, max_ctas=ctas) as net:
        for flags in (0, rac.INCREMENTAL, rac.STOP_ON_WIPEOUT):
            want = oracle_enforce(n, d, net_np.scope, net_np.rel, doms, flags)
            assert_same(gpu_enforce(n, d, net_np.scope, net_np.rel, doms, flags, net=net), want,
                        "cap %d flags %d" % (ctas, flags))
            assert_same(gpu_enforce(n, d, net_np.scope, net_np.rel, doms[:1], flags, net=net),
                        tuple(a[:1] for a in want), "cap %d flags %d one state" % (ctas, flags))
            if flags == 0:
                assert max(want[1]) >= 3  # removals cascade over several sweeps
        out, it, st = rac.enforce_host(net, doms)
        want = oracle_enforce(n, d, net_np.scope, net_np.rel, doms)
        assert np.array_equal(out, want[0]) and list(it) == list(want[1])
        assert list(st) == list(want[2])
        T = torch()
        din = to_dev(doms[0])
        dout = T.empty_like(din)
        its = T.empty(1, dtype=T.int32, device="cuda:0")
        sts = T.empty(1, dtype=T.int32, device="cuda:0")
        rac.enforce_noalloc(net, din, dout, its, sts)
        T.cuda.synchronize()
        assert np.array_equal(from_dev(dout), want[0][0])
        assert (int(its.item()), int(sts.item())) == (want[1][0], want[2][0])


def test_host_entry_point_with_changing_state_counts():
    """rac_enforce_host on one (network, stream) with 3, 1, 2, 3, 1 states in
    turn: the results of up to three states are published with a completion
    number whose place in the pinned buffer moves with the state count; every
    call must wait for its own launch."""
    n, d = 300, 12
    net_np = racgen.random_network(17, 0, n, d, 0.5, 0.5)
    pool = np.array([racgen.assignment_state(17, 0, s, n, d) for s in range(12)])
    want = oracle_enforce(n, d, net_np.scope, net_np.rel, pool)
    with rac.Network(n, d, net_np.scope, net_np.rel) as net:
        pos = 0
        for B in (3, 1, 2, 3, 1, 2):
            sel = np.arange(pos, pos + B) % len(pool)
            pos += B
            out, it, st = rac.enforce_host(net, pool[sel])
            assert np.array_equal(out.reshape(B, n), want[0][sel]), B
            assert list(it) == list(want[1][sel]) and list(st) == list(want[2][sel])
    assert want[1].max() >= 3
