"""The batched persistent launch (many networks of uneven n and d, many
states each, one cooperative launch) against the CPU oracle (GPU)."""
import numpy as np
import pytest

import oracle
import racgen
import paper_2407_11388_b300 as rac
from gpu_helpers import assert_same, from_dev, to_dev, torch

pytestmark = pytest.mark.gpu


def _batch(seed, n_nets, states_per_net, shape=None):
    nets_np, items, offs, doms = [], [], [], []
    pos = 3
    for i in range(n_nets):
        n, d, p, t = shape(i) if shape else racgen.batch_params(seed, i)
        nets_np.append(racgen.random_network(seed, i, n, d, p, t))
    rng = np.random.default_rng(seed)
    order = []
    for i in range(n_nets):
        for s in range(states_per_net):
            order.append((i, s))
    rng.shuffle(order)  # items interleaved over networks, scattered in memory
    for i, s in order:
        x = nets_np[i]
        dom = racgen.assignment_state(seed, i, s, x.n, x.d)
        items.append(i)
        offs.append(pos)
        doms.append(dom)
        pos += x.n + int(rng.integers(0, 3))
    flat = np.zeros(pos + 1, np.uint32)
    for o, dm in zip(offs, doms):
        flat[o:o + dm.size] = dm
    return nets_np, np.array(items, np.int32), np.array(offs, np.int64), doms, flat


def _run(nets, items, offs, flat, flags=0, plan=None, stream=None):
    T = torch()
    din = to_dev(flat)
    dout = T.zeros_like(din)
    it = T.full((len(items),), -7, dtype=T.int32, device="cuda:0")
    st = T.full((len(items),), -7, dtype=T.int32, device="cuda:0")
    if plan is None:
        rac.enforce_batch(nets, items, offs, din, dout, it, st, flags=flags, stream=stream)
    else:
        plan.enforce(din, dout, it, st, flags=flags, stream=stream)
    T.cuda.synchronize()
    return from_dev(dout), it.cpu().numpy(), st.cpu().numpy()


def _check(nets_np, items, offs, doms, got, flags, sample=None):
    out, its, sts = got
    idx = range(len(items)) if sample is None else sample
    for j in idx:
        x = nets_np[items[j]]
        ro, ri, rs = oracle.rac(x.n, x.d, x.scope, x.rel, doms[j],
                                stop_on_wipeout=bool(flags & rac.STOP_ON_WIPEOUT), threads=8)
        o = offs[j]
        assert np.array_equal(out[o:o + x.n], ro) and its[j] == ri and sts[j] == rs, \
            "item %d (net %d): sweeps gpu %d oracle %d, status gpu %d oracle %d" % (
                j, items[j], its[j], ri, sts[j], rs)


@pytest.mark.parametrize("flags", [0, rac.INCREMENTAL, rac.STOP_ON_WIPEOUT,
                                   rac.STOP_ON_WIPEOUT | rac.INCREMENTAL])
def test_uneven_batch_full_parity(flags):
    """24 networks with n in [50, 800], d in [8, 32], density in [0.3, 1],
    tightness in [0.2, 0.4], 6 assignment states each: every item checked."""
    nets_np, items, offs, doms, flat = _batch(5, 24, 6)
    nets = [rac.Network(x.n, x.d, x.scope, x.rel) for x in nets_np]
    got = _run(nets, items, offs, flat, flags)
    _check(nets_np, items, offs, doms, got, flags)


def test_uneven_batch_small_networks_and_widths():
    """Many small networks of every width, a network without constraints and
    single-state jobs in the same launch."""
    def shape(i):
        return (3 + (i * 7) % 60, 1 + i % 32, [0.0, 0.4, 0.9, 1.0][i % 4], 0.45)
    nets_np, items, offs, doms, flat = _batch(9, 40, 3, shape=shape)
    nets = [rac.Network(x.n, x.d, x.scope, x.rel) for x in nets_np]
    for flags in (0, rac.INCREMENTAL | rac.STOP_ON_WIPEOUT):
        got = _run(nets, items, offs, flat, flags)
        _check(nets_np, items, offs, doms, got, flags)


def test_batched_config_256_networks_64_states():
    """The uneven batch at full size: 256 networks (n ~ U[50,800], d ~
    U[8,32], density ~ U[0.3,1], tightness ~ U[0.2,0.4]) x 64 assignment
    states, 16,384 fixpoints in one launch; the oracle checks two random
    items of every network, and every status is a completed one."""
    nets_np, items, offs, doms, flat = _batch(0, 256, 64)
    nets = [rac.Network(x.n, x.d, x.scope, x.rel) for x in nets_np]
    with rac.Plan(nets, items, offs) as plan:
        got = _run(nets, items, offs, flat, 0, plan=plan)
        again = _run(nets, items, offs, flat, 0, plan=plan)  # reuse of the plan's workspace
    assert np.array_equal(got[0], again[0]) and np.array_equal(got[1], again[1])
    assert set(np.unique(got[2]).tolist()) <= {rac.OK, rac.WIPEOUT}
    rng = np.random.default_rng(0)
    sample = []
    for i in range(len(nets_np)):
        mine = np.flatnonzero(items == i)
        sample += [int(j) for j in rng.choice(mine, size=2, replace=False)]
    _check(nets_np, items, offs, doms, got, 0, sample=sample)


def test_plan_in_cuda_graph():
    """A plan launch allocates nothing, so it can be captured and replayed."""
    T = torch()
    nets_np, items, offs, doms, flat = _batch(3, 10, 8)
    nets = [rac.Network(x.n, x.d, x.scope, x.rel) for x in nets_np]
    with rac.Plan(nets, items, offs) as plan:
        din = to_dev(flat)
        dout = T.zeros_like(din)
        it = T.zeros((len(items),), dtype=T.int32, device="cuda:0")
        st = T.zeros((len(items),), dtype=T.int32, device="cuda:0")
        s = T.cuda.Stream()
        with T.cuda.stream(s):
            plan.enforce(din, dout, it, st, stream=s)  # warm-up outside capture
        s.synchronize()
        g = T.cuda.CUDAGraph()
        with T.cuda.graph(g, stream=s):
            plan.enforce(din, dout, it, st, stream=s)
        for _ in range(3):
            dout.zero_()
            it.fill_(-1)
            g.replay()
        T.cuda.synchronize()
        got = (from_dev(dout), it.cpu().numpy(), st.cpu().numpy())
    _check(nets_np, items, offs, doms, got, 0)


@pytest.mark.parametrize("rows", [2, 4, 8, 16, 32])
def test_tile_rows_do_not_change_results(rows):
    """Every admissible tile row count (RAC_LAYOUT_ROWS) gives the oracle's
    domains, sweep counts and statuses: single-network launches, the
    Proposition-2 flag and the multi-network launch."""
    from paper_2407_11388_b300.autotune import admissible_rows

    def shape(i):
        return (40 + 37 * i, [5, 8, 12, 16, 20, 24, 32][i % 7], 0.7, [0.25, 0.3, 0.35][i % 3])
    nets_np, items, offs, doms, flat = _batch(13, 7, 4, shape=shape)
    nets = [rac.Network(x.n, x.d, x.scope, x.rel,
                        rows=rows if rows in admissible_rows(x.d) else None)
            for x in nets_np]
    for x, net in zip(nets_np, nets):
        want = rows if rows in admissible_rows(x.d) else None
        if want is not None:
            assert net.info()["rows_per_slab"] == want
    for flags in (0, rac.INCREMENTAL):
        got = _run(nets, items, offs, flat, flags)
        _check(nets_np, items, offs, doms, got, flags)
        for i in range(len(nets)):  # one network per launch
            sel = np.flatnonzero(items == i)
            got1 = _run([nets[i]], np.zeros(sel.size, np.int32), offs[sel], flat, flags)
            for a, j in enumerate(sel):
                n = nets_np[i].n
                assert np.array_equal(got1[0][offs[j]:offs[j] + n], got[0][offs[j]:offs[j] + n])
                assert got1[1][a] == got[1][j] and got1[2][a] == got[2][j]


@pytest.mark.parametrize("flags", [0, rac.INCREMENTAL, rac.STOP_ON_WIPEOUT])
def test_batch_wipe_split_over_slabs(flags):
    """A domain emptied only by the AND of two slabs' removals (see
    test_parity_gpu._split_wipe_network), batched with a random network, in
    the batched kernel."""
    from test_parity_gpu import _split_wipe_network
    n, d, scope, rel, dom = _split_wipe_network()
    other = racgen.random_network(8, 1, 300, 12, 0.6, 0.3)
    shapes = [(n, d, scope, rel), (other.n, other.d, other.scope, other.rel)]
    doms, items, offs, pos = [], [], [], 0
    for s in range(6):
        i = s % 2
        dm = dom.copy() if i == 0 else racgen.assignment_state(8, 1, s, other.n, other.d)
        if i == 0 and s >= 2:
            dm[7] = 3
        doms.append(dm)
        items.append(i)
        offs.append(pos)
        pos += shapes[i][0]
    flat = np.concatenate(doms).astype(np.uint32)
    items, offs = np.array(items, np.int32), np.array(offs, np.int64)
    nets = [rac.Network(*sh) for sh in shapes]
    with rac.Plan(nets, items, offs) as plan:
        out, its, sts = _run(nets, items, offs, flat, flags, plan=plan)
    for j in range(len(items)):
        nn, dd, sc, rl = shapes[items[j]]
        ro, ri, rs = oracle.rac(nn, dd, sc, rl, doms[j],
                                stop_on_wipeout=bool(flags & rac.STOP_ON_WIPEOUT), threads=8)
        o = offs[j]
        assert np.array_equal(out[o:o + nn], ro) and its[j] == ri and sts[j] == rs, j
        if items[j] == 0:
            assert rs == rac.WIPEOUT and ri == (1 if flags & rac.STOP_ON_WIPEOUT else 3)
