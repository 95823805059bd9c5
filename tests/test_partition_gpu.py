"""The partitioned sweep on the GPU: each rank's one-sweep partial from the
library (rac_enforce with one sweep on its constraints) and the combine
kernel (rac_combine_partials).  Ranks are threads of this process sharing
the GPU and its default stream, so their kernels run one after another and
never wait on one another; the gather is a host barrier.  Domains, sweep
counts and statuses must equal rac_enforce on the whole network and the
oracle (GPU)."""
import threading

import numpy as np
import pytest

import racgen
import paper_2407_11388_b300 as rac
from paper_2407_11388_b300.partition import (GpuShare, ThreadGroup, TorchGroup,
                                             enforce_partitioned, partition_constraints)
from gpu_helpers import assert_same, gpu_enforce, oracle_enforce, to_dev, torch

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n_parts,n_vars", [(1, 1), (2, 31), (3, 1000), (5, 4097), (4, 2000000)])
def test_combine_partials_against_numpy(n_parts, n_vars):
    T = torch()
    rng = np.random.default_rng(n_parts * 7 + n_vars)

    def words(shape):
        return rng.integers(0, 2 ** 32, shape, dtype=np.uint64).astype(np.uint32)

    prev = words(n_vars) | 1                      # no empty domain before
    cases = [prev[None, :] & words((n_parts, n_vars)),            # removals, some empty
             np.repeat(prev[None, :], n_parts, axis=0),           # a fixpoint: nothing changes
             np.repeat(prev[None, :], n_parts, axis=0) & ~np.uint32(1)]  # changes, none empty
    for i, p in enumerate(cases):
        want = prev & np.bitwise_and.reduce(p, axis=0)
        flags = T.full((2,), 7, dtype=T.int32, device="cuda:0")
        out = T.empty(n_vars, dtype=T.int32, device="cuda:0")
        rac.combine_partials(to_dev(p), to_dev(prev), out, flags)
        T.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy().view(np.uint32), want), i
        f = flags.cpu().tolist()
        assert f == [int(np.any(want != prev)), int(np.any(want == 0))], (i, f)


def test_combine_partials_in_place_and_empty():
    T = torch()
    prev = np.array([0b111, 0b10, 0b1], np.uint32)
    parts = np.array([[0b101, 0b10, 0b1], [0b111, 0b10, 0b0]], np.uint32)
    buf = to_dev(prev)
    flags = T.empty(2, dtype=T.int32, device="cuda:0")
    rac.combine_partials(to_dev(parts).reshape(2, 3), buf, buf, flags)
    T.cuda.synchronize()
    assert buf.cpu().numpy().view(np.uint32).tolist() == [0b101, 0b10, 0]
    assert flags.cpu().tolist() == [1, 1]
    empty = T.empty(0, dtype=T.int32, device="cuda:0")
    rac.combine_partials(empty.reshape(2, 0), empty, empty, flags)
    T.cuda.synchronize()
    assert flags.cpu().tolist() == [0, 0]


def _partitioned(n, d, scope, rel, dom, G, flags=0, max_sweeps=0, layout=rac.LAYOUT_BITS):
    parts, _ = partition_constraints(n, scope, G)
    group = ThreadGroup(G)
    res, errs = [None] * G, []

    def body(g):
        try:
            share = GpuShare(n, d, scope, rel, parts[g], layout=layout)
            try:
                out, it, st = enforce_partitioned(share, group.rank_view(g), to_dev(dom),
                                                  max_sweeps=max_sweeps, flags=flags)
                torch().cuda.synchronize()
                res[g] = (out.cpu().numpy().view(np.uint32).copy(), it, st)
            finally:
                share.close()
        except Exception as e:  # noqa: BLE001 - reported below
            errs.append(e)

    ts = [threading.Thread(target=body, args=(g,)) for g in range(G)]
    for t in ts:
        t.start()
    for t in ts:
        t.join(timeout=300)
    assert not errs, errs
    return res


def _check(n, d, x, doms, G, flags=0, max_sweeps=0, layout=rac.LAYOUT_BITS):
    doms = np.asarray(doms, np.uint32).reshape(-1, n)
    want = oracle_enforce(n, d, x.scope, x.rel, doms, flags=flags, max_sweeps=max_sweeps)
    whole = [gpu_enforce(n, d, x.scope, x.rel, doms[s], flags=flags, max_sweeps=max_sweeps)
             for s in range(doms.shape[0])]
    for s in range(doms.shape[0]):
        assert_same(whole[s], tuple(a[s:s + 1] for a in want), "rac_enforce")
        for g, (out, it, st) in enumerate(_partitioned(n, d, x.scope, x.rel, doms[s], G,
                                                       flags, max_sweeps, layout)):
            got = (out[None, :], np.array([it]), np.array([st]))
            assert_same(got, whole[s], "rank %d of %d, state %d" % (g, G, s))
    return want


def test_large_dense_network_over_four_ranks():
    """n = 2000, d = 32, density 0.9, tightness 0.3 (the large dense
    benchmark network), full domains and assignment states."""
    n, d = 2000, 32
    x = racgen.random_network(0, 0, n, d, 0.9, 0.3)
    doms = [racgen.full_domain(n, d)] + [racgen.assignment_state(0, 0, s, n, d) for s in range(2)]
    _check(n, d, x, doms, 4)


@pytest.mark.parametrize("G", [2, 3])
def test_cascades_wipeouts_and_the_cap(G):
    n, d = 600, 16
    x = racgen.random_network(21, 0, n, d, 0.2, 0.62)
    doms = [racgen.assignment_state(21, 0, s, n, d) for s in range(4)]
    want = _check(n, d, x, doms, G)
    assert want[1].max() >= 3
    _check(n, d, x, doms[:2], G, flags=rac.STOP_ON_WIPEOUT)
    _check(n, d, x, doms[:2], G, max_sweeps=2)


def test_packed_shares_over_three_ranks():
    """Each rank's share stored with packed relation rows (d = 20)."""
    n, d = 700, 20
    x = racgen.random_network(33, 0, n, d, 0.5, 0.4)
    doms = [racgen.full_domain(n, d)] + [racgen.assignment_state(33, 0, s, n, d) for s in range(3)]
    _check(n, d, x, doms, 3, layout=rac.LAYOUT_BITS | rac.LAYOUT_PACKED)
    _check(n, d, x, doms[1:3], 3, flags=rac.STOP_ON_WIPEOUT,
           layout=rac.LAYOUT_BITS | rac.LAYOUT_PACKED)


def test_nccl_group_of_one_rank():
    """The torch.distributed path (NCCL all-gather of device words) with a
    single rank: the whole network is its share."""
    import torch.distributed as dist
    T = torch()
    n, d = 300, 12
    x = racgen.random_network(9, 0, n, d, 0.5, 0.5)
    dom = racgen.assignment_state(9, 0, 1, n, d)
    want = oracle_enforce(n, d, x.scope, x.rel, dom)
    dist.init_process_group("nccl", store=dist.HashStore(), rank=0, world_size=1,
                            device_id=T.device("cuda", 0))
    try:
        share = GpuShare(n, d, x.scope, x.rel, np.arange(x.m))
        out, it, st = enforce_partitioned(share, TorchGroup(), to_dev(dom))
        T.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy().view(np.uint32), want[0][0])
        assert (it, st) == (want[1][0], want[2][0])
        share.close()
    finally:
        dist.destroy_process_group()
