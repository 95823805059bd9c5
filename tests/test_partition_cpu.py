"""The partitioned sweep of one network (Eq. 1 with its constraints split over
ranks by row blocks of the store) on CPU ranks: gloo processes and threads,
each rank's one-sweep partial from the oracle restricted to its constraints.
The loop (gather, combine, the stop decisions and the sweep count) must give
exactly the oracle's single-process result, and a rank that stalls must make
the others return RAC_EBARRIER instead of hanging (no GPU)."""
import os
import socket
import threading
import time

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle
import racgen
import paper_2407_11388_b300 as rac
from paper_2407_11388_b300.partition import (ThreadGroup, enforce_partitioned,
                                             partition_constraints)
from partition_helpers import OracleShare


def _chain(n, d):
    """x_0 < x_1 < ... < x_{n-1}: D_ac(x_i) = [i, d-n+i] in exactly n sweeps."""
    scope = np.array([[i, i + 1] for i in range(n - 1)], np.int32)
    rel = np.array([[sum(1 << b for b in range(a + 1, d)) for a in range(d)]] * (n - 1),
                   np.uint32)
    return scope, rel


def _cases():
    """(n, d, scope, rel, dom, flags, max_sweeps): cascades over many sweeps,
    wipe-outs in both modes, the sweep cap, a chain spread over tile rows."""
    out = []
    for seed, (n, d, p, t) in enumerate([(150, 8, 0.3, 0.55), (200, 12, 0.25, 0.6),
                                         (97, 6, 0.5, 0.45)]):
        x = racgen.random_network(40 + seed, 0, n, d, p, t)
        for s in range(3):
            dom = racgen.assignment_state(40 + seed, 0, s, n, d)
            out.append((n, d, x.scope, x.rel, dom, 0, 0))
            out.append((n, d, x.scope, x.rel, dom, rac.STOP_ON_WIPEOUT, 0))
        out.append((n, d, x.scope, x.rel, racgen.full_domain(n, d), 0, 0))
        out.append((n, d, x.scope, x.rel, racgen.assignment_state(40 + seed, 0, 7, n, d), 0, 2))
    # a chain across three tile rows (d < n: wipes out) and one that keeps
    # its closed-form D_ac after exactly n sweeps
    out.append((70, 32, *_chain(70, 32), np.full(70, 0xFFFFFFFF, np.uint32), 0, 0))
    out.append((20, 24, *_chain(20, 24), np.full(20, (1 << 24) - 1, np.uint32), 0, 0))
    return out


def _want(case):
    n, d, scope, rel, dom, flags, cap = case
    return oracle.rac(n, d, scope, rel, dom, stop_on_wipeout=bool(flags & rac.STOP_ON_WIPEOUT),
                      max_sweeps=cap)


def test_row_bands_partition_every_constraint_once():
    for n, p, G in [(2000, 0.9, 4), (1000, 0.3, 8), (100, 1.0, 3), (40, 0.5, 5), (33, 1.0, 2)]:
        x = racgen.random_network(3, 0, n, 4, p, 0.3)
        parts, bounds = partition_constraints(n, x.scope, G)
        allc = np.concatenate(parts)
        assert np.array_equal(np.sort(allc), np.arange(x.m))        # each exactly once
        assert bounds[0] == 0 and bounds[-1] == (n + 31) // 32
        assert all(a <= b for a, b in zip(bounds, bounds[1:]))
        rows = np.minimum(x.scope[:, 0], x.scope[:, 1]) // 32
        per_row = np.bincount(rows, minlength=(n + 31) // 32)
        for g in range(G):                                          # a contiguous band
            r = rows[parts[g]]
            assert r.size == 0 or (r.min() >= bounds[g] and r.max() < bounds[g + 1])
            # balanced: at most one tile row above an even share
            assert len(parts[g]) <= x.m / G + per_row.max() + 1


def test_no_constraints_and_one_rank():
    parts, bounds = partition_constraints(10, np.zeros((0, 2), np.int32), 3)
    assert [len(p) for p in parts] == [0, 0, 0] and bounds == [0, 0, 0, 1]
    x = racgen.random_network(5, 0, 64, 4, 0.5, 0.3)
    parts, _ = partition_constraints(64, x.scope, 1)
    assert np.array_equal(parts[0], np.arange(x.m))


def _run_threads(case, G, timeout_s=30.0, stall=None):
    n, d, scope, rel, dom, flags, cap = case
    parts, _ = partition_constraints(n, scope, G)
    group = ThreadGroup(G)
    res = [None] * G

    class Stalling(OracleShare):
        def __init__(self, *a, rank):
            super().__init__(*a)
            self.rank, self.k = rank, 0

        def sweep(self, dom_):
            self.k += 1
            if stall and self.rank == stall[0] and self.k == stall[1]:
                time.sleep(stall[2])
            return super().sweep(dom_)

    def body(g):
        share = Stalling(n, d, scope, rel, parts[g], rank=g)
        out, it, st = enforce_partitioned(share, group.rank_view(g), dom, max_sweeps=cap,
                                          flags=flags, timeout_s=timeout_s)
        res[g] = (out.numpy().view(np.uint32).copy(), it, st)

    ts = [threading.Thread(target=body, args=(g,)) for g in range(G)]
    for t in ts:
        t.start()
    for t in ts:
        t.join(timeout=120)
    assert all(r is not None for r in res)
    return res


@pytest.mark.parametrize("G", [2, 3, 5])
def test_thread_ranks_match_the_oracle(G):
    for case in _cases():
        want = _want(case)
        for out, it, st in _run_threads(case, G):
            assert np.array_equal(out, want[0]) and (it, st) == (want[1], want[2]), case[:2]


def test_a_stalled_thread_rank_times_out_the_others():
    x = racgen.random_network(41, 0, 200, 12, 0.25, 0.6)
    dom = racgen.assignment_state(41, 0, 0, 200, 12)
    case = (200, 12, x.scope, x.rel, dom, 0, 0)
    want_it = _want(case)[1]
    assert want_it >= 3
    t0 = time.perf_counter()
    res = _run_threads(case, 3, timeout_s=0.5, stall=(1, 2, 2.0))
    assert time.perf_counter() - t0 < 10
    one_sweep = oracle.rac(200, 12, x.scope, x.rel, dom, max_sweeps=1)[0]
    for g, (out, it, st) in enumerate(res):
        assert st == rac.EBARRIER and it == 2
        assert np.array_equal(out, one_sweep)    # the state before the sweep that failed


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _gloo_rank(rank, world, port, q, stall):
    import datetime

    import torch.distributed as dist
    from paper_2407_11388_b300.partition import TorchGroup
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=60))
    group = TorchGroup()
    cases = _cases() if stall is None else [_stall_case()]
    out = []
    for n, d, scope, rel, dom, flags, cap in cases:
        parts, _ = partition_constraints(n, scope, world)

        class Share(OracleShare):
            k = 0

            def sweep(self, dom_):
                self.k += 1
                if stall and rank == stall[0] and self.k == stall[1]:
                    time.sleep(stall[2])
                return super().sweep(dom_)

        share = Share(n, d, scope, rel, parts[rank])
        t0 = time.perf_counter()
        dom_out, it, st = enforce_partitioned(share, group, dom, max_sweeps=cap, flags=flags,
                                              timeout_s=1.0 if stall else 60.0)
        out.append((dom_out.numpy().view(np.uint32).copy(), it, st, time.perf_counter() - t0))
    q.put((rank, out))
    q.close()
    q.join_thread()
    if stall is None:
        dist.barrier()
        dist.destroy_process_group()
    # after a failed gather the group is not torn down collectively: the
    # process ends here without waiting on its peers
    os._exit(0)


def _stall_case():
    x = racgen.random_network(41, 0, 200, 12, 0.25, 0.6)
    return (200, 12, x.scope, x.rel, racgen.assignment_state(41, 0, 0, 200, 12), 0, 0)


def _spawn(world, stall=None):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_gloo_rank, args=(r, world, port, q, stall)) for r in range(world)]
    for p in procs:
        p.start()
    res = {}
    try:
        for _ in range(world):
            r, out = q.get(timeout=240)
            res[r] = out
    finally:
        for p in procs:
            p.join(timeout=30)
            if p.is_alive():
                p.kill()
    return res


@pytest.mark.parametrize("world", [2, 4])
def test_gloo_ranks_match_the_oracle(world):
    res = _spawn(world)
    cases = _cases()
    for i, case in enumerate(cases):
        want = _want(case)
        for r in range(world):
            out, it, st, _ = res[r][i]
            assert np.array_equal(out, want[0]), (r, i)
            assert (it, st) == (want[1], want[2]), (r, i, it, st, want[1:])


def test_a_stalled_gloo_rank_times_out_the_others():
    """Rank 1 of 3 sleeps 4 s before its second sweep; the others' gather of
    that sweep gives up after 1 s and they return RAC_EBARRIER with the state
    after sweep 1; the sleeper then finds its peers gone and returns the same
    status."""
    res = _spawn(3, stall=(1, 2, 4.0))
    n, d, scope, rel, dom, _, _ = _stall_case()
    one_sweep = oracle.rac(n, d, scope, rel, dom, max_sweeps=1)[0]
    for r in range(3):
        out, it, st, el = res[r][0]
        assert st == rac.EBARRIER and it == 2, (r, it, st)
        assert np.array_equal(out, one_sweep)
        if r != 1:
            assert el < 3.5, "the gather's limit is 1 s"
