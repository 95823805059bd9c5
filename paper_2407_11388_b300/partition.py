"""One network's fixpoint split over several ranks (one process per GPU).

Eq. 1 (Sec. 3) computes every D^(k)[x] from D^(k-1) alone, and a sweep keeps
a value (x,a) only if it has a support on every constraint of C_x: an AND over
the constraints.  Split the constraints over G ranks and rank g's one sweep of
its share gives a partial next domain

    P_g = D^(k-1) AND (supports on the constraints of rank g),

and D^(k) = AND_g P_g exactly, whatever the split.  Per sweep every rank
  1. sweeps its share once (rac_enforce with max_sweeps = 1 on a network
     made of its constraints), giving P_g (n words);
  2. all-gathers the partials (G x n words; 8 KB per rank at n = 2000);
  3. combines them (rac_combine_partials): D^(k), plus "some domain changed"
     and "some domain empty", read off the gathered words and hence identical
     on every rank, so the loop needs no second collective.
The loop ends as Algorithm 1 / the listing end it (checked in this order):
with RAC_STOP_ON_WIPEOUT after the first sweep that leaves a domain empty;
after the first sweep that changes nothing (status WIPEOUT iff a domain is
empty); after max_sweeps sweeps (ETIMEOUT).  `iterations` counts every sweep.

The split is by row blocks of the relation store: constraint (x, y) lies in
tile row I = min(x, y) // 32, and each rank takes a contiguous band of tile
rows, the bands balanced by constraint count, so each rank holds about 1/G of
the store and reads it once per sweep.

A gather that does not complete within its time limit (a rank that stalled,
died or left) ends the enforcement on the ranks still running with status
RAC_EBARRIER and the state before that sweep, instead of hanging.

Proposition 2 gating (RAC_INCREMENTAL) is not offered here: a rank's one-sweep
call examines every constraint of its share.
"""
import datetime
import threading

import numpy as np

from . import (EBARRIER, EINVAL, ETIMEOUT, INCREMENTAL, LAYOUT_BITS, OK, STOP_ON_WIPEOUT, WIPEOUT,
               Network, RacError, combine_partials, enforce)


def partition_constraints(n, scope, n_parts):
    """Row-block split of a network's constraints over n_parts ranks.

    Constraint c = (x, y) lies in tile row min(x, y) // 32; rank g takes the
    tile rows [bounds[g], bounds[g+1]).  The bounds put about total / n_parts
    constraints before each cut (a band can exceed that by at most one tile
    row's constraints).  Returns (parts, bounds): parts[g] is the sorted
    index array of rank g's constraints."""
    if n_parts < 1:
        raise ValueError("n_parts must be >= 1")
    scope = np.asarray(scope, dtype=np.int64).reshape(-1, 2)
    nb = (int(n) + 31) // 32
    rows = np.minimum(scope[:, 0], scope[:, 1]) // 32
    counts = np.bincount(rows, minlength=nb) if scope.shape[0] else np.zeros(nb, np.int64)
    cum = np.cumsum(counts)
    total = int(cum[-1]) if nb else 0
    bounds = [0]
    for g in range(1, n_parts):
        # first tile row at which the running count reaches g/n_parts of all
        r = int(np.searchsorted(cum, total * g / n_parts, side="left")) + 1 if total else 0
        bounds.append(min(max(r, bounds[-1]), nb))
    bounds.append(nb)
    order = np.argsort(rows, kind="stable")
    sorted_rows = rows[order]
    parts = []
    for g in range(n_parts):
        lo = np.searchsorted(sorted_rows, bounds[g], side="left")
        hi = np.searchsorted(sorted_rows, bounds[g + 1], side="left")
        parts.append(np.sort(order[lo:hi]))
    return parts, bounds


class GatherTimeout(RuntimeError):
    """A collective did not complete within its limit."""


class TorchGroup:
    """The ranks of a torch.distributed process group (NCCL for GPU tensors,
    gloo for CPU tensors): one all-gather per sweep, waited on with a time
    limit."""

    def __init__(self, group=None):
        import torch.distributed as dist
        self.dist = dist
        self.group = group
        self.rank = dist.get_rank(group)
        self.size = dist.get_world_size(group)

    def all_gather(self, partial, timeout_s):
        import torch
        # a flat output: gloo takes only that, NCCL either
        out = torch.empty(self.size * partial.numel(), dtype=partial.dtype, device=partial.device)
        work = self.dist.all_gather_into_tensor(out, partial.reshape(-1), group=self.group,
                                                async_op=True)
        try:
            work.wait(timeout=datetime.timedelta(seconds=timeout_s))
        except RuntimeError as e:  # timed out, or a peer's connection closed
            raise GatherTimeout(str(e)) from e
        return out.reshape((self.size,) + tuple(partial.shape))


class ThreadGroup:
    """Ranks emulated by threads of one process (each thread one rank, all
    on the same device): the all-gather is a barrier on the host.  Each
    rank's partial is copied out after its stream is synchronised, so the
    ranks' kernels never wait on one another."""

    def __init__(self, size):
        self.size = size
        self._slots = [None] * size
        self._barrier = threading.Barrier(size)

    def rank_view(self, rank):
        """The group as seen by one rank (one view per thread)."""
        return _ThreadRank(self, rank)


class _ThreadRank:
    def __init__(self, group, rank):
        self.g = group
        self.rank = rank
        self.size = group.size

    def all_gather(self, partial, timeout_s):
        import torch
        if partial.is_cuda:
            torch.cuda.current_stream(partial.device).synchronize()
        self.g._slots[self.rank] = partial.clone()
        if partial.is_cuda:
            torch.cuda.current_stream(partial.device).synchronize()
        try:
            self.g._barrier.wait(timeout=timeout_s)       # every partial deposited
            out = torch.stack(self.g._slots)
            if out.is_cuda:
                torch.cuda.current_stream(out.device).synchronize()
            self.g._barrier.wait(timeout=timeout_s)       # every rank has its copy
        except threading.BrokenBarrierError as e:
            raise GatherTimeout("a rank did not arrive within %.3g s" % timeout_s) from e
        return out


class GpuShare:
    """One rank's share of a network on the current CUDA device: its
    constraints as a library network, and the buffers of its sweeps.  All of
    its work goes to torch's current stream of the calling thread."""

    def __init__(self, n, d, scope, rel, cons, layout=LAYOUT_BITS):
        import torch
        scope = np.asarray(scope, dtype=np.int32).reshape(-1, 2)
        rel = np.asarray(rel)
        self.n, self.d = int(n), int(d)
        self.net = Network(n, d, scope[cons], rel[cons], layout=layout)
        dev = torch.device("cuda", torch.cuda.current_device())
        self.partial = torch.empty(self.n, dtype=torch.int32, device=dev)
        self.bufs = [torch.empty(self.n, dtype=torch.int32, device=dev) for _ in range(2)]
        self.it = torch.empty(1, dtype=torch.int32, device=dev)
        self.st = torch.empty(1, dtype=torch.int32, device=dev)
        self.flags = torch.empty(2, dtype=torch.int32, device=dev)
        self._cur = 0

    def load(self, dom_in):
        self.bufs[0].copy_(dom_in.reshape(-1))
        self._cur = 0
        return self.bufs[0]

    def sweep(self, dom):
        """P_g: one sweep of this rank's constraints on dom (the state before
        the sweep)."""
        enforce(self.net, dom, self.partial, self.it, self.st, max_sweeps=1)
        return self.partial

    def combine(self, gathered, dom):
        """(D^(k), some domain changed, some domain empty)."""
        nxt = self.bufs[1 - self._cur]
        combine_partials(gathered.reshape(-1, self.n), dom, nxt, self.flags)
        f = self.flags.cpu()  # the loop's decision: one small copy per sweep
        self._cur = 1 - self._cur
        return nxt, bool(f[0]), bool(f[1])

    def close(self):
        self.net.close()


def enforce_partitioned(share, group, dom_in, max_sweeps=0, flags=0, timeout_s=30.0):
    """Eq. 1 to its fixpoint with the constraints split over the ranks of
    `group`; every rank calls this with its own `share` (GpuShare, or any
    object with the same load / sweep / combine methods) and the same
    dom_in.  Returns (domain, iterations, status), identical on every rank;
    a gather that runs out of time gives status RAC_EBARRIER and the state
    before that sweep."""
    if flags & INCREMENTAL:
        raise RacError(EINVAL, "enforce_partitioned: Proposition 2 gating is not offered here")
    if flags & ~(STOP_ON_WIPEOUT | INCREMENTAL):
        raise RacError(EINVAL, "enforce_partitioned: unknown flag")
    stop = bool(flags & STOP_ON_WIPEOUT)
    dom = share.load(dom_in)
    k = 0
    while True:
        k += 1
        partial = share.sweep(dom)
        try:
            gathered = group.all_gather(partial, timeout_s)
        except GatherTimeout:
            return dom, k, EBARRIER
        dom, changed, empty = share.combine(gathered, dom)
        if stop and empty:
            return dom, k, WIPEOUT
        if not changed:
            return dom, k, WIPEOUT if empty else OK
        if max_sweeps > 0 and k >= max_sweeps:
            return dom, k, ETIMEOUT
