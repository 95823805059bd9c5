"""Backtrack search over the device enforcement (Algorithm 2 of the paper).

`dfs` follows Algorithm 2: enforce arc consistency on the initial domains
(`tensorAC(Vars, all)`), then repeatedly pick a variable, try its values in
order, and after each `assign` enforce with only that variable changed
(`tensorAC(Vars, [idx])`, rac_assign_enforce), descending while no domain is
empty and backtracking otherwise.  The states of the levels stay on the
device; after each enforcement one read brings the child state, its sweep
count and its status back together (the variable-ordering heuristic, which
the paper leaves open, needs the state: smallest domain of size > 1, lowest
index first).  Every assignment's sweep count is recorded: it is the
quantity Table 1 reports as #Recurrence.
"""
from dataclasses import dataclass, field

import numpy as np

from . import OK, assign_enforce, enforce


@dataclass
class SearchResult:
    solution: object = None              # uint32 domain words (all singletons) or None
    steps: list = field(default_factory=list)  # (level, var, value, iterations, status)
    root_iterations: int = 0
    root_status: int = OK
    nodes: int = 0
    exhausted: bool = False              # the node budget ran out

    def mean_sweeps(self):
        return float(np.mean([s[3] for s in self.steps])) if self.steps else 0.0


def choose_variable(dom):
    """Smallest domain of size > 1, lowest index; None when all are singletons."""
    words = np.ascontiguousarray(dom, dtype=np.uint32)
    sizes = np.bitwise_count(words)
    open_vars = np.flatnonzero(sizes > 1)
    if open_vars.size == 0:
        return None
    return int(open_vars[np.argmin(sizes[open_vars])])


def dfs(net, dom0, max_nodes=10_000, stream=None, flags=0, hook=None):
    """Depth-first search of Algorithm 2 on the device.  dom0: host uint32
    words (n).  hook, if given, is called with "before" and "after" around
    each assignment's enforcement launch (to time it on the stream).  Returns
    a SearchResult."""
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    n = net.n
    res = SearchResult()
    # a level's buffer: its n domain words, then the sweep count and status of
    # the enforcement that produced it, so that one read brings all three back
    bufs = [torch.empty(n + 2, dtype=torch.int32, device=dev) for _ in range(n + 1)]
    levels = [b[:n] for b in bufs]
    bufs[0][:n].copy_(torch.from_numpy(np.ascontiguousarray(dom0, dtype=np.uint32).view(np.int32)))
    enforce(net, levels[0], levels[0], bufs[0][n:n + 1], bufs[0][n + 1:], flags=flags,
            stream=stream)
    host = bufs[0].cpu().numpy()
    res.root_iterations = int(host[n])
    res.root_status = int(host[n + 1])
    if res.root_status != OK:
        return res
    doms = {0: host[:n].view(np.uint32)}

    def rec(level):
        dom = doms[level]
        var = choose_variable(dom)
        if var is None:
            res.solution = dom.copy()
            return True
        for value in range(net.d):
            if not (int(dom[var]) >> value) & 1:
                continue
            if res.nodes >= max_nodes:
                res.exhausted = True
                return False
            res.nodes += 1
            if hook:
                hook("before")
            nxt = bufs[level + 1]
            assign_enforce(net, levels[level], levels[level + 1], var, value, nxt[n:n + 1],
                           nxt[n + 1:], flags=flags, stream=stream)
            if hook:
                hook("after")
            host = nxt.cpu().numpy()  # the child state, its sweep count and status
            iters, status = int(host[n]), int(host[n + 1])
            doms[level + 1] = host[:n].view(np.uint32)
            res.steps.append((level, var, value, iters, status))
            if status == OK and rec(level + 1):
                return True
            if res.exhausted:
                return False
        return False

    rec(0)
    return res
