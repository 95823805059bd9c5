"""A CPU stand-in for one rank's share in the partitioned-sweep tests: the
oracle's single Eq. 1 sweep over the rank's constraints gives the partial
next domain, and numpy combines the gathered partials.  The library's own
share (GpuShare) runs the same three steps with its kernels."""
import numpy as np
import torch

import oracle


class OracleShare:
    def __init__(self, n, d, scope, rel, cons):
        scope = np.asarray(scope, dtype=np.int32).reshape(-1, 2)
        self.n, self.d = int(n), int(d)
        self.scope = np.ascontiguousarray(scope[cons])
        self.rel = np.ascontiguousarray(np.asarray(rel, dtype=np.uint32)[cons])

    def load(self, dom_in):
        return torch.from_numpy(np.asarray(dom_in, dtype=np.uint32).view(np.int32).copy())

    def sweep(self, dom):
        d = dom.numpy().view(np.uint32)
        out, _, _ = oracle.rac(self.n, self.d, self.scope, self.rel, d, max_sweeps=1)
        return torch.from_numpy(out.view(np.int32).copy())

    def combine(self, gathered, dom):
        g = gathered.numpy().view(np.uint32).reshape(-1, self.n)
        prev = dom.numpy().view(np.uint32)
        nxt = prev & np.bitwise_and.reduce(g, axis=0)
        return (torch.from_numpy(nxt.view(np.int32).copy()), bool(np.any(nxt != prev)),
                bool(np.any(nxt == 0)))
