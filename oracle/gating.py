"""Plain definitions behind learned gating (TEST INFRASTRUCTURE ONLY).

Only tests/ and the benchmark may import this; it shares no code with the
CUDA library.  It restates, on the network's constraint list and on the
per-sweep domains the oracle's Eq. 1 recurrence records, what the trace of a
gated enforcement must contain:

  slabs(n, scope, rows)   the relation slabs: (I, J, row0) for every group of
                          constraints with lo // 32 == I, hi // 32 == J and
                          (lo % 32) // rows == row0 // rows (lo < hi the
                          constraint's variables);
  candidate(...)          Proposition 2: some variable of the slab's rows or of
                          its column block changed in sweep k-1 (before sweep
                          1 every pair is a candidate, and a variable counts
                          as changed when its input domain is not full);
  label(...)              the evaluation of the slab's constraints on D_{k-1}
                          removes a value: some (x, a) with a in D_{k-1}(x) has
                          no b in D_{k-1}(y) with R_xy[a][b] on one of them
                          (Eq. 1 restricted to those constraints), or the same
                          for some (y, b);
  features(...)           the predictor's eight inputs, as include/rac.h
                          states them.
"""
import numpy as np


def _popcount(words):
    w = np.asarray(words, dtype=np.uint64)
    return np.array([bin(int(v)).count("1") for v in w.reshape(-1)], dtype=np.int64).reshape(w.shape)


class SlabIndex:
    """The constraints of each slab, in the (lo, hi) orientation."""

    def __init__(self, n, d, scope, rel, rows):
        scope = np.asarray(scope, dtype=np.int64).reshape(-1, 2)
        rel = np.asarray(rel, dtype=np.uint64).reshape(-1, d)
        self.n, self.d, self.rows = n, d, rows
        lo = np.minimum(scope[:, 0], scope[:, 1])
        hi = np.maximum(scope[:, 0], scope[:, 1])
        swap = scope[:, 0] > scope[:, 1]
        # relation as a boolean [m, d, d] in (lo, hi) orientation
        bits = ((rel[:, :, None] >> np.arange(d, dtype=np.uint64)[None, None, :]) & 1).astype(bool)
        self.R = np.where(swap[:, None, None], bits.transpose(0, 2, 1), bits)
        self.lo, self.hi = lo, hi
        key = list(zip(lo // 32, hi // 32, ((lo % 32) // rows) * rows))
        self.members = {}
        for c, k in enumerate(key):
            self.members.setdefault((int(k[0]), int(k[1]), int(k[2])), []).append(c)
        self.keys = sorted(self.members)

    def tightness(self, key):
        cs = self.members[key]
        allowed = self.R[cs].sum()
        return 1.0 - allowed / (len(cs) * self.d * self.d)

    def density(self, key):
        return len(self.members[key]) / (self.rows * 32.0)


def _dom_bits(D, d):
    D = np.asarray(D, dtype=np.uint64)
    return ((D[:, None] >> np.arange(d, dtype=np.uint64)[None, :]) & 1).astype(bool)


def label(idx, key, D_prev):
    """Does evaluating the slab on the domain D_prev remove a value?"""
    cs = np.array(idx.members[key])
    Db = _dom_bits(D_prev, idx.d)
    R = idx.R[cs]
    x, y = idx.lo[cs], idx.hi[cs]
    fwd_lost = ~(R & Db[y][:, None, :]).any(2) & Db[x]   # (x, a) with no support in D(y)
    rev_lost = ~(R & Db[x][:, :, None]).any(1) & Db[y]   # (y, b) with no support in D(x)
    return bool(fwd_lost.any() or rev_lost.any())


def slab_rows(idx, key):
    I, J, row0 = key
    xs = [32 * I + row0 + r for r in range(idx.rows) if 32 * I + row0 + r < idx.n]
    ys = [32 * J + j for j in range(32) if 32 * J + j < idx.n]
    return xs, ys


def candidate(idx, key, changed):
    xs, ys = slab_rows(idx, key)
    return bool(changed[xs].any() or changed[ys].any())


def features(idx, key, k, changed, D_prev):
    """The eight inputs of (slab, state) before sweep k (changed: variables
    whose domain changed in sweep k-1; D_prev = D_{k-1})."""
    xs, ys = slab_rows(idx, key)
    d = idx.d
    sz = _popcount(D_prev)
    return np.array([
        min(k, 16) / 16.0,
        changed[xs].sum() / idx.rows,
        changed[ys].sum() / 32.0,
        idx.tightness(key),
        idx.density(key),
        sz[ys].min() / d,
        sz[ys].sum() / (len(ys) * d),
        sz[xs].min() / d,
    ])
