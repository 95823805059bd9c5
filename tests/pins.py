"""Checks that pin the CPU oracle to facts other than itself.

Each function takes an oracle library handle (so the mutation tests can run
the same checks on copies with planted mistakes) and returns a list of
failure messages (empty = pinned).  Sources of truth:
  * hand-derived worked examples under tests/golden/ (Sec. 3 definitions);
  * the chain closed form: x_0 < ... < x_{n-1} on d >= n values has
    D_ac(x_i) = [i, d-n+i] and takes exactly n sweeps (n-1 removing sweeps
    plus the final one);
  * brute force over all subsets (D_ac = union of the arc-consistent subsets,
    Sec. 3) and AC-3 (a different algorithm reaching the same set);
  * properties: the result is arc consistent, enforcement is idempotent,
    sweeps <= |D|+1 (Proposition 1), every sweep only removes, and the
    incremental run removes the same values in every sweep (Proposition 2);
  * the paper's dense tensor form of a sweep (Sec. 4, Fig. 1, Algorithm 1),
    restated in numpy: the same states and sweep counts while no domain is
    empty.
"""
import numpy as np

import oracle
from cases import (chain, chain_closed_form, full_word, golden_names, is_arc_consistent,
                   load_golden, random_tiny, tuned_tightness)


def pin_golden(lib):
    fails = []
    for name in golden_names():
        g = load_golden(name)
        out, it, st = oracle.rac(g["n"], g["d"], g["scope"], g["rel"], g["dom"],
                                 stop_on_wipeout=g["stop"], lib=lib)
        if not np.array_equal(out, g["expected"]) or it != g["iterations"] or st != g["status"]:
            fails.append("golden %s: rac gave %s it=%d st=%d" % (name, out.tolist(), it, st))
        if not g["stop"]:
            o1, _, s1 = oracle.ac3(g["n"], g["d"], g["scope"], g["rel"], g["dom"], lib=lib)
            if not np.array_equal(o1, g["expected"]) or s1 != g["status"]:
                fails.append("golden %s: ac3 gave %s" % (name, o1.tolist()))
            o3, s3 = oracle.bruteforce(g["n"], g["d"], g["scope"], g["rel"], g["dom"], lib=lib)
            if not np.array_equal(o3, g["expected"]) or s3 != g["status"]:
                fails.append("golden %s: bruteforce gave %s" % (name, o3.tolist()))
    return fails


def pin_chain(lib):
    fails = []
    for n in range(2, 11):
        for d in range(n, n + 4):
            for rev in (False, True):
                scope, rel = chain(n, d, reverse_scopes=rev)
                dom = np.full(n, full_word(d), dtype=np.uint32)
                want = chain_closed_form(n, d)
                out, it, st = oracle.rac(n, d, scope, rel, dom, lib=lib)
                if not np.array_equal(out, want) or it != n or st != oracle.OK:
                    fails.append("chain n=%d d=%d rev=%s: rac it=%d" % (n, d, rev, it))
                o1, _, _ = oracle.ac3(n, d, scope, rel, dom, lib=lib)
                if not np.array_equal(o1, want):
                    fails.append("chain n=%d d=%d rev=%s: ac3" % (n, d, rev))
                if n * d <= 16:
                    o3, _ = oracle.bruteforce(n, d, scope, rel, dom, lib=lib)
                    if not np.array_equal(o3, want):
                        fails.append("chain n=%d d=%d: bruteforce" % (n, d))
        # fewer values than variables: no arc-consistent value anywhere
        d = n - 1
        if d >= 1:
            scope, rel = chain(n, d)
            dom = np.full(n, full_word(d), dtype=np.uint32)
            out, it, st = oracle.rac(n, d, scope, rel, dom, lib=lib)
            if out.any() or st != oracle.WIPEOUT:
                fails.append("chain n=%d d=%d should wipe out" % (n, d))
            o1, _, s1 = oracle.ac3(n, d, scope, rel, dom, lib=lib)
            if o1.any() or s1 != oracle.WIPEOUT:
                fails.append("chain n=%d d=%d ac3 should wipe out" % (n, d))
    return fails


def pin_special_cases(lib):
    fails = []
    rng = np.random.default_rng(7)
    # no constraints: nothing changes, one sweep
    for n, d in [(1, 1), (5, 3), (40, 32)]:
        dom = rng.integers(1, 1 << min(d, 31), size=n).astype(np.uint32) & np.uint32(full_word(d))
        dom[dom == 0] = 1
        out, it, st = oracle.rac(n, d, np.zeros((0, 2), np.int32), np.zeros((0, d), np.uint32),
                                 dom, lib=lib)
        if not np.array_equal(out, dom) or it != 1 or st != oracle.OK:
            fails.append("no constraints n=%d d=%d" % (n, d))
    # all-ones relations on a random graph: nothing changes, one sweep
    n, d = 12, 7
    scope = np.array([(x, y) for x in range(n) for y in range(x + 1, n) if (x * 7 + y) % 3],
                     dtype=np.int32)
    rel = np.full((scope.shape[0], d), full_word(d), dtype=np.uint32)
    dom = np.full(n, full_word(d), dtype=np.uint32)
    out, it, st = oracle.rac(n, d, scope, rel, dom, lib=lib)
    if not np.array_equal(out, dom) or it != 1 or st != oracle.OK:
        fails.append("all-ones relations")
    # one all-zero relation: both ends emptied in sweep 1
    for stop, want_it in ((False, 2), (True, 1)):
        out, it, st = oracle.rac(2, 4, np.array([[0, 1]], np.int32), np.zeros((1, 4), np.uint32),
                                 np.full(2, 15, np.uint32), stop_on_wipeout=stop, lib=lib)
        if out.any() or it != want_it or st != oracle.WIPEOUT:
            fails.append("all-zero relation stop=%s it=%d" % (stop, it))
    # a singleton x = a reduces its neighbour y to {b : R[a][b]} in sweep 1
    d = 6
    for a in range(d):
        row = rng.integers(1, 1 << d, size=d).astype(np.uint32)
        scope = np.array([[0, 1]], np.int32)
        dom = np.array([1 << a, full_word(d)], np.uint32)
        out, it, st = oracle.rac(2, d, scope, row[None, :], dom, lib=lib)
        if out[1] != row[a] or out[0] != (1 << a) or st != oracle.OK:
            fails.append("singleton a=%d" % a)
    return fails


def pin_three_way(lib, cases=1500, seed=11):
    """Eq. 1, AC-3 and the brute-force union agree on tiny random networks."""
    fails = []
    rng = np.random.default_rng(seed)
    for i in range(cases):
        n = int(rng.integers(2, 6))
        d = int(rng.integers(1, 5))
        if n * d > 16:
            d = 16 // n
        scope, rel, dom = random_tiny(rng, n, d, rng.uniform(0.3, 1.0), rng.uniform(0.3, 0.9),
                                      restrict=rng.uniform(0.0, 0.4))
        o2, it, s2 = oracle.rac(n, d, scope, rel, dom, lib=lib)
        o1, _, s1 = oracle.ac3(n, d, scope, rel, dom, lib=lib)
        o3, s3 = oracle.bruteforce(n, d, scope, rel, dom, lib=lib)
        if not (np.array_equal(o1, o2) and np.array_equal(o2, o3)) or not (s1 == s2 == s3):
            fails.append("case %d (n=%d d=%d): rac %s ac3 %s bf %s" % (
                i, n, d, o2.tolist(), o1.tolist(), o3.tolist()))
            if len(fails) > 5:
                break
        if it > int(sum(bin(int(w)).count("1") for w in dom)) + 1:
            fails.append("case %d: %d sweeps exceed |D|+1" % (i, it))
    return fails


def pin_invariants(lib, seed=5):
    """Arc consistency of the result, idempotence, monotone sweeps, the final
    sweep removing nothing, |D|+1 bound, and agreement with AC-3 on mid-size
    networks."""
    fails = []
    rng = np.random.default_rng(seed)
    for i in range(12):
        n = int(rng.integers(10, 30))
        d = int(rng.integers(2, 9))
        scope, rel, dom = random_tiny(rng, n, d, rng.uniform(0.1, 0.6), rng.uniform(0.4, 0.8),
                                      restrict=rng.uniform(0.0, 0.5))
        out, it, st, tr, rem = oracle.rac(n, d, scope, rel, dom, trace=True, lib=lib)
        if not is_arc_consistent(n, d, scope, rel, out):
            fails.append("inv %d: result not arc consistent" % i)
        o1, _, _ = oracle.ac3(n, d, scope, rel, dom, lib=lib)
        if not np.array_equal(o1, out):
            fails.append("inv %d: ac3 differs" % i)
        again, it2, _ = oracle.rac(n, d, scope, rel, out, lib=lib)
        if not np.array_equal(again, out) or it2 != 1:
            fails.append("inv %d: not idempotent" % i)
        prev = dom
        for k in range(tr.shape[0]):
            if np.any(tr[k] & ~prev):
                fails.append("inv %d: sweep %d adds values" % (i, k + 1))
            prev = tr[k]
        if tr.shape[0] != it or not np.array_equal(tr[-1], out) or rem[-1] != 0:
            fails.append("inv %d: trace does not end in a removal-free sweep" % i)
        if it > 1 and not np.array_equal(tr[-2], out):
            fails.append("inv %d: last sweep changed the domain" % i)
        if (st == oracle.WIPEOUT) != bool(np.any(out == 0)):
            fails.append("inv %d: status %d vs empty domains" % (i, st))
    return fails


def pin_incremental(lib, seed=9):
    """Proposition 2: restricting sweep k >= 2 to constraints whose far end
    lost a value in sweep k-1 removes exactly the same values every sweep."""
    fails = []
    rng = np.random.default_rng(seed)
    for i in range(15):
        n = int(rng.integers(5, 25))
        d = int(rng.integers(2, 8))
        scope, rel, dom = random_tiny(rng, n, d, rng.uniform(0.1, 0.7), rng.uniform(0.4, 0.85),
                                      restrict=rng.uniform(0.0, 0.5))
        a = oracle.rac(n, d, scope, rel, dom, trace=True, lib=lib)
        b = oracle.rac(n, d, scope, rel, dom, trace=True, incremental=True, lib=lib)
        if a[1] != b[1] or not np.array_equal(a[3], b[3]) or not np.array_equal(a[4], b[4]):
            fails.append("incremental %d differs (%d vs %d sweeps)" % (i, a[1], b[1]))
    # on a chain the plain and restricted runs differ in work, not in result
    scope, rel = chain(8, 9)
    dom = np.full(8, full_word(9), np.uint32)
    b = oracle.rac(8, 9, scope, rel, dom, incremental=True, lib=lib)
    if not np.array_equal(b[0], chain_closed_form(8, 9)) or b[1] != 8:
        fails.append("incremental chain")
    return fails


def pin_stop_and_cap(lib, seed=3):
    """Stop-on-wipeout returns the state of the first sweep with an empty
    domain; a sweep cap returns the capped sweep's state."""
    fails = []
    rng = np.random.default_rng(seed)
    seen = 0
    for i in range(60):
        n = int(rng.integers(4, 15))
        d = int(rng.integers(2, 6))
        scope, rel, dom = random_tiny(rng, n, d, rng.uniform(0.3, 0.9), rng.uniform(0.5, 0.9),
                                      restrict=rng.uniform(0.0, 0.3))
        out, it, st, tr, _ = oracle.rac(n, d, scope, rel, dom, trace=True, lib=lib)
        first = next((k for k in range(tr.shape[0]) if np.any(tr[k] == 0)), None)
        so, sit, sst = oracle.rac(n, d, scope, rel, dom, stop_on_wipeout=True, lib=lib)
        if first is None:
            if sit != it or not np.array_equal(so, out) or sst != oracle.OK:
                fails.append("stop %d: no wipe-out but results differ" % i)
        else:
            seen += 1
            if sit != first + 1 or not np.array_equal(so, tr[first]) or sst != oracle.WIPEOUT:
                fails.append("stop %d: wanted sweep %d got %d" % (i, first + 1, sit))
    if seen < 5:
        fails.append("stop: too few wipe-out cases (%d)" % seen)
    scope, rel = chain(6, 8)
    dom = np.full(6, full_word(8), np.uint32)
    full = oracle.rac(6, 8, scope, rel, dom, trace=True, lib=lib)
    for cap in range(1, 6):
        o, it, st = oracle.rac(6, 8, scope, rel, dom, max_sweeps=cap, lib=lib)
        if it != cap or st != oracle.ETIMEOUT or not np.array_equal(o, full[3][cap - 1]):
            fails.append("cap %d: it=%d st=%d" % (cap, it, st))
    o, it, st = oracle.rac(6, 8, scope, rel, dom, max_sweeps=6, lib=lib)
    if it != 6 or st != oracle.OK:
        fails.append("cap equal to the sweep count must reach the fixpoint")
    return fails


def tensor_form(n, d, scope, rel, dom, stop_on_wipeout):
    """One state enforced in the paper's dense tensor form (Sec. 4, Fig. 1,
    Algorithm 1), in plain numpy:
    - a constraint tensor of n x n blocks of d x d, holding R_xy on a
      constrained pair, its transpose on (y, x), and all ones on an
      unconstrained pair and on the diagonal;
    - the support counts of every value, that tensor times the n x d domain
      mask;
    - each count clamped to {0, 1} and summed over y;
    - (x, a) kept iff the sum reaches n.
    The wipe-out test comes before the no-change test.  The input domains
    must be non-empty.  Returns (domain words, sweeps, status)."""
    cons = np.ones((n, n, d, d), dtype=np.int64)
    bits = np.arange(d)
    for c, (x, y) in enumerate(scope):
        R = (np.asarray(rel[c], dtype=np.int64)[:, None] >> bits[None, :]) & 1  # R[a, b]
        cons[x, y] = R
        cons[y, x] = R.T
    V = ((np.asarray(dom, dtype=np.int64)[:, None] >> bits[None, :]) & 1)  # V[x, a]
    k = 0
    while True:
        k += 1
        counts = np.einsum("xyab,yb->xya", cons, V)
        support = np.minimum(counts, 1).sum(axis=1)  # over y, the diagonal included
        Vn = V * (support == n)
        empty = bool((Vn.sum(axis=1) == 0).any())
        if stop_on_wipeout and empty:
            status = oracle.WIPEOUT
            break
        if (Vn == V).all():
            status = oracle.WIPEOUT if empty else oracle.OK
            break
        V = Vn
    out = (Vn << bits[None, :]).sum(axis=1).astype(np.uint32)
    return out, k, status


def tensor_form_cases(seed, count):
    """Small random networks with non-empty input domains, tightness near the
    point where removals cascade."""
    rng = np.random.default_rng(seed)
    for _ in range(count):
        n = int(rng.integers(2, 11))
        d = int(rng.integers(1, 7))
        density = float(rng.choice([0.3, 0.6, 1.0]))
        tight = tuned_tightness(n, d, density, float(rng.choice([0.1, 0.3, 1.0])))
        scope, rel, dom = random_tiny(rng, n, d, density, tight,
                                      restrict=float(rng.choice([0.0, 0.3])))
        dom[dom == 0] = 1
        yield n, d, scope, rel, dom


def pin_tensor_form(lib, seed=21, cases=400):
    """Eq. 1 over the real constraints against the dense tensor form: while no
    domain is empty an all-ones block supports every value (reading c5), so
    in stop-on-wipeout mode the two agree on every state, sweep count and
    status, and in the default mode on every input whose fixpoint has no
    empty domain."""
    fails = []
    for i, (n, d, scope, rel, dom) in enumerate(tensor_form_cases(seed, cases)):
        for stop in (True, False):
            got = oracle.rac(n, d, scope, rel, dom, stop_on_wipeout=stop, lib=lib)
            if not stop and got[2] != oracle.OK:
                continue
            want = tensor_form(n, d, scope, rel, dom, stop)
            if not np.array_equal(got[0], want[0]) or tuple(got[1:]) != tuple(want[1:]):
                fails.append("tensor form %d (stop %d): sweeps/status %s vs %s" % (
                    i, stop, tuple(got[1:]), tuple(want[1:])))
    return fails


ALL_PINS = [pin_golden, pin_chain, pin_special_cases, pin_three_way, pin_invariants,
            pin_incremental, pin_stop_and_cap, pin_tensor_form]


def run_all(lib, quick=False):
    fails = []
    for p in ALL_PINS:
        if quick and p is pin_three_way:
            fails += pin_three_way(lib, cases=300)
        else:
            fails += p(lib)
    return fails
