"""Small hand-made networks and property checks shared by the tests.

Networks use the boundary's format: scope (m, 2) int32, rel (m, d) uint32
with bit b of rel[c, a] = R[a][b] for scope (x, y) = scope[c]; domains are
uint32 words, bit a = value a."""
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def full_word(d):
    return 0xFFFFFFFF if d >= 32 else (1 << d) - 1


def rel_from_predicate(d, pred):
    rows = np.zeros(d, dtype=np.uint32)
    for a in range(d):
        w = 0
        for b in range(d):
            if pred(a, b):
                w |= 1 << b
        rows[a] = w
    return rows


def chain(n, d, reverse_scopes=False):
    """x_0 < x_1 < ... < x_{n-1} on {0..d-1}."""
    scope, rel = [], []
    for i in range(n - 1):
        if reverse_scopes:
            scope.append((i + 1, i))
            rel.append(rel_from_predicate(d, lambda a, b: a > b))
        else:
            scope.append((i, i + 1))
            rel.append(rel_from_predicate(d, lambda a, b: a < b))
    return (np.array(scope, dtype=np.int32).reshape(-1, 2),
            np.array(rel, dtype=np.uint32).reshape(-1, d))


def chain_closed_form(n, d):
    """D_ac of the chain when d >= n: x_i keeps [i, d-n+i]."""
    out = np.zeros(n, dtype=np.uint32)
    for i in range(n):
        for a in range(i, d - n + i + 1):
            out[i] |= np.uint32(1 << a)
    return out


def random_tiny(rng, n, d, density, tight, restrict=0.0):
    """A random network drawn with numpy (independent of racgen), plus a random
    input domain where each value is dropped with probability `restrict`."""
    scope, rel = [], []
    for x in range(n):
        for y in range(x + 1, n):
            if rng.random() < density:
                xy = (x, y) if rng.random() < 0.5 else (y, x)
                scope.append(xy)
                bits = rng.random((d, d)) >= tight
                rel.append([sum(1 << b for b in range(d) if bits[a, b]) for a in range(d)])
    dom = np.array([sum(1 << a for a in range(d) if rng.random() >= restrict)
                    for _ in range(n)], dtype=np.uint32)
    return (np.array(scope, dtype=np.int32).reshape(-1, 2),
            np.array(rel, dtype=np.uint32).reshape(-1, d), dom)


def is_arc_consistent(n, d, scope, rel, dom):
    """Every (x,a) in dom has, on every constraint on x, an allowed partner in
    the other variable's domain (the definition at the start of Sec. 3)."""
    for c in range(scope.shape[0]):
        x, y = int(scope[c, 0]), int(scope[c, 1])
        for a in range(d):
            if (int(dom[x]) >> a) & 1 and (int(rel[c, a]) & int(dom[y])) == 0:
                return False
        for b in range(d):
            if (int(dom[y]) >> b) & 1:
                if not any(((int(dom[x]) >> a) & 1) and ((int(rel[c, a]) >> b) & 1)
                           for a in range(d)):
                    return False
    return True


def load_golden(name):
    path = os.path.join(GOLDEN, name)
    n = d = None
    cons, doms, exp_dom = [], {}, {}
    mode, it, st = "default", None, None
    with open(path) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            tok = line.split()
            if tok[0] == "n":
                n = int(tok[1])
            elif tok[0] == "d":
                d = int(tok[1])
            elif tok[0] == "con":
                x, y = int(tok[1]), int(tok[2])
                rows = tok[3:]
                assert len(rows) == d and all(len(r) == d for r in rows)
                cons.append(((x, y), [sum(1 << b for b, ch in enumerate(r) if ch == "1")
                                      for r in rows]))
            elif tok[0] == "dom":
                doms[int(tok[1])] = sum(1 << a for a, ch in enumerate(tok[2]) if ch == "1")
            elif tok[0] == "mode":
                mode = tok[1]
            elif tok[0] == "expect_dom":
                exp_dom[int(tok[1])] = sum(1 << a for a, ch in enumerate(tok[2]) if ch == "1")
            elif tok[0] == "expect_iterations":
                it = int(tok[1])
            elif tok[0] == "expect_status":
                st = {"ok": 0, "wipeout": 1}[tok[1]]
            else:
                raise ValueError("bad golden line: " + line)
    scope = np.array([c[0] for c in cons], dtype=np.int32).reshape(-1, 2)
    rel = np.array([c[1] for c in cons], dtype=np.uint32).reshape(-1, d)
    dom = np.array([doms.get(x, full_word(d)) for x in range(n)], dtype=np.uint32)
    expected = np.array([exp_dom[x] for x in range(n)], dtype=np.uint32)
    return dict(n=n, d=d, scope=scope, rel=rel, dom=dom, stop=(mode == "stop"),
                expected=expected, iterations=it, status=st)


def golden_names():
    return sorted(f for f in os.listdir(GOLDEN) if f.endswith(".txt") and f != "README.txt")


def tuned_tightness(n, d, density, c):
    """Tightness at which a full-domain value lacks a support on about c of
    its ~n*density constraints: near the point where removals start to
    cascade, so that enforcement runs for several sweeps."""
    return min(0.95, (c / max(1.0, n * density)) ** (1.0 / d))


def mixed_states(rng, n, d):
    """Three input domains: every variable randomly restricted (no empty
    domain), four variables restricted and the rest full, and all full."""
    full = np.full(n, full_word(d), np.uint32)
    a = random_tiny(rng, n, d, 0.0, 0.0, restrict=0.3)[2]
    a[a == 0] = 1
    b = full.copy()
    for x in rng.choice(n, size=min(n, 4), replace=False):
        b[x] = np.uint32(int(rng.integers(1, 1 << min(d, 31))) & full_word(d))
    return np.array([a, b, full], dtype=np.uint32)


# (n, density, c) of the per-width parity cases
WIDTH_CASES = [(37, 0.5, 0.3), (70, 0.15, 0.03), (33, 1.0, 0.01)]


def width_cases(d):
    rng = np.random.default_rng(1000 + d)
    for n, dens, c in WIDTH_CASES:
        scope, rel, _ = random_tiny(rng, n, d, dens, tuned_tightness(n, d, dens, c))
        yield n, scope, rel, mixed_states(rng, n, d)
