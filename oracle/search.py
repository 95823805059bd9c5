"""Backtrack search of Algorithm 2 on the CPU oracle (TEST INFRASTRUCTURE ONLY).

Only tests/ and the benchmark's CPU legs may import this; it shares no code
with the CUDA library.  `dfs` follows Algorithm 2 (Sec. 4): enforce the
initial domains with Eq. 1, then pick a variable, try its values in order,
and after each assignment enforce again (the plain recurrence over every
constraint: by Proposition 2 it equals the seeded enforcement the library
runs from an arc-consistent state), descending while no domain is empty and
backtracking otherwise.  The variable-ordering heuristic, which the paper
leaves open, is the one the library's driver uses: the smallest domain of
size > 1, lowest index first.
"""
import numpy as np

from . import OK, rac


def choose_variable(dom):
    """Smallest domain of size > 1, lowest index; None when all are singletons."""
    best, best_size = None, None
    for x, w in enumerate(dom):
        size = bin(int(w)).count("1")
        if size > 1 and (best_size is None or size < best_size):
            best, best_size = x, size
    return best


def dfs(n, d, scope, rel, dom0, max_nodes, threads=1):
    """Returns {"root": (iterations, status), "steps": [(level, var, value,
    iterations, status)], "nodes", "solution", "exhausted"}."""
    out = {"steps": [], "nodes": 0, "solution": None, "exhausted": False}
    root, rit, rst = rac(n, d, scope, rel, dom0, threads=threads)
    out["root"] = (rit, rst)
    if rst != OK:
        return out

    def rec(level, dom):
        var = choose_variable(dom)
        if var is None:
            out["solution"] = dom.copy()
            return True
        for value in range(d):
            if not (int(dom[var]) >> value) & 1:
                continue
            if out["nodes"] >= max_nodes:
                out["exhausted"] = True
                return False
            out["nodes"] += 1
            nxt = dom.copy()
            nxt[var] = np.uint32(1 << value)
            res, it, st = rac(n, d, scope, rel, nxt, threads=threads)
            out["steps"].append((level, var, value, it, st))
            if st == OK and rec(level + 1, res):
                return True
            if out["exhausted"]:
                return False
        return False

    rec(0, np.ascontiguousarray(root, dtype=np.uint32))
    return out
