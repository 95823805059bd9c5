"""Autotuned tile table of the relation layout.

A network's relations are stored in tiles ("slabs") of 32 column variables by
`rows` row variables of one block pair; the kernels stream one tile at a time
through shared memory (rac_create_network, RAC_LAYOUT_ROWS).  Small tiles
spread uneven networks more evenly over the CTAs of a batched launch and let
Proposition 2 skip finer pieces; large tiles pay the per-tile overhead
(stage hand-off, domain staging, pipeline latency) fewer times.  The best
size depends on d, the density and the GPU, so it is measured:

    python -m paper_2407_11388_b300.autotune [--out FILE] [--runs 20]

times every admissible row count on seeded synthetic batches of each
(d, density) bucket -- several networks with 64 assignment states each,
enforced in one batched launch through a rac_plan, CUDA events, L2 flushed
between runs -- and writes the fastest per bucket to a JSON table.
Network() consults that table (tile_table.json next to this file) when no
row count is given.
"""
import argparse
import json
import os
import time

HERE = os.path.dirname(os.path.abspath(__file__))
TABLE = os.path.join(HERE, "tile_table.json")
D_BUCKETS = [(1, 8), (9, 16), (17, 24), (25, 32)]
DENSITY_BUCKETS = [(0.0, 0.6), (0.6, 1.0)]
STAGE_BYTES = 32768  # relation bytes of one tile the kernels can stage

_table = None


def admissible_rows(d):
    dp = (d + 3) & ~3
    return [r for r in (2, 4, 8, 16, 32) if r * 32 * dp * 4 <= STAGE_BYTES]


def load_table(path=TABLE):
    global _table
    if _table is None or path != TABLE:
        try:
            with open(path) as f:
                t = json.load(f)
        except (OSError, ValueError):
            t = {"entries": []}
        if path != TABLE:
            return t
        _table = t
    return _table


def table_rows(d, density, path=TABLE):
    """The tuned tile rows for this shape, or None (library default)."""
    for e in load_table(path).get("entries", []):
        if e["d_lo"] <= d <= e["d_hi"] and e["dens_lo"] <= density <= e["dens_hi"]:
            r = int(e["rows"])
            return r if r in admissible_rows(d) else None
    return None


def _bucket_batch(d_lo, d_hi, dens_lo, dens_hi, seed, states):
    """Seeded representatives of a bucket: networks of 120, 360 and 700
    variables at the bucket's middle d and density, tightness 0.3."""
    import racgen
    d = (d_lo + d_hi + 1) // 2
    dens = 0.5 * (dens_lo + dens_hi)
    nets = []
    for i, n in enumerate((120, 360, 700)):
        net = racgen.random_network(seed, 100 + i, n, d, dens, 0.3)
        doms = [racgen.assignment_state(seed, 100 + i, s, n, d) for s in range(states)]
        nets.append((net, doms))
    return d, dens, nets


def time_rows(nets, rows, runs):
    """Median time (ms) of one batched enforcement of all states of all
    networks with tiles of `rows` rows."""
    import numpy as np
    import torch
    from . import Network, Plan
    handles = [Network(x.n, x.d, x.scope, x.rel, rows=rows) for x, _ in nets]
    items, offs, flat, pos = [], [], [], 0
    for i, (x, doms) in enumerate(nets):
        for dom in doms:
            items.append(i)
            offs.append(pos)
            flat.append(dom)
            pos += x.n
    flat = np.concatenate(flat).astype(np.uint32)
    din = torch.from_numpy(flat.view(np.int32)).cuda()
    dout = torch.empty_like(din)
    it = torch.empty(len(items), dtype=torch.int32, device="cuda")
    st = torch.empty_like(it)
    plan = Plan(handles, np.array(items, np.int32), np.array(offs, np.int64))
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.int32, device="cuda")
    ts = []
    for r in range(runs + 3):
        flush.fill_(r)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        plan.enforce(din, dout, it, st)
        b.record()
        torch.cuda.synchronize()
        if r >= 3:
            ts.append(a.elapsed_time(b))
    plan.close()
    for h in handles:
        h.close()
    return float(np.median(ts))


def tune(runs=20, states=64, seed=7, out=TABLE, log=print):
    import torch
    entries = []
    for d_lo, d_hi in D_BUCKETS:
        for dens_lo, dens_hi in DENSITY_BUCKETS:
            d, dens, nets = _bucket_batch(d_lo, d_hi, dens_lo, dens_hi, seed, states)
            times = {r: time_rows(nets, r, runs) for r in admissible_rows(d)}
            best = min(times, key=times.get)
            log("d %2d-%2d density %.1f-%.1f: %s -> rows %d" % (
                d_lo, d_hi, dens_lo, dens_hi,
                " ".join("%d:%.3fms" % (r, t) for r, t in sorted(times.items())), best))
            entries.append({"d_lo": d_lo, "d_hi": d_hi, "dens_lo": dens_lo, "dens_hi": dens_hi,
                            "rows": best, "ms": {str(r): round(t, 4) for r, t in times.items()}})
    table = {"version": 1, "device": torch.cuda.get_device_name(0), "states": states,
             "runs": runs, "seed": seed, "created": time.strftime("%Y-%m-%d %H:%M:%S"),
             "entries": entries}
    with open(out, "w") as f:
        json.dump(table, f, indent=1)
    global _table
    _table = None
    return table


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=TABLE)
    ap.add_argument("--runs", type=int, default=20)
    ap.add_argument("--states", type=int, default=64)
    a = ap.parse_args()
    import sys
    sys.path.insert(0, os.path.dirname(HERE))
    tune(a.runs, a.states, out=a.out)
