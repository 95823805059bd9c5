"""Autotuned launch table: tile rows, grid cap and relation layout per (d,
density, states).

A network's relations are stored in tiles ("slabs") of 32 column variables by
`rows` row variables of one block pair; the kernels stream one tile at a time
through shared memory (rac_create_network, RAC_LAYOUT_ROWS), and CTA c of a
persistent launch owns tiles c, c + G, ...  (RAC_LAYOUT_MAX_CTAS caps G).
Small tiles spread the work more evenly over the CTAs and let Proposition 2
skip finer pieces; large tiles pay the per-tile overhead (stage hand-off,
domain staging, pipeline latency) fewer times.  A smaller grid makes each
sweep's grid barrier cheaper and leaves each CTA more tiles to overlap.
Packed relation rows (RAC_LAYOUT_PACKED, d <= 28) move fewer bytes per sweep
and let taller tiles fit a stage, for one more instruction per row of every
support test.  The best choice depends on d, the density, the number of
states per launch and the GPU, so it is measured:

    python -m paper_2407_11388_b300.autotune [--out FILE] [--runs 20]

For every (d, density, states) bucket -- one-state buckets also split at
SIZE_SPLIT constraints -- it times every admissible row count, grid cap and
relation layout on seeded synthetic networks of the bucket (120, 360 and 700
variables at the bucket's middle d and density, tightness 0.3, assignment
states; for one state 120, 250 and 400 variables below the split, 1000 and
2000 above it; one launch per network -- rac_enforce for one state,
rac_enforce_batch for more -- CUDA events, L2 flushed before each launch,
median of `runs`),
and, for networks enforced together, every row count and layout of one
multi-network plan launch of the three networks with 64 states each; it writes the
fastest choice per bucket to a JSON table.  Network() consults that table
(tile_table.json next to this file) for what its caller leaves open.
"""
import argparse
import json
import os
import time

HERE = os.path.dirname(os.path.abspath(__file__))
TABLE = os.path.join(HERE, "tile_table.json")
# one bucket per relation width q = ceil(d / 4): every d of a bucket runs the
# same kernel instance and has the same tile sizes in both layouts
D_BUCKETS = [(4 * q - 3, 4 * q) for q in range(1, 9)]
DENSITY_BUCKETS = [(0.0, 0.6), (0.6, 1.0)]
STATE_BUCKETS = [(1, 1), (2, 16), (17, 1 << 30)]
# One-state launches are also split by size (constraints): a network of a few
# hundred tiles is done in one round of the CTAs' static tiles, a large one
# streams most of its tiles through the dynamic claims, and the two regimes
# prefer different tiles and layouts.  Representatives per class: networks of
# these variable counts at the bucket's middle d and density.
SIZE_SPLIT = 100_000
SIZE_CLASSES = [(0, SIZE_SPLIT - 1, (120, 250, 400)), (SIZE_SPLIT, 1 << 62, (1000, 2000))]
MULTI_STATE_SIZES = (120, 360, 700)
STATES_TIMED = {(1, 1): 1, (2, 16): 8, (17, 1 << 30): 32}
PLAN_STATES = 64  # states per network in the multi-network plans timed
CTA_CAPS = (None, 74, 37)  # every resident CTA (capped at the tile count), or fewer
STAGE_BYTES = 32768  # relation bytes of one tile the kernels can stage

_table = None


def words_per_relation(d, packed=False):
    """Stored words of one relation: a word per row (round_up(d, 4) rows), or
    packed rows (4q rows of 4q bits, q = ceil(d / 4)) for d <= 28."""
    q = (d + 3) // 4
    return (16 * q * q + 31) // 32 if packed and q < 8 else 4 * q


def admissible_rows(d, packed=False):
    w = words_per_relation(d, packed)
    return [r for r in (2, 4, 8, 16, 32) if r * 32 * w * 4 <= STAGE_BYTES]


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


def _entry(d, density, states, path, kind, m=None):
    for e in load_table(path).get("entries", []):
        if e.get("kind", "single") != kind:
            continue
        if not (e["d_lo"] <= d <= e["d_hi"] and e["dens_lo"] <= density <= e["dens_hi"]):
            continue
        if not e.get("st_lo", 1) <= states <= e.get("st_hi", 1 << 30):
            continue
        if m is not None and not e.get("m_lo", 0) <= m <= e.get("m_hi", 1 << 62):
            continue
        return e
    return None


def table_choice(d, density, states=1, path=TABLE, kind="single", packed=False, m=None):
    """(rows, max_ctas) tuned for this shape; None for what the table does
    not fix (the library default).  kind: "single" for a network enforced in
    launches of its own, "plan" for one enforced in multi-network plans;
    packed: the relation layout the network is created with (the tuned rows
    are taken only when they fit its tiles); m: the number of constraints
    (None: the first entry of any size)."""
    e = _entry(d, density, states, path, kind, m)
    if e is None:
        return None, None
    r = int(e["rows"])
    return (r if r in admissible_rows(d, packed) else None), e.get("max_ctas")


def table_packed(d, density, states=1, path=TABLE, kind="single", m=None):
    """Whether the table found packed relation rows faster for this shape
    (False where it has no entry or did not time them)."""
    e = _entry(d, density, states, path, kind, m)
    return bool(e and e.get("packed", False))


def table_rows(d, density, states=1, path=TABLE, kind="single"):
    """The tuned tile rows for this shape, or None (library default)."""
    return table_choice(d, density, states, path, kind)[0]


def _bucket_networks(d_lo, d_hi, dens_lo, dens_hi, seed, states, sizes=MULTI_STATE_SIZES):
    """Seeded representatives of a bucket: networks of `sizes` variables at
    the bucket's middle d and density, tightness 0.3, with `states`
    assignment states each."""
    import racgen
    d = (d_lo + d_hi + 1) // 2
    dens = 0.5 * (dens_lo + dens_hi)
    nets = []
    for i, n in enumerate(sizes):
        net = racgen.random_network(seed, 100 + i, n, d, dens, 0.3)
        doms = [racgen.assignment_state(seed, 100 + i, s, n, d) for s in range(states)]
        nets.append((net, doms))
    return d, dens, nets


def time_choice(nets, rows, max_ctas, runs, packed=False):
    """Median over runs of the summed time (ms) of one launch per network
    (all of its states) with this tile height, grid cap and relation layout."""
    import numpy as np
    import torch
    from . import Network, enforce, enforce_batch
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.int32, device="cuda")
    total = 0.0
    for x, doms in nets:
        with Network(x.n, x.d, x.scope, x.rel, rows=rows, packed=packed,
                     max_ctas=max_ctas if max_ctas is not None else 65535) as h:
            B = len(doms)
            din = torch.from_numpy(np.concatenate(doms).astype(np.uint32).view(np.int32)).cuda()
            dout = torch.empty_like(din)
            it = torch.empty(B, dtype=torch.int32, device="cuda")
            st = torch.empty_like(it)
            items = np.zeros(B, np.int32)
            offs = np.arange(B, dtype=np.int64) * x.n

            def launch():
                if B == 1:
                    enforce(h, din, dout, it, st)
                else:
                    enforce_batch([h], items, offs, din, dout, it, st)

            ts = []
            for r in range(runs + 3):
                flush.fill_(r)
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record()
                launch()
                b.record()
                torch.cuda.synchronize()
                if r >= 3:
                    ts.append(a.elapsed_time(b))
            total += float(np.median(ts))
    return total


def time_plan(nets, rows, runs, packed=False):
    """Median time (ms) of one multi-network plan launch of all states of all
    networks with tiles of `rows` rows (the batched kernel) in the given
    relation layout."""
    import numpy as np
    import torch
    from . import Network, Plan
    handles = [Network(x.n, x.d, x.scope, x.rel, rows=rows, max_ctas=65535, packed=packed)
               for x, _ in nets]
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


MARGIN = 0.01  # a choice replaces the library default only when this much faster


def select(times, default):
    """The fastest choice, unless the library default is within MARGIN of it
    (timing noise should not move a network off the default)."""
    best = min(times, key=times.get)
    return default if times[default] <= times[best] * (1.0 + MARGIN) else best


def _layouts(d):
    """Relation layouts worth timing: packed rows differ only for d <= 28."""
    return (False, True) if d <= 28 else (False,)


def tune(runs=20, seed=7, out=TABLE, log=print):
    import torch
    entries = []
    for st_lo, st_hi in STATE_BUCKETS:
        states = STATES_TIMED[(st_lo, st_hi)]
        classes = SIZE_CLASSES if st_hi == 1 else [(None, None, MULTI_STATE_SIZES)]
        for m_lo, m_hi, sizes in classes:
            for d_lo, d_hi in D_BUCKETS:
                for dens_lo, dens_hi in DENSITY_BUCKETS:
                    d, dens, nets = _bucket_networks(d_lo, d_hi, dens_lo, dens_hi, seed, states,
                                                     sizes)
                    # the grid cap only for networks too small to fill every
                    # CTA with tiles of their own
                    caps = CTA_CAPS if not m_lo else (None,)
                    times = {(r, c, pk): time_choice(nets, r, c, runs, pk)
                             for pk in _layouts(d) for r in admissible_rows(d, pk)
                             for c in caps}
                    best = select(times, (max(admissible_rows(d)), None, False))
                    default = times[(max(admissible_rows(d)), None, False)]
                    log("states %d%s d %2d-%2d density %.1f-%.1f: best rows %d ctas %s %s "
                        "(%.3f ms; library default %.3f ms)"
                        % (states, "" if m_lo is None else " m %d-%d" % (m_lo, min(m_hi, 10**9)),
                           d_lo, d_hi, dens_lo, dens_hi, best[0], best[1],
                           "packed" if best[2] else "words", times[best], default))
                    e = {"d_lo": d_lo, "d_hi": d_hi, "dens_lo": dens_lo, "dens_hi": dens_hi,
                         "st_lo": st_lo, "st_hi": st_hi, "rows": best[0], "max_ctas": best[1],
                         "packed": best[2], "sizes": list(sizes),
                         "ms": {"%d/%s/%s" % (r, c if c is not None else "all",
                                              "packed" if pk else "words"): round(t, 4)
                                for (r, c, pk), t in times.items()}}
                    if m_lo is not None:
                        e["m_lo"], e["m_hi"] = m_lo, m_hi
                    entries.append(e)
    # networks enforced together in multi-network plans (the batched kernel:
    # its grid is every resident CTA, so only the tile rows are tuned)
    for d_lo, d_hi in D_BUCKETS:
        for dens_lo, dens_hi in DENSITY_BUCKETS:
            d, dens, nets = _bucket_networks(d_lo, d_hi, dens_lo, dens_hi, seed, PLAN_STATES)
            times = {(r, pk): time_plan(nets, r, runs, pk)
                     for pk in _layouts(d) for r in admissible_rows(d, pk)}
            best = select(times, (max(admissible_rows(d)), False))
            log("plan, %d states each: d %2d-%2d density %.1f-%.1f: best rows %d %s (%.3f ms; "
                "library default %.3f ms)" % (PLAN_STATES, d_lo, d_hi, dens_lo, dens_hi, best[0],
                                              "packed" if best[1] else "words", times[best],
                                              times[(max(admissible_rows(d)), False)]))
            entries.append({"kind": "plan", "d_lo": d_lo, "d_hi": d_hi, "dens_lo": dens_lo,
                            "dens_hi": dens_hi, "st_lo": 1, "st_hi": 1 << 30, "rows": best[0],
                            "max_ctas": None, "packed": best[1],
                            "ms": {"%d/%s" % (r, "packed" if pk else "words"): round(t, 4)
                                   for (r, pk), t in times.items()}})
    table = {"version": 2, "device": torch.cuda.get_device_name(0),
             "states_timed": {"%d-%d" % k: v for k, v in STATES_TIMED.items()},
             "runs": runs, "seed": seed, "created": time.strftime("%Y-%m-%d %H:%M:%S"),
             "key": "ms: 'rows/grid cap/relation rows' -> summed median launch time of the "
                    "bucket's networks (their variable counts under 'sizes'; plans: 120, "
                    "360 and 700)",
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
    a = ap.parse_args()
    import sys
    sys.path.insert(0, os.path.dirname(HERE))
    tune(a.runs, out=a.out)
