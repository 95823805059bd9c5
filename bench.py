"""Benchmark: recurrent arc consistency (Eq. 1) to its fixpoint on B300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
                    [--impl ours|reference]

One step = one enforcement to the fixpoint (every sweep of the hot path:
support test, AND-reduction over C_x, change and wipe-out flags, the
device-side fixpoint loop) of one batch of domain states of the workload,
through the C ABI, with the network already resident on the device.  The L2
cache is flushed between timed steps (outside the timed events); each step is
timed with CUDA events on the stream it runs on.

Prints ONE JSON line.  Under torchrun every rank runs its own replica of the
workload (the fixpoints are independent), `value` is the units of all ranks
over the slowest rank's time.  `--impl reference` times the CPU oracle (the
literal Eq. 1 recurrence) on the same workload instead.
"""
import argparse
import gc
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "RAC fixpoints/s and relation-bits/s vs plain GPU RAC; % of HBM/tensor roofline"

# Synthetic workloads (random binary CSPs of the experiments' model, Sec. 5:
# every pair of variables constrained with probability `density`, every value
# pair of a constraint disallowed with probability `tightness`).
WORKLOADS = {
    "dense_n500_d20": dict(n=500, d=20, density=1.0, tightness=0.35, states="full", n_states=1),
    "rb_n50_d10": dict(n=50, d=10, density=0.5, tightness=0.3, states="full", n_states=1),
    "dense_n2000_d32": dict(n=2000, d=32, density=0.9, tightness=0.3, states="full", n_states=1),
    # the same graph at narrower domains: single-state launches that stream a
    # store larger than L2, where packed relation rows (--layout packed) read
    # 13 / 18 words per relation instead of 20 / 24
    "dense_n2000_d20": dict(n=2000, d=20, density=0.9, tightness=0.3, states="full", n_states=1),
    "dense_n2000_d24": dict(n=2000, d=24, density=0.9, tightness=0.3, states="full", n_states=1),
    "n1000_d24_b32": dict(n=1000, d=24, density=0.8, tightness=0.3, states="assign",
                          n_states=32),
    "n1000_d24_b64": dict(n=1000, d=24, density=0.8, tightness=0.3, states="assign",
                          n_states=64),
    "n1000_d24_b128": dict(n=1000, d=24, density=0.8, tightness=0.3, states="assign",
                           n_states=128),
    # the same network and states with learned active-block gating: the
    # predictor is trained first (GPU traces of the n=500/2000 dense and batch
    # generators, other seeds), then the gated enforcement is timed
    "learned_n1000_d24_b32": dict(n=1000, d=24, density=0.8, tightness=0.3, states="assign",
                                  n_states=32, learned=True),
    # 256 networks, n ~ U{50..800}, d ~ U{8..32}, density ~ U[0.3,1],
    # tightness ~ U[0.2,0.4], 64 assignment states each: one launch per step
    "batch256_x64": dict(batch=True, networks=256, states_per_net=64),
    # the same generator at a size small enough for full profiler captures
    "batch32_x16": dict(batch=True, networks=32, states_per_net=16),
    # Algorithm 2 on the n=500 d=20 network: a step is one assignment and its
    # seeded enforcement (rac_assign_enforce) inside the device-state search
    "search_n500_d20": dict(n=500, d=20, density=1.0, tightness=0.35, states="full", n_states=1,
                            search=True),
}
# the largest single-state configuration (n=2000, d=32, density 0.9,
# tightness 0.3: a 230 MB relation store, larger than L2)
DEFAULT_WORKLOAD = "dense_n2000_d32"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10000)
    p.add_argument("--warmup", type=int, default=20)
    p.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--seed", type=int, default=0)
    p.add_argument("--flags", type=int, default=0, help="enforce flags (1 stop, 2 incremental)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--layout", default="auto", choices=["auto", "words", "packed"],
                   help="relation rows: the tuned table's choice, a word per row, or packed")
    p.add_argument("--rows", type=int, default=None,
                   help="tile rows (a power of two); default: the tuned table's choice")
    return p.parse_args()


def profile_key(args):
    """The traffic.json entry of this run's workload and relation layout."""
    return args.workload + ("+packed" if getattr(args, "packed", False) else "")


def make_inputs(wl, seed):
    import racgen
    spec = WORKLOADS[wl]
    net = racgen.random_network(seed, 0, spec["n"], spec["d"], spec["density"], spec["tightness"])
    if spec["states"] == "full":
        doms = np.tile(racgen.full_domain(spec["n"], spec["d"]), (spec["n_states"], 1))
    else:
        doms = np.array([racgen.assignment_state(seed, 0, s, spec["n"], spec["d"])
                         for s in range(spec["n_states"])])
    return spec, net, doms


def make_batch(seed, networks, states_per_net):
    """Uneven batch: networks with racgen.batch_params shapes, assignment
    states interleaved over networks and stored back to back."""
    import racgen
    nets = [racgen.random_network(seed, i, *racgen.batch_params(seed, i)) for i in range(networks)]
    items, offs, doms = [], [], []
    pos = 0
    for s in range(states_per_net):
        for i, x in enumerate(nets):
            dom = racgen.assignment_state(seed, i, s, x.n, x.d)
            items.append(i)
            offs.append(pos)
            doms.append(dom)
            pos += x.n
    flat = np.concatenate(doms).astype(np.uint32)
    return nets, np.array(items, np.int32), np.array(offs, np.int64), doms, flat


L2_NOTE = ("flushed between timed steps: a 256 MB buffer written, then another 256 MB read, "
           "so L2 holds no line of the workload and none left dirty by the flush")


def config_of(wl, spec, net, flush):
    return {"workload": wl, "n": spec["n"], "d": spec["d"], "density": spec["density"],
            "tightness": spec["tightness"], "constraints": net.m, "states": spec["n_states"],
            "state_kind": spec["states"], "seed_generated": True,
            "l2": L2_NOTE if flush else "inputs larger than L2"}


class L2Flush:
    """Evicts the workload from the 126 MB L2 between timed steps, outside the
    timed events: writes a 256 MB buffer, then reads a second 256 MB buffer, so
    the lines the write left dirty are written back to HBM before the next
    step rather than during it."""

    def __init__(self, torch, dev):
        self.w = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
        self.r = torch.ones(64 << 20, dtype=torch.int32, device=dev)

    def __call__(self):
        self.w.zero_()
        self.r.max()


def _code_only(text):
    """C/C++ source without its comments and blank runs: edits to comments
    leave the kernels (and so the recorded counters) unchanged."""
    out, i, n = [], 0, len(text)
    while i < n:
        if text.startswith("//", i):
            j = text.find("\n", i)
            i = n if j < 0 else j
        elif text.startswith("/*", i):
            j = text.find("*/", i + 2)
            i = n if j < 0 else j + 2
        elif text[i] in "\"'":
            q, j = text[i], i + 1
            while j < n and text[j] != q:
                j += 2 if text[j] == "\\" else 1
            out.append(text[i:j + 1])
            i = j + 1
        else:
            out.append(text[i])
            i += 1
    return "\n".join(ln.rstrip() for ln in "".join(out).splitlines() if ln.strip())


# The sources a kernel's recorded counters depend on: the kernel, the device
# helpers and the host code that lays out the relation store and launches it.
KERNEL_SOURCES = {
    "rac_bits_kernel": ("rac_bits_kernel.cu", "rac_bits_packed.cu", "rac_device.cuh",
                        "rac_internal.h", "rac_mlp.cuh", "rac_api.cu"),
    "rac_batch_kernel": ("rac_batch_kernel.cu", "rac_plan.cu", "rac_device.cuh",
                         "rac_internal.h", "rac_api.cu"),
}


def source_hash(kernel=None):
    """Hash of the code (comments excluded) of the kernel's sources under
    csrc/ (every file there when kernel is None)."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2407_11388_b300", "csrc")
    files = sorted(os.listdir(csrc)) if kernel is None else sorted(KERNEL_SOURCES[kernel])
    for f in files:
        h.update(f.encode())
        h.update(_code_only(open(os.path.join(csrc, f), encoding="utf-8").read()).encode())
    return h.hexdigest()[:16]


def profile_entry(wl):
    """The committed ncu counters of one launch of the workload's kernel
    (DRAM bytes, warp instructions), if they were taken on the kernel's
    current sources (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        data = json.load(open(path))
    except (OSError, ValueError):
        return None
    ent = data.get(wl)
    if not ent:
        return None
    kernel = ent.get("kernel")
    if ent.get("source_hash") != (source_hash(kernel) if kernel in KERNEL_SOURCES else source_hash()):
        return None
    return ent


def traffic_from_profiles(wl):
    """DRAM bytes per launch from a committed ncu summary, if it was taken on
    the current kernel sources (else None)."""
    ent = profile_entry(wl)
    return None if ent is None else ent.get("dram_bytes_per_launch")


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return None


class ClockSampler:
    """SM clock and throttle reasons sampled while the timed region runs:
    NVML when the pynvml module is importable, else `nvidia-smi -lms`."""

    FIELDS = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")
    NAMES = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.samples = []
        self.reasons = set()
        self.max_mhz = None
        self._stop = threading.Event()
        self._t = None
        self._proc = None
        self.error = None
        self.source = None

    def __enter__(self):
        try:
            import pynvml
            pynvml.nvmlInit()
            self._h = pynvml.nvmlDeviceGetHandleByIndex(self.index)
            self.max_mhz = pynvml.nvmlDeviceGetMaxClockInfo(self._h, pynvml.NVML_CLOCK_SM)
            self._nv = pynvml
            self.source = "nvml"
            self._t = threading.Thread(target=self._run_nvml, daemon=True)
            self._t.start()
            return self
        except Exception as e:  # noqa: BLE001 - fall back to nvidia-smi
            self.error = "nvml: %s" % e
        try:
            self._proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.source = "nvidia-smi"
            first = self._proc.stdout.readline()  # the sampler is running before timing starts
            self._parse(first)
            self._t = threading.Thread(target=self._run_smi, daemon=True)
            self._t.start()
        except Exception as e:  # noqa: BLE001
            self.error = (self.error or "") + "; nvidia-smi: %s" % e
        return self

    def _parse(self, line):
        parts = [p.strip() for p in line.strip().split(",")]
        if len(parts) < 6:
            return
        try:
            self.samples.append(float(parts[0]))
            self.max_mhz = float(parts[1])
        except ValueError:
            return
        for name, val in zip(self.NAMES, parts[2:6]):
            if val.lower() == "active":
                self.reasons.add(name)

    def _run_smi(self):
        for line in self._proc.stdout:
            self._parse(line)
            if self._stop.is_set():
                break

    def _run_nvml(self):
        nv = self._nv
        names = {
            "hw_slowdown": getattr(nv, "nvmlClocksEventReasonHwSlowdown", 0x8),
            "hw_thermal_slowdown": getattr(nv, "nvmlClocksEventReasonHwThermalSlowdown", 0x40),
            "sw_thermal_slowdown": getattr(nv, "nvmlClocksEventReasonSwThermalSlowdown", 0x20),
            "sw_power_cap": getattr(nv, "nvmlClocksEventReasonSwPowerCap", 0x4),
        }
        fn = getattr(nv, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            nv.nvmlDeviceGetCurrentClocksThrottleReasons
        while not self._stop.is_set():
            try:
                self.samples.append(nv.nvmlDeviceGetClockInfo(self._h, nv.NVML_CLOCK_SM))
                r = fn(self._h)
                for k, bit in names.items():
                    if r & bit:
                        self.reasons.add(k)
            except Exception as e:  # noqa: BLE001
                self.error = str(e)
                break
            time.sleep(0.005)

    def __exit__(self, *exc):
        self._stop.set()
        if self._proc is not None:
            time.sleep(0.06)  # one more sample after the timed region
            self._proc.terminate()
            try:
                self._proc.wait(timeout=2)
            except Exception:  # noqa: BLE001
                self._proc.kill()
        if self._t:
            self._t.join(timeout=2)

    def summary(self):
        med = float(np.median(self.samples)) if self.samples else None
        out = {"sm_mhz": med, "sm_max_mhz": self.max_mhz, "reasons": sorted(self.reasons),
               "samples": len(self.samples), "source": self.source}
        if self.error and not self.samples:
            out["error"] = self.error
        return out


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def cpu_baseline(W, budget_s=15.0):
    """The oracle (literal Eq. 1 sweeps, OpenMP over variables) on a bounded
    sample of the same workload: whole fixpoints of its items, in order,
    until the time budget is used."""
    import oracle
    threads = os.cpu_count() or 1
    t0 = time.perf_counter()
    done = 0
    sweeps = 0
    while True:
        j = done % W.B
        x = W.nets_np[int(W.items[j])]
        _, it, _ = oracle.rac(x.n, x.d, x.scope, x.rel, W.doms[j], threads=threads)
        done += 1
        sweeps += it
        el = time.perf_counter() - t0
        if el >= budget_s or done >= 4000:
            break
    return {"value": done / el, "unit": "fixpoints/s", "cores": threads, "kind": "oracle",
            "sample": "%d whole fixpoints (%d sweeps) of this workload's items, %.1f s" % (
                done, sweeps, el)}, sweeps / done


def run_reference(args):
    """The reference arm: the CPU oracle (literal Eq. 1) on this workload's
    items, one whole fixpoint per step, on all host cores; the step count is
    capped so the run ends within a few minutes."""
    world, rank, _ = dist_setup(args)
    if rank != 0:
        return
    import oracle
    spec = WORKLOADS[args.workload]
    if spec.get("search"):
        run_reference_search(args, spec)
        return
    if spec.get("batch"):
        nets_np, items, _, doms, _ = make_batch(args.seed, spec["networks"], spec["states_per_net"])
        cfg = {"workload": args.workload, "networks": spec["networks"],
               "states_per_network": spec["states_per_net"]}
    else:
        _, net, dm = make_inputs(args.workload, args.seed)
        nets_np, items, doms = [net], np.zeros(dm.shape[0], np.int32), list(dm)
        cfg = config_of(args.workload, spec, net, True)
    threads = os.cpu_count() or 1

    def one(j):
        x = nets_np[int(items[j % len(items)])]
        return oracle.rac(x.n, x.d, x.scope, x.rel, doms[j % len(items)], threads=threads)[1]

    t0 = time.perf_counter()
    one(0)
    est = time.perf_counter() - t0
    steps = max(1, min(args.steps, int(150.0 / max(est, 1e-6))))
    warm = max(0, min(args.warmup, 3))
    for w in range(warm):
        one(w)
    sweeps = 0
    bits = 0.0
    t0 = time.perf_counter()
    for j in range(steps):
        it = one(j)
        x = nets_np[int(items[j % len(items)])]
        sweeps += it
        bits += float(x.m) * x.d * x.d * it
    el = time.perf_counter() - t0
    value = steps / el
    line = {"metric": METRIC, "value": value, "unit": "fixpoints/s", "impl": "reference",
            "n_gpus": args.gpus, "steps": steps, "warmup": warm,
            "ms_per_step": 1000.0 * el / steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u8", "data": "synthetic", "config": cfg,
            "relation_bits_per_s": bits / el,
            "cpu_baseline": {"value": value, "unit": "fixpoints/s", "cores": threads,
                             "kind": "oracle",
                             "sample": "%d whole fixpoints (requested %d steps)" % (steps, args.steps)},
            "e2e": {"value": value, "unit": "fixpoints/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_reference_search(args, spec):
    """The reference arm of a search workload: the oracle's Algorithm 2 on the
    same network, the root enforcement and up to --steps assignments (each a
    whole Eq. 1 enforcement on all host cores), capped to a few minutes."""
    from oracle.search import dfs as oracle_dfs
    _, x, _ = make_inputs(args.workload, args.seed)
    threads = os.cpu_count() or 1
    t0 = time.perf_counter()
    oracle_dfs(x.n, x.d, x.scope, x.rel, racgen_full(x), 2, threads=threads)
    est = (time.perf_counter() - t0) / 3.0
    steps = max(1, min(args.steps, int(150.0 / max(est, 1e-6))))
    t0 = time.perf_counter()
    out = oracle_dfs(x.n, x.d, x.scope, x.rel, racgen_full(x), steps, threads=threads)
    el = time.perf_counter() - t0
    fix = out["nodes"] + 1  # the root enforcement is a fixpoint too
    value = fix / el
    line = {"metric": METRIC, "value": value, "unit": "fixpoints/s", "impl": "reference",
            "n_gpus": args.gpus, "steps": fix, "warmup": 0, "ms_per_step": 1000.0 * el / fix,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
            "data": "synthetic",
            "config": {"workload": args.workload, "n": x.n, "d": x.d, "density": spec["density"],
                       "tightness": spec["tightness"], "constraints": int(x.m),
                       "state_kind": "search (Algorithm 2: assign, then enforce)"},
            "sweeps_per_fixpoint": float(np.mean([s[3] for s in out["steps"]])) if out["steps"] else 0.0,
            "cpu_baseline": {"value": value, "unit": "fixpoints/s", "cores": threads,
                             "kind": "oracle",
                             "sample": "the root and %d assignments of the oracle's search"
                                       % out["nodes"]},
            "e2e": {"value": value, "unit": "fixpoints/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# untimed steps right before the timed ones (after the clock sampler starts)
RESUME_STEPS = 10

# a slab's 32-state group is scored only with at least this many gated
# candidates (fewer are evaluated unscored: measured faster on B300)
LEARNED_MIN_SCORED = 28


def train_predictor(rac, torch, seed, recall=0.995, log=None):
    """The active-block predictor trained on the GPU from Proposition-2 traces
    of other networks: the n=500 d=20 and n=2000 d=32 dense generators and the
    batch generator (assignment states, seeds disjoint from the workload's).
    Returns (predictor, logit threshold, training summary)."""
    import racgen
    from paper_2407_11388_b300 import learned
    t0 = time.perf_counter()
    specs = [(seed + 1000, 0, 500, 20, 1.0, 0.35, 32), (seed + 1000, 1, 500, 20, 1.0, 0.35, 32),
             (seed + 1000, 0, 2000, 32, 0.9, 0.3, 16)]
    specs += [(seed + 1000, i) + tuple(racgen.batch_params(seed + 1000, i)) + (16,)
              for i in range(12)]
    items, keep = [], []
    for sd, inst, n, d, p, t, B in specs:
        x = racgen.random_network(sd, inst, n, d, p, t)
        doms = np.array([racgen.assignment_state(sd, inst, s, n, d) for s in range(B)], np.uint32)
        net = rac.Network(x.n, x.d, x.scope, x.rel)
        keep.append(net)
        items.append((net, torch.from_numpy(doms.view(np.int32)).cuda()))
    x, y, _ = learned.collect_traces(items)
    for net in keep:
        net.close()
    pred = learned.train(x, y, steps=4000, batch=4096, lr=2e-3, pos_weight=4.0, seed=seed + 1)
    thr = learned.choose_threshold(pred, x, y, recall=recall)
    info = {"records": int(x.shape[0]), "positive_rate": float(y.mean()), "recall_target": recall,
            "threshold_logit": thr, "train_s": time.perf_counter() - t0,
            "traces": "Proposition-2 sweeps of n=500 d=20 (2x32 states), n=2000 d=32 (16), "
                      "12 batch-generator networks (16 each), seed %d" % (seed + 1000)}
    return pred, thr, info


class Prepared:
    """The workload resident on the device, and how one step enforces it."""

    def __init__(self, args, rac, torch, dev):
        spec = WORKLOADS[args.workload]
        self.spec = spec
        if spec.get("batch"):
            nets_np, items, offs, doms, flat = make_batch(args.seed, spec["networks"],
                                                          spec["states_per_net"])
            self.cfg = {"workload": args.workload, "networks": spec["networks"],
                        "states_per_network": spec["states_per_net"],
                        "n": "U{50..800}", "d": "U{8..32}", "density": "U[0.3,1.0]",
                        "tightness": "U[0.2,0.4]", "constraints": int(sum(x.m for x in nets_np)),
                        "state_kind": "assign", "seed_generated": True,
                        "l2": L2_NOTE}
        else:
            _, net_np, dm = make_inputs(args.workload, args.seed)
            nets_np = [net_np]
            B = dm.shape[0]
            items = np.zeros(B, np.int32)
            offs = np.arange(B, dtype=np.int64) * net_np.n
            doms = list(dm)
            flat = dm.reshape(-1)
            self.cfg = config_of(args.workload, spec, net_np, True)
        self.nets_np, self.items, self.offs, self.doms = nets_np, items, offs, doms
        self.B = len(items)
        per_launch = spec.get("states_per_net", spec.get("n_states", 1))
        layout = rac.LAYOUT_BITS | (rac.LAYOUT_PACKED if args.layout == "packed" else 0)
        self.nets = [rac.Network(x.n, x.d, x.scope, x.rel, layout=layout, states=per_launch,
                                 plan=len(nets_np) > 1, rows=args.rows,
                                 packed=None if args.layout == "auto" else args.layout == "packed")
                     for x in nets_np]
        args.packed = any(net.info()["words_per_relation"] < (x.d + 3) // 4 * 4
                          for net, x in zip(self.nets, nets_np))
        self.cfg["relation_rows"] = "packed" if args.packed else "a word per row"
        self.cfg["tile_rows"] = sorted({int(net.info()["rows_per_slab"]) for net in self.nets})
        self.flat = flat
        self.din = torch.from_numpy(np.ascontiguousarray(flat).view(np.int32)).to(dev)
        self.dout = torch.empty_like(self.din)
        self.it = torch.empty(self.B, dtype=torch.int32, device=dev)
        self.st = torch.empty(self.B, dtype=torch.int32, device=dev)
        self.plan = rac.Plan(self.nets, items, offs) if len(self.nets) > 1 else None
        self.rac = rac
        self.torch = torch
        self.dev = dev
        self.pred = None
        if spec.get("learned"):
            self.pred, self.thr, self.train_info = train_predictor(rac, torch, args.seed)
            self.cfg["gating"] = ("learned (rac_enforce_learned, pending-pair verification, "
                                  "min_scored %d)" % LEARNED_MIN_SCORED)

    def capture(self, flags):
        """Batches of several networks: record the plan's launch (it
        allocates nothing) in a CUDA graph once; each step replays it."""
        if self.plan is None:
            return
        torch = self.torch
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self.plan.enforce(self.din, self.dout, self.it, self.st, flags=flags)
        torch.cuda.synchronize()
        self.cfg["launch"] = "CUDA graph replay of the plan's one persistent launch"

    def step(self, flags, stream):
        rac = self.rac
        if getattr(self, "graph", None) is not None:
            self.graph.replay()
        elif self.pred is not None:
            rac.enforce_learned(self.nets[0], self.din, self.dout, self.it, self.st,
                                predictor=self.pred, threshold=self.thr, flags=flags,
                                stream=stream, min_scored=LEARNED_MIN_SCORED)
        elif self.plan is not None:
            self.plan.enforce(self.din, self.dout, self.it, self.st, flags=flags, stream=stream)
        elif self.B == 1:
            rac.enforce(self.nets[0], self.din, self.dout, self.it, self.st, flags=flags,
                        stream=stream)
        else:
            rac.enforce_batch(self.nets, self.items, self.offs, self.din, self.dout, self.it,
                              self.st, flags=flags, stream=stream)

    def plain_step(self, stream, ptr_in, ptr_out, it_ptr, st_ptr):
        """Plain GPU RAC on the same items: one single-state launch per item."""
        L = self.rac.lib()
        sh = stream.cuda_stream
        for j in range(self.B):
            net = self.nets[int(self.items[j])]
            o = int(self.offs[j]) * 4
            rc = L.rac_enforce(net.handle, ptr_in + o, ptr_out + o, it_ptr + 4 * j, st_ptr + 4 * j,
                               0, 0, sh)
            if rc != 0:
                raise self.rac.RacError(rc, self.rac.last_error())

    def alg_bytes(self, its):
        """m d^2 / 8 bytes per network per sweep that any of its states ran:
        a launch reads each relation once per sweep for all of its states."""
        per_net = {}
        for j in range(self.B):
            k = int(self.items[j])
            per_net[k] = max(per_net.get(k, 0), int(its[j]))
        return float(sum(self.nets_np[k].m * self.nets_np[k].d ** 2 / 8.0 * sw
                         for k, sw in per_net.items()))

    def plain_bits(self, its):
        """Relation bits of the plain recurrence: m d^2 per state per sweep."""
        return float(sum(self.nets_np[int(self.items[j])].m * self.nets_np[int(self.items[j])].d ** 2
                         * int(its[j]) for j in range(self.B)))


def compare_learned(W, args, stream, flush, per_step_s, world):
    """Learned gating against plain and Proposition-2 RAC on the same states:
    the same batch through rac_enforce_batch (flags 0 and RAC_INCREMENTAL),
    CUDA-event timed like the main loop; (slab, state) evaluations from the
    trace counters; the learned result checked against the plain one."""
    torch, rac = W.torch, W.rac
    B = W.B
    net = W.nets[0]
    out_p = torch.empty_like(W.din)
    it_p = torch.empty(B, dtype=torch.int32, device=W.dev)
    st_p = torch.empty_like(it_p)

    def timed(fn, reps):
        tot = 0.0
        for _ in range(reps):
            flush()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            torch.cuda.synchronize()
            tot += a.elapsed_time(b) / 1000.0
        return tot / reps

    reps = max(3, min(20, args.steps))
    res = {}
    for name, fl in (("plain", 0), ("proposition2", rac.INCREMENTAL)):
        def run(fl=fl):
            rac.enforce_batch([net], W.items, W.offs, W.din, out_p, it_p, st_p, flags=fl,
                              stream=stream)
        run()
        t = timed(run, reps)
        res[name] = {"value": world * B / t, "unit": "fixpoints/s", "ms_per_step": t * 1000.0}
    torch.cuda.synchronize()
    plain_its = it_p.cpu().numpy()
    if not (torch.equal(out_p, W.dout) and np.array_equal(st_p.cpu().numpy(), W.st.cpu().numpy())):
        raise SystemExit("learned gating disagrees with plain RAC")
    tr = rac.Trace(0)
    rac.enforce_learned(net, W.din, out_p, it_p, st_p, predictor=W.pred, threshold=W.thr,
                        trace=tr, stream=stream, min_scored=LEARNED_MIN_SCORED)
    torch.cuda.synchronize()
    learned_evals = tr.evaluated()
    learned_sweeps = it_p.cpu().numpy()
    rac.enforce_learned(net, W.din, out_p, it_p, st_p, predictor=None, trace=tr, stream=stream)
    torch.cuda.synchronize()
    p2_evals = tr.evaluated()
    slabs = net.info()["n_slabs"]
    res.update({
        "evaluations": {"plain": int(plain_its.sum()) * slabs, "proposition2": p2_evals,
                        "learned": learned_evals, "unit": "(slab, state) evaluations per step"},
        "sweeps_per_fixpoint_plain": float(plain_its.mean()),
        "sweeps_per_fixpoint_learned": float(learned_sweeps.mean()),
        "max_sweeps": {"plain": int(plain_its.max()), "learned": int(learned_sweeps.max())},
        "speedup_vs_plain": res["plain"]["ms_per_step"] / (per_step_s * 1000.0),
        "speedup_vs_proposition2": res["proposition2"]["ms_per_step"] / (per_step_s * 1000.0),
        "_plain_iterations": plain_its})
    return res


def tensor_roofline(W, its, per_step_s, kernel):
    """The tensor-core kernel's algorithmic MMA work -- per state and sweep,
    every relation's forward and reverse counts, 2 x d x d multiply-adds
    each (4 d^2 flops) -- over the launch's CUDA-event time, against the
    dense FP8 peak measured on this machine (profiles/fp8_peak.json)."""
    flops = sum(4.0 * W.nets_np[int(W.items[j])].m * W.nets_np[int(W.items[j])].d ** 2 * int(its[j])
                for j in range(W.B))
    try:
        peak = float(json.load(open(os.path.join(ROOT, "profiles", "fp8_peak.json")))
                     ["fp8_e4m3_tflops_burst"])
        src = "measured (profiles/fp8_peak.json: cuBLASLt E4M3 GEMM)"
    except (OSError, ValueError, KeyError):
        peak, src = 4500.0, "nominal dense FP8"
    achieved = flops / per_step_s / 1e12
    return {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": None, "peak_source": src, "kernel": kernel,
            "alg_flops_per_launch": flops}


def issue_roofline(wl, per_step_s, torch, dev, peaks, kernel):
    """Warp instructions per launch (ncu smsp__inst_executed.sum, recorded on
    the kernel's current sources) over the live CUDA-event time of a launch,
    against the SM issue peak: SMs x 4 schedulers x 1 warp instruction per
    cycle at the maximum SM clock."""
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz = float(peaks["sm_max_mhz"]) if peaks and "sm_max_mhz" in peaks else 2032.0
    peak = sms * 4 * mhz * 1e6 / 1e12
    ent = profile_entry(wl) or {}
    inst = ent.get("inst_executed")
    achieved = inst / per_step_s / 1e12 if inst else None
    return {"bound": "issue", "achieved": achieved, "peak": peak,
            "unit": "T warp-instructions/s", "frac": achieved / peak if inst else None,
            "inst_per_launch": inst, "traffic": ent.get("dram_bytes_per_launch"),
            "peak_source": "derived: %d SMs x 4 schedulers x %.0f MHz (maximum SM clock)"
                           % (sms, mhz),
            "kernel": kernel}


def run_ours(args):
    import torch
    import paper_2407_11388_b300 as rac
    from paper_2407_11388_b300.dist import max_over_ranks

    world, rank, local = dist_setup(args)
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
        pg = dist

    W = Prepared(args, rac, torch, dev)
    B = W.B
    stream = torch.cuda.current_stream()
    flush = L2Flush(torch, dev)
    # at least 20 untimed steps (each is microseconds to milliseconds): the
    # first launches after the set-up run slower (clock ramp, first touches
    # of the store's pages), and a short run would average them in
    warm = max(20, args.warmup)
    for _ in range(warm):
        W.step(args.flags, stream)
        flush()
    torch.cuda.synchronize()
    its = W.it.cpu().numpy()
    W.capture(args.flags)
    for _ in range(3):  # the replayed graph gives the eager launch's results
        W.step(args.flags, stream)
        flush()
    torch.cuda.synchronize()
    if not np.array_equal(W.it.cpu().numpy(), its):
        raise SystemExit("the replayed graph disagrees with the eager launch")
    statuses = W.st.cpu().numpy()
    total_sweeps = int(its.sum())

    K = args.steps
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    # the interpreter's cyclic collector stays off inside timed loops (its
    # passes over the live objects would land in the host-timed ones)
    gc.collect()
    gc.disable()
    with ClockSampler(local) as clk:
        # the sampler's start-up leaves the GPU idle for a while: a few more
        # untimed steps bring its clock back up before the timed ones
        for _ in range(RESUME_STEPS):
            W.step(args.flags, stream)
            flush()
        w0 = time.perf_counter()
        for i in range(K):
            starts[i].record(stream)
            W.step(args.flags, stream)
            ends[i].record(stream)
            flush()
        torch.cuda.synchronize()
        wall = time.perf_counter() - w0
    gc.enable()
    if pg:
        pg.barrier()
    dev_ms = max_over_ranks(float(sum(s.elapsed_time(e) for s, e in zip(starts, ends))))
    del starts, ends
    gc.collect()
    per_step_s = dev_ms / 1000.0 / K
    value = world * B / per_step_s

    learned_cmp = None
    if W.pred is not None:
        learned_cmp = compare_learned(W, args, stream, flush, per_step_s, world)
        its = learned_cmp.pop("_plain_iterations")
    # plain GPU RAC on the same items (only where the step is a batch)
    plain = None
    if B > 1 and W.pred is None:
        pin, pout = W.din.data_ptr(), W.dout.data_ptr()
        pit = torch.empty(B, dtype=torch.int32, device=dev)
        pst = torch.empty(B, dtype=torch.int32, device=dev)
        W.plain_step(stream, pin, pout, pit.data_ptr(), pst.data_ptr())
        torch.cuda.synchronize()
        if not (np.array_equal(pit.cpu().numpy(), its) and np.array_equal(pst.cpu().numpy(), statuses)):
            raise SystemExit("plain per-item launches disagree with the batched launch")
        ps = max(1, min(3, K))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t_plain = 0.0
        for _ in range(ps):
            flush()
            e0.record(stream)
            W.plain_step(stream, pin, pout, pit.data_ptr(), pst.data_ptr())
            e1.record(stream)
            torch.cuda.synchronize()
            t_plain += e0.elapsed_time(e1) / 1000.0
        t_plain = max_over_ranks(t_plain) / ps
        plain = {"value": world * B / t_plain, "unit": "fixpoints/s", "steps": ps,
                 "how": "one single-state rac_enforce launch per item (kernel (a)), same items",
                 "speedup_of_this_form": (world * B / per_step_s) / (world * B / t_plain)}

    # the tensor-core kernel against kernel (a) on the same states (one
    # batched launch each, the same flags otherwise)
    kernel_a = None
    if args.flags & 0x10:
        fl_a = args.flags & ~0x10
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        W.step(fl_a, stream)
        torch.cuda.synchronize()
        reps, t_a = max(3, min(20, K)), 0.0
        for _ in range(reps):
            flush()
            e0.record(stream)
            W.step(fl_a, stream)
            e1.record(stream)
            torch.cuda.synchronize()
            t_a += e0.elapsed_time(e1) / 1000.0
        t_a = max_over_ranks(t_a) / reps
        kernel_a = {"ms_per_step": t_a * 1000.0, "value": world * B / t_a, "unit": "fixpoints/s",
                    "how": "kernel (a) (bit-packed) on the same states, same launch shape",
                    "tensor_speedup_over_it": t_a / per_step_s}

    # end to end through the host entry point (copies inside the timed region)
    e2e = None
    if not args.no_e2e and len(W.nets) == 1 and W.pred is None:
        host_in = torch.from_numpy(np.ascontiguousarray(W.flat).view(np.int32).copy()).pin_memory()
        host_out = torch.empty_like(host_in).pin_memory()
        hit = torch.empty(B, dtype=torch.int32).pin_memory()
        hst = torch.empty(B, dtype=torch.int32).pin_memory()
        L = rac.lib()
        sh = stream.cuda_stream
        net = W.nets[0]

        def host_step():
            rc = L.rac_enforce_host(net.handle, B, host_in.data_ptr(), host_out.data_ptr(),
                                    hit.data_ptr(), hst.data_ptr(), 0, args.flags, sh)
            if rc != 0:
                raise rac.RacError(rc, rac.last_error())

        for _ in range(20):
            host_step()
        Ke = max(100, min(K, 500))  # host calls: at least 100 even in a short run
        if pg:
            pg.barrier()
        gc.collect()
        gc.disable()
        t0 = time.perf_counter()
        for _ in range(Ke):
            host_step()
        el = time.perf_counter() - t0
        gc.enable()
        el = max_over_ranks(el)
        if not np.array_equal(host_out.numpy().view(np.uint32), W.dout.cpu().numpy().view(np.uint32)):
            raise SystemExit("host entry point disagrees with the device entry point")
        e2e = {"value": world * B * Ke / el, "unit": "fixpoints/s",
               "h2d_bytes_per_step": int(W.flat.size * 4), "d2h_bytes_per_step": int(W.flat.size * 4 + B * 8),
               "steps": Ke}
    elif not args.no_e2e:
        # batches and learned gating: pinned host states copied in, the step's
        # launch, results copied out
        host_in = torch.from_numpy(np.ascontiguousarray(W.flat).view(np.int32).copy()).pin_memory()
        host_out = torch.empty_like(host_in).pin_memory()
        hit = torch.empty(B, dtype=torch.int32).pin_memory()
        Ke = max(3, min(K, 20))
        torch.cuda.synchronize()
        gc.collect()
        gc.disable()
        t0 = time.perf_counter()
        for _ in range(Ke):
            W.din.copy_(host_in, non_blocking=True)
            W.step(args.flags, stream)
            host_out.copy_(W.dout, non_blocking=True)
            hit.copy_(W.it, non_blocking=True)
            torch.cuda.synchronize()
        el = time.perf_counter() - t0
        gc.enable()
        el = max_over_ranks(el)
        e2e = {"value": world * B * Ke / el, "unit": "fixpoints/s",
               "h2d_bytes_per_step": int(W.flat.size * 4), "d2h_bytes_per_step": int(W.flat.size * 4 + B * 4),
               "steps": Ke}

    peaks = measured_peaks()
    hbm_peak = float(peaks["hbm_gbs"]) if peaks and "hbm_gbs" in peaks else 6400.0
    alg_bytes_per_launch = W.alg_bytes(its)
    achieved = alg_bytes_per_launch / per_step_s / 1e9
    traffic = traffic_from_profiles(profile_key(args))
    clocks = clk.summary()
    kernel = "rac_batch_kernel" if W.plan is not None else (
        "rac_tc_kernel" if args.flags & 0x10 else "rac_bits_kernel")

    hbm_line = {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                "frac": achieved / hbm_peak, "traffic": traffic,
                "peak_source": "measured" if peaks else "fallback",
                "kernel": kernel, "alg_bytes_per_launch": alg_bytes_per_launch}
    roof = hbm_line
    if args.flags & 0x10:
        # the tensor-core kernel: its MMAs against the measured FP8 peak
        roof = tensor_roofline(W, its, per_step_s, kernel="rac_tc_kernel")
        roof["hbm"] = hbm_line
    elif B > 1:
        # many states: the per-state support tests bound the launch, not the
        # one read of the store per sweep; the binding roofline is the SM
        # issue rate (one warp instruction per cycle per scheduler)
        roof = issue_roofline(profile_key(args), per_step_s, torch, dev, peaks, kernel)
        roof["hbm"] = hbm_line
    line = {"metric": METRIC, "value": value, "unit": "fixpoints/s", "n_gpus": world,
            "steps": K, "warmup": warm + RESUME_STEPS, "ms_per_step": per_step_s * 1000.0,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic (seeded random binary CSP, generated in-process)",
            "config": W.cfg,
            "relation_bits_per_s": world * W.plain_bits(its) / per_step_s,
            "sweeps_per_fixpoint": total_sweeps / B,
            "status_counts": {str(k): int(v) for k, v in zip(*np.unique(statuses, return_counts=True))},
            "wall_s_timed_region": wall,
            "roofline": roof,
            "clocks": clocks,
            "gpu_launches": K,
            "e2e": e2e}
    if plain is not None:
        line["plain_gpu_rac"] = plain
    if kernel_a is not None:
        line["kernel_a_same_states"] = kernel_a
    if learned_cmp is not None:
        line["learned"] = learned_cmp
        line["learned"]["training"] = W.train_info
        line["sweeps_per_fixpoint"] = learned_cmp["sweeps_per_fixpoint_learned"]
    if rank == 0 and not args.no_cpu_baseline:
        cb, _ = cpu_baseline(W)
        line["cpu_baseline"] = cb
    if rank == 0:
        print(json.dumps(line), flush=True)
    if W.plan is not None:
        W.plan.close()
    for n in W.nets:
        n.close()
    if pg:
        pg.destroy_process_group()


def _search_alg_bytes(x, steps):
    """Algorithmic bytes of the timed assignments: the seeded first sweep reads
    the assigned variable's constraints, every later sweep the whole store
    (m d^2 / 8 bytes)."""
    deg = np.bincount(np.asarray(x.scope).reshape(-1), minlength=x.n)
    return sum(deg[var] * x.d * x.d / 8.0 + (it - 1) * x.m * x.d * x.d / 8.0
               for _, var, _, it, _ in steps)


def cpu_search_baseline(x, budget_s=15.0):
    """The oracle's Algorithm 2 on the same network: assignments per second
    (each a whole Eq. 1 enforcement on all host cores) for about budget_s."""
    from oracle.search import dfs as oracle_dfs
    threads = os.cpu_count() or 1
    nodes, el = 8, 0.0
    while True:
        t0 = time.perf_counter()
        out = oracle_dfs(x.n, x.d, x.scope, x.rel, racgen_full(x), nodes, threads=threads)
        el = time.perf_counter() - t0
        if el >= budget_s or out["nodes"] < nodes or nodes >= 4096:
            break
        nodes = int(nodes * max(2.0, min(8.0, budget_s / max(el, 1e-3))))
    done = max(1, out["nodes"])
    return {"value": done / el, "unit": "fixpoints/s", "cores": threads, "kind": "oracle",
            "sample": "the first %d assignments of the oracle's Algorithm 2 search on this "
                      "network (each a whole Eq. 1 enforcement), %.1f s" % (done, el)}


def racgen_full(x):
    import racgen
    return racgen.full_domain(x.n, x.d)


def run_search(args):
    """One step = one assignment of Algorithm 2's search and its seeded
    enforcement, timed on the device (CUDA events around each launch, L2
    flushed before each, outside the events); the whole search's wall time
    per assignment (the host's variable choice reads each child state back)
    is the end-to-end figure."""
    import torch
    import paper_2407_11388_b300 as rac
    from paper_2407_11388_b300.dist import max_over_ranks
    from paper_2407_11388_b300.search import dfs

    world, rank, local = dist_setup(args)
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if world > 1:  # every rank searches its own network (weak scaling)
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
        pg = dist
    spec, x, _ = make_inputs(args.workload, args.seed + rank)
    net = rac.Network(x.n, x.d, x.scope, x.rel)
    stream = torch.cuda.current_stream()
    flush = L2Flush(torch, dev)
    W, K = max(3, args.warmup), args.steps
    events = []

    def hook(phase):
        if phase == "before":
            flush()
            events.append([torch.cuda.Event(enable_timing=True),
                           torch.cuda.Event(enable_timing=True)])
            events[-1][0].record(stream)
        else:
            events[-1][1].record(stream)

    gc.collect()
    gc.disable()
    with ClockSampler(local) as clk:
        res = dfs(net, racgen_full(x), max_nodes=W + K, stream=stream, flags=args.flags, hook=hook)
        torch.cuda.synchronize()
    gc.enable()
    timed = res.steps[W:]
    if not timed:
        raise SystemExit("the search ended after %d assignments: no step to time" % res.nodes)
    dev_s = sum(a.elapsed_time(b) for a, b in events[W:]) / 1000.0
    per_step_s = max_over_ranks(dev_s / len(timed))
    # end to end: the same search from the host domains through the
    # library's own search loop (rac_search), no flushes, wall clock
    gc.collect()
    gc.disable()
    t0 = time.perf_counter()
    res2 = rac.run_search(net, racgen_full(x), max_nodes=W + K, flags=args.flags, stream=stream)
    wall = time.perf_counter() - t0
    gc.enable()
    wall_per_step = max_over_ranks(wall / max(1, res2["nodes"]))
    if [tuple(int(v) for v in r) for r in res2["steps"]] != \
            [tuple(int(v) for v in r) for r in res.steps]:
        raise SystemExit("the library's search took other steps than the timed one")
    peaks = measured_peaks()
    hbm_peak = float(peaks["hbm_gbs"]) if peaks and "hbm_gbs" in peaks else 6400.0
    alg = _search_alg_bytes(x, timed) / len(timed)
    its = [s[3] for s in timed]
    line = {"metric": METRIC, "value": world / per_step_s, "unit": "fixpoints/s", "n_gpus": world,
            "steps": len(timed), "warmup": W, "ms_per_step": per_step_s * 1000.0,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic (seeded random binary CSP, generated in-process)",
            "config": {"workload": args.workload, "n": x.n, "d": x.d, "density": spec["density"],
                       "tightness": spec["tightness"], "constraints": int(x.m),
                       "state_kind": "search (Algorithm 2: assign, then seeded enforcement)",
                       "seed_generated": True, "l2": L2_NOTE},
            "sweeps_per_fixpoint": float(np.mean(its)),
            "search": {"assignments": res.nodes, "root_sweeps": res.root_iterations,
                       "solution_found": res.solution is not None,
                       "wipeouts": int(sum(1 for s in timed if s[4] == rac.WIPEOUT)),
                       "sweeps_per_assignment": float(np.mean(its)),
                       "paper_table1_range": "3.44-4.83 sweeps per assignment (its own networks)"},
            "roofline": {"bound": "hbm", "achieved": alg / per_step_s / 1e9, "peak": hbm_peak,
                         "unit": "GB/s", "frac": alg / per_step_s / 1e9 / hbm_peak,
                         "traffic": traffic_from_profiles(args.workload),
                         "peak_source": "measured" if peaks else "fallback",
                         "kernel": "rac_bits_kernel", "alg_bytes_per_launch": alg},
            "clocks": clk.summary(),
            "gpu_launches": len(timed),
            "e2e": {"value": world / wall_per_step, "unit": "fixpoints/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": int(x.n * 4 + 8), "steps": res2["nodes"],
                    "note": "the whole search on the host's clock through rac_search: an "
                            "assignment's inputs are launch parameters (the parent state stays "
                            "on the device); the kernel writes the child state, its sweep count "
                            "and status into pinned memory for the next choice"}}
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_search_baseline(x)
    if rank == 0:
        print(json.dumps(line), flush=True)
    net.close()
    if pg:
        pg.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif WORKLOADS[args.workload].get("search"):
        run_search(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
