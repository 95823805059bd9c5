"""Host logic of bench.py that needs no GPU: the code hash that ties the
recorded DRAM traffic to the kernel sources, and the JSON line of the
reference arm (the CPU oracle)."""
import json
import os
import subprocess
import sys

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_code_only_drops_comments_and_keeps_strings():
    src = 'int a = 1; // one\n/* block\n comment */ const char *s = "a // b /* c */";\n'
    out = bench._code_only(src)
    assert "one" not in out and "block" not in out
    assert '"a // b /* c */"' in out and "int a = 1;" in out


def test_comment_edits_keep_the_hash(monkeypatch, tmp_path):
    """The traffic figures stay valid across comment edits, not across code
    edits."""
    csrc = tmp_path / "paper_2407_11388_b300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "k.cu").write_text("__global__ void k() { int x = 1; }  // note\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h0 = bench.source_hash()
    (csrc / "k.cu").write_text("// a new comment\n__global__ void k() { int x = 1; }\n")
    assert bench.source_hash() == h0
    (csrc / "k.cu").write_text("__global__ void k() { int x = 2; }\n")
    assert bench.source_hash() != h0


def test_traffic_needs_the_recorded_hash(monkeypatch):
    data = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    ent = data["dense_n500_d20"]
    monkeypatch.setattr(bench, "source_hash", lambda kernel=None: ent["source_hash"])
    assert bench.traffic_from_profiles("dense_n500_d20") == ent["dram_bytes_per_launch"]
    monkeypatch.setattr(bench, "source_hash", lambda kernel=None: "0" * 16)
    assert bench.traffic_from_profiles("dense_n500_d20") is None
    assert bench.traffic_from_profiles("no_such_workload") is None


def test_reference_arm_line():
    """`--impl reference` runs the oracle and prints the contract's line: the
    arm's metric and config, impl, a cpu_baseline describing the run and an
    e2e with no device copies."""
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "2",
                          "--warmup", "3", "--workload", "rb_n50_d10"],
                         cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config"):
        assert key in line, key
    assert line["impl"] == "reference" and line["steps"] == 2 and line["warmup"] == 3
    assert line["config"]["workload"] == "rb_n50_d10" and line["higher_is_better"] is True
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == line["value"] and cb["cores"] >= 1
    e = line["e2e"]
    assert e["value"] == line["value"] and e["unit"] == line["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0
