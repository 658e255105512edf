"""Host-side arithmetic of the benchmark (no GPU): the roofline figures and
the lookup of ncu DRAM traffic, which is reported only for the kernel source
and the workload it was captured on."""
import hashlib
import os
import types

import bench


def _tree(tmp_path, source_text, counters):
    src = tmp_path / "paper_2510_06562_gb300" / "csrc"
    src.mkdir(parents=True)
    (src / "k.cu").write_text(source_text)
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "k.md").write_text("# summary\n\n" + counters + "\n")
    return str(tmp_path), hashlib.sha256(source_text.encode()).hexdigest()


def test_traffic_reported_for_the_captured_source_and_workload(tmp_path):
    text = "__global__ void k() {}\n"
    sha = hashlib.sha256(text.encode()).hexdigest()
    root, _ = _tree(tmp_path, text,
                    f"counters: kernel=k<64,16> source_sha256={sha} dram_bytes_per_launch=1234 pairs=100000")
    assert bench.captured_traffic("k<64,16>", "k.cu", 100000, root) == 1234.0
    assert bench.captured_traffic("k<64,16>", "k.cu", 100900, root) == 1234.0   # same box, dynamics drift
    assert bench.captured_traffic("k<64,16>", "k.cu", 102000, root) is None     # another workload
    assert bench.captured_traffic("k<64,8>", "k.cu", 100000, root) is None      # another kernel
    assert bench.captured_traffic("k<64,16>", "missing.cu", 100000, root) is None


def test_traffic_withdrawn_when_the_source_changes(tmp_path):
    root, sha = _tree(tmp_path, "__global__ void k() {}\n",
                      "counters: kernel=k source_sha256=0000 dram_bytes_per_launch=1 pairs=10")
    assert bench.captured_traffic("k", "k.cu", 10, root) is None
    prof = os.path.join(root, "profiles", "k.md")
    with open(prof, "w") as f:
        f.write(f"counters: kernel=k source_sha256={sha} dram_bytes_per_launch=1\n")   # no pair count
    assert bench.captured_traffic("k", "k.cu", 10, root) is None


def test_committed_counters_lines_are_well_formed():
    pdir = os.path.join(bench.ROOT, "profiles")
    seen = 0
    for name in os.listdir(pdir):
        for line in open(os.path.join(pdir, name), errors="replace"):
            if not line.startswith("counters:"):
                continue
            fields = dict(kv.split("=", 1) for kv in line.split()[1:])
            assert {"kernel", "source_sha256", "dram_bytes_per_launch"} <= set(fields), line
            assert len(fields["source_sha256"]) == 64
            assert int(fields["dram_bytes_per_launch"]) > 0
            seen += 1
    assert seen >= 2


def test_roofline_arithmetic():
    D = types.SimpleNamespace(FP32=0, BF16_MLP=1)
    arch = types.SimpleNamespace(n_radial=16, n_feat=64)
    stages = {"edge_fwd_l0": 0.05, "edge_bwd_l1": 0.1, "atom_fwd_l0": 0.2, "neighbors": 0.3}
    E = 640_000
    # BF16: the MMAs issued per pair, K padded to 16: 2 (2 * 16 F + 2 F^2) flop in the backward pass
    r = bench.roofline_of(D, D.BF16_MLP, stages, E, arch)
    assert r["kernel"].startswith("edge_bwd_l1")          # the slowest edge pass, not the slowest stage
    assert r["algorithmic_flop_per_launch"] == 2 * (2 * 16 * 64 + 2 * 64 * 64) * E
    assert abs(r["achieved"] - 20480 * E / 1e-4 / 1e12) < 1e-9
    assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-15
    assert r["bound"] == "tensor" and r["unit"] == "TFLOP/s"
    # the algorithm's work per pair whichever the layer (the layer-0 kernel issues fewer MMAs than that)
    r = bench.roofline_of(D, D.BF16_MLP, {"edge_fwd_l0": 0.05, "edge_bwd_l0": 0.1}, E, arch)
    assert r["algorithmic_flop_per_launch"] == 2 * (2 * 16 * 64 + 2 * 64 * 64) * E
    # FP32: the run-time K, and the SIMT peak derived from the SM count and clock
    arch8 = types.SimpleNamespace(n_radial=8, n_feat=64)
    r = bench.roofline_of(D, D.FP32, {"edge_fwd_l0": 0.2, "edge_bwd_l0": 0.1}, E, arch8)
    assert r["algorithmic_flop_per_launch"] == 2 * (8 * 64 + 64 * 64) * E
    assert r["bound"] == "alu"
    assert abs(r["peak"] - 152 * 128 * 2 * 2.07e9 / 1e12) < 1e-9


def _run_bench(*argv, env=None):
    import subprocess
    import sys
    e = dict(os.environ, **(env or {}))
    r = subprocess.run([sys.executable, os.path.join(bench.ROOT, "bench.py"), *argv], capture_output=True,
                       text=True, timeout=600, env=e)
    assert r.returncode == 0, r.stderr[-2000:]
    return r.stdout


def test_reference_arm_line_on_the_small_box():
    """The reference arm times the FP64 oracle on the host cores and prints
    the same metric, unit and workload as the CUDA arm, with its own
    cpu_baseline and an e2e that moves no bytes."""
    import json
    out = _run_bench("--impl", "reference", "--workload", "water192", "--steps", "1", "--warmup", "0")
    lines = [ln for ln in out.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == "ns/day"
    assert d["higher_is_better"] is True and d["dtype"] == "f64" and d["steps"] == 1
    assert d["value"] > 0 and abs(d["ms_per_step"] - 3.0 / d["value"] * 86.4) < 1e-6 * d["ms_per_step"]
    assert d["config"]["workload"].startswith("water192: 64 rigid waters, 192 atoms, L=12.4 A")
    assert d["config"]["n_inner"] == 3 and d["config"]["inner_fs"] == 1.0
    import argparse
    from paper_2510_06562_gb300 import inputs as I
    ns = argparse.Namespace(workload="water192", outer_fs=3.0, n_inner=3)
    assert d["config"] == bench.step_config(ns, I.water_192(0), 1)     # the CUDA arm's config, key for key
    assert d["warmup"] == 3                                              # at least 3 untimed steps
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and "192-atom" in cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "ns/day", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_print_nothing():
    out = _run_bench("--impl", "reference", "--workload", "water192", "--steps", "1",
                     env={"RANK": "1", "WORLD_SIZE": "2"})
    assert out.strip() == ""
