"""Host logic of bench.py that decides what its JSON line reports: figures
taken from the committed ncu summaries only when those were captured on the
current kernel source, and the issue-slot roofline built from them."""
import os

import pytest

import bench


def test_profile_figures_follow_the_kernel_source(tmp_path, monkeypatch):
    """A summary whose kernel_source_sha256_16 matches the current sources
    yields its figures; a stale one (or a missing key) yields None."""
    prof = tmp_path / "profiles"
    prof.mkdir()
    cur = bench.kernel_source_hash()
    (prof / bench.PROFILES["cfg2"]).write_text(
        f"kernel_source_sha256_16: {cur}\n"
        "   dram_bytes_per_full_launch: 1.5e6\n"
        "   warp_instructions_per_path_step: 3.5   (comment)\n")
    (prof / bench.PROFILES["cfg4"]).write_text(
        "kernel_source_sha256_16: 0000000000000000\n"
        "   dram_bytes_per_full_launch: 2.0e8\n")
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: cur)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.profiled_traffic("cfg2") == 1.5e6
    assert bench.profiled_value("cfg2", "warp_instructions_per_path_step") == 3.5
    assert bench.profiled_value("cfg2", "no_such_key") is None
    assert bench.profiled_traffic("cfg4") is None          # stale source hash
    assert bench.profiled_traffic("e1") is None            # no summary for this workload


def test_issue_roofline_arithmetic(monkeypatch):
    """achieved = path-steps/s x warp instructions per path-step; peak = 152
    SMs x 4 schedulers x one warp instruction per cycle at the max SM clock."""
    monkeypatch.setattr(bench, "profiled_value", lambda config, key: 4.0)
    r = bench.issue_roofline("cfg2", 1.0e11, 2000.0)
    assert r["achieved_warp_inst_per_s"] == pytest.approx(4.0e11)
    assert r["peak_warp_inst_per_s"] == pytest.approx(152 * 4 * 2000e6)
    assert r["frac"] == pytest.approx(4.0e11 / (152 * 4 * 2000e6))
    monkeypatch.setattr(bench, "profiled_value", lambda config, key: None)
    assert bench.issue_roofline("cfg2", 1.0e11, 2000.0) is None


def test_committed_profiles_parse():
    """The committed summaries carry a source hash and the figures bench.py
    reads (whether or not they match the sources of this checkout)."""
    import re
    for name in bench.PROFILES.values():
        txt = open(os.path.join(bench.ROOT, "profiles", name)).read()
        assert re.search(r"kernel_source_sha256_16:\s*[0-9a-f]{16}", txt), name
        assert re.search(r"dram_bytes_per_full_launch:\s*[0-9.eE+]+", txt), name


def test_source_hash_covers_the_path_kernel_include_closure():
    """The hash gating the committed figures spans exactly the files compiled
    into the path kernel: every csrc/ file that instantiates the template, and
    every csrc/ header reachable from path_kernel.cuh by #include."""
    import re
    csrc = os.path.join(bench.ROOT, "paper_2301_05780_gb300", "csrc")

    def local_includes(name):
        txt = open(os.path.join(csrc, name)).read()
        return [f for f in re.findall(r'#include\s+"([^"]+)"', txt)
                if os.path.exists(os.path.join(csrc, f))]

    closure, todo = set(), ["path_kernel.cuh"]
    while todo:
        f = todo.pop()
        if f not in closure:
            closure.add(f)
            todo.extend(local_includes(f))
    users = {f for f in os.listdir(csrc) if f.endswith(".cu")
             and "&path_kernel<" in open(os.path.join(csrc, f)).read()}
    assert len(users) == 6
    assert set(bench.PATH_KERNEL_SOURCES) == closure | users


def test_reference_arm_prints_its_line():
    """`bench.py --impl reference` times the oracle on the host cores and prints
    one JSON line with the keys the comparison needs (config 1: a sample of
    under a second)."""
    import json
    import subprocess
    import sys
    out = subprocess.run([sys.executable, os.path.join(bench.ROOT, "bench.py"), "--impl",
                          "reference", "--config", "cfg1", "--steps", "2", "--warmup", "1"],
                         capture_output=True, text=True, timeout=600, check=True)
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == "path-steps/s"
    assert line["value"] > 0 and line["steps"] == 2 and line["higher_is_better"] is True
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"] == {"value": line["value"], "unit": "path-steps/s",
                           "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert line["config"]["workload"] == "cfg1_laplace_2x2"


def test_reference_arm_default_is_the_batched_workload():
    """With no --config the reference arm times the oracle on the default
    workload, the 16-problem batch (config 3), on a bounded sample per step."""
    import json
    import subprocess
    import sys
    out = subprocess.run([sys.executable, os.path.join(bench.ROOT, "bench.py"), "--impl",
                          "reference", "--steps", "1", "--warmup", "0"],
                         capture_output=True, text=True, timeout=600, check=True)
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["config"]["workload"] == "cfg3_batch16"
    assert line["value"] > 0 and line["steps"] == 1
    assert 0 < line["config"]["sample_budget_fraction"] <= 1
    assert "16 problems" in line["cpu_baseline"]["sample"]
