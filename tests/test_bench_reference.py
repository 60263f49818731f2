"""bench.py's reference arm (the FP64 oracle on the host cores) runs without a GPU and
prints one JSON line with the contract's keys, in the main arm's metric and unit."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_the_contract_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "3"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads([l for l in r.stdout.splitlines() if l.startswith("{")][-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["n_gpus"] == 1
    assert line["unit"] == "updates/s" and line["higher_is_better"] is True
    assert line["metric"].startswith("DVM cell-velocity updates/s")
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["cpu_baseline"]["cores"] >= 1 and line["cpu_baseline"]["sample"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
    assert line["config"]["n_cells"] == 20000 and line["config"]["order"] == 2


def test_recorded_traffic_is_reported_only_for_the_captured_sources(tmp_path):
    """roofline.traffic comes from a recorded ncu capture and is null once the kernel
    sources differ from those the capture ran."""
    sys.path.insert(0, ROOT)
    import bench
    csrc = tmp_path / "csrc"
    csrc.mkdir()
    for name in bench.KERNEL_SOURCES:
        (csrc / name).write_text("// " + name + "\n")
    digest = bench.kernel_sources_sha256(str(csrc))
    rec = tmp_path / "capture.md"
    rec.write_text("summary\n\ntraffic_bytes_per_launch_pair: 1651000000\nkernel_sources_sha256: %s\n" % digest)
    assert bench.sweep_traffic("fp32", 2, str(rec), str(csrc)) == (1651000000.0, "ncu capture of these kernel sources")
    assert bench.sweep_traffic("fp64", 2, str(rec), str(csrc))[0] is None
    (csrc / bench.KERNEL_SOURCES[0]).write_text("// changed\n")
    t, note = bench.sweep_traffic("fp32", 2, str(rec), str(csrc))
    assert t is None and "changed" in note
    assert bench.sweep_traffic("fp32", 2, str(tmp_path / "missing.md"), str(csrc))[0] is None
