"""Host logic of bench.py that needs no GPU: the clock record keeps only samples taken
inside the timed region and names every throttle reason seen there; the wavefront
traffic figure is withheld once the kernel sources differ from the profiled ones; the
reference arm prints one well-formed JSON line."""
import json
import os
import subprocess
import sys

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ACTIVE, IDLE = "Active", "Not Active"


def _line(sm, reasons=(IDLE, IDLE, IDLE, IDLE)):
    return f"{sm}, 2070, 700, 0x0, " + ", ".join(reasons)


def test_clock_record_keeps_the_timed_region_only():
    c = bench.ClockSampler(0)
    c.lines = [(0.9, _line(1000, (ACTIVE, IDLE, IDLE, IDLE))),   # warm-up: not in the record
               (1.1, _line(2070)), (1.3, _line(2000, (IDLE, IDLE, IDLE, ACTIVE))), (1.5, _line(2040)),
               (3.0, _line(500, (IDLE, ACTIVE, IDLE, IDLE)))]     # after the region
    c.t0, c.t1 = 1.0, 1.5
    s = c.summary()
    assert s == {"sm_mhz": 2040.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    c.t0 = c.t1 = None
    assert c.summary()["samples"] == 0


def test_traffic_is_withheld_for_other_sources(monkeypatch):
    import hashlib
    assert bench.wave_traffic(128) is None                   # another workload size
    got = bench.wave_traffic(256)
    assert got is None or got == bench.WAVE_TRAFFIC_BYTES
    # a figure taken on the current sources is reported; one taken on other sources is not
    rel = "paper_2406_00878_gb300/csrc/pit_kernels.cuh"
    with open(os.path.join(ROOT, rel), "rb") as f:
        digest = hashlib.sha256(f.read()).hexdigest()
    monkeypatch.setattr(bench, "WAVE_TRAFFIC_BYTES", 1.0e8)
    monkeypatch.setattr(bench, "WAVE_TRAFFIC_SOURCES", {rel: digest})
    assert bench.wave_traffic(256) == 1.0e8
    monkeypatch.setattr(bench, "WAVE_TRAFFIC_SOURCES", {rel: "0" * 64})
    assert bench.wave_traffic(256) is None


def test_reference_arm_prints_one_json_line():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0",
                          "--ref-levels", "2"], cwd=ROOT, capture_output=True, text=True, timeout=600, check=True)
    lines = [l for l in out.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "DOF/s" and d["value"] > 0 and d["higher_is_better"]
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
