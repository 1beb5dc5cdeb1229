"""Host logic of bench.py without a GPU: the default launch (one GPU, K and W
that finish within minutes, W >= 3), the clock summary of nvidia-smi samples
(median under load, throttle reasons), the measured peaks, the workload
description, and the reference arm's JSON line (the oracle timed on the
host cores) on a small detector."""
import io
import json
import sys
from contextlib import redirect_stdout

import bench
from paper_2203_14354_gb300 import geometry as g


def test_default_launch(monkeypatch):
    monkeypatch.setattr(sys, "argv", ["bench.py"])
    a = bench.parse()
    assert a.gpus == 1 and a.impl == "ours" and a.warmup >= 3 and 1 <= a.steps <= 10
    assert a.photons == 1e8


def test_clock_summary():
    c = bench.ClockSampler(0)
    c.rows = [["0", "2070", "2070", "500.1", "Not Active", "Not Active", "Not Active", "Not Active"],
              ["0", "1980", "2070", "900.0", "Not Active", "Not Active", "Not Active", "Active"],
              ["0", "2070", "2070", "[N/A]", "Not Active", "Not Active", "Not Active", "Not Active"]]
    s = c.summary()
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0 and s["samples"] == 3
    assert s["reasons"] == ["sw_power_cap"]
    assert bench.ClockSampler(0).summary()["reasons"] == ["unavailable"]


def test_measured_peaks_and_workload():
    peaks, kind = bench.measured_peaks()
    assert kind in ("measured", "fallback") and peaks["hbm_gbs"] > 1000
    cfg = bench.workload_config(100_000_000, 2, 17_927_640)
    assert cfg["photons_per_step"] == 200_000_000 and cfg["photons_per_rank"] == 100_000_000
    assert cfg["triangles"] == 17_927_640 and "1.79e7" in cfg["workload"]


def test_reference_arm_line(monkeypatch):
    monkeypatch.setattr(g, "darwin", lambda **kw: g.small_tpc())
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--steps", "2", "--warmup", "1",
                                      "--cpu-seconds", "0.2"])
    a = bench.parse()
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.run_reference(a, 0, 1)
    line = json.loads(buf.getvalue().strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["steps"] == 2 and line["warmup"] == 1
    assert line["metric"] == bench.METRIC and line["unit"] == "photons/s" and line["higher_is_better"]
    assert line["value"] > 0 and line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"] == {"value": line["value"], "unit": "photons/s", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    # other ranks print nothing
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.run_reference(a, 1, 2)
    assert buf.getvalue() == ""


def test_pmt_rings_of_the_50cm_tpc():
    """The ring aggregates of the adjoint check: per array, the hexagonal
    rings 0..4 of the 80 mm window lattice, 1 + 6 + 12 + 18 + 24 windows."""
    import bench
    from paper_2203_14354_gb300 import geometry as g
    labels, masks, pitch = bench.pmt_rings(g.scaled_tpc())
    assert pitch == 80.0
    assert [int(m.sum()) for m in masks] == [1, 6, 12, 18, 24] * 2
    assert labels[0].startswith("top ring 0") and labels[5].startswith("bottom ring 0")
    import numpy as np
    together = np.sum(masks, axis=0)
    assert np.all(together == 1)


def test_kernel_signature_reads_the_build_log():
    """The staleness check of the ncu-derived constants: the timed kernel's
    registers and spills come from the library's ptxas log, its sources'
    hash from the files."""
    from paper_2203_14354_gb300 import build
    build.build()
    sig = bench.kernel_signature()
    assert isinstance(sig["registers"], int) and 16 <= sig["registers"] <= 255
    assert isinstance(sig["spill_stores"], int) and isinstance(sig["spill_loads"], int)
    assert len(sig["sources_sha256"]) == 64
    assert set(sig) == set(bench.CAPTURED_KERNEL)


def test_adjoint_summary_is_compact():
    """The bench line's adjoint field: the cost ratio and the finite-
    difference summary, taking each parameter at the step it was resolved
    with (the wide step for noisy ones)."""
    def agg(rel, z, fd, se):
        return {"rel_diff": rel, "z": z, "fd": fd, "fd_se": se, "adjoint": fd, "adjoint_se": se}
    fd = {"photons": 10 ** 9, "h_rel": 1e-3, "params": ["a", "b"], "seconds": 1.0,
          "total": agg([0.01, 0.9], [1.0, 0.5], [100.0, 1.0], [1.0, 5.0]),
          "top": agg([0.012, 0.5], [1.1, 0.4], [50.0, 1.0], [0.5, 5.0]),
          "bottom": agg([0.011, 0.5], [0.9, 0.3], [50.0, 1.0], [0.5, 5.0]),
          "per_pmt": {"z": [0.5, -1.0]}, "rings": {"z_max": [1.5, 2.0]},
          "wide_step": {"h_rel": 3e-2, "params": ["b"], "total": agg([0.5], [0.2], [1.0], [1.0]),
                        "top": agg([0.015], [0.4], [100.0], [1.0]), "bottom": agg([0.012], [0.3], [100.0], [1.0])}}
    s = bench.adjoint_summary({"ratio": 1.16, "fwd_ms": 10.0, "fwd_adjoint_ms": 11.6, "fd_check": fd})
    assert s["ratio"] == 1.16 and s["fd"]["wide_params"] == ["b"]
    # resolved: a on all three aggregates, b on top and bottom at the wide step
    assert s["fd"]["max_rel_diff_resolved"] == 0.015
    assert len(json.dumps(s)) < 600
