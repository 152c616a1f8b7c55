"""The algorithmic bytes behind the bench's roofline fractions, checked against their per-unit
definitions: the decode writes 16 bytes of cache and 4 of residual and reads 4 of samples per voxel,
plus the control points, the 72-byte descriptor and the 8-byte RMSE sum per block; the apron fill reads
and writes 16 bytes per apron voxel, and the apron voxels of an n^3 brick are the (n+1)^3 cube less
its n^3 interior."""

import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_fill_bytes_cover_the_three_apron_planes():
    n = bench.BRICK
    planes = (n + 1) ** 2 + (n + 1) * n + n * n  # x = n (with its edges), then y = n, then z = n
    assert planes == (n + 1) ** 3 - n ** 3
    assert bench.algorithmic_bytes(4096, True)["fill"] == 4096 * planes * 32
    assert bench.algorithmic_bytes(4096, False)["fill"] == 0


def test_decode_and_contraction_bytes_per_block():
    vox, cp = bench.BRICK ** 3, bench.NCP ** 3
    b = bench.algorithmic_bytes(1, True)
    assert b["decode"] == vox * (16 + 4 + 4) + cp * 4 + 72 + 8
    assert b["encode"] == vox * 4 + cp * 4
    assert b["adjoint"] == vox * 4 + cp * 4 + 72
    # the step's 4096 blocks of 32^3 at C = 12: 24.2 bytes per voxel through the decode
    assert abs(bench.algorithmic_bytes(4096, True)["decode"] / (4096 * vox) - 24.2) < 0.05


def test_reduced_step_field_is_for_profiling_only():
    """A step on another field than 512^3 needs the oracle checks and baselines off (they are written for the
    512^3 field), and the field must be a multiple of 32 of at least 64; both refusals come before any GPU
    work."""
    import subprocess
    run = lambda *a: subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *a], capture_output=True,
                                    text=True, cwd=ROOT, timeout=300)
    r = run("--field", "384")
    assert r.returncode != 0 and "--no-check --no-cpu-baseline" in r.stderr
    r = run("--field", "100", "--no-check", "--no-cpu-baseline")
    assert r.returncode != 0 and "multiple of 32" in r.stderr


def test_clock_sampler_reads_clocks_and_throttle_reasons(tmp_path, monkeypatch):
    """The clock record of a timed region: median SM clock, the maximum clock, and every throttle reason
    that was Active in any sample (here hw_slowdown in one row and sw_power_cap in another), from
    nvidia-smi's CSV rows (a stand-in script prints three samples, then waits to be stopped)."""
    import time
    fake = tmp_path / "nvidia-smi"
    rows = ["0, 2032, 2032, 800.5, 0x0, Not Active, Not Active, Not Active, Not Active",
            "0, 1980, 2032, 1100.2, 0x4, Not Active, Not Active, Not Active, Active",
            "0, 2032, 2032, 900.0, 0x8, Active, Not Active, Not Active, Not Active"]
    fake.write_text("#!/bin/sh\n" + "".join(f"echo '{r}'\n" for r in rows) + "exec sleep 30\n")
    fake.chmod(0o755)
    monkeypatch.setenv("PATH", f"{tmp_path}{os.pathsep}{os.environ.get('PATH', '')}")
    s = bench.ClockSampler(0)
    s.start()
    time.sleep(0.5)
    r = s.stop()
    assert r["samples"] == 3 and r["sm_mhz"] == 2032.0 and r["sm_max_mhz"] == 2032.0
    assert r["reasons"] == ["hw_slowdown", "sw_power_cap"]


def test_clock_rejection_rule():
    """A timed region is measured again when a hardware or thermal slowdown was active, or when the SM clock
    sat well below its maximum with no reason (a leftover clock lock); sw_power_cap alone is kept."""
    ok = {"sm_mhz": 2032.0, "sm_max_mhz": 2032.0, "reasons": []}
    assert not bench.clocks_rejected(ok)
    assert not bench.clocks_rejected(dict(ok, sm_mhz=1900.0, reasons=["sw_power_cap"]))
    for r in ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"):
        assert bench.clocks_rejected(dict(ok, reasons=[r]))
    assert bench.clocks_rejected(dict(ok, sm_mhz=1200.0))  # locked low, no reason given
    assert not bench.clocks_rejected({"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]})
