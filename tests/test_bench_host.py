"""Host-side parts of bench.py that need no GPU: the oracle leg (the
reference arm and cpu_baseline) on a small sample, with and without the
NEXT-4 solver variants, and the JSON line of the reference arm."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


@pytest.fixture
def bench():
    import bench as b
    saved = dict(b.VARIANT)
    yield b
    b.VARIANT.clear()
    b.VARIANT.update(saved)


@pytest.mark.parametrize("variant", [{}, {"jacobian": 1}, {"cf": True}])
def test_oracle_sample_runs_the_variants(bench, variant):
    bench.VARIANT.clear()
    bench.VARIANT.update(variant)
    w = bench.WORKLOADS["2d-40x40"]
    v, dt, st, sample = bench.oracle_sample(w, 0, sub=(20, 20, 1))
    assert st.converged and v > 0 and dt > 0
    assert sample.startswith("20x20x1 corner box")


def test_reference_arm_line(bench):
    class Args:
        seed, steps, warmup = 0, 1, 0
    bench.VARIANT.clear()
    bench.VARIANT["jacobian"] = 1
    w = bench.WORKLOADS["2d-40x40"]
    out = bench.run_reference(Args, w, 0, 1)
    assert out["impl"] == "reference" and out["unit"] == bench.UNIT
    assert out["config"]["workload"].endswith("full-Jacobian Newton")
    assert out["e2e"]["h2d_bytes_per_step"] == 0 and out["cpu_baseline"]["kind"] == "oracle"
    assert bench.run_reference(Args, w, 1, 2) is None          # only rank 0 runs it


def test_class_rooflines(bench):
    """Per-class achieved bandwidth: algorithmic bytes of one launch group
    over its average time, against the peak; classes without a byte count
    or without launches are left out."""
    prof = {"residual": (10, 5.0, 20), "ilu_fwd": (50, 40.0, 50), "coarse_solve": (45, 17.0, 45),
            "restrict": (0, 0.0, 0)}
    out = bench.class_rooflines(prof, 4_000_000, 0, 6800.0)
    assert set(out) == {"residual", "ilu_fwd"}
    r = out["residual"]
    assert r["launches"] == 10 and abs(r["avg_ms"] - 0.5) < 1e-12
    assert abs(r["gbs"] - 56 * 4e6 / 0.5e-3 / 1e9) < 1e-9 and abs(r["frac"] - r["gbs"] / 6800.0) < 1e-12
    mixed = bench.class_rooflines(prof, 4_000_000, 1, 6800.0)
    assert mixed["ilu_fwd"]["gbs"] < out["ilu_fwd"]["gbs"]        # 4-byte operands in mixed precision


def test_restriction_override_reaches_the_oracle_leg(bench):
    class Args:
        seed, steps, warmup = 0, 1, 0
    bench.VARIANT.clear()
    w = bench.WORKLOADS["2d-40x40"].with_(restriction=2)
    out = bench.run_reference(Args, w, 0, 1)
    assert out["config"]["restriction"] == "MSFE+closing MSFV"


def test_measured_traffic_matches_the_launch_list_profile(bench):
    """The DRAM traffic the bench line reports for the mixed 4M-cell
    smoother classes is the committed launch list's read + write per launch
    (profiles/launch_list_3d-200x200x100-mixed.md), to the 0.1 MB the table
    prints."""
    import re
    path = os.path.join(ROOT, "profiles", "launch_list_3d-200x200x100-mixed.md")
    rows = {}
    for line in open(path):
        m = re.match(r"\| (k_\S+(?:\\<[^|]*)?) \| (\d+) \| [\d.]+ \| [\d.]+% \| ([\d.]+) MB \| ([\d.]+) MB \|", line)
        if m:
            rows[m.group(1).replace("\\<", "<").strip()] = float(m.group(3)) + float(m.group(4))
    kernels = {"ilu_fwd": "k_sweep_warp<FwdSolve<float>, 0>",
               "ilu_bwd": "k_sweep_warp<BwdSolve<float>, 1>",
               "ilu_resid": "k_resid_scaled<float, float, 0>",
               "ilu_apply": "k_apply_z<float>"}
    for cls, kern in kernels.items():
        assert kern in rows, kern
        got = bench.MEASURED_TRAFFIC[("3d-200x200x100-mixed", cls)] / 1e6
        assert abs(got - rows[kern]) <= 0.15, (cls, got, rows[kern])
