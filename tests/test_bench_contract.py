"""bench.py's output contract and its host-side helpers, on CPU.

The reference arm (`--impl reference`, the FP64 oracle on the host cores) runs
here on the smallest workload and must print one JSON line with the keys the
benchmark contract names; the helpers that pick the roofline kernel and read its
committed small-case profile are checked against the sources in the tree.
"""
import json
import subprocess
import sys
from pathlib import Path

ROOT = Path(__file__).resolve().parents[1]


def test_reference_arm_prints_one_contract_line():
    r = subprocess.run([sys.executable, str(ROOT / "bench.py"), "--impl", "reference", "--workload", "c1",
                        "--steps", "1", "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [x for x in r.stdout.splitlines() if x.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["higher_is_better"] is False and d["value"] > 0
    assert d["config"]["workload"].startswith("c1")
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_roofline_kernel_variant_and_profile():
    sys.path.insert(0, str(ROOT))
    import bench
    # the E' kernel instance of the largest tile list names the roofline line
    rep = [{"tiles": 990, "pipeline": 1}, {"tiles": 49141, "pipeline": 0}]
    assert bench.syrk_variant(rep) == "syrk_tc_kernel<64, 3>"
    assert bench.syrk_variant([{"tiles": 5, "pipeline": 1}]) == "syrk_tc_kernel<32, 6>"
    assert bench.syrk_variant([]) == "syrk_tc_kernel<64, 3>"
    # the committed small-case capture of that instance matches the kernel's current
    # source, so the bench line's traffic comes from it (scaled by the launch's flops)
    t, prof = bench.profile_traffic("syrk_tc_kernel<64, 3>", 1.0e12)
    assert prof is not None and 1e8 < t < 1e11
    assert bench.profile_traffic("syrk_tc_kernel<32, 6>", 1.0e12) == (None, None)
