"""bench.py's JSON contract, on the CPU through its reference arm.

The reference arm times the FP64 oracle on a bounded sample of the workload
on the host cores; it must print one JSON line with the keys the benchmark
contract names (and exit 0 without output on ranks other than 0).
"""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(env_extra=None):
    env = dict(os.environ, **(env_extra or {}))
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--config", "c1", "--steps", "1", "--warmup", "0"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    return [l for l in p.stdout.splitlines() if l.startswith("{")]


def test_reference_line_has_the_contract_keys():
    lines = _run()
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "impl",
              "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["higher_is_better"] is False
    assert d["steps"] == 1 and d["warmup"] == 0 and d["value"] > 0
    assert d["config"]["workload"].startswith("c1")
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_reference_arm_is_silent_off_rank_zero():
    assert _run({"RANK": "1", "WORLD_SIZE": "2"}) == []


class _Done:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def test_clock_record_median_max_and_reasons(tmp_path):
    # nvidia-smi's CSV (noheader, nounits) in the order of ClockSampler.FIELDS:
    # the record keeps the median SM clock under load, the largest maximum, and
    # every throttle reason seen active in any sample.
    sys.path.insert(0, ROOT)
    import bench
    rows = ["0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
            "0, 1980, 2070, 1390.5, 0x4, Not Active, Not Active, Not Active, Active",
            "0, 2055, 2070, 1200.0, 0x0, Not Active, Not Active, Not Active, Not Active",
            "garbage line",
            "0, N/A, 2070, 1.0, 0x0, Not Active, Not Active, Not Active, Not Active"]
    path = tmp_path / "clocks.csv"
    path.write_text("\n".join(rows) + "\n")
    cs = bench.ClockSampler(0)
    cs.path, cs.proc = str(path), _Done()
    rec = cs.stop()
    assert rec["sm_mhz"] == 2055.0 and rec["sm_max_mhz"] == 2070.0 and rec["samples"] == 3
    assert rec["reasons"] == ["sw_power_cap"]
    assert not path.exists()
