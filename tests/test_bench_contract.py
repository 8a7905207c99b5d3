"""The benchmark's JSON contract, checked on the CPU through its reference arm
(the oracle timed on the host cores): one JSON line with the keys and types the
benchmark promises, and nothing from the non-zero ranks of a multi-process
launch."""
import json
import os
import subprocess
import sys

from tests.conftest import ROOT

BENCH = os.path.join(ROOT, "bench.py")


def _run(extra_env=None, *args):
    env = dict(os.environ)
    env.update(extra_env or {})
    r = subprocess.run([sys.executable, BENCH, "--impl", "reference", "--workload", "small512", "--steps", "2",
                        "--warmup", "1", "--cpu-budget", "1.5", *args],
                       capture_output=True, text=True, env=env, cwd=ROOT, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    return [line for line in r.stdout.splitlines() if line.startswith("{")]


def test_reference_arm_prints_one_contract_line():
    lines = _run()
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key, typ in [("impl", str), ("metric", str), ("value", float), ("unit", str), ("n_gpus", int),
                     ("steps", int), ("warmup", int), ("ms_per_step", float), ("higher_is_better", bool),
                     ("scaling", str), ("dtype", str), ("data", str), ("config", dict), ("cpu_baseline", dict),
                     ("e2e", dict)]:
        assert isinstance(d[key], typ), key
    assert d["impl"] == "reference" and d["steps"] == 2 and d["warmup"] == 1 and d["n_gpus"] == 1
    assert d["higher_is_better"] is False and d["unit"] == "s/matrix" and d["vs_baseline"] is None
    assert d["value"] > 0 and abs(d["ms_per_step"] - 1e3 * d["value"]) <= 1e-9 * d["ms_per_step"]
    assert "workload" in d["config"] and "512x256" in d["config"]["workload"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert cb["measured_s"] > 0 and cb["measured_psteps"] >= 1
    assert d["e2e"] == {"value": d["value"], "unit": "s/matrix", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_is_silent_on_other_ranks():
    assert _run({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"}) == []


def test_clock_sampler_parses_nvidia_smi_lines():
    """The clocks record of the benchmark line: median SM clock under load, the
    maximum, and the throttle reasons seen in any sample."""
    sys.path.insert(0, ROOT)
    import bench

    class FakeProc:
        def terminate(self):
            pass

        def communicate(self, timeout=None):
            lines = ["2070, 2070, 900.5, 0x0, Not Active, Not Active, Not Active, Not Active",
                     "2055, 2070, 1300.0, 0x4, Not Active, Not Active, Not Active, Active",
                     "2070, 2070, 1250.0, 0x0, Not Active, Not Active, Not Active, Not Active",
                     "[N/A], 2070, 10.0, 0x0, Not Active, Not Active, Not Active, Not Active",
                     "garbage"]
            return "\n".join(lines), ""

    cs = bench.ClockSampler(0)
    cs.proc = FakeProc()
    rec = cs.stop()
    assert rec == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    cs2 = bench.ClockSampler(0)
    assert cs2.stop() is None                                   # no sampler ran
