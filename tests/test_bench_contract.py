"""bench.py's JSON line contract, checked on the CPU through the reference
arm (the FP64 oracle timed on the host): one line with the contract's keys
and types, the reference marker, a CPU baseline describing the run and an
end-to-end entry with no copies."""

import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
KEYS = {"metric": str, "value": float, "unit": str, "n_gpus": int, "steps": int,
        "warmup": int, "ms_per_step": float, "higher_is_better": bool, "scaling": str,
        "dtype": str, "data": str, "config": dict, "impl": str, "cpu_baseline": dict,
        "e2e": dict}


@pytest.mark.parametrize("workload", ["kinect", "swap"])
def test_reference_arm_prints_one_contract_line(workload):
    env = dict(os.environ)
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        env.pop(k, None)
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", workload,
                        "--steps", "1", "--warmup", "0", "--frames", "3", "--cpu-seconds", "2"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    out = json.loads(lines[0])
    for k, t in KEYS.items():
        assert k in out, k
        assert isinstance(out[k], t) or (t is float and isinstance(out[k], int)), (k, out[k])
    assert out["impl"] == "reference" and out["value"] > 0 and out["higher_is_better"]
    assert "vs_baseline" in out and out["vs_baseline"] is None
    assert out["cpu_baseline"]["kind"] == "oracle" and out["cpu_baseline"]["cores"] >= 1
    assert out["cpu_baseline"]["value"] == out["value"]
    assert out["e2e"]["h2d_bytes_per_step"] == 0 and out["e2e"]["d2h_bytes_per_step"] == 0
    assert "workload" in out["config"]
