"""bench.py's output contract, on the host: the reference arm (the FP64 oracle timed on the host
cores) prints one JSON line with the keys the measurement contract names, and the bench modes
parse.  The GPU arms print the same kind of line; they need a GB300 and are run there."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    # one integration of a 10-integration W-projection track: 351 x 64 x 4 visibilities
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0",
                          "--n-int", "10", "--cpu-sample-every", "10"],
                         cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    rec = json.loads(lines[0])
    assert rec["impl"] == "reference"
    assert rec["metric"] == "gridded+degridded visibilities/s" and rec["unit"] == "visibilities/s"
    assert rec["higher_is_better"] is True and rec["value"] > 0 and rec["steps"] == 1
    cb = rec["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == rec["value"]
    assert "351 rows x 64 channels x 4 pols" in cb["sample"]
    e2e = rec["e2e"]
    assert e2e["value"] == rec["value"] and e2e["unit"] == rec["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


@pytest.mark.parametrize("argv,flag", [(["--forward-model"], "forward_model"), (["--calibrate"], "calibrate"),
                                       (["--minor-cycle"], "minor_cycle"), (["--mosaic"], "mosaic")])
def test_bench_modes_parse(monkeypatch, argv, flag):
    import bench
    monkeypatch.setattr(sys, "argv", ["bench.py", *argv])
    args = bench.parse()
    assert getattr(args, flag) is True
    assert (args.gpus, args.steps, args.warmup, args.impl) == (1, 5, 3, "ours")
