"""The benchmark's contract pieces that run without a GPU: the reference arm
(the FP64 oracle on the host cores) prints one JSON line with every key the
contract names, and the roofline numerators are the per-kernel algorithmic
figures of the workload."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_2409_02912_b300 import synth  # noqa: E402


def test_reference_arm_prints_the_contract_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "1"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC and line["unit"] == "REs/s"
    assert line["n_gpus"] == 1 and line["steps"] == 1 and line["warmup"] == 1
    assert line["value"] > 0 and line["higher_is_better"] is True and line["vs_baseline"] is None
    assert line["config"]["workload"] == bench.WORKLOAD and line["data"] == "synthetic"
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
    # one 273-PRB slot per step: REs/s = REs per slot / seconds per step
    res = synth.NUM_SYMBOLS * 12 * 273
    assert abs(line["value"] - res / (line["ms_per_step"] * 1e-3)) <= 1e-6 * line["value"]


def test_roofline_numerators_of_the_workload():
    """Algorithmic FLOPs per RE-user and DRAM bytes per launch (C=64, B=4, R=2,
    m_max=6; 8 slots x 4 users x 14 x 3276 REs, 16-bit activations)."""
    w = synth.WORKLOADS[bench.WORKLOAD]
    f = bench.nrx_flops_per_re_ue(w.net)
    C = 64
    assert f["residual_block"] == 2 * (2 * 9 * C + 2 * C * C) == 18688
    assert f["message_passing"] == 2 * (2 * C * C + (2 * C + 2) * C)
    assert f["state_init"] == 2 * (18 * C + 9 * C)
    act = 8 * 4 * 14 * 3276 * C * 2  # one 16-bit activation tensor, 188 MB
    bits = [[6, 6, 6, 6]] * 8
    b = bench.kernel_bytes_per_launch(w, 8, bits, 2)
    assert act == 187_858_944
    assert b["residual_block"] == (2 * (2 - 1) + 3) * act / 2  # non-last: z in, z out; last: + state
    assert b["message_passing"] == 2 * act


def test_traffic_record_matches_the_kernel_source():
    """The committed DRAM traffic of the dominant kernel is keyed to the hash of its
    source and the CUDA headers; the bench reports null once they change, so a
    kernel edit without a new capture (or a stated re-keying) fails here first."""
    for prec in ("bf16", "fp16"):
        t = bench.traffic_for("residual_block", prec)
        assert t is not None, prec
        # between 50% and 150% of the algorithmic bytes of one launch (2.5 tensors of 188 MB)
        assert 0.5 * 2.5 * 187_858_944 < t < 1.5 * 2.5 * 187_858_944
