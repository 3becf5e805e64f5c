"""The bench's reference arm, byte model and packed batch layout, on the host (no GPU).

The reference arm times the FP64 oracle itself and must print one JSON line with the
fields of the bench contract; the algorithmic bytes of a contraction launch follow
from the layout of the split operands (every part read once, written once)."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_the_contract_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--workload", "ac2d_n64_expeuler", "--steps", "2", "--warmup", "1"],
                         capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert out.returncode == 0, out.stderr
    line = json.loads(out.stdout.strip().splitlines()[-1])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["value"] > 0 and line["higher_is_better"] is True
    assert line["config"]["workload"] == "ac2d_n64_expeuler"
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]


def test_contraction_byte_model():
    sys.path.insert(0, ROOT)
    import bench
    from paper_2304_02327_gb300 import workloads as wl
    p = wl.workload("adr3d_n320_etd2rk")
    N = p.N
    # BF16x3: three 2-byte parts in and out per element for modes 1-2, FP32 out for
    # mode 3, plus the phi parts (3 x 2 x 320^2 bytes); averaged over the six launches
    phi = 3 * 2 * 320 * 320
    expect = (4 * (6 * N + phi + 6 * N) + 2 * (6 * N + phi + 4 * N)) / 6
    assert bench.mixed_bytes_per_launch(p, "bf16x3") == pytest.approx(expect)
    # TF32x3: two 4-byte parts
    phi4 = 3 * 4 * 320 * 320
    expect4 = (4 * (8 * N + phi4 + 8 * N) + 2 * (8 * N + phi4 + 4 * N)) / 6
    assert bench.mixed_bytes_per_launch(p, "tf32x3") == pytest.approx(expect4)


def test_flat_offsets_pack_states_on_16_byte_boundaries():
    """The packed state layout of a batch: each state starts on a 16-byte boundary
    (an even number of doubles), states do not overlap, the total covers them all."""
    from paper_2304_02327_gb300 import api, workloads as wl
    probs = wl.batched_allen_cahn(count=7, seed=3, steps=1, sizes=(48, 64, 96))
    rng = np.random.default_rng(1)
    A1, A2 = wl.fd_matrix(5, 0.02), wl.fd_matrix(3, 0.02)
    probs.append(wl.Problem(name="odd", A=[A1, A2], u0=rng.uniform(-1, 1, (3, 5)), tau=1e-3))
    offs, total = api.flat_offsets(probs)
    assert all(o % 2 == 0 for o in offs)
    ends = [o + p.u0.size for o, p in zip(offs, probs)]
    assert all(e <= o2 for e, o2 in zip(ends, offs[1:]))
    assert ends[-1] <= total and total - ends[-1] <= 1
