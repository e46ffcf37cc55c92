"""bench.py's brute-force mode on a reduced workload: one JSON line with the
contract's keys, the tensor-core path taken, and a tensor roofline whose
achieved rate is below the measured peak."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a GPU", allow_module_level=True)

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.parametrize("rows", [0, 500])
def test_bruteforce_bench_line(rows):
    r = subprocess.run([sys.executable, "bench.py", "--bruteforce", "--workload", "mixture_n1m_d128",
                        "--n", "20000", "--rows", str(rows), "--steps", "2", "--warmup", "3", "--no-cpu"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "config", "e2e", "gpu_launches", "roofline", "clocks"):
        assert key in line, key
    assert line["config"]["path"] == "tensor cores"
    assert line["config"]["queries"] == (rows or 20000)
    roof = line["roofline"]
    assert roof["bound"] == "tensor" and 0 < roof["frac"] < 1.2
    assert 0 < roof["share_of_call"] <= 1
    assert line["e2e"]["h2d_bytes_per_step"] >= 20000 * 128 * 4
    assert line["gpu_launches"] >= 7 * 2


def test_l2_read_rate_is_measured():
    """The L2 read rate the roofline of L2-resident kernels is reported
    against: positive, and a small buffer read many times is served from L2,
    above the HBM copy rate."""
    import json as _json
    import paper_2112_06630_gb300 as knng
    g = knng.measure_l2_read(32 << 20, 100)
    assert g > 0
    peaks = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(peaks):
        assert g > _json.load(open(peaks))["hbm_gbs"]
    with pytest.raises(knng.KnngError):
        knng.measure_l2_read(1024, 10)
