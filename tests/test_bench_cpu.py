"""bench.py pieces that need no GPU: the reference arm's JSON line (the
oracle timed on the host, a bounded sample) and the roofline bookkeeping."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_the_contract_line():
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0"], env=env, capture_output=True, text=True, timeout=900, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "config",
              "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["value"] > 0 and line["higher_is_better"] is True
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["value"] == line["value"] and line["e2e"]["h2d_bytes_per_step"] == 0
    assert line["config"]["workload"] == "batch64_n4096_k64_l16384"


def test_roofline_bookkeeping():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.levinson_flops(100) == 8.0 * 100 * 100
    assert bench.fft_flops(1024) == 5.0 * 1024 * 10
    assert bench.pow2_at_least(1000) == 1024 and bench.pow2_at_least(1024) == 1024
    # a leaf-sized factorisation: one leaf of n - 1 <= 32 orders plus the refinement FFTs
    assert bench.schur_flops(33) == 8.0 * 4 * 32 * 32 + 9 * bench.fft_flops(128)
    # the superfast count grows like n log^2 n: far below the Levinson count at large n
    assert bench.schur_flops(65536) < 0.05 * bench.levinson_flops(65536)
    assert bench.schur_flops(1 << 14) / bench.schur_flops(1 << 13) < 2.5
    # direct sums below 32 frequencies, the non-uniform FFT from 32 on
    n = 4096
    assert bench.eval_flops(n, 31) - bench.eval_flops(n, 0) == 8.0 * n * 31 + 7 * 8.0 * n * 31
    # the traffic figure is reported only for the sources it was measured on
    assert len(bench.sources_digest()) == 64
    d = bench.sources_digest(bench.FIT_SOURCES)
    t = bench.fit_traffic(64)
    if bench.FIT_TRAFFIC["sources_sha256"] == d:
        assert t == 64 * bench.FIT_TRAFFIC["bytes_per_instance"]
    else:
        assert t is None
