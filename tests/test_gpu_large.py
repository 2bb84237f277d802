"""Large, ill-conditioned grid evaluations against the dense oracle at sampled
grid points (Sec. III-A, III-D; App. B).

N = 8192, K = 128, L = 32768, |alpha| log-uniform over 30 dB at 15 and 30 dB
SNR, at the true state: kappa(C) <= 1 + N gamma_max / beta reaches ~1e7 here.
On the double-float path an instance this large runs its generator recursion
with the vectors in global memory, shared by a cluster of blocks, and the
grid (L above the on-chip FFT limit) on the global-memory grid kernel; the
FP64 path runs the FP64 recursion and the FP64 global-memory grid kernel.
The oracle evaluates the dense model (Cholesky of the 8192 x 8192 C) in a
subprocess that may use every host core.
Tolerances as for the smaller grids: 1e-4 normwise on every output (over the
sampled points) for both paths; s pointwise 1e-4 on the FP64 path.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_1705_06073_gb300 import synth
from tests.gpu_util import grid_errors

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
N, K, L = 8192, 128, 32768
FIELDS = ("q", "dq", "d2q", "s", "ds", "d2s")


@pytest.fixture(scope="module")
def dense_ref(tmp_path_factory):
    cache = {}

    def get(snr, seed):
        if (snr, seed) not in cache:
            out = str(tmp_path_factory.mktemp("dense") / f"n{N}_{int(snr)}.npz")
            env = dict(os.environ)
            nproc = str(os.cpu_count() or 1)
            env.update(OPENBLAS_NUM_THREADS=nproc, OMP_NUM_THREADS=nproc, MKL_NUM_THREADS=nproc,
                       CUDA_VISIBLE_DEVICES="")
            subprocess.run([sys.executable, "-m", "tests.dense_points", str(N), str(K), str(L), str(snr), str(seed),
                            out], cwd=ROOT, env=env, check=True, timeout=1500)
            with np.load(out) as z:
                cache[(snr, seed)] = {k: z[k] for k in z.files}
        return cache[(snr, seed)]
    return get


@pytest.mark.parametrize("snr,seed", [(15.0, 8801), (30.0, 8802)])
@pytest.mark.parametrize("pname", ["mixed_df", "fp64"])
def test_grid_n8192_l32768_sampled_vs_dense_oracle(dense_ref, pname, snr, seed):
    from paper_1705_06073_gb300 import build, lse
    build.build()
    ref = dense_ref(snr, seed)
    inst = synth.make_instance(N, K, snr, seed, law="loguniform30")
    gamma = np.abs(inst.alpha) ** 2
    f64 = pname == "fp64"
    prec = lse.LSE_PREC_FP64 if f64 else lse.LSE_PREC_MIXED_DF
    ctx = lse.lse_create(lse.lse_config_default(precision=prec))
    try:
        got = lse.lse_eval_grid(ctx, inst.y, inst.theta, gamma, inst.beta, L, f64=f64)
    finally:
        lse.lse_destroy(ctx)
    pts = ref["points"]
    sub = {f: got[f][pts] for f in FIELDS}
    err = grid_errors(sub, {f: ref[f] for f in FIELDS}, N)
    kappa = 1.0 + N * gamma.max() / inst.beta
    print(f"{pname} snr={snr} kappa<={kappa:.2e} errors={err}")
    assert max(err.values()) < 1e-4, err
    if f64:
        assert np.all(np.abs(sub["s"] - ref["s"]) <= 1e-4 * ref["s"])
