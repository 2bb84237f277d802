"""Full-size checks, in the launch configuration bench.py times.

- The 64 x N=4096 batch of the benchmark is fitted in one launch; instance 0
  is compared with a complete dense-oracle fit (about a minute of CPU).
- The grid of every instance of that batch at its true state is evaluated in
  one batched launch; sampled grid points are compared with the dense oracle.
- The maximum size, N = 65536 with L = 2N, is checked against the closed form
  of a single sinusoid (Sherman-Morrison: C^{-1} = (I - g a a^H/(b + g N))/b),
  exact at any size; the reference uses numpy's FFT for the sums over n.
"""
import os

import numpy as np
import pytest

from oracle import dense as dn
from paper_1705_06073_gb300 import synth
from tests.gpu_util import grid_errors, wrapdist

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def lse_mod():
    from paper_1705_06073_gb300 import build, lse
    build.build()
    return lse


def _oracle_fit_subprocess(y, L):
    """The dense oracle's fit in a child process with every host core for BLAS
    (this test process keeps one BLAS thread); returns (theta, gamma, beta, K,
    n_evals)."""
    import json
    import subprocess
    import sys
    import tempfile
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    with tempfile.TemporaryDirectory() as td:
        np.save(os.path.join(td, "y.npy"), y)
        code = ("import sys, json, numpy as np; sys.path.insert(0, %r); from oracle import fit as f; "
                "r = f.fit(np.load(%r), %d); "
                "print(json.dumps(dict(theta=r.theta.tolist(), gamma=r.gamma.tolist(), beta=r.beta, K=r.K, "
                "n_evals=r.n_evals)))") % (root, os.path.join(td, "y.npy"), L)
        env = dict(os.environ, OPENBLAS_NUM_THREADS=str(os.cpu_count() or 1), CUDA_VISIBLE_DEVICES="")
        out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=1200)
        assert out.returncode == 0, out.stderr[-2000:]
        return json.loads(out.stdout.strip().splitlines()[-1])


@pytest.fixture(scope="module")
def oracle_fit0(batch):
    insts, ys, offs = batch
    return _oracle_fit_subprocess(ys[0], 16384)


@pytest.fixture(scope="module")
def batch():
    insts = synth.batch64_n4096()
    ys = [i.y for i, _ in insts]
    offs = np.concatenate([[0], np.cumsum([len(y) for y in ys])]).astype(np.int64)
    return insts, ys, offs


@pytest.mark.parametrize("prec", ["mixed_df", "fp64"])
def test_bench_batch_fit_matches_oracle_on_instance0(lse_mod, batch, oracle_fit0, prec):
    import torch
    lse = lse_mod
    insts, ys, offs = batch
    P = {"mixed_df": lse.LSE_PREC_MIXED_DF, "fp64": lse.LSE_PREC_FP64}[prec]
    ctx = lse.lse_create(lse.lse_config_default(precision=P, grid_size=16384))
    try:
        out = lse.alloc_batch_out(offs)
        lse.lse_fit_batch_d(ctx, torch.from_numpy(np.concatenate(ys)).cuda(), offs, out)
        torch.cuda.synchronize()
    finally:
        lse.lse_destroy(ctx)
    assert int(out["status"].abs().sum()) == 0
    K = int(out["K"][0])
    th = out["theta"][:K].cpu().numpy()
    ga = out["gamma"][:K].cpu().numpy()
    ref = oracle_fit0
    assert K == ref["K"]
    assert np.all(wrapdist(th, np.array(ref["theta"])) < 1e-6)
    assert np.allclose(ga, ref["gamma"], rtol=1e-6)
    assert abs(float(out["beta"][0]) - ref["beta"]) <= 1e-6 * ref["beta"]
    assert int(out["n_evals"][0]) == ref["n_evals"]


@pytest.mark.parametrize("prec", ["mixed_df", "fp64"])
def test_bench_batch_grid_sampled_points(lse_mod, batch, prec):
    import torch
    lse = lse_mod
    insts, ys, offs = batch
    f64 = prec == "fp64"
    P = {"mixed_df": lse.LSE_PREC_MIXED_DF, "fp64": lse.LSE_PREC_FP64}[prec]
    B, L = len(ys), 16384
    th = [i.theta for i, _ in insts]
    ga = [np.abs(i.alpha) ** 2 for i, _ in insts]
    be = [i.beta for i, _ in insts]
    ko = np.concatenate([[0], np.cumsum([len(t) for t in th])]).astype(np.int64)
    dev = torch.device("cuda")
    ct = torch.complex128 if f64 else torch.complex64
    rt = torch.float64 if f64 else torch.float32
    outs = {f: torch.zeros(B * L, dtype=ct if f in ("q", "dq", "d2q") else rt, device=dev)
            for f in ("q", "dq", "d2q", "s", "ds", "d2s")}
    ctx = lse.lse_create(lse.lse_config_default(precision=P))
    try:
        lse.lse_eval_grid_batch_d(ctx, torch.from_numpy(np.concatenate(ys)).to(dev), offs,
                                  torch.from_numpy(np.concatenate(th)).to(dev), torch.from_numpy(np.concatenate(ga)).to(dev),
                                  ko, torch.tensor(be, dtype=torch.float64, device=dev), np.full(B, L, np.int32), outs, f64)
        torch.cuda.synchronize()
    finally:
        lse.lse_destroy(ctx)
    rng = np.random.default_rng(5)
    for b in (0, 37, 63):
        pts = np.sort(rng.choice(L, 48, replace=False))
        ev = dn.DenseEval(ys[b], th[b], ga[b], be[b])
        ref = ev.grid(L, derivatives=True, points=pts / L)
        got = {f: outs[f][b * L:(b + 1) * L].cpu().numpy()[pts] for f in outs}
        # normwise over the sample, relative to the full-grid scale of each output
        err = grid_errors(got, ref, len(ys[b]))
        assert max(err.values()) < (1e-8 if f64 else 1e-4), (b, err)


@pytest.mark.parametrize("prec", ["mixed_df", "fp64"])
def test_max_size_grid_single_sinusoid_closed_form(lse_mod, prec):
    lse = lse_mod
    N, L = 65536, 131072
    f64 = prec == "fp64"
    P = {"mixed_df": lse.LSE_PREC_MIXED_DF, "fp64": lse.LSE_PREC_FP64}[prec]
    inst = synth.make_instance(N, 1, 15.0, 301)
    th1, g, b = float(inst.theta[0]), float(abs(inst.alpha[0]) ** 2), inst.beta
    ctx = lse.lse_create(lse.lse_config_default(precision=P))
    try:
        got = lse.lse_eval_grid(ctx, inst.y, [th1], [g], b, L, f64=f64)
    finally:
        lse.lse_destroy(ctx)
    n = np.arange(N)
    y = inst.y.astype(np.complex128)
    a1 = dn.unit_phase(n, np.array([th1]))[:, 0]
    w = 2 * np.pi * n
    # D_k(theta) = sum_n (-j w_n)^k a1_n e^{-j 2 pi n theta}: derivatives of a(theta)^H a1
    D0 = np.fft.fft(a1, L)
    D1 = np.fft.fft(-1j * w * a1, L)
    D2 = np.fft.fft(-(w ** 2) * a1, L)
    Y0 = np.fft.fft(y, L)
    Y1 = np.fft.fft(-1j * w * y, L)
    Y2 = np.fft.fft(-(w ** 2) * y, L)
    den = b + g * N
    a1y = np.vdot(a1, y)
    c = g / (b * den)
    ref = {
        "s": (N - g * np.abs(D0) ** 2 / den) / b,
        "ds": -c * 2 * np.real(np.conj(D0) * D1),
        "d2s": -c * 2 * (np.abs(D1) ** 2 + np.real(np.conj(D0) * D2)),
        "q": (Y0 - g * D0 * a1y / den) / b,
        "dq": (Y1 - g * D1 * a1y / den) / b,
        "d2q": (Y2 - g * D2 * a1y / den) / b,
    }
    err = grid_errors(got, ref, N)
    assert max(err.values()) < (1e-8 if f64 else 1e-4), err


def test_big_cluster_factorisation_matches_one_block(lse_mod):
    """Double-float eval-grid at N = 65536 with the Levinson recursion
    (LSE_FLAG_LEVINSON; too large for shared memory, a single instance runs it
    on a cluster of eight blocks through global memory) against the same
    evaluation with one block (LSE_FLAG_NO_CLUSTER), and against the default
    superfast recursion: the grids agree to the FP32 output precision."""
    lse = lse_mod
    inst = synth.single_n65536()[0][0]
    N, L = inst.N, 2 * inst.N
    th = inst.theta
    ga = np.abs(inst.alpha) ** 2
    got = {}
    lev = lse.LSE_FLAG_LEVINSON
    for flags in (lev, lev | lse.LSE_FLAG_NO_CLUSTER, 0):
        ctx = lse.lse_create(lse.lse_config_default(precision=lse.LSE_PREC_MIXED_DF, flags=flags))
        try:
            got[flags] = lse.lse_eval_grid(ctx, inst.y, th, ga, inst.beta, L, f64=False)
        finally:
            lse.lse_destroy(ctx)
    err = grid_errors(got[lev], got[lev | lse.LSE_FLAG_NO_CLUSTER], N)
    assert max(err.values()) < 1e-5, err
    err = grid_errors(got[0], got[lev | lse.LSE_FLAG_NO_CLUSTER], N)
    assert max(err.values()) < 1e-5, err
