"""Batched fits of uneven N: one persistent launch, a plan, and its CUDA graph.

Every instance is fitted by one thread block with the arithmetic of a lone
fit, so the batched, planned and graph-replayed results must equal the
single-instance ones exactly, and each must match the oracle's fit.
"""
import numpy as np
import pytest

from oracle import fit as ofit
from paper_1705_06073_gb300 import synth
from tests.gpu_util import wrapdist

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lse_mod():
    from paper_1705_06073_gb300 import build, lse
    build.build()
    return lse


def ragged(n=12, seed0=9100):
    """Uneven N (non-powers of two included), K = max(1, N // 64), SNR in [0, 30] dB:
    the ragged-batch workload at sizes the oracle finishes quickly."""
    rs = synth.Stream(seed0)
    insts = []
    for i in range(n):
        u = rs.uniform(2)
        N = 40 + int(u[0] * 400)
        insts.append(synth.make_instance(N, max(1, N // 64), 30.0 * float(u[1]), seed0 + i))
    return insts


def as_np(out):
    return {k: v.cpu().numpy() for k, v in out.items()}


@pytest.mark.parametrize("prec", ["mixed_df", "fp64"])
def test_plan_and_graph_equal_direct_and_single(lse_mod, prec):
    import torch
    lse = lse_mod
    P = {"mixed_df": lse.LSE_PREC_MIXED_DF, "fp64": lse.LSE_PREC_FP64}[prec]
    insts = ragged()
    ys = [i.y for i in insts]
    offs = np.concatenate([[0], np.cumsum([len(y) for y in ys])]).astype(np.int64)
    y_d = torch.from_numpy(np.concatenate(ys)).cuda()
    ctx = lse.lse_create(lse.lse_config_default(precision=P))
    try:
        direct = lse.alloc_batch_out(offs)
        lse.lse_fit_batch_d(ctx, y_d, offs, direct)
        plan = lse.lse_plan_fit(ctx, offs)
        try:
            planned = lse.alloc_batch_out(offs)
            lse.lse_plan_launch(plan, y_d, planned)
            graphed = lse.alloc_batch_out(offs)
            for _ in range(3):  # capture once, replay
                graphed["K"].zero_()
                lse.lse_plan_launch(plan, y_d, graphed, graph=True)
            torch.cuda.synchronize()
        finally:
            lse.lse_plan_destroy(plan)
        singles = [lse.lse_fit(ctx, y) for y in ys]
    finally:
        lse.lse_destroy(ctx)
    d, p, g = as_np(direct), as_np(planned), as_np(graphed)
    for k in ("K", "beta", "objective", "iters", "n_evals", "status"):
        assert np.array_equal(d[k], p[k]) and np.array_equal(d[k], g[k]), k
    for k in ("theta", "gamma", "alpha"):
        assert np.array_equal(d[k], p[k]) and np.array_equal(d[k], g[k]), k
    for b, (y, s) in enumerate(zip(ys, singles)):
        K = int(d["K"][b])
        assert K == s["K"]
        assert np.array_equal(d["theta"][offs[b]:offs[b] + K], s["theta"])
        assert d["beta"][b] == s["beta"]
    # and against the oracle (a few instances)
    for b in (0, 5, 11):
        ref = ofit.fit(ys[b], synth.default_grid_size(len(ys[b])))
        K = int(d["K"][b])
        assert K == ref.K
        assert np.all(wrapdist(d["theta"][offs[b]:offs[b] + K], ref.theta) < 1e-6)


def test_fit_batch_d_captured_in_cuda_graph(lse_mod):
    """lse_fit_batch_d captured in a CUDA graph after one uncaptured call with
    the same offsets replays to the direct call's results exactly."""
    import torch
    lse = lse_mod
    insts = ragged(n=6, seed0=9400)
    ys = [i.y for i in insts]
    offs = np.concatenate([[0], np.cumsum([len(y) for y in ys])]).astype(np.int64)
    y_d = torch.from_numpy(np.concatenate(ys)).cuda()
    ctx = lse.lse_create(lse.lse_config_default(precision=lse.LSE_PREC_MIXED_DF))
    try:
        st = torch.cuda.Stream()
        st.wait_stream(torch.cuda.current_stream())
        direct = lse.alloc_batch_out(offs)
        lse.lse_fit_batch_d(ctx, y_d, offs, direct, st)
        st.synchronize()
        graphed = lse.alloc_batch_out(offs)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=st, capture_error_mode="thread_local"):
            lse.lse_fit_batch_d(ctx, y_d, offs, graphed, st)
        for _ in range(2):
            for v in graphed.values():
                v.zero_()
            g.replay()
            torch.cuda.synchronize()
            for k in direct:
                assert torch.equal(graphed[k], direct[k]), k
    finally:
        lse.lse_destroy(ctx)
