"""Multiple-measurement-vector fits (Sec. V) on the GPU through the C ABI
against the oracle (oracle/mmv.py).

Bar (the same as the single-snapshot fits): equal K, every frequency within
1e-6 cycles of the oracle's, gamma, alpha, beta and the objective within 1e-6
relative.  G = 1 must reproduce lse_fit bit for bit, and a ragged batch the
single fits of its instances.
"""
import numpy as np
import pytest

from oracle import dense as dn
from oracle import mmv as omv
from paper_1705_06073_gb300 import synth
from tests.gpu_util import wrapdist

pytestmark = pytest.mark.gpu

PRECS = ["fp64", "mixed", "mixed_df"]


@pytest.fixture(scope="module")
def lse_mod():
    from paper_1705_06073_gb300 import build, lse
    build.build()
    return lse


def prec_of(lse, name):
    return {"fp64": lse.LSE_PREC_FP64, "mixed": lse.LSE_PREC_MIXED, "mixed_df": lse.LSE_PREC_MIXED_DF}[name]


def check(gpu, ref, tol=1e-6):
    assert gpu["K"] == ref.K, (gpu["K"], ref.K)
    if ref.K:
        assert wrapdist(gpu["theta"], ref.theta).max() < tol
        assert np.allclose(gpu["gamma"], ref.gamma, rtol=tol)
        assert np.allclose(gpu["alpha"], ref.alpha, rtol=tol, atol=tol * np.abs(ref.alpha).max())
    assert abs(gpu["beta"] - ref.beta) <= tol * ref.beta
    assert abs(gpu["objective"] - ref.objective) <= tol * max(1.0, abs(ref.objective))


@pytest.mark.parametrize("prec", PRECS)
def test_one_snapshot_is_the_single_fit_bit_for_bit(lse_mod, prec):
    inst = synth.make_instance(200, 6, 15.0, 8101)
    ctx = lse_mod.lse_create(lse_mod.lse_config_default(precision=prec_of(lse_mod, prec)))
    try:
        a = lse_mod.lse_fit(ctx, inst.y)
        b = lse_mod.lse_fit_mmv(ctx, inst.y[None, :])
    finally:
        lse_mod.lse_destroy(ctx)
    assert a["K"] == b["K"] and a["n_evals"] == b["n_evals"] and a["iters"] == b["iters"]
    assert np.array_equal(a["theta"], b["theta"]) and np.array_equal(a["gamma"], b["gamma"])
    assert np.array_equal(a["alpha"], b["alpha"][:, 0])
    assert a["beta"] == b["beta"] and a["objective"] == b["objective"]


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("N,K,G,snr,seed", [(64, 3, 3, 20.0, 1), (96, 4, 4, 10.0, 2), (128, 8, 2, 15.0, 3),
                                            (45, 2, 5, 5.0, 4), (256, 8, 8, 12.0, 5)])
def test_fit_against_oracle(lse_mod, N, K, G, snr, seed, prec):
    inst = synth.make_mmv_instance(N, K, G, snr, 8200 + seed)
    L = synth.default_grid_size(N)
    ctx = lse_mod.lse_create(lse_mod.lse_config_default(precision=prec_of(lse_mod, prec)))
    try:
        gpu = lse_mod.lse_fit_mmv(ctx, inst.Y)
    finally:
        lse_mod.lse_destroy(ctx)
    ref = omv.fit(inst.Y.T, L)
    check(gpu, ref)
    assert gpu["n_evals"] == ref.n_evals and gpu["n_grid"] == ref.n_grid_evals


def test_close_components_resolved_with_snapshots(lse_mod):
    """Two components 0.6/N apart at 10 dB: the G = 16 fit on the GPU
    resolves both, as the oracle does."""
    N, G = 64, 16
    inst = synth.make_mmv_instance(N, 2, G, 10.0, 17, min_sep=0.5 / N)
    inst.theta[:] = [0.3, 0.3 + 0.6 / N]
    H = np.stack([synth.sum_of_sinusoids(N, inst.theta, inst.alpha[g]) for g in range(G)])
    noise = np.sqrt(inst.beta) * np.stack([synth.Stream(900 + g).cnormal(N) for g in range(G)])
    Y = (H + noise).astype(np.complex64)
    ctx = lse_mod.lse_create(lse_mod.lse_config_default(precision=lse_mod.LSE_PREC_MIXED_DF))
    try:
        gpu = lse_mod.lse_fit_mmv(ctx, Y)
    finally:
        lse_mod.lse_destroy(ctx)
    ref = omv.fit(Y.T.astype(np.complex128), 8 * N)
    check(gpu, ref)
    assert gpu["K"] == 2


@pytest.mark.parametrize("prec", ["fp64", "mixed_df"])
def test_batch_ragged_matches_single_fits(lse_mod, prec):
    import torch
    G = 4
    insts = [synth.make_mmv_instance(N, max(1, N // 24), G, 15.0, 8300 + i)
             for i, N in enumerate((96, 150, 64, 211, 128))]
    offs = np.concatenate([[0], np.cumsum([m.N for m in insts])]).astype(np.int64)
    y = np.concatenate([m.Y.reshape(-1) for m in insts])  # instance b: G x N_b snapshot-major
    dev = torch.device("cuda:0")
    ctx = lse_mod.lse_create(lse_mod.lse_config_default(precision=prec_of(lse_mod, prec),
                                                        flags=lse_mod.LSE_FLAG_NO_CLUSTER))
    try:
        out = lse_mod.alloc_batch_out(offs, device=dev, G=G)
        lse_mod.lse_fit_mmv_batch_d(ctx, torch.from_numpy(y).to(dev), offs, G, out)
        torch.cuda.synchronize()
        singles = [lse_mod.lse_fit_mmv(ctx, m.Y) for m in insts]
    finally:
        lse_mod.lse_destroy(ctx)
    K = out["K"].cpu().numpy()
    th = out["theta"].cpu().numpy()
    al = out["alpha"].cpu().numpy()
    for b, (m, r) in enumerate(zip(insts, singles)):
        assert K[b] == r["K"]
        o, n = int(offs[b]), m.N
        assert np.array_equal(th[o:o + K[b]], r["theta"])
        for g in range(G):
            s0 = G * o + g * n
            assert np.array_equal(al[s0:s0 + K[b]], r["alpha"][:, g])
        assert out["beta"].cpu().numpy()[b] == r["beta"]


def test_bench_shape_objective_matches_a_dense_evaluation(lse_mod):
    """At the benchmark's shape (N = 1024, G = 8, K = 32; eight instances of the
    64-instance batch, too large for whole oracle fits) the objective each fit
    reports is eq. (L_MMV) at its returned state, evaluated densely by the
    oracle, and the fits find the true frequencies."""
    import torch
    work = synth.mmv_batch(B=8)
    G = work[0][0].G
    offs = np.concatenate([[0], np.cumsum([m.N for m, _ in work])]).astype(np.int64)
    y = np.concatenate([m.Y.reshape(-1) for m, _ in work])
    dev = torch.device("cuda:0")
    ctx = lse_mod.lse_create(lse_mod.lse_config_default(precision=lse_mod.LSE_PREC_MIXED_DF))
    try:
        out = lse_mod.alloc_batch_out(offs, device=dev, G=G)
        lse_mod.lse_fit_mmv_batch_d(ctx, torch.from_numpy(y).to(dev), offs, G, out)
        torch.cuda.synchronize()
    finally:
        lse_mod.lse_destroy(ctx)
    K = out["K"].cpu().numpy()
    th = out["theta"].cpu().numpy()
    ga = out["gamma"].cpu().numpy()
    be = out["beta"].cpu().numpy()
    obj = out["objective"].cpu().numpy()
    st = out["status"].cpu().numpy()
    for b, (m, _L) in enumerate(work):
        assert st[b] in (0, 5)
        o = int(offs[b])
        t, g = th[o:o + K[b]], ga[o:o + K[b]]
        ev = omv.MMVDenseEval(m.Y.T.astype(np.complex128), t, g, be[b])
        data = ev.data_term()
        # the reported objective is the data term minus the prior term at the
        # fit's last zeta = min(0.5, K'/N), K' the count after its last activation
        errs = [abs(obj[b] - (data - dn.prior_term(int(K[b]), m.N, dn.zeta_update(k2, m.N))))
                for k2 in range(int(K[b]), int(K[b]) + 4)]
        assert min(errs) <= 1e-9 * abs(data)
        # most true frequencies are found (weak ones may drop at 0 dB)
        d = np.array([wrapdist(t0, t).min() for t0 in m.theta])
        assert np.mean(d < 0.5 / m.N) > 0.75
