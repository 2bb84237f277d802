"""The semifast evaluation of incomplete observations (Sec. IV) on the GPU
through the C ABI, against the dense incomplete-data oracle
(oracle/incomplete.py).

Bar: ln|C|, y^H C^-1 y and eqs. (q)-(x) at the active frequencies within
1e-8 relative (normwise per quantity); the grid q normwise and s pointwise
within 1e-8 on the FP64 path and 1e-6 on the double-float path (whose grid
outputs are rounded to FP32, 6e-8)."""
import numpy as np
import pytest

from oracle import incomplete as oi
from paper_1705_06073_gb300 import synth
from tests.gpu_util import rel_inf

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lse_mod():
    from paper_1705_06073_gb300 import build, lse
    build.build()
    return lse


def run(lse, insts, states, Ls, prec, grid=True):
    import torch
    dev = torch.device("cuda:0")
    f64 = prec == "fp64"
    p = lse.LSE_PREC_FP64 if f64 else lse.LSE_PREC_MIXED_DF
    B = len(insts)
    moff = np.concatenate([[0], np.cumsum([len(m.y) for m in insts])]).astype(np.int64)
    koff = np.concatenate([[0], np.cumsum([len(t) for t, _g, _b in states])]).astype(np.int64)
    y = torch.from_numpy(np.concatenate([m.y for m in insts])).to(dev)
    obs = torch.from_numpy(np.concatenate([m.obs for m in insts]).astype(np.int32)).to(dev)
    th = torch.from_numpy(np.concatenate([t for t, _g, _b in states] + [np.zeros(1)])).to(dev)
    ga = torch.from_numpy(np.concatenate([g for _t, g, _b in states] + [np.zeros(1)])).to(dev)
    be = torch.tensor([b for _t, _g, b in states], dtype=torch.float64, device=dev)
    scal = torch.zeros(2 * B, dtype=torch.float64, device=dev)
    vec = torch.zeros(max(1, 7 * int(koff[-1])), dtype=torch.complex128, device=dev)
    status = torch.full((B,), -1, dtype=torch.int32, device=dev)
    G = int(np.sum(Ls))
    q = torch.zeros(G, dtype=torch.complex128 if f64 else torch.complex64, device=dev) if grid else None
    s = torch.zeros(G, dtype=torch.float64 if f64 else torch.float32, device=dev) if grid else None
    ctx = lse.lse_create(lse.lse_config_default(precision=p))
    try:
        lse.lse_eval_semifast_batch_d(ctx, y, obs, moff, [m.N for m in insts], th, ga, koff, be, Ls, scal, vec, status,
                                      q=q, s=s, f64=f64)
        torch.cuda.synchronize()
    finally:
        lse.lse_destroy(ctx)
    out = dict(scal=scal.cpu().numpy(), vec=vec.cpu().numpy(), status=status.cpu().numpy(), koff=koff)
    if grid:
        out["q"] = q.cpu().numpy().astype(np.complex128)
        out["s"] = s.cpu().numpy().astype(np.float64)
    return out


def true_state(m):
    return np.asarray(m.theta, float), np.abs(m.alpha) ** 2, float(m.beta)


def check_instance(out, b, m, state, L, g0, grid_tol):
    th, ga, be = state
    ev = oi.IncompleteDenseEval(m.y, m.obs, m.N, th, ga, be)
    assert out["status"][b] == 0
    assert abs(out["scal"][2 * b] - ev.logdet) <= 1e-8 * max(1.0, abs(ev.logdet))
    assert abs(out["scal"][2 * b + 1] - ev.yCy) <= 1e-8 * abs(ev.yCy)
    K = len(th)
    if K:
        ref = ev.active_vectors()
        v = out["vec"][7 * out["koff"][b]:7 * (out["koff"][b] + K)].reshape(K, 7)
        for j, name in enumerate(("q", "r", "u", "s", "t", "v", "x")):
            got = v[:, j].real if name in ("s", "x") else v[:, j]
            assert rel_inf(got, ref[name]) < 1e-8, (name, rel_inf(got, ref[name]))
    if "q" in out:
        gr = ev.grid(L)
        assert rel_inf(out["q"][g0:g0 + L], gr["q"]) < grid_tol
        assert np.max(np.abs(out["s"][g0:g0 + L] - gr["s"]) / gr["s"]) < grid_tol


@pytest.mark.parametrize("prec", ["fp64", "mixed_df"])
def test_batch_against_dense_oracle(lse_mod, prec):
    insts = [synth.make_incomplete_instance(N, M, K, snr, 9400 + i)
             for i, (N, M, K, snr) in enumerate([(64, 48, 3, 20.0), (200, 150, 8, 10.0), (37, 30, 2, 30.0),
                                                 (512, 384, 16, 20.0), (128, 100, 0, 20.0)])]
    states = [true_state(m) if len(m.theta) else (np.zeros(0), np.zeros(0), 1.0) for m in insts]
    Ls = [synth.default_grid_size(m.N) for m in insts]
    out = run(lse_mod, insts, states, Ls, prec)
    g0 = 0
    for b, m in enumerate(insts):
        check_instance(out, b, m, states[b], Ls[b], g0, 1e-8 if prec == "fp64" else 1e-6)
        g0 += Ls[b]


def test_perturbed_state_and_grid_size(lse_mod):
    """An off-truth state (frequencies moved, variances scaled) and L = 2N,
    the smallest grid, on the double-float path."""
    m = synth.make_incomplete_instance(300, 225, 10, 15.0, 9410)
    r = np.random.default_rng(1)
    th = np.mod(m.theta + r.normal(0, 0.3 / 300, 10), 1.0)
    ga = np.abs(m.alpha) ** 2 * (0.5 + r.random(10))
    st = (th, ga, 1.7 * m.beta)
    L = 1024
    out = run(lse_mod, [m], [st], [L], "mixed_df")
    check_instance(out, 0, m, st, L, 0, 1e-6)


def test_not_positive_definite_is_reported(lse_mod):
    """A tiny negative variance (1/gamma = -1e8 on the diagonal of
    Sigma^-1 = A^H A/beta + Gamma^-1, beyond anything A^H A/beta adds) makes
    Sigma^-1 indefinite: that instance reports LSE_ENUMERIC, the other of the
    launch is unaffected."""
    a = synth.make_incomplete_instance(96, 72, 4, 20.0, 9420)
    b = synth.make_incomplete_instance(80, 60, 3, 20.0, 9421)
    sa = true_state(a)
    sa = (sa[0], np.where(np.arange(4) == 1, -1e-8, sa[1]), sa[2])
    sb = true_state(b)
    out = run(lse_mod, [a, b], [sa, sb], [1024, 1024], "fp64", grid=False)
    assert out["status"][0] == lse_mod.LSE_ENUMERIC
    check_instance(out, 1, b, sb, 1024, 0, 1e-8)


@pytest.mark.slow
def test_bench_shape_sampled_against_dense_oracle(lse_mod):
    """One instance of the benchmark's incomplete-data batch (N = 4096,
    M = 3072, K = 16, L = 16384): scalars and eqs. (q)-(x) in full, the grid
    at 64 sampled points (a dense M x M factorisation)."""
    m, L = synth.incomplete_batch(B=1)[0]
    st = true_state(m)
    out = run(lse_mod, [m], [st], [L], "mixed_df")
    ev = oi.IncompleteDenseEval(m.y, m.obs, m.N, *st)
    assert abs(out["scal"][0] - ev.logdet) <= 1e-8 * abs(ev.logdet)
    assert abs(out["scal"][1] - ev.yCy) <= 1e-8 * abs(ev.yCy)
    ref = ev.active_vectors()
    v = out["vec"].reshape(-1, 7)
    for j, name in enumerate(("q", "r", "u", "s", "t", "v", "x")):
        got = v[:, j].real if name in ("s", "x") else v[:, j]
        assert rel_inf(got, ref[name]) < 1e-8, name
    idx = np.random.default_rng(2).choice(L, 64, replace=False)
    gr = ev.grid(0, points=idx / L)
    assert rel_inf(out["q"][idx], gr["q"]) < 1e-6
    assert np.max(np.abs(out["s"][idx] - gr["s"]) / gr["s"]) < 1e-6


# ------------------------------------------------------------------ fits ---

def fit_check(gpu, ref, tol=1e-6):
    assert gpu["K"] == ref.K, (gpu["K"], ref.K)
    if ref.K:
        from tests.gpu_util import wrapdist
        assert wrapdist(gpu["theta"], ref.theta).max() < tol
        assert np.allclose(gpu["gamma"], ref.gamma, rtol=tol)
        assert np.allclose(gpu["alpha"], ref.alpha, rtol=tol, atol=tol * np.abs(ref.alpha).max())
    assert abs(gpu["beta"] - ref.beta) <= tol * ref.beta
    assert abs(gpu["objective"] - ref.objective) <= tol * max(1.0, abs(ref.objective))


@pytest.mark.parametrize("prec", ["fp64", "mixed_df"])
@pytest.mark.parametrize("N,M,K,snr,seed", [(64, 48, 3, 20.0, 1), (128, 96, 5, 15.0, 2), (100, 80, 4, 25.0, 3),
                                            (256, 192, 8, 20.0, 4)])
def test_incomplete_fit_against_oracle(lse_mod, N, M, K, snr, seed, prec):
    lse = lse_mod
    m = synth.make_incomplete_instance(N, M, K, snr, 9500 + seed)
    p = lse.LSE_PREC_FP64 if prec == "fp64" else lse.LSE_PREC_MIXED_DF
    ctx = lse.lse_create(lse.lse_config_default(precision=p))
    try:
        gpu = lse.lse_fit_incomplete(ctx, m.y, m.obs, N)
    finally:
        lse.lse_destroy(ctx)
    ref = oi.fit(m.y, m.obs, N, synth.default_grid_size(N))
    assert gpu["status"] == 0
    fit_check(gpu, ref)


def test_incomplete_batch_matches_single_fits(lse_mod):
    import torch
    lse = lse_mod
    insts = [synth.make_incomplete_instance(N, M, K, 20.0, 9600 + i)
             for i, (N, M, K) in enumerate([(96, 70, 4), (160, 120, 6), (64, 50, 3)])]
    moff = np.concatenate([[0], np.cumsum([len(m.y) for m in insts])]).astype(np.int64)
    dev = torch.device("cuda:0")
    y = torch.from_numpy(np.concatenate([m.y for m in insts])).to(dev)
    obs = torch.from_numpy(np.concatenate([m.obs for m in insts]).astype(np.int32)).to(dev)
    ctx = lse.lse_create(lse.lse_config_default(precision=lse.LSE_PREC_MIXED_DF))
    try:
        out = lse.alloc_batch_out(moff, device=dev)
        lse.lse_fit_incomplete_batch_d(ctx, y, obs, moff, [m.N for m in insts], out)
        torch.cuda.synchronize()
        singles = [lse.lse_fit_incomplete(ctx, m.y, m.obs, m.N) for m in insts]
    finally:
        lse.lse_destroy(ctx)
    K = out["K"].cpu().numpy()
    th = out["theta"].cpu().numpy()
    for b, r in enumerate(singles):
        assert K[b] == r["K"] and out["status"].cpu().numpy()[b] == r["status"]
        o = int(moff[b])
        assert np.array_equal(th[o:o + K[b]], r["theta"])
        assert out["beta"].cpu().numpy()[b] == r["beta"]
