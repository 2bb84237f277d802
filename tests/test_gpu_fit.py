"""Whole fits on the GPU through the C ABI against the oracle's fits.

Bar: equal K and every frequency within 1e-6 cycles (wrap distance) of the
oracle's.  gamma, alpha, beta and the objective agree to 1e-6 relative: on
every path the Newton sums, the objective and the updates are FP64 (or the
48-bit double-float recursion), so the iterates follow the oracle's.
"""
import numpy as np
import pytest

from oracle import fit as ofit
from paper_1705_06073_gb300 import synth
from tests.gpu_util import match_fit, wrapdist

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lse_mod():
    from paper_1705_06073_gb300 import build, lse
    build.build()
    return lse


def make_ctx(lse, L=0, **kw):
    return lse.lse_create(lse.lse_config_default(grid_size=L, **kw))


def tol_for(prec):
    return 1e-6


def check(gpu, ref, tol_theta=1e-6, tol_rel=1e-6):
    assert match_fit(gpu, ref) < tol_theta
    if ref.K:
        assert np.allclose(gpu["gamma"], ref.gamma, rtol=tol_rel)
        assert np.allclose(gpu["alpha"], ref.alpha, rtol=tol_rel, atol=tol_rel * np.abs(ref.alpha).max())
    assert abs(gpu["beta"] - ref.beta) <= tol_rel * ref.beta
    assert abs(gpu["objective"] - ref.objective) <= tol_rel * max(1.0, abs(ref.objective))


PRECS = ["fp64", "mixed", "mixed_df"]


def prec_of(lse, name):
    return {"fp64": lse.LSE_PREC_FP64, "mixed": lse.LSE_PREC_MIXED, "mixed_df": lse.LSE_PREC_MIXED_DF}[name]


@pytest.mark.parametrize("prec", PRECS)
def test_fit_single_n256(lse_mod, prec):
    inst, L = synth.single_n256()[0]
    ctx = make_ctx(lse_mod, L, precision=prec_of(lse_mod, prec))
    try:
        gpu = lse_mod.lse_fit(ctx, inst.y)
    finally:
        lse_mod.lse_destroy(ctx)
    ref = ofit.fit(inst.y, L)
    check(gpu, ref, tol_rel=tol_for(prec))
    assert gpu["iters"] == ref.iters
    assert gpu["n_evals"] == ref.n_evals
    assert gpu["n_grid"] == ref.n_grid_evals


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("N,K,snr,seed", [(64, 3, 25.0, 1), (100, 4, 15.0, 2), (128, 10, 20.0, 3), (37, 2, 30.0, 4),
                                          (200, 6, 10.0, 5), (1024, 16, 25.0, 6)])
def test_fit_small_instances(lse_mod, N, K, snr, seed, prec):
    inst = synth.make_instance(N, K, snr, 7000 + seed)
    L = synth.default_grid_size(N)
    ctx = make_ctx(lse_mod, precision=prec_of(lse_mod, prec))
    try:
        gpu = lse_mod.lse_fit(ctx, inst.y)
    finally:
        lse_mod.lse_destroy(ctx)
    ref = ofit.fit(inst.y, L)
    check(gpu, ref, tol_rel=tol_for(prec))


@pytest.mark.parametrize("prec", PRECS)
def test_fit_batch_ragged_matches_single_fits(lse_mod, prec):
    """One launch over instances of different N; each equals the oracle's fit."""
    specs = [(48, 2), (130, 5), (77, 3), (256, 8), (33, 1), (160, 4)]
    insts = [synth.make_instance(N, K, 20.0, 8000 + i) for i, (N, K) in enumerate(specs)]
    ctx = make_ctx(lse_mod, precision=prec_of(lse_mod, prec))
    try:
        res = lse_mod.lse_fit_batch(ctx, [i.y for i in insts])
    finally:
        lse_mod.lse_destroy(ctx)
    for inst, gpu in zip(insts, res):
        ref = ofit.fit(inst.y, synth.default_grid_size(inst.N))
        check(gpu, ref, tol_rel=tol_for(prec))


def test_fit_degenerate_inputs(lse_mod):
    ctx = make_ctx(lse_mod)
    try:
        r = lse_mod.lse_fit(ctx, np.zeros(16, np.complex64))
        assert r["K"] == 0 and r["beta"] == 0.0
        # pure noise: the oracle decides; typically nothing is activated
        y = synth.Stream(5).cnormal(32).astype(np.complex64)
        gpu = lse_mod.lse_fit(ctx, y)
        check(gpu, ofit.fit(y, synth.default_grid_size(32)))
        # smallest N
        y2 = np.array([1 + 1j, 0.5 - 0.2j], np.complex64)
        gpu = lse_mod.lse_fit(ctx, y2)
        check(gpu, ofit.fit(y2, synth.default_grid_size(2)))
        with pytest.raises(lse_mod.LseError):
            lse_mod.lse_fit(ctx, np.ones(1, np.complex64))
    finally:
        lse_mod.lse_destroy(ctx)


def test_fit_capacity_error(lse_mod):
    inst, L = synth.single_n256()[0]
    ctx = make_ctx(lse_mod, L)
    try:
        r = lse_mod.lse_fit_batch(ctx, [inst.y], K_cap=2)[0]
        assert r["status"] == lse_mod.LSE_ECAPACITY and r["K"] == 8 and r["theta"] is None
    finally:
        lse_mod.lse_destroy(ctx)


def test_cluster_recursion_matches_one_block():
    """Double-float path with the Levinson recursion (LSE_FLAG_LEVINSON): the
    same batch fitted with clusters of two blocks (the default for a batch
    smaller than half the SMs) and with one block per instance
    (LSE_FLAG_NO_CLUSTER) gives the same fits to rounding: the two differ only
    in the order the inner products of the recursion are summed."""
    from paper_1705_06073_gb300 import build, lse
    build.build()
    specs = [(256, 8), (1000, 16), (2048, 32), (4096, 64), (37, 2), (600, 9), (3000, 40), (5000, 70)]
    insts = [synth.make_instance(N, K, 20.0, 8100 + i) for i, (N, K) in enumerate(specs)]
    res = {}
    for flags in (0, lse.LSE_FLAG_NO_CLUSTER):
        ctx = lse.lse_create(lse.lse_config_default(precision=lse.LSE_PREC_MIXED_DF,
                                                    flags=flags | lse.LSE_FLAG_LEVINSON))
        try:
            res[flags] = lse.lse_fit_batch(ctx, [i.y for i in insts])
        finally:
            lse.lse_destroy(ctx)
    for a, b in zip(res[0], res[lse.LSE_FLAG_NO_CLUSTER]):
        assert a["status"] == b["status"] and a["status"] in (0, lse.LSE_ENOTCONV)
        assert a["K"] == b["K"] and a["n_evals"] == b["n_evals"] and a["iters"] == b["iters"]
        if a["K"]:
            assert np.all(wrapdist(a["theta"], b["theta"]) < 1e-9)
            assert np.allclose(a["gamma"], b["gamma"], rtol=1e-8)
        assert abs(a["beta"] - b["beta"]) <= 1e-9 * b["beta"]


def test_big_cluster_recursion_matches_one_block():
    """Double-float Levinson path, instances too large for the shared-memory
    recursion: a small batch runs each recursion on a cluster of eight blocks
    sharing c and a in global memory; the fits equal the one-block fits to
    rounding."""
    from paper_1705_06073_gb300 import build, lse
    build.build()
    insts = [synth.make_instance(N, K, 20.0, 8200 + i) for i, (N, K) in enumerate([(8192, 64), (6500, 40)])]
    res = {}
    for flags in (0, lse.LSE_FLAG_NO_CLUSTER):
        ctx = lse.lse_create(lse.lse_config_default(precision=lse.LSE_PREC_MIXED_DF,
                                                    flags=flags | lse.LSE_FLAG_LEVINSON))
        try:
            res[flags] = lse.lse_fit_batch(ctx, [i.y for i in insts])
        finally:
            lse.lse_destroy(ctx)
    for a, b in zip(res[0], res[lse.LSE_FLAG_NO_CLUSTER]):
        assert a["status"] == b["status"] and a["status"] in (0, lse.LSE_ENOTCONV)
        assert a["K"] == b["K"] and a["n_evals"] == b["n_evals"] and a["iters"] == b["iters"]
        if a["K"]:
            assert np.all(wrapdist(a["theta"], b["theta"]) < 1e-9)
            assert np.allclose(a["gamma"], b["gamma"], rtol=1e-8)
        assert abs(a["beta"] - b["beta"]) <= 1e-9 * b["beta"]


@pytest.mark.parametrize("prec", PRECS)
def test_levinson_path_matches_oracle(lse_mod, prec):
    """The O(N^2) Levinson recursion (LSE_FLAG_LEVINSON) against the oracle's
    fits: the N = 256 instance and a ragged batch of small instances."""
    lse = lse_mod
    inst, L = synth.single_n256()[0]
    ctx = make_ctx(lse, L, precision=prec_of(lse, prec), flags=lse.LSE_FLAG_LEVINSON)
    try:
        gpu = lse.lse_fit(ctx, inst.y)
    finally:
        lse.lse_destroy(ctx)
    ref = ofit.fit(inst.y, L)
    check(gpu, ref)
    assert gpu["n_evals"] == ref.n_evals
    insts = [synth.make_instance(N, K, snr, 8300 + i) for i, (N, K, snr) in
             enumerate([(100, 4, 15.0), (128, 10, 20.0), (300, 6, 25.0)])]
    ctx = make_ctx(lse, 0, precision=prec_of(lse, prec), flags=lse.LSE_FLAG_LEVINSON)
    try:
        res = lse.lse_fit_batch(ctx, [i.y for i in insts])
    finally:
        lse.lse_destroy(ctx)
    for g, i in zip(res, insts):
        check(g, ofit.fit(i.y, synth.default_grid_size(len(i.y))))


def test_superfast_matches_levinson():
    """The superfast Schur recursion (default) and the Levinson recursion give
    the same fits: equal K and evaluation counts, frequencies within 1e-8
    cycles, on instances where the superfast recursion runs several levels of
    merges (N up to 8192, 10-30 dB)."""
    from paper_1705_06073_gb300 import build, lse
    build.build()
    specs = [(64, 3, 25.0), (1000, 16, 30.0), (4096, 64, 10.0), (4096, 64, 30.0), (8192, 64, 20.0), (3001, 40, 15.0)]
    insts = [synth.make_instance(N, K, snr, 8400 + i) for i, (N, K, snr) in enumerate(specs)]
    res = {}
    for flags in (0, lse.LSE_FLAG_LEVINSON | lse.LSE_FLAG_NO_CLUSTER):
        ctx = lse.lse_create(lse.lse_config_default(precision=lse.LSE_PREC_MIXED_DF, flags=flags))
        try:
            res[flags] = lse.lse_fit_batch(ctx, [i.y for i in insts])
        finally:
            lse.lse_destroy(ctx)
    for a, b in zip(res[0], res[lse.LSE_FLAG_LEVINSON | lse.LSE_FLAG_NO_CLUSTER]):
        assert a["status"] == b["status"] and a["status"] in (0, lse.LSE_ENOTCONV)
        assert a["K"] == b["K"] and a["n_evals"] == b["n_evals"]
        if a["K"]:
            assert np.all(wrapdist(a["theta"], b["theta"]) < 1e-8)
            assert np.allclose(a["gamma"], b["gamma"], rtol=1e-6)
        assert abs(a["beta"] - b["beta"]) <= 1e-8 * b["beta"]


@pytest.mark.parametrize("prec", ["mixed_df", "fp64", "mixed"])
def test_superfast_pair_matches_one_block(prec):
    """A small batch runs every superfast recursion on a two-block cluster:
    the second block takes half of every pass of the FFT stages kept in
    global memory, of the refinement and of the Gohberg-Semencul applies.
    Each butterfly is computed as by one block, so the fits equal the
    one-block fits bit for bit (instances whose recursion has one, two and
    three global-memory levels, and a ragged N), on every precision path."""
    from paper_1705_06073_gb300 import build, lse
    build.build()
    specs = [(1200, 12, 25.0), (2049, 24, 15.0), (4096, 64, 20.0), (8192, 64, 30.0), (300, 6, 20.0)]
    insts = [synth.make_instance(N, K, snr, 8600 + i) for i, (N, K, snr) in enumerate(specs)]
    res = {}
    for flags in (0, lse.LSE_FLAG_NO_CLUSTER):
        ctx = lse.lse_create(lse.lse_config_default(precision=prec_of(lse, prec), flags=flags))
        try:
            res[flags] = lse.lse_fit_batch(ctx, [i.y for i in insts])
            res[flags] = (res[flags], lse.lse_fit_batch(ctx, [i.y for i in insts]))  # twice: no state left behind
        finally:
            lse.lse_destroy(ctx)
    for run in range(2):
        for a, b in zip(res[0][run], res[lse.LSE_FLAG_NO_CLUSTER][0]):
            assert a["status"] == b["status"] and a["status"] in (0, lse.LSE_ENOTCONV)
            assert a["K"] == b["K"] and a["n_evals"] == b["n_evals"] and a["iters"] == b["iters"]
            for key in ("theta", "gamma", "alpha"):
                assert np.array_equal(a[key], b[key]), key
            assert a["beta"] == b["beta"] and a["objective"] == b["objective"]
