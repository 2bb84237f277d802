"""The L-BFGS update of Sec. II-C1 (LSE_FLAG_LBFGS; readings L1-L4) on the
GPU against the oracle's L-BFGS fits (oracle/fit.py, update="lbfgs").

Bar: the fit bar (equal K, frequencies within 1e-6 cycles, gamma, alpha,
beta and the objective within 1e-6 relative) and equal evaluation counts."""
import numpy as np
import pytest

from oracle import fit as ofit
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


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("N,K,snr,seed", [(64, 3, 25.0, 1), (128, 10, 20.0, 2), (200, 6, 12.0, 3), (256, 8, 20.0, 4)])
def test_lbfgs_fit_against_oracle(lse_mod, N, K, snr, seed, prec):
    lse = lse_mod
    inst = synth.make_instance(N, K, snr, 9700 + seed)
    L = synth.default_grid_size(N)
    ctx = lse.lse_create(lse.lse_config_default(precision=prec_of(lse, prec), flags=lse.LSE_FLAG_LBFGS))
    try:
        gpu = lse.lse_fit(ctx, inst.y)
    finally:
        lse.lse_destroy(ctx)
    ref = ofit.fit(inst.y, L, update="lbfgs")
    assert gpu["K"] == ref.K
    assert wrapdist(gpu["theta"], ref.theta).max() < 1e-6
    assert np.allclose(gpu["gamma"], ref.gamma, rtol=1e-6)
    assert np.allclose(gpu["alpha"], ref.alpha, rtol=1e-6, atol=1e-6 * np.abs(ref.alpha).max())
    assert abs(gpu["beta"] - ref.beta) <= 1e-6 * ref.beta
    assert abs(gpu["objective"] - ref.objective) <= 1e-6 * max(1.0, abs(ref.objective))
    assert gpu["n_evals"] == ref.n_evals


def test_lbfgs_and_newton_reach_the_same_fit(lse_mod):
    lse = lse_mod
    inst = synth.make_instance(1024, 16, 25.0, 9710)
    res = {}
    for name, flags in (("newton", 0), ("lbfgs", lse.LSE_FLAG_LBFGS)):
        ctx = lse.lse_create(lse.lse_config_default(precision=lse.LSE_PREC_MIXED_DF, flags=flags))
        try:
            res[name] = lse.lse_fit(ctx, inst.y)
        finally:
            lse.lse_destroy(ctx)
    a, b = res["newton"], res["lbfgs"]
    assert a["K"] == b["K"]
    assert wrapdist(a["theta"], b["theta"]).max() < 1e-6
    assert abs(a["objective"] - b["objective"]) <= 1e-6 * abs(a["objective"])
