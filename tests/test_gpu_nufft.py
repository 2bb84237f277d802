"""Off-grid sums by the non-uniform FFT (Sec. III-B footnote) inside whole
fits on the GPU, against the oracle (whose sums are dense solves, eqs. q-x)
and against the same fits with the direct O(N K) sums (LSE_FLAG_DIRECT_SUMS).

The fits below hold K >= 32 components, so their Newton sums, and the
re-scoring of grid candidates, go through the non-uniform FFT.  Bar: the
single-snapshot fit bar (equal K, frequencies within 1e-6 cycles, gamma,
alpha, beta, objective within 1e-6 relative)."""
import numpy as np
import pytest

from oracle import fit as ofit
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
    assert wrapdist(gpu["theta"], ref.theta).max() < tol
    assert np.allclose(gpu["gamma"], ref.gamma, rtol=tol)
    a = np.asarray(ref.alpha)
    assert np.allclose(gpu["alpha"], a, rtol=tol, atol=tol * np.abs(a).max())
    assert abs(gpu["beta"] - ref.beta) <= tol * ref.beta
    assert abs(gpu["objective"] - ref.objective) <= tol * max(1.0, abs(ref.objective))


def fit(lse, y, prec, flags=0, mmv=False):
    ctx = lse.lse_create(lse.lse_config_default(precision=prec_of(lse, prec), flags=flags))
    try:
        return lse.lse_fit_mmv(ctx, y) if mmv else lse.lse_fit(ctx, y)
    finally:
        lse.lse_destroy(ctx)


@pytest.mark.parametrize("prec", PRECS)
def test_fit_with_nufft_sums_matches_oracle(lse_mod, prec):
    inst = synth.make_instance(512, 40, 20.0, 9101)
    gpu = fit(lse_mod, inst.y, prec)
    assert gpu["K"] >= 32  # the sums of every Newton step go through the non-uniform FFT
    ref = ofit.fit(inst.y, synth.default_grid_size(512))
    check(gpu, ref)
    assert gpu["n_evals"] == ref.n_evals


@pytest.mark.parametrize("prec", ["fp64", "mixed_df"])
def test_nufft_and_direct_sums_agree(lse_mod, prec):
    inst = synth.make_instance(1024, 48, 15.0, 9102)
    a = fit(lse_mod, inst.y, prec)
    b = fit(lse_mod, inst.y, prec, flags=lse_mod.LSE_FLAG_DIRECT_SUMS)
    assert a["K"] == b["K"] >= 32
    assert wrapdist(a["theta"], b["theta"]).max() < 1e-8
    assert np.allclose(a["gamma"], b["gamma"], rtol=1e-7)
    assert abs(a["objective"] - b["objective"]) <= 1e-9 * abs(b["objective"])


def test_mmv_fit_with_nufft_sums_matches_oracle(lse_mod):
    inst = synth.make_mmv_instance(256, 36, 3, 15.0, 9103)
    gpu = fit(lse_mod, inst.Y, "mixed_df", mmv=True)
    assert gpu["K"] >= 32
    ref = omv.fit(inst.Y.T, synth.default_grid_size(256))
    check(gpu, ref)
