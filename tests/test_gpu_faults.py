"""Fault handling without faulting the GPU: an instance whose data are not
finite (a NaN or an infinity in y) makes the factorisation meet a
non-finite pivot, so that instance ends with LSE_ENUMERIC while the other
instances of the same launch finish normally, with the result they have
alone."""
import numpy as np
import pytest

from paper_1705_06073_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lse_mod():
    from paper_1705_06073_gb300 import build, lse
    build.build()
    return lse


@pytest.mark.parametrize("prec", ["fp64", "mixed_df"])
def test_non_finite_instance_fails_alone(lse_mod, prec):
    lse = lse_mod
    p = {"fp64": lse.LSE_PREC_FP64, "mixed_df": lse.LSE_PREC_MIXED_DF}[prec]
    good = synth.make_instance(200, 5, 20.0, 9301).y
    bad_nan = synth.make_instance(150, 4, 20.0, 9302).y.copy()
    bad_nan[17] = np.nan
    bad_inf = synth.make_instance(128, 3, 20.0, 9303).y.copy()
    bad_inf[5] = np.inf
    ctx = lse.lse_create(lse.lse_config_default(precision=p, flags=lse.LSE_FLAG_NO_CLUSTER))
    try:
        res = lse.lse_fit_batch(ctx, [bad_nan, good, bad_inf])
        alone = lse.lse_fit(ctx, good)
    finally:
        lse.lse_destroy(ctx)
    assert res[0]["status"] == lse.LSE_ENUMERIC and res[2]["status"] == lse.LSE_ENUMERIC
    assert res[1]["status"] == lse.LSE_OK
    assert res[1]["K"] == alone["K"] and np.array_equal(res[1]["theta"], alone["theta"])
    assert res[1]["beta"] == alone["beta"]
