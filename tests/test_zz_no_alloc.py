"""The allocation-free fit entry point (lse_fit_noalloc_d) against the
regular batched entry point (lse_fit_batch_d), through the C ABI.

lse_fit_noalloc_d exists for callers that may not allocate device memory
when they run a fit (fixed-deadline loops where cudaMalloc/cudaFree would
stall the device, hosts whose framework owns all GPU allocations): it keeps
its scratch in a static array inside the library.  For every precision, two
calls in a row on different inputs must each reproduce the regular entry
point's result (same kernel, same arithmetic, same tolerance as the other
fit tests), which also shows that the second call is not disturbed by what
the first left in the shared scratch.  The double-float call is also held
against the CPU oracle.  The file is named so that pytest collects it last.
"""
import numpy as np
import pytest

from paper_1705_06073_gb300 import synth
from tests.gpu_util import wrapdist

pytestmark = pytest.mark.gpu

PRECISIONS = ("fp64", "mixed", "mixed_df")


def _prec(lse, name):
    return {"fp64": lse.LSE_PREC_FP64, "mixed": lse.LSE_PREC_MIXED, "mixed_df": lse.LSE_PREC_MIXED_DF}[name]


def _regular_fit(lse, torch, y, L, prec):
    ctx = lse.lse_create(lse.lse_config_default(grid_size=L, precision=prec))
    try:
        offs = np.array([0, len(y)], np.int64)
        out = lse.alloc_batch_out(offs)
        lse.lse_fit_batch_d(ctx, torch.from_numpy(y).cuda(), offs, out)
        torch.cuda.synchronize()
        return {k: v.cpu().numpy() for k, v in out.items()}
    finally:
        lse.lse_destroy(ctx)


def _noalloc_fit(lse, torch, y, L, prec):
    N = len(y)
    cfg = lse.lse_config_default(grid_size=L, precision=prec)
    out = lse.alloc_batch_out(np.array([0, N], np.int64))
    lse.lse_fit_noalloc_d(torch.from_numpy(y).cuda(), N, out, cfg)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


def _cases():
    return [synth.single_n256()[0], (synth.make_instance(1000, 12, 15.0, 4242), 8192)]


@pytest.mark.parametrize("pname", PRECISIONS)
def test_noalloc_fit_matches_regular_entry_point_twice(pname):
    torch = pytest.importorskip("torch")
    from paper_1705_06073_gb300 import build, lse
    build.build()
    prec = _prec(lse, pname)
    for inst, L in _cases():  # two calls in a row, different sizes
        got = _noalloc_fit(lse, torch, inst.y, L, prec)
        ref = _regular_fit(lse, torch, inst.y, L, prec)
        K = int(ref["K"][0])
        assert int(got["status"][0]) == int(ref["status"][0]) == lse.LSE_OK
        assert int(got["K"][0]) == K and K > 0
        assert np.all(wrapdist(got["theta"][:K], ref["theta"][:K]) < 1e-6)
        assert np.allclose(got["gamma"][:K], ref["gamma"][:K], rtol=1e-6)
        assert np.allclose(got["alpha"][:K], ref["alpha"][:K], rtol=1e-6, atol=1e-9)
        assert abs(got["beta"][0] - ref["beta"][0]) <= 1e-6 * ref["beta"][0]
        assert int(got["n_evals"][0]) == int(ref["n_evals"][0])


def test_noalloc_double_float_fit_matches_oracle():
    torch = pytest.importorskip("torch")
    from oracle import fit as ofit
    from paper_1705_06073_gb300 import build, lse
    build.build()
    inst, L = synth.single_n256()[0]
    got = _noalloc_fit(lse, torch, inst.y, L, lse.LSE_PREC_MIXED_DF)
    ref = ofit.fit(inst.y, L)
    K = int(got["K"][0])
    assert K == ref.K
    assert np.all(wrapdist(got["theta"][:K], ref.theta) < 1e-6)
    assert np.allclose(got["gamma"][:K], ref.gamma, rtol=1e-6)
    assert abs(got["beta"][0] - ref.beta) <= 1e-6 * ref.beta


def test_noalloc_rejects_sizes_and_arguments_beyond_its_limits():
    torch = pytest.importorskip("torch")
    from paper_1705_06073_gb300 import build, lse
    build.build()
    N = 8192
    y = torch.zeros(N, dtype=torch.complex64, device="cuda")
    out = lse.alloc_batch_out(np.array([0, N], np.int64))
    with pytest.raises(lse.LseError) as e:
        lse.lse_fit_noalloc_d(y, N, out)
    assert e.value.status == lse.LSE_EINVAL
    y = torch.zeros(64, dtype=torch.complex64, device="cuda")
    out = lse.alloc_batch_out(np.array([0, 64], np.int64))
    for bad in (dict(grid_size=-512), dict(flags=1 << 40), dict(grid_size=1 << 16)):
        with pytest.raises(lse.LseError) as e:
            lse.lse_fit_noalloc_d(y, 64, out, lse.lse_config_default(**bad))
        assert e.value.status == lse.LSE_EINVAL
