"""The allocation-free fit entry point (lse_fit_noalloc_d) against the
regular batched entry point (lse_fit_batch_d), through the C ABI.

lse_fit_noalloc_d exists for callers that may not allocate device memory
when they run a fit (fixed-deadline loops, hosts whose framework owns all
GPU allocations): it keeps its scratch in a static array inside the library.
Two calls in a row on different inputs must each reproduce the regular
entry point's result (same kernel, same arithmetic), which also shows that
the second call is not disturbed by what the first left in the shared
scratch.  The file is named so that pytest collects it last.
"""
import numpy as np
import pytest

from paper_1705_06073_gb300 import synth

pytestmark = pytest.mark.gpu


def _regular_fit(lse, torch, y, L):
    ctx = lse.lse_create(lse.lse_config_default(grid_size=L))
    try:
        offs = np.array([0, len(y)], np.int64)
        out = lse.alloc_batch_out(offs)
        lse.lse_fit_batch_d(ctx, torch.from_numpy(y).cuda(), offs, out)
        torch.cuda.synchronize()
        return {k: v.cpu().numpy() for k, v in out.items()}
    finally:
        lse.lse_destroy(ctx)


def test_noalloc_fit_matches_regular_entry_point_twice():
    torch = pytest.importorskip("torch")
    from paper_1705_06073_gb300 import build, lse
    build.build()
    cases = [synth.single_n256()[0], (synth.make_instance(1000, 12, 15.0, 4242), 8192)]
    for inst, L in cases:  # two calls in a row, different sizes
        y = inst.y
        N = len(y)
        cfg = lse.lse_config_default(grid_size=L)
        out = lse.alloc_batch_out(np.array([0, N], np.int64))
        lse.lse_fit_noalloc_d(torch.from_numpy(y).cuda(), N, out, cfg)
        torch.cuda.synchronize()
        got = {k: v.cpu().numpy() for k, v in out.items()}
        ref = _regular_fit(lse, torch, y, L)
        K = int(ref["K"][0])
        assert int(got["status"][0]) == int(ref["status"][0]) == lse.LSE_OK
        assert int(got["K"][0]) == K and K > 0
        d = np.abs(got["theta"][:K] - ref["theta"][:K])
        assert np.all(np.minimum(d, 1 - d) < 1e-6)
        assert np.allclose(got["gamma"][:K], ref["gamma"][:K], rtol=1e-6)
        assert np.allclose(got["alpha"][:K], ref["alpha"][:K], rtol=1e-6, atol=1e-9)
        assert abs(got["beta"][0] - ref["beta"][0]) <= 1e-6 * ref["beta"][0]
        assert int(got["n_evals"][0]) == int(ref["n_evals"][0])


def test_noalloc_rejects_sizes_beyond_its_static_scratch():
    torch = pytest.importorskip("torch")
    from paper_1705_06073_gb300 import build, lse
    build.build()
    N = 8192
    y = torch.zeros(N, dtype=torch.complex64, device="cuda")
    out = lse.alloc_batch_out(np.array([0, N], np.int64))
    with pytest.raises(lse.LseError) as e:
        lse.lse_fit_noalloc_d(y, N, out)
    assert e.value.status == lse.LSE_EINVAL
