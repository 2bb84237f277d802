"""GPU grid evaluation (Sec. III-D) through the C ABI against the dense FP64
oracle, element by element.

Tolerances: FP64 path 1e-8 normwise (and 1e-8 pointwise for s): the
Levinson recursion and FFT convolutions lose about kappa(C) * 1e-16, and the
states here have kappa(C) <= 1e6.  Mixed path (FP32 spectra): 1e-4
normwise, the bound the hot path is specified to meet.
"""
import numpy as np
import pytest

from oracle import dense as dn
from paper_1705_06073_gb300 import synth
from tests.gpu_util import grid_errors, s_fp32_bound

pytestmark = pytest.mark.gpu

FIELDS = ("q", "dq", "d2q", "s", "ds", "d2s")


@pytest.fixture(scope="module")
def ctxs():
    from paper_1705_06073_gb300 import build, lse
    build.build()
    c64 = lse.lse_create(lse.lse_config_default(precision=lse.LSE_PREC_FP64))
    cmx = lse.lse_create(lse.lse_config_default(precision=lse.LSE_PREC_MIXED))
    cdf = lse.lse_create(lse.lse_config_default(precision=lse.LSE_PREC_MIXED_DF))
    yield c64, cmx, cdf
    for c in (c64, cmx, cdf):
        lse.lse_destroy(c)


def state(N, K, seed):
    inst = synth.make_instance(N, K, 20.0, seed) if K else synth.make_instance(N, 0, 20.0, seed)
    r = np.random.default_rng(seed)
    gamma = np.abs(inst.alpha) ** 2 + 0.05 if K else np.zeros(0)
    theta = np.mod(inst.theta + 1e-3 * r.standard_normal(K), 1.0) if K else np.zeros(0)
    beta = inst.beta if K else 0.3
    return inst.y, theta, gamma, beta


CASES = [(2, 0, 4), (2, 1, 4), (7, 2, 16), (16, 1, 32), (33, 3, 128), (64, 4, 128), (100, 5, 256),
         (256, 8, 2048), (300, 12, 1024), (512, 16, 1024)]


@pytest.mark.parametrize("N,K,L", CASES)
def test_grid_fp64_matches_oracle(ctxs, N, K, L):
    from paper_1705_06073_gb300 import lse
    y, th, ga, be = state(N, K, 1000 + N)
    got = lse.lse_eval_grid(ctxs[0], y, th, ga, be, L, f64=True)
    ref = dn.DenseEval(y, th, ga, be).grid(L, derivatives=True)
    err = grid_errors(got, ref, N)
    assert max(err.values()) < 1e-8, err
    assert np.all(np.abs(got["s"] - ref["s"]) <= 1e-8 * ref["s"])


@pytest.mark.parametrize("which", [1, 2])
@pytest.mark.parametrize("N,K,L", CASES)
def test_grid_mixed_matches_oracle(ctxs, N, K, L, which):
    """FP32 spectra: 1e-4 normwise on every output, and s pointwise within
    1e-4 s(l) plus the FP32 FFT's own error bound (tests.gpu_util.s_fp32_bound):
    near a strong component s dips to ~1/gamma while the transform's rounding
    error scales with the whole sequence, so a pure 1e-4 s(l) bound is out of
    FP32's reach there."""
    from paper_1705_06073_gb300 import lse
    y, th, ga, be = state(N, K, 2000 + N)
    got = lse.lse_eval_grid(ctxs[which], y, th, ga, be, L, f64=False)
    ev = dn.DenseEval(y, th, ga, be)
    ref = ev.grid(L, derivatives=True)
    err = grid_errors(got, ref, N)
    assert max(err.values()) < 1e-4, err
    bound = 1e-4 * ref["s"] + s_fp32_bound(ev, L)
    assert np.all(np.abs(got["s"] - ref["s"]) <= bound), float(np.max(np.abs(got["s"] - ref["s"]) / bound))


def test_grid_batch_ragged_device(ctxs):
    """Several instances of different N, K and L in one batched launch, each
    against the oracle."""
    import torch
    from paper_1705_06073_gb300 import lse
    specs = [(37, 2, 128), (128, 0, 256), (250, 6, 512), (64, 3, 512)]
    ys, ths, gas, bes = [], [], [], []
    for i, (N, K, L) in enumerate(specs):
        y, th, ga, be = state(N, K, 3000 + i)
        ys.append(y); ths.append(th); gas.append(ga); bes.append(be)
    yo = np.concatenate([[0], np.cumsum([len(y) for y in ys])])
    ko = np.concatenate([[0], np.cumsum([len(t) for t in ths])])
    Ls = np.array([s[2] for s in specs], np.int32)
    dev = torch.device("cuda:0")
    y_d = torch.from_numpy(np.concatenate(ys)).to(dev)
    th_d = torch.from_numpy(np.concatenate(ths + [np.zeros(1)])).to(dev)
    ga_d = torch.from_numpy(np.concatenate(gas + [np.zeros(1)])).to(dev)
    be_d = torch.tensor(bes, dtype=torch.float64, device=dev)
    G = int(Ls.sum())
    outs = {f: torch.zeros(G, dtype=torch.complex128 if f in ("q", "dq", "d2q") else torch.float64, device=dev)
            for f in FIELDS}
    lse.lse_eval_grid_batch_d(ctxs[0], y_d, yo, th_d, ga_d, ko, be_d, Ls, outs, f64=True)
    torch.cuda.synchronize()
    g0 = 0
    for i, (N, K, L) in enumerate(specs):
        ref = dn.DenseEval(ys[i], ths[i], gas[i], bes[i]).grid(L, derivatives=True)
        got = {f: outs[f][g0:g0 + L].cpu().numpy() for f in FIELDS}
        err = grid_errors(got, ref, N)
        assert max(err.values()) < 1e-8, (i, err)
        g0 += L


def test_grid_rejects_bad_arguments(ctxs):
    from paper_1705_06073_gb300 import lse
    y = np.ones(8, np.complex64)
    with pytest.raises(lse.LseError) as e:
        lse.lse_eval_grid(ctxs[0], y, [], [], 1.0, 12, f64=True)  # L not a power of two
    assert e.value.status == lse.LSE_EINVAL
    with pytest.raises(lse.LseError):
        lse.lse_eval_grid(ctxs[0], y, [], [], 1.0, 8, f64=True)  # L < 2N
    with pytest.raises(lse.LseError):
        lse.lse_eval_grid(ctxs[0], y, [], [], 0.0, 16, f64=True)  # beta <= 0
    with pytest.raises(lse.LseError):
        lse.lse_eval_grid(ctxs[0], y, [], [], 1.0, 16, f64=False)  # dtype mismatch


@pytest.mark.parametrize("which", [0, 2])
def test_grid_batch_captured_in_cuda_graph(ctxs, which):
    """The factorisation and grid kernels of lse_eval_grid_batch_d captured in
    a CUDA graph (after one uncaptured call of the same shapes) replay to the
    direct call's outputs, bit for bit; the call itself does not wait for the
    device (it returns while the kernels are still queued)."""
    import torch
    from paper_1705_06073_gb300 import lse
    f64 = which == 0
    specs = [(37, 2, 128), (128, 0, 256), (250, 6, 512), (64, 3, 512)]
    ys, ths, gas, bes = [], [], [], []
    for i, (N, K, L) in enumerate(specs):
        y, th, ga, be = state(N, K, 3100 + i)
        ys.append(y); ths.append(th); gas.append(ga); bes.append(be)
    yo = np.concatenate([[0], np.cumsum([len(y) for y in ys])])
    ko = np.concatenate([[0], np.cumsum([len(t) for t in ths])])
    Ls = np.array([s[2] for s in specs], np.int32)
    dev = torch.device("cuda:0")
    y_d = torch.from_numpy(np.concatenate(ys)).to(dev)
    th_d = torch.from_numpy(np.concatenate(ths + [np.zeros(1)])).to(dev)
    ga_d = torch.from_numpy(np.concatenate(gas + [np.zeros(1)])).to(dev)
    be_d = torch.tensor(bes, dtype=torch.float64, device=dev)
    G = int(Ls.sum())
    ct, rt = (torch.complex128, torch.float64) if f64 else (torch.complex64, torch.float32)

    def alloc():
        return {f: torch.zeros(G, dtype=ct if f in ("q", "dq", "d2q") else rt, device=dev) for f in FIELDS}

    st = torch.cuda.Stream(device=dev)
    st.wait_stream(torch.cuda.current_stream())
    direct = alloc()
    with torch.cuda.stream(st):
        lse.lse_eval_grid_batch_d(ctxs[which], y_d, yo, th_d, ga_d, ko, be_d, Ls, direct, f64, stream=st)
    st.synchronize()
    graphed = alloc()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=st, capture_error_mode="thread_local"):
        lse.lse_eval_grid_batch_d(ctxs[which], y_d, yo, th_d, ga_d, ko, be_d, Ls, graphed, f64, stream=st)
    for _ in range(2):
        for v in graphed.values():
            v.zero_()
        g.replay()
        torch.cuda.synchronize()
        for f in FIELDS:
            assert torch.equal(graphed[f], direct[f]), f


@pytest.mark.parametrize("which", [0, 2])
def test_grid_batch_mixing_on_chip_and_four_step_sizes(ctxs, which):
    """One batched launch whose grids are partly small enough for the on-chip
    FFT kernel and partly larger (the four-step kernels: L above 16384 points
    in FP32, 8192 in FP64), with two equal large instances whose s'' shares a
    transform; every instance against the dense oracle at sampled points."""
    import torch
    from paper_1705_06073_gb300 import lse
    f64 = which == 0
    specs = [(200, 4, 512), (1000, 8, 32768), (1000, 6, 32768), (300, 5, 65536), (2000, 12, 16384), (64, 2, 128)]
    ys, ths, gas, bes = [], [], [], []
    for i, (N, K, L) in enumerate(specs):
        y, th, ga, be = state(N, K, 3300 + i)
        ys.append(y); ths.append(th); gas.append(ga); bes.append(be)
    yo = np.concatenate([[0], np.cumsum([len(y) for y in ys])])
    ko = np.concatenate([[0], np.cumsum([len(t) for t in ths])])
    Ls = np.array([s[2] for s in specs], np.int32)
    dev = torch.device("cuda:0")
    y_d = torch.from_numpy(np.concatenate(ys)).to(dev)
    th_d = torch.from_numpy(np.concatenate(ths + [np.zeros(1)])).to(dev)
    ga_d = torch.from_numpy(np.concatenate(gas + [np.zeros(1)])).to(dev)
    be_d = torch.tensor(bes, dtype=torch.float64, device=dev)
    G = int(Ls.sum())
    ct, rt = (torch.complex128, torch.float64) if f64 else (torch.complex64, torch.float32)
    outs = {f: torch.zeros(G, dtype=ct if f in ("q", "dq", "d2q") else rt, device=dev) for f in FIELDS}
    lse.lse_eval_grid_batch_d(ctxs[which], y_d, yo, th_d, ga_d, ko, be_d, Ls, outs, f64)
    torch.cuda.synchronize()
    g0 = 0
    r = np.random.default_rng(77)
    for i, (N, K, L) in enumerate(specs):
        pts = np.unique(np.concatenate([r.integers(0, L, 150), np.mod(np.round(ths[i] * L).astype(int), L)]))
        ref = dn.DenseEval(ys[i], ths[i], gas[i], bes[i]).grid(L, derivatives=True, points=pts / L)
        got = {f: outs[f][g0:g0 + L].cpu().numpy()[pts] for f in FIELDS}
        err = grid_errors(got, ref, N)
        assert max(err.values()) < (1e-8 if f64 else 1e-4), (i, err)
        g0 += L


@pytest.mark.parametrize("prec", ["mixed_df", "fp64", "mixed"])
def test_grid_superfast_pair_matches_one_block(prec):
    """A launch whose instances all take the superfast recursion runs on
    two-block clusters (every precision path): the second block takes
    half of every pass of the recursion's global-memory FFT stages, its
    refinement, the Gohberg-Semencul apply and the omega_s transforms.  Each
    butterfly is computed as by one block, so the grid outputs equal those of
    the one-block launch bit for bit (ragged N and L, twice in a row), and
    they meet the grid bound of the path against the oracle."""
    import torch
    from paper_1705_06073_gb300 import build, lse
    build.build()
    specs = [(1200, 10, 4096), (4096, 32, 16384), (300, 4, 1024), (2049, 16, 8192)]
    ys, ths, gas, bes = [], [], [], []
    for i, (N, K, L) in enumerate(specs):
        y, th, ga, be = state(N, K, 3100 + i)
        ys.append(y); ths.append(th); gas.append(ga); bes.append(be)
    yo = np.concatenate([[0], np.cumsum([len(y) for y in ys])])
    ko = np.concatenate([[0], np.cumsum([len(t) for t in ths])])
    Ls = np.array([s[2] for s in specs], np.int32)
    dev = torch.device("cuda:0")
    y_d = torch.from_numpy(np.concatenate(ys)).to(dev)
    th_d = torch.from_numpy(np.concatenate(ths)).to(dev)
    ga_d = torch.from_numpy(np.concatenate(gas)).to(dev)
    be_d = torch.tensor(bes, dtype=torch.float64, device=dev)
    G = int(Ls.sum())
    f64 = prec == "fp64"  # an FP64 context writes FP64 spectra, the others FP32
    ct, rt = (torch.complex128, torch.float64) if f64 else (torch.complex64, torch.float32)
    precision = {"mixed_df": lse.LSE_PREC_MIXED_DF, "fp64": lse.LSE_PREC_FP64, "mixed": lse.LSE_PREC_MIXED}[prec]
    res = {}
    for flags in (0, lse.LSE_FLAG_NO_CLUSTER):
        ctx = lse.lse_create(lse.lse_config_default(precision=precision, flags=flags))
        try:
            runs = []
            for _ in range(2):
                outs = {f: torch.zeros(G, dtype=ct if f in ("q", "dq", "d2q") else rt, device=dev) for f in FIELDS}
                lse.lse_eval_grid_batch_d(ctx, y_d, yo, th_d, ga_d, ko, be_d, Ls, outs, f64=f64)
                torch.cuda.synchronize()
                runs.append({f: outs[f].cpu().numpy() for f in FIELDS})
            res[flags] = runs
        finally:
            lse.lse_destroy(ctx)
    for run in res[0]:
        for f in FIELDS:
            assert np.array_equal(run[f], res[lse.LSE_FLAG_NO_CLUSTER][0][f]), f
    # and the paired launch still meets the oracle at the smallest instance
    ref = dn.DenseEval(ys[2], ths[2], gas[2], bes[2]).grid(int(Ls[2]), derivatives=True)
    g0 = int(Ls[0] + Ls[1])
    got = {f: res[0][0][f][g0:g0 + Ls[2]] for f in FIELDS}
    err = grid_errors(got, ref, specs[2][0])
    assert max(err.values()) < (1e-8 if f64 else 1e-4), err
