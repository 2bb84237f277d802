"""Helpers shared by the GPU parity tests."""
import numpy as np


def wrapdist(a, b):
    d = np.abs(np.asarray(a) - np.asarray(b)) % 1.0
    return np.minimum(d, 1.0 - d)


def rel_inf(got, ref, floor=0.0):
    """Normwise relative error ||got - ref||_inf / max(||ref||_inf, floor)."""
    got = np.asarray(got)
    ref = np.asarray(ref)
    den = max(float(np.abs(ref).max()), floor)
    return float(np.abs(got - ref).max() / (den if den > 0 else 1.0))


def grid_errors(got, ref, N):
    """Normwise errors of the six grid outputs.  A theta-derivative of order k
    is measured against max(||ref||, (2 pi N)^k ||f||) with f its undifferentiated
    function: when the exact derivative vanishes (e.g. s' with no active
    component) the reference is rounding noise and the natural scale of a
    k-th derivative of a degree-N trigonometric polynomial is the bound."""
    w = 2 * np.pi * N
    out = {}
    for f, base, k in (("q", "q", 0), ("dq", "q", 1), ("d2q", "q", 2), ("s", "s", 0), ("ds", "s", 1), ("d2s", "s", 2)):
        if f in got:
            out[f] = rel_inf(got[f], ref[f], floor=1e-3 * w ** k * float(np.abs(ref[base]).max()) if k else 0.0)
    return out


def match_fit(gpu, ref):
    """Compare a GPU fit with the oracle's: equal K and matched frequencies.
    Both return components sorted by frequency; the match is by sorted order
    after checking that the cyclic shift with the smallest distance is 0."""
    assert gpu["K"] == ref.K, (gpu["K"], ref.K)
    if ref.K == 0:
        return 0.0
    d = wrapdist(gpu["theta"], ref.theta)
    return float(d.max())


def s_fp32_bound(ev, L):
    """Pointwise error bound of an FP32 grid s (the reading of the 1e-4 bar on
    the FP32-grid paths): s(theta) = sum_{|i|<N} w(i) e^{j 2 pi i theta} with
    w(i) = sum_{q-p=i} [C^{-1}]_{pq} (the lag sums of C^{-1}, App. B), and a
    length-L FFT in FP32 gives each output to within about
    (log2 L + 3) rounding errors of the running sums, each at most
    u32 * sum_i |w(i)| (a complex operation contributes up to ~4 u32).  So
    |s_gpu(l) - s(l)| <= 1e-4 s(l) + 4 (log2 L + 3) 2^-24 ||w||_1.
    Returns the second term; ev is the oracle's DenseEval."""
    Cinv = ev.solve(np.eye(ev.N, dtype=complex))
    w1 = sum(abs(np.trace(Cinv, offset=i)) for i in range(-(ev.N - 1), ev.N))
    return 4.0 * (np.log2(L) + 3.0) * 2.0 ** -24 * w1
