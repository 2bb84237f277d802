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
