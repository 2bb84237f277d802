"""CPU checks of the mathematics the GPU's non-uniform FFT sums rely on
(csrc/lse_nufft.cuh), independent of its code: the Kaiser-Bessel
window/transform pair against numerical quadrature, and the error of the
type-2 scheme built from them (width 16, M >= 2N, the Beatty et al. beta)
against the direct sums, written out here in numpy."""
import numpy as np
import pytest
from scipy import integrate, special

W = 16


def beta_of(N, M):
    sg = M / N
    return np.pi * np.sqrt(W * W * (sg - 0.5) ** 2 / sg ** 2 - 0.8)


def kb(t, beta):
    return special.i0(beta * np.sqrt(np.maximum(0.0, 1.0 - (2.0 * t / W) ** 2)))


def kb_transform(nu, M, beta):
    """int psi(u) e^{j 2 pi nu u} du for psi(u) = kb(u M): (W/M) sinh(r)/r."""
    a = np.pi * W * nu / M
    r = np.sqrt(beta * beta - a * a)
    return W / M * np.sinh(r) / r


@pytest.mark.parametrize("N,M", [(64, 128), (1000, 2048), (4096, 8192), (300, 1024)])
def test_kaiser_bessel_transform_pair(N, M):
    beta = beta_of(N, M)
    for nu in (0, 1, N // 4, N // 2, -N // 2):
        ref, _ = integrate.quad(lambda u: kb(u * M, beta) * np.cos(2 * np.pi * nu * u), -W / (2 * M), W / (2 * M),
                                limit=400, epsabs=0, epsrel=1e-13)
        assert abs(kb_transform(nu, M, beta) - ref) <= 1e-11 * abs(ref)


def nufft_sums(f, thetas):
    """The scheme of lse_nufft.cuh in numpy (FP64)."""
    N = len(f)
    M = 1 << int(np.ceil(np.log2(2 * N)))
    n0 = N // 2
    beta = beta_of(N, M)
    npr = np.arange(N) - n0
    a = np.pi * W * npr / M
    r = np.sqrt(beta * beta - a * a)
    c = special.i0(beta) * r / np.sinh(r)  # the stored deconvolution factors
    g = np.zeros(M, complex)
    g[npr % M] = f * c
    F = np.fft.fft(g)
    out = []
    for th in thetas:
        x = th * M
        m0 = int(np.floor(x - W / 2)) + 1
        ms = np.arange(m0, m0 + W)
        w = kb(x - ms, beta) / (W * special.i0(beta))
        out.append(np.exp(-2j * np.pi * n0 * th) * np.sum(F[ms % M] * w))
    return np.array(out)


@pytest.mark.parametrize("N", [64, 333, 1000, 4096])
def test_type2_scheme_matches_direct_sums(N):
    r = np.random.default_rng(N)
    f = r.standard_normal(N) + 1j * r.standard_normal(N)
    th = np.concatenate([r.random(40), [0.0, 1 - 2 ** -40, 0.5, 1.0 / 3.0]])
    ref = np.exp(-2j * np.pi * np.outer(th, np.arange(N))) @ f
    got = nufft_sums(f, th)
    assert np.abs(got - ref).max() <= 1e-13 * np.abs(f).sum()
