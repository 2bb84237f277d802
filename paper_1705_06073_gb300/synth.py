"""Seeded synthetic inputs shaped like the paper's experiments (Sec. VI-A).

This module holds only the data model of eq. (model) -- sums of complex
sinusoids plus white circular Gaussian noise -- and the random draws that
build them.  It contains none of the estimator's arithmetic, so both the
CUDA path and the CPU oracle may use it.

Random numbers come from a counter-based generator: SplitMix64 (Steele, Lea,
Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014) maps a
64-bit counter to a 64-bit output; uniforms take its top 53 bits, and complex
normals use the Box-Muller transform.  Every instance owns one seed and its
draws are taken from consecutive counter values, so an instance is
reproducible on its own, independent of batch composition.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, counters: np.ndarray) -> np.ndarray:
    """SplitMix64 output for ``seed`` at each counter value (uint64 array)."""
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + (counters.astype(np.uint64) + np.uint64(1)) * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


class Stream:
    """Sequential draws from one seed: uniforms on [0,1) and CN(0,1) normals."""

    def __init__(self, seed: int):
        self.seed = int(seed)
        self.counter = 0

    def uniform(self, n: int) -> np.ndarray:
        c = np.arange(self.counter, self.counter + n, dtype=np.uint64)
        self.counter += n
        return (splitmix64(self.seed, c) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)

    def cnormal(self, n: int) -> np.ndarray:
        """Circularly-symmetric complex normals with unit variance (E|z|^2 = 1)."""
        u = self.uniform(2 * n)
        u1, u2 = u[0::2], u[1::2]
        r = np.sqrt(-np.log1p(-u1))  # sqrt(-2 ln(1-u)) / sqrt(2)
        return r * np.exp(2j * np.pi * u2)


def wrap_distance(a, b):
    """Wrap-around distance on [0,1): d(x,y) = min(|x-y|, 1-|x-y|) (Sec. II-E footnote)."""
    d = np.abs(np.asarray(a, dtype=np.float64) - np.asarray(b, dtype=np.float64)) % 1.0
    return np.minimum(d, 1.0 - d)


def draw_frequencies(stream: Stream, K: int, min_sep: float) -> np.ndarray:
    """Frequencies drawn one after another, each uniform on the part of [0,1)
    farther than ``min_sep`` from all earlier ones (Sec. VI-A), by rejection."""
    out: list[float] = []
    tries = 0
    while len(out) < K:
        u = float(stream.uniform(1)[0])
        tries += 1
        if tries > 10000 * (K + 1):
            raise RuntimeError("cannot place frequencies with this separation")
        if out and np.min(wrap_distance(u, np.asarray(out))) <= min_sep:
            continue
        out.append(u)
    return np.asarray(out)


def draw_amplitudes(stream: Stream, K: int, law: str) -> np.ndarray:
    if law == "cn":  # alpha ~ CN(0, 1)
        return stream.cnormal(K)
    if law == "paper":  # a ~ CN with std 0.8, alpha = a + 0.2 e^{j arg a} (Sec. VI-A)
        a = 0.8 * stream.cnormal(K)
        return a + 0.2 * np.exp(1j * np.angle(a))
    if law.startswith("loguniform"):  # |alpha| log-uniform over a dB range, uniform phase
        rng_db = float(law[len("loguniform"):] or 30.0)
        u = stream.uniform(2 * K)
        mag = 10.0 ** (-u[0::2] * rng_db / 20.0)
        return mag * np.exp(2j * np.pi * u[1::2])
    raise ValueError(law)


@dataclasses.dataclass
class Instance:
    y: np.ndarray  # complex64 [N]
    theta: np.ndarray  # true frequencies
    alpha: np.ndarray  # true coefficients
    beta: float  # true noise variance
    snr_db: float
    seed: int

    @property
    def N(self) -> int:
        return int(self.y.shape[0])


def sum_of_sinusoids(N: int, theta: np.ndarray, alpha: np.ndarray) -> np.ndarray:
    """h_n = sum_k alpha_k exp(j 2 pi theta_k n), n = 0..N-1.  With n = 64 a + b
    the phase splits into two small tables, so h is one (N/64 x K)(K x 64)
    matrix product instead of N K complex exponentials."""
    if len(theta) == 0:
        return np.zeros(N, complex)
    Bn = 64
    A = (N + Bn - 1) // Bn
    t1 = np.exp(2j * np.pi * np.outer(theta, np.arange(A, dtype=np.float64) * Bn)) * alpha[:, None]
    t2 = np.exp(2j * np.pi * np.outer(theta, np.arange(Bn, dtype=np.float64)))
    return (t1.T @ t2).reshape(-1)[:N]


def make_instance(N: int, K: int, snr_db: float, seed: int, *, law: str = "cn",
                  min_sep: float | None = None, noise: bool = True) -> Instance:
    """y = sum_k alpha_k e^{j 2 pi theta_k n} + w, n = 0..N-1 (eq. model, Phi = I).

    The noise variance is set from SNR = ||Psi alpha||^2 / (N beta) (Sec. VI-A).
    """
    st = Stream(seed)
    sep = (2.0 / N) if min_sep is None else min_sep
    theta = draw_frequencies(st, K, sep)
    alpha = draw_amplitudes(st, K, law)
    h = sum_of_sinusoids(N, theta, alpha)
    beta = float(np.vdot(h, h).real / (N * 10.0 ** (snr_db / 10.0))) if K else 1.0
    w = math.sqrt(beta) * st.cnormal(N) if noise else 0.0
    y = (h + w).astype(np.complex64)
    return Instance(y=y, theta=theta, alpha=alpha, beta=beta, snr_db=snr_db, seed=seed)


@dataclasses.dataclass
class MMVInstance:
    Y: np.ndarray  # complex64 [G, N]: snapshot g is Y[g] (snapshot-major, as the C ABI)
    theta: np.ndarray  # true frequencies, shared by the snapshots
    alpha: np.ndarray  # true coefficients [G, K]
    beta: float  # true noise variance
    snr_db: float
    seed: int

    @property
    def N(self) -> int:
        return int(self.Y.shape[1])

    @property
    def G(self) -> int:
        return int(self.Y.shape[0])


def make_mmv_instance(N: int, K: int, G: int, snr_db: float, seed: int, *, law: str = "cn",
                      min_sep: float | None = None) -> MMVInstance:
    """y^(g) = sum_k alpha_k^(g) e^{j 2 pi theta_k n} + w^(g), g = 1..G (the
    multiple-measurement-vector model of Sec. V): the frequencies are shared,
    each snapshot draws its own coefficients and noise.  The noise variance
    is set from the mean per-snapshot SNR, sum_g ||Psi alpha^(g)||^2 / (G N beta)."""
    st = Stream(seed)
    sep = (2.0 / N) if min_sep is None else min_sep
    theta = draw_frequencies(st, K, sep)
    alpha = np.stack([draw_amplitudes(st, K, law) for _ in range(G)])
    H = np.stack([sum_of_sinusoids(N, theta, alpha[g]) for g in range(G)])
    beta = float(np.sum(np.abs(H) ** 2) / (G * N * 10.0 ** (snr_db / 10.0))) if K else 1.0
    W = np.stack([math.sqrt(beta) * st.cnormal(N) for _ in range(G)])
    return MMVInstance(Y=(H + W).astype(np.complex64), theta=theta, alpha=alpha, beta=beta,
                       snr_db=snr_db, seed=seed)


@dataclasses.dataclass
class IncompleteInstance:
    y: np.ndarray  # complex64 [M]: the observed samples
    obs: np.ndarray  # int32 [M]: their indices n_m in [0, N), ascending
    N: int
    theta: np.ndarray
    alpha: np.ndarray
    beta: float
    snr_db: float
    seed: int


def draw_subset(stream: Stream, N: int, M: int) -> np.ndarray:
    """M of the indices 0..N-1 uniformly without replacement (a partial
    Fisher-Yates shuffle driven by the stream), ascending."""
    idx = np.arange(N)
    u = stream.uniform(M)
    for i in range(M):
        j = i + int(u[i] * (N - i))
        idx[i], idx[j] = idx[j], idx[i]
    return np.sort(idx[:M]).astype(np.int32)


def make_incomplete_instance(N: int, M: int, K: int, snr_db: float, seed: int, *, law: str = "cn",
                             min_sep: float | None = None) -> IncompleteInstance:
    """The model of eq. (model) observed at M of its N samples (Phi a row
    selection, Sec. IV): the signal and noise as make_instance, the SNR over
    the observed samples, ||Phi Psi alpha||^2 / (M beta)."""
    st = Stream(seed)
    sep = (2.0 / N) if min_sep is None else min_sep
    theta = draw_frequencies(st, K, sep)
    alpha = draw_amplitudes(st, K, law)
    obs = draw_subset(st, N, M)
    h = sum_of_sinusoids(N, theta, alpha)[obs]
    beta = float(np.vdot(h, h).real / (M * 10.0 ** (snr_db / 10.0))) if K else 1.0
    y = (h + math.sqrt(beta) * st.cnormal(M)).astype(np.complex64)
    return IncompleteInstance(y=y, obs=obs, N=N, theta=theta, alpha=alpha, beta=beta, snr_db=snr_db, seed=seed)


def default_grid_size(N: int) -> int:
    """L = 8N rounded to the nearest power of two (Sec. II-D footnote)."""
    return 1 << int(round(math.log2(8 * N)))


# ----------------------------------------------------------------------------
# The workloads: each returns a list of (Instance, L).
# ----------------------------------------------------------------------------

def single_n256(seed: int = 101):
    """One instance, N=256, K=8, separation 2/N, alpha ~ CN(0,1), 20 dB, L=8N."""
    return [(make_instance(256, 8, 20.0, seed), 2048)]


def batch64_n4096(seed0: int = 201, B: int = 64):
    """B instances, N=4096, K=64, SNR uniform on [10,30] dB per instance, L=4N."""
    out = []
    for i in range(B):
        snr = 10.0 + 20.0 * float(Stream(seed0 + i + 7919 * 1000003).uniform(1)[0])
        out.append((make_instance(4096, 64, snr, seed0 + i), 16384))
    return out


def single_n65536(seed: int = 301):
    """One instance, N=65536, K=512, separation 1.5/N, |alpha| log-uniform over
    30 dB, 15 dB SNR, L=2N."""
    N = 65536
    return [(make_instance(N, 512, 15.0, seed, law="loguniform30", min_sep=1.5 / N), 2 * N)]


def ragged1024(seed0: int = 401, B: int = 1024):
    """B instances, N uniform on [128, 8192], K = max(1, N // 64), SNR uniform
    on [0,30] dB, L = 8N rounded to the nearest power of two."""
    out = []
    for i in range(B):
        u = Stream(seed0 + i + 7919 * 1000003).uniform(2)
        N = 128 + int(u[0] * (8192 - 128 + 1))
        K = max(1, N // 64)
        out.append((make_instance(N, K, 30.0 * float(u[1]), seed0 + i), default_grid_size(N)))
    return out


def serving_stream(rate_hz: float = 2000.0, duration_s: float = 60.0, seed: int = 501,
                   n_max: int | None = None):
    """Poisson arrivals; each request N log-uniform on [256, 32768], K uniform on
    [4, N/32], SNR uniform on [5,25] dB.  Returns (arrival times, request specs);
    the instances themselves are built lazily by ``make_request``."""
    st = Stream(seed)
    t = 0.0
    times, specs = [], []
    while True:
        t += -math.log1p(-float(st.uniform(1)[0])) / rate_hz
        if t >= duration_s or (n_max is not None and len(times) >= n_max):
            break
        u = st.uniform(3)
        N = int(round(2.0 ** (8.0 + 7.0 * float(u[0]))))
        K = 4 + int(u[1] * (N // 32 - 4 + 1))
        times.append(t)
        specs.append((N, K, 5.0 + 20.0 * float(u[2]), seed * 1000003 + len(times)))
    return np.asarray(times), specs


def make_request(spec):
    N, K, snr, s = spec
    return make_instance(N, K, snr, s), default_grid_size(N)


def paper_accuracy_n128(trial: int, seed0: int = 601):
    """N=128, K=10, 20 dB, the paper's amplitude law (Sec. VI-A, Fig. 2)."""
    return make_instance(128, 10, 20.0, seed0 + trial, law="paper"), 1024


def mmv_batch(seed0: int = 701, B: int = 64, N: int = 1024, G: int = 8, K: int = 32):
    """B multiple-measurement-vector instances (Sec. V): N = 1024 samples, G = 8
    snapshots sharing K = 32 frequencies (separation 2/N, alpha ~ CN(0,1) per
    snapshot), SNR uniform on [0, 20] dB per instance, L = 8N."""
    out = []
    for i in range(B):
        snr = 20.0 * float(Stream(seed0 + i + 7919 * 1000003).uniform(1)[0])
        out.append((make_mmv_instance(N, K, G, snr, seed0 + i), default_grid_size(N)))
    return out


def incomplete_batch(seed0: int = 801, B: int = 64, N: int = 4096, M: int = 3072, K: int = 16):
    """B instances observed at M = 3N/4 of N = 4096 samples (the paper's
    incomplete-data setting, Sec. VI: a random subset, K = 16, 20 dB),
    L = 4N."""
    return [(make_incomplete_instance(N, M, K, 20.0, seed0 + i), 4 * N) for i in range(B)]
