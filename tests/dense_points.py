"""Dense-oracle grid values at sampled points for a large instance, run as a
separate process so that the O(N^3) Cholesky can use every host core (the
test process keeps BLAS single-threaded).

    python -m tests.dense_points N K L SNR SEED OUT.npz

The instance is the seeded synthetic one (|alpha| log-uniform over 30 dB,
separation 2/N) and the state is its true one: theta, gamma = |alpha|^2,
beta.  The sampled grid points are 32 pseudo-random ones and the grid points
nearest the 32 strongest components (deep nulls of s).  Writes the points'
indices and the oracle's q, s and their theta-derivatives there.
"""
import os
import sys

import numpy as np


def sample_points(theta, gamma, L, seed):
    r = np.random.default_rng(seed)
    strong = np.argsort(-np.asarray(gamma))[:32]
    near = np.mod(np.round(np.asarray(theta)[strong] * L).astype(np.int64), L)
    rand = r.integers(0, L, 32)
    return np.unique(np.concatenate([near, rand]))


def main(argv):
    N, K, L = (int(a) for a in argv[:3])
    snr, seed, out = float(argv[3]), int(argv[4]), argv[5]
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    from oracle import dense
    from paper_1705_06073_gb300 import synth
    inst = synth.make_instance(N, K, snr, seed, law="loguniform30")
    gamma = np.abs(inst.alpha) ** 2
    pts = sample_points(inst.theta, gamma, L, seed)
    ev = dense.DenseEval(inst.y, inst.theta, gamma, inst.beta)
    g = ev.grid(L, derivatives=True, points=pts / L)
    np.savez(out, points=pts, **g)


if __name__ == "__main__":
    main(sys.argv[1:])
