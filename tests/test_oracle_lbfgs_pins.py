"""Pins of the oracle's L-BFGS update (Sec. II-C1, readings L1-L4 in
oracle/fit.py) against facts that do not come from it: the dense BFGS
inverse-Hessian formula, the secant condition, the diagonal Newton step when
nothing is saved, the memory rules, and whole fits (objective never rises,
noise-free recovery, the same optimum as the Newton update)."""
import numpy as np

from oracle import fit as of
from paper_1705_06073_gb300 import synth


def dense_bfgs_inverse(h, S, Y):
    """H_0 = diag(1/h); H <- (I - rho s y^T) H (I - rho y s^T) + rho s s^T for
    each pair, oldest first (Nocedal and Wright, eq. 6.17), as a matrix."""
    n = len(h)
    H = np.diag(1.0 / np.asarray(h, float))
    I = np.eye(n)
    for s, y in zip(S, Y):
        rho = 1.0 / np.dot(y, s)
        H = (I - rho * np.outer(s, y)) @ H @ (I - rho * np.outer(y, s)) + rho * np.outer(s, s)
    return H


def random_pairs(n, m, seed):
    r = np.random.default_rng(seed)
    A = r.standard_normal((n, n))
    A = A @ A.T + n * np.eye(n)  # a positive definite Hessian gives s.y > 0
    S = [r.standard_normal(n) for _ in range(m)]
    Y = [A @ s for s in S]
    return S, Y, r.standard_normal(n), 0.5 + r.random(n)


def test_two_loop_recursion_is_the_dense_bfgs_inverse():
    for n, m, seed in ((6, 3, 1), (10, 10, 2), (4, 1, 3)):
        S, Y, g, h = random_pairs(n, m, seed)
        d = of.lbfgs_direction(g, h, S, Y)
        ref = -dense_bfgs_inverse(h, S, Y) @ g
        assert np.allclose(d, ref, rtol=1e-10, atol=1e-12 * np.abs(ref).max())


def test_secant_condition_holds_for_the_newest_pair():
    S, Y, _g, h = random_pairs(7, 4, 5)
    # H y_last = s_last: the direction for g = -y_last is s_last
    d = of.lbfgs_direction(-Y[-1], h, S, Y)
    assert np.allclose(d, S[-1], rtol=1e-10)


def test_no_saved_pair_is_the_diagonal_newton_step():
    g = np.array([1.0, -2.0, 0.5])
    h = np.array([4.0, 0.5, 2.0])
    assert np.array_equal(of.lbfgs_direction(g, h, [], []), -g / h)


def test_memory_keeps_curvature_pairs_only_and_at_most_J():
    mem = of.LbfgsMemory(J=3)
    g0 = np.zeros(2)
    for i in range(5):
        mem.pending = (np.array([1.0, 0.0]), g0)
        mem.absorb(np.array([1.0 + i, 0.0]))  # s.y = 1 + i > 0
    assert len(mem.S) == 3 and mem.Y[0][0] == 3.0 and mem.Y[-1][0] == 5.0
    mem.pending = (np.array([1.0, 0.0]), g0)
    mem.absorb(np.array([-1.0, 0.0]))  # s.y < 0: dropped
    assert len(mem.S) == 3 and mem.pending is None
    mem.reset()
    assert mem.S == [] and mem.Y == [] and mem.pending is None


def test_lbfgs_fit_objective_never_increases():
    inst, L = synth.single_n256()[0]
    r = of.fit(inst.y, L, trace=True, update="lbfgs")
    obj = np.array([o for _, o in r.trace])
    assert np.all(np.diff(obj) <= 1e-9 * np.abs(obj[:-1]).max())
    assert r.converged and r.K == 8


def test_lbfgs_fit_recovers_noise_free_frequencies_and_matches_newton():
    inst = synth.make_instance(64, 3, 80.0, 7, min_sep=4 / 64)
    r = of.fit(inst.y, 512, update="lbfgs")
    assert r.K == 3
    assert np.all(synth.wrap_distance(np.sort(inst.theta), r.theta) < 1e-6)
    for N, K, snr, seed in ((128, 10, 20.0, 12), (100, 5, 15.0, 14)):
        inst = synth.make_instance(N, K, snr, seed)
        a = of.fit(inst.y, 4 * N)
        b = of.fit(inst.y, 4 * N, update="lbfgs")
        assert a.K == b.K
        assert np.max(synth.wrap_distance(a.theta, b.theta)) < 1e-6
        assert abs(a.objective - b.objective) < 1e-6 * abs(a.objective)
