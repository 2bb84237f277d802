"""Pins of the incomplete-observation oracle (oracle/incomplete.py) against
facts that do not come from it: the semifast identities of Sec. IV (Woodbury
for C^-1, the matrix determinant lemma for ln|C|, the K x K forms of the
vectors and of the grid s), finite differences of the dense objective, the
complete-data oracle when every sample is observed, and noise-free
recovery from a subset of the samples."""
import numpy as np
import pytest

from oracle import dense as dn
from oracle import fit as of
from oracle import incomplete as oi
from paper_1705_06073_gb300 import synth


def rand_state(N, M, K, seed, beta=0.1, gmax=2.0):
    r = np.random.default_rng(seed)
    obs = np.sort(r.choice(N, M, replace=False))
    theta = r.random(K)
    gamma = 0.1 + gmax * r.random(K)
    y = r.standard_normal(M) + 1j * r.standard_normal(M)
    return y, obs, theta, gamma, beta


def semifast_forms(y, obs, N, theta, gamma, beta):
    """Sec. IV written out: Sigma^-1 = A^H A / beta + Gamma^-1 = L L^H,
    C^-1 = I/beta - A Sigma A^H / beta^2, and every quantity through K x K
    matrices (G_a = A_{D^a}^H A) and h_a = A_{D^a}^H y."""
    A = dn.steering(N, theta)[obs]
    d = 2 * np.pi * obs.astype(float)
    M = len(obs)
    G0 = A.conj().T @ A
    G1 = (d[:, None] * A).conj().T @ A
    G2 = (d[:, None] ** 2 * A).conj().T @ A
    h0 = A.conj().T @ y
    h1 = (d[:, None] * A).conj().T @ y
    h2 = (d[:, None] ** 2 * A).conj().T @ y
    Sinv = G0 / beta + np.diag(1 / gamma)
    Lc = np.linalg.cholesky(Sinv)
    Li = np.linalg.inv(Lc)
    Sh = np.linalg.solve(Sinv, h0)
    Z0, Z1, Z2 = Li @ G0, Li @ G1.conj().T, Li @ G2.conj().T
    out = dict(
        logdet=M * np.log(beta) + np.sum(np.log(gamma)) + 2 * np.sum(np.log(np.diag(Lc).real)),
        yCy=(np.vdot(y, y).real - np.vdot(h0, Sh).real / beta) / beta,
        q=(h0 - G0 @ Sh / beta) / beta, r=(h1 - G1 @ Sh / beta) / beta, u=(h2 - G2 @ Sh / beta) / beta,
        s=(np.diag(G0).real - np.sum(np.abs(Z0) ** 2, axis=0) / beta) / beta,
        t=(np.diag(G1) - np.sum(Z1.conj() * Z0, axis=0) / beta) / beta,
        v=(np.diag(G2) - np.sum(Z2.conj() * Z0, axis=0) / beta) / beta,
        x=(np.diag(G2).real - np.sum(np.abs(Z1) ** 2, axis=0) / beta) / beta)
    return out, A, Lc, Sh


def test_semifast_identities_reproduce_the_dense_oracle():
    N, M, K = 48, 36, 4
    y, obs, th, g, b = rand_state(N, M, K, 3)
    ev = oi.IncompleteDenseEval(y, obs, N, th, g, b)
    ref, A, Lc, Sh = semifast_forms(y, obs, N, th, g, b)
    assert abs(ev.logdet - ref["logdet"]) < 1e-10 * abs(ref["logdet"])
    assert abs(ev.yCy - ref["yCy"]) < 1e-10 * abs(ref["yCy"])
    vec = ev.active_vectors()
    for k in "qrsuvtx":
        assert np.allclose(vec[k], ref[k], rtol=1e-9, atol=1e-9 * np.abs(ref[k]).max()), k
    # grid: q = A(theta_l)^H C^-1 y, s = M/beta - ||L^-1 b_l||^2 / beta^2 with b_l = A^H a(theta_l)
    L = 128
    gr = ev.grid(L)
    P = dn.steering(N, np.arange(L) / L)[obs]
    x = (y - A @ Sh / b) / b
    assert np.allclose(gr["q"], P.conj().T @ x, rtol=0, atol=1e-10 * np.abs(gr["q"]).max())
    Bm = A.conj().T @ P
    s_ref = M / b - np.sum(np.abs(np.linalg.solve(Lc, Bm)) ** 2, axis=0) / b ** 2
    assert np.allclose(gr["s"], s_ref, rtol=1e-9)


def test_every_sample_observed_is_the_complete_oracle():
    for N, K, snr, seed in ((64, 3, 25.0, 21), (80, 4, 12.0, 22)):
        inst = synth.make_instance(N, K, snr, seed)
        a = of.fit(inst.y, 4 * N)
        b = oi.fit(inst.y, np.arange(N), N, 4 * N)
        assert a.K == b.K and a.n_evals == b.n_evals and a.iters == b.iters
        assert np.max(synth.wrap_distance(a.theta, b.theta)) < 1e-12
        assert np.allclose(a.gamma, b.gamma, rtol=1e-10) and abs(a.beta - b.beta) < 1e-10 * a.beta


def test_derivatives_match_finite_differences():
    N, M = 40, 30
    y, obs, _th, g, b = rand_state(N, M, 3, 5, beta=0.3, gmax=1.0)
    th = np.array([0.13, 0.5, 0.77])
    ev = oi.IncompleteDenseEval(y, obs, N, th, g, b)
    gt, gg, ht, hg = dn.derivatives(ev.active_vectors(), g, N)

    def d12(fun, h):
        f = [fun(j * h) for j in (-2, -1, 0, 1, 2)]
        return ((f[0] - 8 * f[1] + 8 * f[3] - f[4]) / (12 * h),
                (-f[0] + 16 * f[1] - 30 * f[2] + 16 * f[3] - f[4]) / (12 * h * h))
    for k in range(3):
        e = np.zeros(3)
        e[k] = 1.0
        d1, d2 = d12(lambda dt: oi.IncompleteDenseEval(y, obs, N, th + dt * e, g, b).data_term(), 3e-5)
        assert abs(d1 - gt[k]) < 1e-7 * max(1, abs(gt[k]))
        assert abs(d2 - ht[k]) < 1e-5 * max(1, abs(ht[k]))
        d1, d2 = d12(lambda dg: oi.IncompleteDenseEval(y, obs, N, th, g + dg * e, b).data_term(), 1e-3 * g[k])
        assert abs(d1 - gg[k]) < 1e-7 * max(1, abs(gg[k]))
        assert abs(d2 - hg[k]) < 1e-5 * max(1, abs(hg[k]))


def test_grid_derivatives_match_finite_differences():
    N, M = 30, 21
    y, obs, th, g, b = rand_state(N, M, 2, 7)
    ev = oi.IncompleteDenseEval(y, obs, N, th, g, b)
    pts = np.array([0.07, 0.33, 0.62, 0.91])
    h = 1e-5
    c = ev.grid(0, derivatives=True, points=pts)
    p = ev.grid(0, derivatives=True, points=pts + h)
    m = ev.grid(0, derivatives=True, points=pts - h)
    for f, df in (("q", "dq"), ("s", "ds"), ("dq", "d2q"), ("ds", "d2s")):
        fd = (p[f] - m[f]) / (2 * h)
        assert np.all(np.abs(fd - c[df]) < 1e-6 * np.abs(c[df]).max()), f


def test_delta_objective_and_deactivation_are_dense_changes():
    N, M = 36, 27
    y, obs, th, g, b = rand_state(N, M, 3, 9)
    ev = oi.IncompleteDenseEval(y, obs, N, th, g, b)
    zeta = 0.2
    pts = np.array([0.21, 0.58])
    gr = ev.grid(0, points=pts)
    dl = dn.delta_objective(gr["q"], gr["s"], g.mean(), zeta)
    for i, t in enumerate(pts):
        ev2 = oi.IncompleteDenseEval(y, obs, N, np.append(th, t), np.append(g, g.mean()), b)
        ref = ev2.objective(zeta) - ev.objective(zeta)
        assert abs(dl[i] - ref) < 1e-9 * max(1, abs(ref))
    vec = ev.active_vectors()
    stat = dn.deactivation_statistic(vec["q"], vec["s"], g)
    for k in range(3):
        keep = np.arange(3) != k
        evk = oi.IncompleteDenseEval(y, obs, N, th[keep], g[keep], b)
        assert abs(stat[k] - (evk.data_term() - ev.data_term())) < 1e-9 * max(1, abs(stat[k]))


def test_beta_update_against_the_explicit_posterior():
    N, M = 32, 24
    y, obs, th, g, b = rand_state(N, M, 3, 11)
    ev = oi.IncompleteDenseEval(y, obs, N, th, g, b)
    new = oi.beta_update(ev, ev.active_vectors()["s"], 1e-12)
    A = ev.A
    Sigma = np.linalg.inv(A.conj().T @ A / b + np.diag(1 / g))
    mu = Sigma @ A.conj().T @ y / b
    ref = (np.trace(Sigma @ A.conj().T @ A).real + np.linalg.norm(y - A @ mu) ** 2) / M
    assert abs(new - ref) < 1e-10 * ref


def test_fit_recovers_noise_free_frequencies_from_three_quarters_of_the_samples():
    N = 64
    inst = synth.make_instance(N, 3, 80.0, 13, min_sep=4 / N)
    obs = np.sort(np.random.default_rng(1).choice(N, 48, replace=False))
    r = oi.fit(inst.y[obs], obs, N, 8 * N)
    assert r.K == 3
    assert np.all(synth.wrap_distance(np.sort(inst.theta), r.theta) < 1e-6)
