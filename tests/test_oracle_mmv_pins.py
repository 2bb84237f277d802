"""Pins of the multiple-measurement-vector oracle (Sec. V, readings M1-M8)
against facts that do not come from it: finite differences and dense changes
of the MMV objective eq. (L_MMV), its minimiser over gamma, the explicit
posterior for beta, the single-snapshot oracle at G = 1, phase-rotated copies
of one snapshot, and noise-free recovery."""
import numpy as np
import pytest

from oracle import dense as dn
from oracle import fit as of
from oracle import mmv
from paper_1705_06073_gb300 import synth


def rand_state(N, K, G, seed, beta=0.05, gmax=3.0):
    r = np.random.default_rng(seed)
    theta = r.random(K)
    gamma = 0.1 + gmax * r.random(K)
    Y = r.standard_normal((N, G)) + 1j * r.standard_normal((N, G))
    return Y, theta, gamma, beta


def mmv_objective(Y, theta, gamma, beta, zeta):
    """eq. (L_MMV) straight from its definition: sum_g [ln|C| + y_g^H C^-1 y_g]
    minus the prior term, with C formed and inverted densely."""
    N, G = Y.shape
    C = dn.covariance(N, theta, gamma, beta)
    _sign, logdet = np.linalg.slogdet(C)
    Ci = np.linalg.inv(C)
    tot = sum(logdet + np.vdot(Y[:, g], Ci @ Y[:, g]).real for g in range(G))
    return tot - dn.prior_term(len(theta), N, zeta)


def test_data_term_is_the_definition():
    Y, th, g, b = rand_state(20, 3, 4, 1)
    ev = mmv.MMVDenseEval(Y, th, g, b)
    ref = mmv_objective(Y, th, g, b, 0.3) + dn.prior_term(3, 20, 0.3)
    assert abs(ev.data_term() - ref) < 1e-10 * abs(ref)


def test_derivatives_match_finite_differences():
    """M1 against 5-point differences of G ln|C| + sum_g y_g^H C^-1 y_g."""
    N, G = 36, 3
    Y, _th, g, b = rand_state(N, 3, G, 21, beta=0.2, gmax=1.0)
    th = np.array([0.12, 0.47, 0.71])
    ev = mmv.MMVDenseEval(Y, th, g, b)
    gt, gg, ht, hg = mmv.derivatives(ev.active_vectors(), g, N)

    def d12(fun, h):
        f = [fun(j * h) for j in (-2, -1, 0, 1, 2)]
        return ((f[0] - 8 * f[1] + 8 * f[3] - f[4]) / (12 * h),
                (-f[0] + 16 * f[1] - 30 * f[2] + 16 * f[3] - f[4]) / (12 * h * h))
    for k in range(3):
        e = np.zeros(3)
        e[k] = 1.0
        d1, d2 = d12(lambda dt: mmv.MMVDenseEval(Y, th + dt * e, g, b).data_term(), 3e-5)
        assert abs(d1 - gt[k]) < 1e-7 * max(1, abs(gt[k]))
        assert abs(d2 - ht[k]) < 1e-5 * max(1, abs(ht[k]))
        d1, d2 = d12(lambda dg: mmv.MMVDenseEval(Y, th, g + dg * e, b).data_term(), 1e-3 * g[k])
        assert abs(d1 - gg[k]) < 1e-7 * max(1, abs(gg[k]))
        assert abs(d2 - hg[k]) < 1e-5 * max(1, abs(hg[k]))


def test_rotated_copies_scale_the_single_snapshot_derivatives():
    """Snapshots y e^{j phi_g} share every |q|, so each derivative is G times
    the single-snapshot one (eqs. derivative, derivative2)."""
    N, G = 30, 5
    Y, th, g, b = rand_state(N, 4, 1, 23)
    y = Y[:, 0]
    phi = np.random.default_rng(3).random(G) * 2 * np.pi
    Yr = y[:, None] * np.exp(1j * phi)[None, :]
    d1 = dn.derivatives(dn.DenseEval(y, th, g, b).active_vectors(), g, N)
    dG = mmv.derivatives(mmv.MMVDenseEval(Yr, th, g, b).active_vectors(), g, N)
    for a, c in zip(d1, dG):
        assert np.allclose(c, G * a, rtol=1e-9, atol=1e-9 * np.abs(a).max())


def test_delta_objective_is_the_objective_change():
    """M2: Delta L equals eq. (L_MMV) with the component minus without it."""
    N, G = 28, 3
    Y, th, g, b = rand_state(N, 3, G, 41)
    ev = mmv.MMVDenseEval(Y, th, g, b)
    zeta = 0.15
    pts = np.array([0.2, 0.55, 0.81])
    gr = ev.grid(0, points=pts)
    gbar = g.mean()
    dl = mmv.delta_objective(mmv.q_power(gr["q"]), gr["s"], gbar, zeta, G)
    for i, t in enumerate(pts):
        ref = mmv_objective(Y, np.append(th, t), np.append(g, gbar), b, zeta) - mmv_objective(Y, th, g, b, zeta)
        assert abs(dl[i] - ref) < 1e-9 * max(1, abs(ref))


def test_activation_criterion_is_the_sign_of_the_objective_change():
    """M4 with tau = 0 holds exactly where activating lowers eq. (L_MMV)."""
    N, G = 22, 4
    # noise variance near the snapshots' power: activation helps at some points only
    Y, th, g, b = rand_state(N, 2, G, 43, beta=0.4)
    ev = mmv.MMVDenseEval(Y, th, g, b)
    pts = np.linspace(0.0, 1.0, 33, endpoint=False)
    gr = ev.grid(0, points=pts)
    Q = mmv.q_power(gr["q"])
    checked, outcomes = 0, set()
    for zeta in (0.05, 0.2, 0.45):
        base = mmv_objective(Y, th, g, b, zeta)
        for gbar in (0.3, 2.0, 9.0):
            ok = mmv.activation_test(Q, gr["s"], gbar, zeta, G, 0.0)
            for i, t in enumerate(pts):
                d = mmv_objective(Y, np.append(th, t), np.append(g, gbar), b, zeta) - base
                if abs(d) > 1e-9:
                    assert bool(ok[i]) == (d < 0.0), (zeta, gbar, t, d)
                    checked += 1
                    outcomes.add(bool(ok[i]))
            # tau is a margin on the mean per-snapshot ratio Q / (G s)
            gs = gbar * gr["s"]
            rhs = (1 + 1 / gs) * (np.log1p(gs) + dn.log_prior_odds(zeta) / G)
            assert np.array_equal(mmv.activation_test(Q, gr["s"], gbar, zeta, G, 5.0), Q / G / gr["s"] > rhs + 5.0)
    assert checked > 250 and outcomes == {True, False}


def test_activate_gamma_minimises_objective():
    """M3 against a bounded scalar minimisation of the dense objective."""
    from scipy.optimize import minimize_scalar
    N, G = 26, 3
    Y, th, g, b = rand_state(N, 2, G, 51)
    Y = Y + 3 * np.exp(2j * np.pi * 0.6 * np.arange(N))[:, None] * np.exp(1j * np.arange(G))[None, :]
    ev = mmv.MMVDenseEval(Y, th, g, b)
    gr = ev.grid(0, points=np.array([0.6]))
    ghat = float(mmv.activate_gamma(mmv.q_power(gr["q"])[0], gr["s"][0], G))
    assert ghat > 0
    res = minimize_scalar(lambda gm: mmv.MMVDenseEval(Y, np.append(th, 0.6), np.append(g, gm), b).data_term(),
                          bounds=(1e-6, 50 * ghat), method="bounded", options={"xatol": 1e-10})
    assert abs(res.x - ghat) < 1e-4 * ghat
    assert mmv.activate_gamma(0.3, 2.0, 3) == 0.0


def test_deactivation_statistic_is_the_dense_removal():
    """M5: the statistic equals the data-term change of removing component k."""
    N, G = 26, 3
    Y, th, g, b = rand_state(N, 4, G, 61)
    ev = mmv.MMVDenseEval(Y, th, g, b)
    vec = ev.active_vectors()
    stat = mmv.deactivation_statistic(vec["q"], vec["s"], g)
    for k in range(4):
        keep = np.arange(4) != k
        evk = mmv.MMVDenseEval(Y, th[keep], g[keep], b)
        assert abs(stat[k] - (evk.data_term() - ev.data_term())) < 1e-9 * max(1, abs(stat[k]))


def test_beta_update_against_the_explicit_posterior():
    """M6 against tr(Sigma A^H A)/N + sum_g ||y_g - A mu_g||^2 / (G N) with
    Sigma, mu_g formed explicitly (eqs. bSigma, bmu with y -> y_g), and the
    EM property: the data term does not increase."""
    N, G = 24, 3
    Y, th, g, b = rand_state(N, 3, G, 71)
    ev = mmv.MMVDenseEval(Y, th, g, b)
    s = ev.active_vectors()["s"]
    new = mmv.beta_update(ev, s, 1e-12)
    A = ev.A
    Sigma = np.linalg.inv(A.conj().T @ A / b + np.diag(1 / g))
    mu = Sigma @ A.conj().T @ Y / b
    ref = np.trace(Sigma @ A.conj().T @ A).real / N + np.linalg.norm(Y - A @ mu) ** 2 / (G * N)
    assert abs(new - ref) < 1e-10 * ref
    assert np.allclose(mu, g[:, None] * ev.active_vectors()["q"], rtol=1e-9)
    assert mmv.MMVDenseEval(Y, th, g, new).data_term() <= ev.data_term() + 1e-12


def test_grid_is_the_single_snapshot_grid_per_column():
    N, G = 20, 3
    Y, th, g, b = rand_state(N, 2, G, 81)
    m = mmv.MMVDenseEval(Y, th, g, b).grid(64, derivatives=True)
    for gi in range(G):
        o = dn.DenseEval(Y[:, gi], th, g, b).grid(64, derivatives=True)
        for k in ("q", "dq", "d2q"):
            assert np.allclose(m[k][:, gi], o[k], rtol=0, atol=1e-12 * np.abs(o[k]).max())
        for k in ("s", "ds", "d2s"):
            assert np.allclose(m[k], o[k], rtol=0, atol=1e-12 * np.abs(o[k]).max())


def test_one_snapshot_is_the_single_snapshot_fit():
    """With G = 1 every reading reduces to the single-snapshot rule."""
    for N, K, snr, seed in ((64, 3, 25.0, 11), (96, 5, 12.0, 12)):
        inst = synth.make_instance(N, K, snr, seed)
        a = of.fit(inst.y, 4 * N)
        b = mmv.fit(inst.y[:, None], 4 * N)
        assert a.K == b.K and a.n_evals == b.n_evals and a.n_grid_evals == b.n_grid_evals
        assert np.max(synth.wrap_distance(a.theta, b.theta)) < 1e-12
        assert np.allclose(a.gamma, b.gamma, rtol=1e-9)
        assert np.allclose(a.alpha, b.alpha[:, 0], rtol=1e-9)
        assert abs(a.beta - b.beta) < 1e-9 * a.beta


def test_fit_recovers_noise_free_frequencies_and_coefficients():
    inst = synth.make_mmv_instance(48, 3, 4, 80.0, 7, min_sep=4 / 48)
    r = mmv.fit(inst.Y.T, 384)
    assert r.K == 3
    d = synth.wrap_distance(np.sort(inst.theta), r.theta)
    assert np.all(d < 1e-6)
    order = np.argsort(inst.theta)
    assert np.allclose(r.alpha, inst.alpha[:, order].T, rtol=1e-3)


def test_snapshots_separate_what_one_snapshot_cannot():
    """Two components 0.6/N apart at 10 dB: more snapshots give more evidence
    per frequency, so G = 16 resolves both while the estimate from the first
    snapshot alone does not (the point of Sec. V)."""
    N = 64
    inst = synth.make_mmv_instance(N, 2, 16, 10.0, 17, min_sep=0.5 / N)
    inst.theta[:] = [0.3, 0.3 + 0.6 / N]
    H = np.stack([synth.sum_of_sinusoids(N, inst.theta, inst.alpha[g]) for g in range(16)])
    noise = np.sqrt(inst.beta) * np.stack([synth.Stream(900 + g).cnormal(N) for g in range(16)])
    Y = (H + noise).T
    r16 = mmv.fit(Y, 8 * N)
    r1 = mmv.fit(Y[:, :1], 8 * N)
    assert r16.K == 2
    assert np.all(synth.wrap_distance(np.sort(inst.theta), r16.theta) < 0.1 / N)
    assert r1.K < 2


def test_fit_objective_never_increases_across_outer_iterations():
    """Theorem 1 carried over: the objective after each outer iteration, for
    increasing iteration caps, never rises."""
    inst = synth.make_mmv_instance(40, 3, 3, 15.0, 19)
    objs = [mmv.fit(inst.Y.T, 320, max_outer=m).objective for m in (1, 2, 3, 4, 6)]
    assert np.all(np.diff(objs) <= 1e-9 * np.abs(objs).max())


def test_zero_signal_is_degenerate():
    r = mmv.fit(np.zeros((16, 3), np.complex64), 128)
    assert r.K == 0 and r.beta == 0.0 and r.alpha.shape == (0, 3)


@pytest.mark.parametrize("G", [2, 5])
def test_mmv_instance_model(G):
    inst = synth.make_mmv_instance(32, 2, G, 30.0, 3)
    assert inst.Y.shape == (G, 32) and inst.alpha.shape == (G, 2)
    H = np.stack([synth.sum_of_sinusoids(32, inst.theta, inst.alpha[g]) for g in range(G)])
    snr = np.sum(np.abs(H) ** 2) / (G * 32 * inst.beta)
    assert abs(10 * np.log10(snr) - 30.0) < 1e-9
