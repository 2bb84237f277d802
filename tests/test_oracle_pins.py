"""Pins of the FP64 CPU oracle against facts that do not come from the oracle.

Each test checks one oracle function against a closed form, exact or
high-precision arithmetic, finite differences of the objective it claims to
differentiate, the objective change it claims to predict, or a library
routine solving the same mathematical problem a different way.
"""
import fractions
import json
import math
import os

import numpy as np
import pytest

from oracle import dense as dn
from oracle import fit as of
from paper_1705_06073_gb300 import synth

HERE = os.path.dirname(os.path.abspath(__file__))


def rand_state(N, K, seed, beta=0.05, gmax=3.0):
    r = np.random.default_rng(seed)
    theta = r.random(K)
    gamma = 0.1 + gmax * r.random(K)
    y = r.standard_normal(N) + 1j * r.standard_normal(N)
    return y, theta, gamma, beta


# ---------------------------------------------------------------- steering ---

def test_unit_phase_exact_reduction():
    """exp(j 2 pi n theta) against n*theta mod 1 in exact rational arithmetic."""
    r = np.random.default_rng(0)
    for theta in list(r.random(20)) + [1 - 2 ** -53, 2 ** -40, 0.5]:
        for n in (1, 7, 4095, 65535, 3 * 10 ** 6):
            f = (fractions.Fraction(theta) * n) % 1
            ref = complex(math.cos(2 * math.pi * float(f)), math.sin(2 * math.pi * float(f)))
            got = dn.unit_phase(np.array([n]), np.array([theta]))[0, 0]
            assert abs(got - ref) < 4e-15, (n, theta)


def test_covariance_is_hermitian_toeplitz_with_first_column():
    """C of eq. (py) is Hermitian Toeplitz and its first column is c_m (Sec. III)."""
    y, th, g, b = rand_state(17, 4, 1)
    C = dn.covariance(17, th, g, b)
    c = dn.first_column(17, th, g, b)
    assert np.allclose(C, C.conj().T, atol=1e-13)
    for m in range(17):
        for n in range(17):
            ref = c[m - n] if m >= n else np.conj(c[n - m])
            assert abs(C[m, n] - ref) < 1e-12
    assert abs(c[0] - (b + g.sum())) < 1e-12


# --------------------------------------------------- Sherman-Morrison case ---

def test_single_sinusoid_closed_form():
    """One component: C^{-1} = (I - gamma a a^H / (beta + gamma N)) / beta."""
    N, L = 32, 128
    th, g, b = np.array([0.3137]), np.array([2.5]), 0.07
    y = np.random.default_rng(2).standard_normal(N) + 1j * np.random.default_rng(3).standard_normal(N)
    ev = dn.DenseEval(y, th, g, b)
    n = np.arange(N)
    a1 = np.exp(2j * np.pi * n * th[0])
    den = b + g[0] * N
    assert abs(ev.logdet - ((N - 1) * math.log(b) + math.log(den))) < 1e-11
    x_ref = (y - g[0] * a1 * np.vdot(a1, y) / den) / b
    assert np.allclose(ev.x, x_ref, rtol=1e-12, atol=1e-12)
    grid = ev.grid(L)
    thetas = np.arange(L) / L
    P = np.exp(2j * np.pi * np.outer(n, thetas))
    dk = P.conj().T @ a1  # a(theta)^H a_1
    s_ref = (N - g[0] * np.abs(dk) ** 2 / den) / b
    q_ref = (P.conj().T @ y - g[0] * dk * np.vdot(a1, y) / den) / b
    assert np.allclose(grid["s"], s_ref, rtol=1e-11)
    assert np.allclose(grid["q"], q_ref, rtol=1e-11, atol=1e-11 * np.abs(q_ref).max())
    vec = ev.active_vectors()
    assert abs(vec["s"][0] - N / den) < 1e-12 * N / den
    assert abs(vec["q"][0] - np.vdot(a1, y) / den) < 1e-12 * abs(np.vdot(a1, y) / den)


def test_no_component_reduces_to_periodogram():
    """K = 0: C = beta I, s = N/beta, q = DFT_L(y)/beta (numpy FFT), rho = e_{N-1}, delta = beta."""
    N, L, b = 24, 96, 0.3
    y = np.random.default_rng(4).standard_normal(N) + 1j * np.random.default_rng(5).standard_normal(N)
    ev = dn.DenseEval(y, [], [], b)
    grid = ev.grid(L, derivatives=True)
    assert np.allclose(grid["s"], N / b, rtol=1e-13)
    assert np.allclose(grid["q"], np.fft.fft(y, L) / b, rtol=1e-12, atol=1e-12)
    n = np.arange(N)
    assert np.allclose(grid["dq"], np.fft.fft(-2j * np.pi * n * y, L) / b, atol=1e-10)
    assert np.allclose(grid["d2q"], np.fft.fft(-(2 * np.pi * n) ** 2 * y, L) / b, atol=1e-8)
    assert np.allclose(grid["ds"], 0.0, atol=1e-9)
    assert np.allclose(grid["d2s"], 0.0, atol=1e-6)
    rho, delta = ev.gs_generators()
    e = np.zeros(N)
    e[-1] = 1
    assert np.allclose(rho, e, atol=1e-14)
    assert np.allclose(delta, b, rtol=1e-13)


# ---------------------------------------------------- Gohberg-Semencul -----

@pytest.mark.parametrize("N", [7, 12, 33, 64])
def test_gohberg_semencul_reproduces_inverse(N):
    """eq. (gohberg-semencul) built from the oracle's rho, delta equals inv(C)."""
    y, th, g, b = rand_state(N, 4, N)
    ev = dn.DenseEval(y, th, g, b)
    rho, delta = ev.gs_generators()
    assert abs(rho[-1] - 1) < 1e-14
    T0 = np.zeros((N, N), complex)
    T1 = np.zeros((N, N), complex)
    for i in range(N):
        for k in range(N):
            if 0 <= i - k - 1 <= N - 1:
                T0[i, k] = rho[i - k - 1]
            if 0 <= N - 1 + i - k <= N - 1:
                T1[i, k] = rho[N - 1 + i - k]
    Ci = (T1.conj().T @ T1 - T0 @ T0.conj().T) / delta[-1]
    ref = np.linalg.inv(ev.C)
    assert np.abs(Ci - ref).max() < 1e-10 * np.abs(ref).max()
    # the pivots give the log-determinant (Sec. III-A)
    assert abs(np.sum(np.log(delta)) - np.linalg.slogdet(ev.C)[1]) < 1e-10 * N


# ---------------------------------------------- high-precision brute force --

def test_brute_force_high_precision():
    """N <= 10: every dense quantity against 40-digit Gauss-Jordan (mpmath)."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    N, L = 9, 20
    y, th, g, b = rand_state(N, 3, 11)
    ev = dn.DenseEval(y, th, g, b)
    two_pi = 2 * mp.pi

    def a(theta):
        return mp.matrix([mp.expj(two_pi * n * mp.mpf(theta)) for n in range(N)])

    A = [a(t) for t in th]
    C = mp.matrix(N, N)
    for i in range(N):
        for j in range(N):
            C[i, j] = (b if i == j else 0) + sum(g[k] * A[k][i] * mp.conj(A[k][j]) for k in range(3))
    Ci = mp.inverse(C)
    Y = mp.matrix([mp.mpc(complex(v)) for v in y])
    X = Ci * Y
    assert abs(complex(mp.log(mp.det(C)).real) - ev.logdet) < 1e-12
    assert max(abs(complex(X[i]) - ev.x[i]) for i in range(N)) < 1e-12 * max(abs(complex(X[i])) for i in range(N))
    D = [two_pi * n for n in range(N)]
    vec = ev.active_vectors()
    for k in range(3):
        ak = A[k]

        def form(wl, wr):
            return complex(sum(mp.conj(ak[m]) * wl[m] * Ci[m, n] * wr[n] * ak[n] for m in range(N) for n in range(N)))
        one = [1] * N
        ref = dict(
            q=complex(sum(mp.conj(ak[m]) * X[m] for m in range(N))),
            r=complex(sum(mp.conj(ak[m]) * D[m] * X[m] for m in range(N))),
            u=complex(sum(mp.conj(ak[m]) * D[m] ** 2 * X[m] for m in range(N))),
            s=form(one, one), t=form(D, one), v=form([d * d for d in D], one), x=form(D, D))
        for key, val in ref.items():
            assert abs(vec[key][k] - val) < 1e-10 * max(1.0, abs(val)), key
    grid = ev.grid(L)
    for l in range(L):
        al = a(l / L)
        s_ref = complex(sum(mp.conj(al[m]) * Ci[m, n] * al[n] for m in range(N) for n in range(N))).real
        q_ref = complex(sum(mp.conj(al[m]) * X[m] for m in range(N)))
        assert abs(grid["s"][l] - s_ref) < 1e-11 * s_ref
        assert abs(grid["q"][l] - q_ref) < 1e-11 * max(1.0, abs(q_ref))


# ------------------------------------------------------- derivatives -------

def test_objective_derivatives_match_finite_differences():
    """eqs. (derivative), (derivative2) against 5-point differences of ln|C| + y^H C^-1 y."""
    N = 40
    y, th, g, b = rand_state(N, 3, 21, beta=0.2, gmax=1.0)
    th = np.array([0.11, 0.43, 0.77])
    ev = dn.DenseEval(y, th, g, b)
    gt, gg, ht, hg = dn.derivatives(ev.active_vectors(), g, N)

    def d12(fun, h):
        f = [fun(j * h) for j in (-2, -1, 0, 1, 2)]
        d1 = (f[0] - 8 * f[1] + 8 * f[3] - f[4]) / (12 * h)
        d2 = (-f[0] + 16 * f[1] - 30 * f[2] + 16 * f[3] - f[4]) / (12 * h * h)
        return d1, d2
    for k in range(3):
        e = np.zeros(3)
        e[k] = 1.0
        d1, d2 = d12(lambda dt: dn.DenseEval(y, th + dt * e, g, b).data_term(), 3e-5)
        assert abs(d1 - gt[k]) < 1e-7 * max(1, abs(gt[k]))
        assert abs(d2 - ht[k]) < 1e-5 * max(1, abs(ht[k]))
        d1, d2 = d12(lambda dg: dn.DenseEval(y, th, g + dg * e, b).data_term(), 1e-3 * g[k])
        assert abs(d1 - gg[k]) < 1e-7 * max(1, abs(gg[k]))
        assert abs(d2 - hg[k]) < 1e-5 * max(1, abs(hg[k]))


def test_grid_derivatives_match_finite_differences():
    N = 24
    y, th, g, b = rand_state(N, 2, 31)
    ev = dn.DenseEval(y, th, g, b)
    pts = np.array([0.05, 0.3, 0.61, 0.9])
    h = 1e-5
    c = ev.grid(0, derivatives=True, points=pts)
    p = ev.grid(0, derivatives=True, points=pts + h)
    m = ev.grid(0, derivatives=True, points=pts - h)
    for f, df in (("q", "dq"), ("s", "ds"), ("dq", "d2q"), ("ds", "d2s")):
        fd = (p[f] - m[f]) / (2 * h)
        assert np.all(np.abs(fd - c[df]) < 1e-6 * np.abs(c[df]).max()), f
    # s is real and positive; s(theta) = sum of |G^-1 psi|^2
    assert np.all(c["s"] > 0)


# ------------------------------------------- single-component algebra -------

def test_delta_objective_is_the_objective_change():
    """eq. (delta_L) equals L(with component) - L(without) computed densely."""
    N = 30
    y, th, g, b = rand_state(N, 3, 41)
    ev = dn.DenseEval(y, th, g, b)
    zeta = 0.15
    pts = np.array([0.2, 0.55, 0.81])
    gr = ev.grid(0, points=pts)
    gbar = g.mean()
    dl = dn.delta_objective(gr["q"], gr["s"], gbar, zeta)
    for i, t in enumerate(pts):
        ev2 = dn.DenseEval(y, np.append(th, t), np.append(g, gbar), b)
        ref = ev2.objective(zeta) - ev.objective(zeta)
        assert abs(dl[i] - ref) < 1e-9 * max(1, abs(ref))


def test_activation_criterion_is_the_sign_of_the_objective_change():
    """Eq. (activate_derived) rearranges Delta L < 0 of eq. (delta_L): with the
    dense objective change as the reference, the criterion with tau = 0 holds
    exactly where activating lowers the objective; tau shifts the threshold
    of |q|^2 / s (eq. activate_criterion)."""
    N = 24
    y, th, g, b = rand_state(N, 2, 43)
    ev = dn.DenseEval(y, th, g, b)
    pts = np.linspace(0.0, 1.0, 41, endpoint=False)
    gr = ev.grid(0, points=pts)
    checked, outcomes = 0, set()
    for zeta in (0.05, 0.2, 0.45):
        for gbar in (0.3, 2.0, 9.0):
            ok = dn.activation_test(gr["q"], gr["s"], gbar, zeta, 0.0)
            for i, t in enumerate(pts):
                ev2 = dn.DenseEval(y, np.append(th, t), np.append(g, gbar), b)
                d = ev2.objective(zeta) - ev.objective(zeta)
                if abs(d) > 1e-9:  # away from the boundary
                    assert bool(ok[i]) == (d < 0.0), (zeta, gbar, t, d)
                    checked += 1
                    outcomes.add(bool(ok[i]))
            ratio = np.abs(gr["q"]) ** 2 / gr["s"]
            rhs = dn.activation_rhs(gr["s"], gbar, zeta)
            assert np.array_equal(dn.activation_test(gr["q"], gr["s"], gbar, zeta, 5.0), ratio > rhs + 5.0)
    assert checked > 300 and outcomes == {True, False}


def test_activate_gamma_minimises_objective():
    from scipy.optimize import minimize_scalar
    N = 30
    y, th, g, b = rand_state(N, 2, 51)
    y = y + 4 * np.exp(2j * np.pi * 0.6 * np.arange(N))
    ev = dn.DenseEval(y, th, g, b)
    gr = ev.grid(0, points=np.array([0.6]))
    ghat = float(dn.activate_gamma(gr["q"][0], gr["s"][0]))
    assert ghat > 0
    res = minimize_scalar(lambda gm: dn.DenseEval(y, np.append(th, 0.6), np.append(g, gm), b).data_term(),
                          bounds=(1e-6, 50 * ghat), method="bounded", options={"xatol": 1e-10})
    assert abs(res.x - ghat) < 1e-4 * ghat
    # no decrease available -> 0
    assert dn.activate_gamma(0.1, 2.0) == 0.0


def test_leave_one_out_and_deactivation_statistic():
    """Woodbury q_{~k}, s_{~k} and the deactivation statistic of eq. (deactivate)
    against densely removing component k."""
    N = 28
    y, th, g, b = rand_state(N, 4, 61)
    ev = dn.DenseEval(y, th, g, b)
    vec = ev.active_vectors()
    qt, st = dn.leave_one_out(vec["q"], vec["s"], g)
    stat = dn.deactivation_statistic(vec["q"], vec["s"], g)
    for k in range(4):
        keep = np.arange(4) != k
        evk = dn.DenseEval(y, th[keep], g[keep], b)
        gr = evk.grid(0, points=th[k:k + 1])
        assert abs(gr["q"][0] - qt[k]) < 1e-10 * abs(qt[k])
        assert abs(gr["s"][0] - st[k]) < 1e-10 * st[k]
        assert abs(stat[k] - (evk.data_term() - ev.data_term())) < 1e-9 * max(1, abs(stat[k]))


def test_beta_update_is_em_and_does_not_increase_objective():
    """eq. (betaUpdate) against the explicit posterior (eqs. bmu, bSigma)."""
    N = 26
    y, th, g, b = rand_state(N, 3, 71)
    ev = dn.DenseEval(y, th, g, b)
    s = ev.active_vectors()["s"]
    new = dn.beta_update(ev, s, 1e-12)
    A = ev.A
    Sigma = np.linalg.inv(A.conj().T @ A / b + np.diag(1 / g))
    mu = Sigma @ A.conj().T @ y / b
    ref = (np.trace(Sigma @ A.conj().T @ A).real + np.linalg.norm(y - A @ mu) ** 2) / N
    assert abs(new - ref) < 1e-10 * ref
    assert np.allclose(mu, g * ev.active_vectors()["q"], rtol=1e-9)
    assert dn.DenseEval(y, th, g, new).data_term() <= ev.data_term() + 1e-12


def test_zeta_update_minimises_prior_term():
    N = 50
    for K in (0, 3, 20, 40):
        z = dn.zeta_update(K, N)
        grid = np.linspace(1e-6, 0.5, 20001)
        vals = [-dn.prior_term(K, N, zz) for zz in grid]
        zbest = grid[int(np.argmin(vals))]
        assert abs(z - (zbest if K else 0.0)) < 1e-4 or (K == 0 and z == 0.0)


# --------------------------------------------------------- whole fits -------

def test_fit_objective_never_increases():
    """Theorem 1: every block update is non-increasing in eq. (obj)."""
    inst, L = synth.single_n256()[0]
    r = of.fit(inst.y, L, trace=True)
    obj = np.array([o for _, o in r.trace])
    assert np.all(np.diff(obj) <= 1e-9 * np.abs(obj[:-1]).max())
    assert r.converged and r.K == 8


def test_fit_recovers_noise_free_frequencies():
    inst = synth.make_instance(64, 3, 80.0, 7, min_sep=4 / 64)
    r = of.fit(inst.y, 512)
    assert r.K == 3
    d = synth.wrap_distance(np.sort(inst.theta), r.theta)
    assert np.all(d < 1e-6)
    order = np.argsort(inst.theta)
    assert np.allclose(r.alpha, inst.alpha[order], rtol=1e-3)


def test_fit_zero_signal_is_degenerate():
    r = of.fit(np.zeros(16, np.complex64), 128)
    assert r.K == 0 and r.beta == 0.0


def _nmse_db(inst, r):
    n = np.arange(inst.N)
    h = np.exp(2j * np.pi * np.outer(n, inst.theta)) @ inst.alpha
    hh = np.exp(2j * np.pi * np.outer(n, r.theta)) @ r.alpha if r.K else 0 * h
    return np.linalg.norm(hh - h) ** 2 / np.linalg.norm(h) ** 2


@pytest.mark.slow
def test_accuracy_near_paper_at_20db():
    """Statistical pin: BSR, CSR, NMSE of Sec. VI-C (Fig. 2) at N=128, K=10, 20 dB."""
    from scipy.optimize import linear_sum_assignment
    gold = json.load(open(os.path.join(HERE, "golden", "paper_accuracy_n128.json")))["points"]["20"]
    trials = 40
    bsr = csr = 0.0
    nmse = []
    for t in range(trials):
        inst, L = synth.paper_accuracy_n128(t)
        r = of.fit(inst.y, L)
        N = inst.N
        d = synth.wrap_distance(inst.theta[:, None], r.theta[None, :]) if r.K else np.ones((10, 1))
        if r.K == 10:
            ri, ci = linear_sum_assignment(d ** 2)
            bsr += float(d[ri, ci].max() < 0.5 / N)
        csr += (np.sum(d.min(axis=0) < 0.5 / N) + np.sum(d.min(axis=1) < 0.5 / N)) / (r.K + 10)
        nmse.append(_nmse_db(inst, r))
    bsr /= trials
    csr /= trials
    nmse_db = 10 * np.log10(np.mean(nmse))
    assert bsr >= gold["bsr"] - 0.08
    assert csr >= gold["csr"] - 0.01
    assert abs(nmse_db - gold["nmse_db"]) < 1.5
