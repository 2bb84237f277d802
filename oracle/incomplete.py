"""Incomplete observations (Sec. II with Phi != I; the semifast method's
setting, Sec. IV) with dense linear algebra (oracle; test infrastructure
only: nothing on the product path imports it).

Phi selects the M observed samples y_m = (Phi z)_m = z_{n_m} of an N-sample
signal (0 <= n_0 < ... < n_{M-1} < N; Sec. IV footnote, unit weights), so
A(theta) = Phi Psi(theta) is Psi's rows n_m and C = beta I_M + A Gamma A^H is
M x M (eq. py).  The vectors of eqs. (q)-(x) carry D's entries 2 pi n_m at
the observed rows.  The estimator is that of oracle/fit.py with the paper's
M where it counts observations: K_max = M (footnote to eq. estModel),
zeta = min(1/2, K/M) (eq. zetaUpdate), beta divided by M (eq. betaUpdate),
initial beta 0.01 ||y||^2/M and eps_beta 1e-12 ||y||^2/M (R7 with M), and the
thresholds M 1e-7 (termination) and M 1e-8 (Newton decrement) of Sec. II-D;
N stays where it measures frequency resolution: the (50N)^2 Hessian
fallback of Sec. II-C1 and the 0.05/N spacing of Sec. II-E.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.linalg as sla

from . import dense as dn
from . import fit as of

EPS_L = of.EPS_L


class IncompleteDenseEval:
    """All quantities at one state from a dense Cholesky of the M x M C."""

    def __init__(self, y, obs, N: int, theta, gamma, beta: float):
        self.y = np.asarray(y, dtype=np.complex128)
        self.obs = np.asarray(obs, dtype=np.int64)
        self.N = int(N)
        self.M = self.obs.shape[0]
        self.theta = np.asarray(theta, dtype=np.float64).copy()
        self.gamma = np.asarray(gamma, dtype=np.float64).copy()
        self.beta = float(beta)
        self.A = dn.steering(self.N, self.theta)[self.obs]
        self.C = self.beta * np.eye(self.M, dtype=np.complex128) + (self.A * self.gamma) @ self.A.conj().T
        self.G = sla.cholesky(self.C, lower=True, check_finite=False)
        self.logdet = float(2.0 * np.sum(np.log(np.diag(self.G).real)))
        self.x = self.solve(self.y)
        self.yCy = float(np.vdot(self.y, self.x).real)

    def solve(self, b):
        z = sla.solve_triangular(self.G, b, lower=True, check_finite=False)
        return sla.solve_triangular(self.G.conj().T, z, lower=False, check_finite=False)

    def whiten(self, b):
        return sla.solve_triangular(self.G, b, lower=True, check_finite=False)

    def data_term(self) -> float:
        """ln|C| + y^H C^-1 y (eq. obj without the prior)."""
        return self.logdet + self.yCy

    def objective(self, zeta: float) -> float:
        """eq. (obj) with K_max = M."""
        return self.data_term() - dn.prior_term(self.theta.shape[0], self.M, zeta)

    def weights(self):
        """D's diagonal at the observed rows: 2 pi n_m."""
        return dn.index_weights(self.N)[self.obs]

    def active_vectors(self):
        """eqs. (q)-(x) with Phi the row selection."""
        A = self.A
        d = self.weights()[:, None]
        W = self.solve(A)
        DW = self.solve(d * A)
        AH = A.conj()
        q = AH.T @ self.x
        r = AH.T @ (d[:, 0] * self.x)
        u = AH.T @ (d[:, 0] ** 2 * self.x)
        s = np.sum(AH * W, axis=0)
        t = np.sum(AH * d * W, axis=0)
        v = np.sum(AH * d ** 2 * W, axis=0)
        xx = np.sum(AH * d * DW, axis=0)
        return dict(q=q, r=r, s=s.real, t=t, u=u, v=v, x=xx.real)

    def grid(self, L: int, derivatives: bool = False, chunk: int = 4096, points=None):
        """q(theta) = psi^H Phi^H C^-1 y and s(theta) = psi^H Phi^H C^-1 Phi psi
        (Sec. IV, evaluating q and s on the grid) and their theta-derivatives,
        straight from the definitions."""
        thetas = (np.arange(L, dtype=np.float64) / L) if points is None else np.asarray(points, np.float64)
        d = self.weights()[:, None]
        keys = ("q", "s", "dq", "d2q", "ds", "d2s") if derivatives else ("q", "s")
        out = {k: [] for k in keys}
        for a in range(0, thetas.shape[0], chunk):
            P = dn.steering(self.N, thetas[a:a + chunk])[self.obs]
            V0 = self.whiten(P)
            out["s"].append(np.sum(np.abs(V0) ** 2, axis=0))
            out["q"].append(P.conj().T @ self.x)
            if derivatives:
                P1 = 1j * d * P
                P2 = -(d ** 2) * P
                V1 = self.whiten(P1)
                V2 = self.whiten(P2)
                out["dq"].append(P1.conj().T @ self.x)
                out["d2q"].append(P2.conj().T @ self.x)
                out["ds"].append(2.0 * np.real(np.sum(V0.conj() * V1, axis=0)))
                out["d2s"].append(2.0 * np.real(np.sum(V0.conj() * V2, axis=0)) + 2.0 * np.sum(np.abs(V1) ** 2, axis=0))
        return {k: np.concatenate(v) for k, v in out.items()}


def beta_update(ev: IncompleteDenseEval, s, eps_beta: float) -> float:
    """eq. (betaUpdate) with the Woodbury forms of Sec. II-C3, divided by M."""
    b = ev.beta
    num = b * float(np.sum(np.asarray(s) * ev.gamma)) + b * b * float(np.vdot(ev.x, ev.x).real)
    return max(eps_beta, num / ev.M)


@dataclasses.dataclass
class IncompleteFitResult:
    theta: np.ndarray
    gamma: np.ndarray
    alpha: np.ndarray
    beta: float
    zeta: float
    objective: float
    iters: int
    converged: bool
    n_evals: int
    n_grid_evals: int

    @property
    def K(self) -> int:
        return int(self.theta.shape[0])


class _State:
    def __init__(self, y, obs, N, L, tau):
        self.y = np.asarray(y, dtype=np.complex128)
        self.obs = np.asarray(obs, dtype=np.int64)
        self.N = int(N)
        self.M = self.obs.shape[0]
        self.L = int(L)
        self.tau = float(tau)
        yy = float(np.vdot(self.y, self.y).real)
        self.beta = 0.01 * yy / self.M
        self.eps_beta = 1e-12 * yy / self.M
        self.zeta = 0.2
        self.theta = np.zeros(0)
        self.gamma = np.zeros(0)
        self.n_evals = 0
        self.n_grid = 0
        self.ev = self.evaluate()

    @property
    def K(self):
        return self.theta.shape[0]

    def evaluate(self, theta=None, gamma=None):
        self.n_evals += 1
        return IncompleteDenseEval(self.y, self.obs, self.N, self.theta if theta is None else theta,
                                   self.gamma if gamma is None else gamma, self.beta)

    def refresh(self):
        self.ev = self.evaluate()

    def objective(self):
        return self.ev.objective(self.zeta)

    def grid_delta(self):
        self.n_grid += 1
        g = self.ev.grid(self.L)
        q, s = g["q"], g["s"]
        gbar = np.mean(self.gamma) if self.K else dn.activate_gamma(q, s)
        return q, s, gbar, dn.delta_objective(q, s, gbar, self.zeta)

    def add(self, theta, gamma):
        self.theta = np.append(self.theta, theta)
        self.gamma = np.append(self.gamma, gamma)


def _exact_activation(st: _State, first=None):
    n = 0
    while st.K < st.M and st.zeta > 0.0:
        q, s, gbar, dl = first if first is not None else st.grid_delta()
        first = None
        l = int(np.argmin(dl))
        ghat = float(dn.activate_gamma(q[l], s[l]))
        gb = float(gbar if np.ndim(gbar) == 0 else gbar[l])
        if not (ghat > 0.0 and dl[l] < -EPS_L and dn.activation_test(q[l], s[l], gb, st.zeta, st.tau)):
            break
        st.add(l / st.L, ghat)
        st.refresh()
        n += 1
    return n


def _approximate_activation(st: _State):
    if st.zeta <= 0.0 or st.K >= st.M:
        return 0, None
    grid = st.grid_delta()
    q, s, gbar, dl = grid
    taken = of.approximate_activation_select(dl, q, s, gbar, st.zeta, st.theta, st.N, st.L, st.M - st.K)
    for l, gh in taken:
        st.add(l / st.L, gh)
    if taken:
        st.refresh()
    return len(taken), grid


def _newton_iteration(st: _State):
    N, M = st.N, st.M
    vec = st.ev.active_vectors()
    gt, gg, ht, hg = dn.derivatives(vec, st.gamma, N)
    ht = np.where(ht > 0.0, ht, (50.0 * N) ** 2)
    hg = np.where(hg > 0.0, hg, 1.0 / st.gamma ** 2)
    dt = -gt / ht
    dg = -gg / hg
    dec = float(np.sum(gt * gt / ht) + np.sum(gg * gg / hg))
    if dec < M * 1e-8:
        return dec
    slope = float(np.sum(gt * dt) + np.sum(gg * dg))
    alpha = 1.0
    neg = dg < 0.0
    if np.any(neg):
        alpha = min(1.0, 0.99 * float(np.min(st.gamma[neg] / -dg[neg])))
    f0 = st.ev.data_term()
    for _ in range(31):
        th = np.mod(st.theta + alpha * dt, 1.0)
        th = np.where(th >= 1.0, th - 1.0, th)
        gm = st.gamma + alpha * dg
        ev = st.evaluate(th, gm)
        if ev.data_term() <= f0 + 1e-4 * alpha * slope:
            st.theta, st.gamma, st.ev = th, gm, ev
            return dec
        alpha *= 0.5
    return dec


def _deactivation(st: _State):
    n = 0
    while st.K > 0:
        vec = st.ev.active_vectors()
        stat = dn.deactivation_statistic(vec["q"], vec["s"], st.gamma)
        k = of.deactivation_pick(stat, dn.log_prior_odds(st.zeta))
        if k is None:
            break
        st.theta = np.delete(st.theta, k)
        st.gamma = np.delete(st.gamma, k)
        st.refresh()
        n += 1
    return n


def fit(y, obs, N: int, L: int, tau: float = 5.0, max_outer: int = 200, max_inner: int = 5,
        approx_iters: int = 10) -> IncompleteFitResult:
    """The estimator of Sec. II on the observed samples y (y_m = z_{obs[m]})."""
    y = np.asarray(y, dtype=np.complex128)
    M = y.shape[0]
    if float(np.vdot(y, y).real) == 0.0:
        return IncompleteFitResult(np.zeros(0), np.zeros(0), np.zeros(0, complex), 0.0, 0.0, 0.0, 0, True, 0, 0)
    st = _State(y, obs, N, L, tau)
    L_prev = st.objective()
    approx = approx_iters > 0
    converged = False
    it = 0
    for it in range(1, max_outer + 1):
        if approx and it <= approx_iters:
            n, grid = _approximate_activation(st)
            if n == 0:
                approx = False
                _exact_activation(st, first=grid)
        else:
            _exact_activation(st)
        st.zeta = dn.zeta_update(st.K, M)
        s = st.ev.active_vectors()["s"] if st.K else np.zeros(0)
        st.beta = beta_update(st.ev, s, st.eps_beta)
        st.refresh()
        for _ in range(max_inner):
            if st.K == 0:
                break
            dec = _newton_iteration(st)
            _deactivation(st)
            if dec < M * 1e-8:
                break
        L_cur = st.objective()
        if abs(L_cur - L_prev) < M * 1e-7:
            converged = True
            break
        L_prev = L_cur
    K = st.K
    q = st.ev.active_vectors()["q"] if K else np.zeros(0, complex)
    order = np.argsort(st.theta, kind="stable")
    return IncompleteFitResult(theta=st.theta[order], gamma=st.gamma[order], alpha=(st.gamma * q)[order],
                               beta=st.beta, zeta=st.zeta, objective=st.objective(), iters=it,
                               converged=converged, n_evals=st.n_evals, n_grid_evals=st.n_grid)
