"""Multiple measurement vectors (Sec. V) with dense linear algebra (oracle;
test infrastructure only: nothing on the product path imports it).

G snapshots y^(g) share one model (frequencies, variances, noise variance,
activation probability) and one covariance C (eq. py); each snapshot has its
own coefficients alpha^(g).  The objective is eq. (L_MMV):
  G ln|C| + sum_g y^(g)H C^-1 y^(g) - prior(z; zeta).
Sec. V derives the updates from the single-snapshot ones and omits the
details of (de)activation; the readings below fill them in, each reducing
to the single-snapshot rule of oracle/fit.py when G = 1:

M1  Derivatives in theta_k, gamma_k: the sum over g of eqs. (derivative),
    (derivative2) with y replaced by y^(g) (as Sec. V states).
M2  Single-component objective eq. (singlecomp-mmv): with Q = sum_g |q_g|^2,
    Delta L(theta) = G ln(1 + gb s) + ln((1 - zeta)/zeta) - gb Q / (1 + gb s).
M3  gamma-hat, the minimiser of eq. (singlecomp-mmv) over gamma:
    (Q/G - s) / s^2 when Q/(G s) > 1, else 0.
M4  Activation test: Delta L < 0 at gamma-bar, written per snapshot as
    Q/(G s) > (1 + 1/(gb s)) (ln(1 + gb s) + ln((1 - zeta)/zeta)/G) + tau,
    i.e. eq. (activate_criterion) with kappa the mean per-snapshot SNR and
    tau the same margin on it.
M5  Deactivation (eq. deactivate from eq. singlecomp-mmv): remove when
    gamma Q~/(1 + gamma s~) - G ln(1 + gamma s~) < ln((1 - zeta)/zeta), with
    q~_g = q_g/(1 - gamma s), s~ = s/(1 - gamma s) (Woodbury, as Sec. II-C4).
M6  beta (the Sec. V update with the Woodbury forms of Sec. II-C3):
    max(eps_beta, (beta sum_k s_k gamma_k + beta^2 sum_g ||C^-1 y_g||^2 / G) / N).
M7  Scales that grow with the data: initial beta = 0.01 ||Y||_F^2 / (G N),
    eps_beta = 1e-12 ||Y||_F^2 / (G N); the termination threshold G N 1e-7
    and the Newton-decrement threshold G N 1e-8 (both sums over snapshots).
M8  alpha^(g) = gamma * q_g (eq. bmu with y replaced by y^(g)).
Everything else (grid, step rules, order of the blocks) is as in
oracle/fit.py (readings R1-R11).
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import dense as dn
from . import fit as of

EPS_L = of.EPS_L


class MMVDenseEval(dn.DenseEval):
    """All quantities at one state for Y = [y^(1) ... y^(G)] (N x G)."""

    def __init__(self, Y, theta, gamma, beta: float):
        Y = np.asarray(Y, dtype=np.complex128)
        if Y.ndim == 1:
            Y = Y[:, None]
        super().__init__(Y, theta, gamma, beta)  # x = C^-1 Y column by column
        self.n_snap = Y.shape[1]  # (self.G is the Cholesky factor)
        # sum_g y_g^H C^-1 y_g
        self.yCy = float(np.sum(np.conj(Y) * self.x).real)

    def data_term(self) -> float:
        """G ln|C| + sum_g y_g^H C^-1 y_g (eq. L_MMV without the prior)."""
        return self.n_snap * self.logdet + self.yCy

    def active_vectors(self):
        """eqs. (q)-(x) at the active frequencies: q, r, u are K x G (one column
        per snapshot), s, t, v, x are shared."""
        A = self.A
        d = dn.index_weights(self.N)[:, None]
        W = self.solve(A)
        DW = self.solve(d * A)
        AH = A.conj()
        q = AH.T @ self.x
        r = AH.T @ (d * self.x)
        u = AH.T @ (d ** 2 * self.x)
        s = np.sum(AH * W, axis=0)
        t = np.sum(AH * d * W, axis=0)
        v = np.sum(AH * d ** 2 * W, axis=0)
        xx = np.sum(AH * d * DW, axis=0)
        return dict(q=q, r=r, s=s.real, t=t, u=u, v=v, x=xx.real)

    def grid(self, L: int, derivatives: bool = False, chunk: int = 4096, points=None):
        """s (and s', s'') as for one snapshot; q (and q', q'') per snapshot,
        shape (points, G), straight from the definitions (Sec. III-D)."""
        N = self.N
        thetas = (np.arange(L, dtype=np.float64) / L) if points is None else np.asarray(points, np.float64)
        d = dn.index_weights(N)[:, None]
        keys = ("q", "s", "dq", "d2q", "ds", "d2s") if derivatives else ("q", "s")
        out = {k: [] for k in keys}
        for a in range(0, thetas.shape[0], chunk):
            P = dn.steering(N, thetas[a:a + chunk])
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


def snapshot_vectors(vec, g: int):
    """The single-snapshot vectors of eqs. (q)-(x) for snapshot g."""
    return dict(q=vec["q"][:, g], r=vec["r"][:, g], u=vec["u"][:, g],
                s=vec["s"], t=vec["t"], v=vec["v"], x=vec["x"])


def derivatives(vec, gamma, N: int):
    """M1: first and second derivatives of eq. (L_MMV) in theta_k, gamma_k, the
    sums over snapshots of eqs. (derivative), (derivative2)."""
    G = vec["q"].shape[1]
    tot = None
    for g in range(G):
        d = dn.derivatives(snapshot_vectors(vec, g), gamma, N)
        tot = d if tot is None else tuple(a + b for a, b in zip(tot, d))
    return tot


def q_power(q) -> np.ndarray:
    """Q = sum_g |q_g|^2 over the last axis."""
    return np.sum(np.abs(np.asarray(q)) ** 2, axis=-1)


def delta_objective(Q, s, gamma_bar, zeta: float, G: int):
    """M2: change of eq. (L_MMV) when a component of variance gamma_bar is
    activated where s_{~k} = s and sum_g |q_{~k}^(g)|^2 = Q (eq. singlecomp-mmv)."""
    gb = np.asarray(gamma_bar, dtype=np.float64)
    s = np.asarray(s, dtype=np.float64)
    return G * np.log1p(gb * s) + dn.log_prior_odds(zeta) - gb * np.asarray(Q) / (1.0 + gb * s)


def activate_gamma(Q, s, G: int):
    """M3: minimiser of eq. (singlecomp-mmv) over gamma."""
    s = np.asarray(s, dtype=np.float64)
    Qg = np.asarray(Q, dtype=np.float64) / G
    return np.where(Qg > s, (Qg - s) / (s * s), 0.0)


def activation_test(Q, s, gamma_bar, zeta: float, G: int, tau: float = 0.0):
    """M4: eq. (activate_criterion) for G snapshots (tau = 0: Delta L < 0)."""
    s = np.asarray(s, dtype=np.float64)
    gs = np.asarray(gamma_bar, dtype=np.float64) * s
    with np.errstate(divide="ignore"):
        rhs = (1.0 + 1.0 / gs) * (np.log1p(gs) + dn.log_prior_odds(zeta) / G)
    return np.asarray(Q) / G / s > rhs + tau


def deactivation_statistic(q, s, gamma):
    """M5: left-hand side of eq. (deactivate) for G snapshots; q is K x G."""
    q = np.asarray(q)
    G = q.shape[1]
    g = np.asarray(gamma, dtype=np.float64)
    den = 1.0 - g * np.asarray(s)
    st = np.asarray(s) / den
    Qt = q_power(q / den[:, None])
    return g * Qt / (1.0 + g * st) - G * np.log1p(g * st)


def beta_update(ev: MMVDenseEval, s, eps_beta: float) -> float:
    """M6: the Sec. V beta update, tr(Sigma A^H A) = beta sum_k s_k gamma_k and
    ||y_g - A mu_g||^2 = beta^2 ||C^-1 y_g||^2 (Sec. II-C3)."""
    b = ev.beta
    xx = float(np.sum(np.abs(ev.x) ** 2))
    num = b * float(np.sum(np.asarray(s) * ev.gamma)) + b * b * xx / ev.n_snap
    return max(eps_beta, num / ev.N)


@dataclasses.dataclass
class MMVFitResult:
    theta: np.ndarray
    gamma: np.ndarray
    alpha: np.ndarray  # K x G
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
    def __init__(self, Y, L, tau):
        self.Y = np.asarray(Y, dtype=np.complex128)
        self.N, self.G = self.Y.shape
        self.L = int(L)
        self.tau = float(tau)
        yy = float(np.sum(np.abs(self.Y) ** 2))
        self.beta = 0.01 * yy / (self.G * self.N)
        self.eps_beta = 1e-12 * yy / (self.G * self.N)
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
        return MMVDenseEval(self.Y, self.theta if theta is None else theta,
                            self.gamma if gamma is None else gamma, self.beta)

    def refresh(self):
        self.ev = self.evaluate()

    def objective(self):
        return self.ev.data_term() - dn.prior_term(self.K, self.N, self.zeta)

    def grid_delta(self):
        """Grid Q, s and Delta L (M2) with gamma-bar per R4."""
        self.n_grid += 1
        g = self.ev.grid(self.L)
        Q, s = q_power(g["q"]), g["s"]
        gbar = np.mean(self.gamma) if self.K else activate_gamma(Q, s, self.G)
        return Q, s, gbar, delta_objective(Q, s, gbar, self.zeta, self.G)

    def add(self, theta, gamma):
        self.theta = np.append(self.theta, theta)
        self.gamma = np.append(self.gamma, gamma)


def _exact_activation(st: _State, first=None):
    n = 0
    while st.K < st.N and st.zeta > 0.0:
        Q, s, gbar, dl = first if first is not None else st.grid_delta()
        first = None
        l = int(np.argmin(dl))
        ghat = float(activate_gamma(Q[l], s[l], st.G))
        gb = float(gbar if np.ndim(gbar) == 0 else gbar[l])
        if not (ghat > 0.0 and dl[l] < -EPS_L and activation_test(Q[l], s[l], gb, st.zeta, st.G, st.tau)):
            break
        st.add(l / st.L, ghat)
        st.refresh()
        n += 1
    return n


def _approximate_activation(st: _State):
    if st.zeta <= 0.0 or st.K >= st.N:
        return 0, None
    grid = st.grid_delta()
    Q, s, gbar, dl = grid
    with np.errstate(divide="ignore", invalid="ignore"):
        ghat = activate_gamma(Q, s, st.G)
        gb = np.broadcast_to(np.asarray(gbar, dtype=np.float64), s.shape)
        passes = activation_test(Q, s, gb, st.zeta, st.G, 0.0)
    taken = of.select_candidates(dl, ghat, passes, st.theta, st.N, st.L, st.N - st.K)
    for l, gh in taken:
        st.add(l / st.L, gh)
    if taken:
        st.refresh()
    return len(taken), grid


def _newton_iteration(st: _State):
    N, G = st.N, st.G
    vec = st.ev.active_vectors()
    gt, gg, ht, hg = derivatives(vec, st.gamma, N)
    ht = np.where(ht > 0.0, ht, (50.0 * N) ** 2)
    hg = np.where(hg > 0.0, hg, 1.0 / st.gamma ** 2)
    dt = -gt / ht
    dg = -gg / hg
    dec = float(np.sum(gt * gt / ht) + np.sum(gg * gg / hg))
    if dec < G * N * 1e-8:
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
        stat = deactivation_statistic(vec["q"], vec["s"], st.gamma)
        k = of.deactivation_pick(stat, dn.log_prior_odds(st.zeta))
        if k is None:
            break
        st.theta = np.delete(st.theta, k)
        st.gamma = np.delete(st.gamma, k)
        st.refresh()
        n += 1
    return n


def fit(Y, L: int, tau: float = 5.0, max_outer: int = 200, max_inner: int = 5,
        approx_iters: int = 10) -> MMVFitResult:
    """Run the estimator of Sec. II with the Sec. V updates on Y (N x G)."""
    Y = np.asarray(Y, dtype=np.complex128)
    if Y.ndim == 1:
        Y = Y[:, None]
    N, G = Y.shape
    if float(np.sum(np.abs(Y) ** 2)) == 0.0:  # R11
        return MMVFitResult(np.zeros(0), np.zeros(0), np.zeros((0, G), complex), 0.0, 0.0, 0.0, 0, True, 0, 0)
    st = _State(Y, L, tau)
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
        st.zeta = dn.zeta_update(st.K, N)
        s = st.ev.active_vectors()["s"] if st.K else np.zeros(0)
        st.beta = beta_update(st.ev, s, st.eps_beta)
        st.refresh()
        for _ in range(max_inner):
            if st.K == 0:
                break
            dec = _newton_iteration(st)
            _deactivation(st)
            if dec < G * N * 1e-8:
                break
        L_cur = st.objective()
        if abs(L_cur - L_prev) < G * N * 1e-7:
            converged = True
            break
        L_prev = L_cur
    K = st.K
    q = st.ev.active_vectors()["q"] if K else np.zeros((0, G), complex)
    order = np.argsort(st.theta, kind="stable")
    return MMVFitResult(theta=st.theta[order], gamma=st.gamma[order], alpha=(st.gamma[:, None] * q)[order],
                        beta=st.beta, zeta=st.zeta, objective=st.objective(), iters=it,
                        converged=converged, n_evals=st.n_evals, n_grid_evals=st.n_grid)
