"""Dense FP64 evaluation of the estimation model (oracle; test infrastructure).

Every function cites the passage of Hansen, Fleury & Rao, "Superfast Line
Spectral Estimation" (IEEE TSP 2018) it follows.  Indices n run over
0..N-1, so [psi(theta)]_n = exp(j 2 pi n theta), the paper's (n-1) for
n = 1..N (Sec. II, eq. model).

Parity status: every function here is pinned by a test in
``tests/test_oracle_pins.py`` against something other than itself (closed
forms, finite differences, exact arithmetic, brute force or the defining
objective).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

TWO_PI = 2.0 * np.pi


def unit_phase(n, theta):
    """exp(j 2 pi n theta) with n*theta reduced modulo 1 without rounding error.

    theta is split as hi + lo with hi a multiple of 2^-27, so n*hi is exact
    for integer n < 2^26 and only the tiny n*lo term is rounded.  This keeps
    the phase accurate to ~1e-16 cycles even for n*theta ~ 1e4.
    """
    n = np.asarray(n, dtype=np.float64)
    theta = np.asarray(theta, dtype=np.float64)
    hi = np.floor(theta * 134217728.0) / 134217728.0
    lo = theta - hi
    ph = np.mod(np.multiply.outer(n, hi), 1.0) + np.multiply.outer(n, lo)
    ph = np.mod(ph, 1.0)
    return np.exp(1j * TWO_PI * ph)


def steering(N: int, theta) -> np.ndarray:
    """Psi(theta) = [psi(theta_1) ... psi(theta_K)], N x K (Sec. II, eq. model)."""
    return unit_phase(np.arange(N), np.atleast_1d(theta))


def index_weights(N: int) -> np.ndarray:
    """Diagonal of D = diag(0, 2pi, ..., 2pi(N-1)) (Sec. II-C, after eq. x)."""
    return TWO_PI * np.arange(N, dtype=np.float64)


def covariance(N: int, theta, gamma, beta: float) -> np.ndarray:
    """C = beta I + A Gamma A^H for the active components (eq. py)."""
    A = steering(N, theta)
    g = np.asarray(gamma, dtype=np.float64)
    return beta * np.eye(N, dtype=np.complex128) + (A * g) @ A.conj().T


def first_column(N: int, theta, gamma, beta: float) -> np.ndarray:
    """c_m = [C]_{m,0} = beta delta_{m0} + sum_k gamma_k e^{j 2 pi m theta_k}.

    C is Hermitian Toeplitz in the complete-data case (Sec. III intro); this is
    the column that defines it.
    """
    A = steering(N, theta)
    c = A @ np.asarray(gamma, dtype=np.complex128) if A.shape[1] else np.zeros(N, complex)
    c[0] += beta
    return c


class DenseEval:
    """All quantities of the method at one state, from a dense Cholesky of C.

    C = G G^H (library Cholesky); ln|C| = 2 sum ln G_ii; x = C^{-1} y.
    """

    def __init__(self, y, theta, gamma, beta: float):
        self.y = np.asarray(y, dtype=np.complex128)
        self.N = N = self.y.shape[0]
        self.theta = np.asarray(theta, dtype=np.float64).copy()
        self.gamma = np.asarray(gamma, dtype=np.float64).copy()
        self.beta = float(beta)
        self.A = steering(N, self.theta)
        self.C = self.beta * np.eye(N, dtype=np.complex128) + (self.A * self.gamma) @ self.A.conj().T
        self.G = sla.cholesky(self.C, lower=True, check_finite=False)
        self.logdet = float(2.0 * np.sum(np.log(np.diag(self.G).real)))
        self.x = self.solve(self.y)
        self.yCy = float(np.vdot(self.y, self.x).real)

    # C^{-1} b through the two triangular solves of the Cholesky factor
    def solve(self, b):
        z = sla.solve_triangular(self.G, b, lower=True, check_finite=False)
        return sla.solve_triangular(self.G.conj().T, z, lower=False, check_finite=False)

    def whiten(self, b):
        """G^{-1} b, so that b^H C^{-1} b' = (G^{-1} b)^H (G^{-1} b')."""
        return sla.solve_triangular(self.G, b, lower=True, check_finite=False)

    # ---- objective (eq. obj) ------------------------------------------------
    def data_term(self) -> float:
        """ln|C| + y^H C^{-1} y: the part of eq. (obj) that depends on C."""
        return self.logdet + self.yCy

    def objective(self, zeta: float) -> float:
        """Eq. (obj) with K_max = N and 0 ln 0 = 0."""
        K = self.theta.shape[0]
        return self.data_term() - prior_term(K, self.N, zeta)

    # ---- the vectors of Sec. II-C, eqs. (q)-(x) -----------------------------
    def active_vectors(self):
        """q, r, s, t, u, v, x at the active frequencies (eqs. q-x, Phi = I)."""
        A = self.A
        d = index_weights(self.N)[:, None]
        W = self.solve(A)  # C^{-1} A
        DW = self.solve(d * A)  # C^{-1} D A
        AH = A.conj()
        q = AH.T @ self.x
        r = AH.T @ (d[:, 0] * self.x)
        u = AH.T @ (d[:, 0] ** 2 * self.x)
        s = np.sum(AH * W, axis=0)
        t = np.sum(AH * d * W, axis=0)
        v = np.sum(AH * d ** 2 * W, axis=0)
        xx = np.sum(AH * d * DW, axis=0)
        return dict(q=q, r=r, s=s.real, t=t, u=u, v=v, x=xx.real)

    # ---- grid quantities (Sec. III-D), taken straight from the definitions ---
    def grid(self, L: int, derivatives: bool = False, chunk: int = 4096, points=None):
        """q(theta), s(theta) on theta_l = l/L (or at ``points``), and optionally
        their first and second theta-derivatives.

        q(theta) = psi^H C^{-1} y and s(theta) = psi^H C^{-1} psi (Sec. III-D);
        with psi' = jD psi and psi'' = -D^2 psi the product rule gives
        q' = psi'^H C^{-1} y, q'' = psi''^H C^{-1} y,
        s' = 2 Re(psi^H C^{-1} psi'), s'' = 2 Re(psi^H C^{-1} psi'') + 2 psi'^H C^{-1} psi'.
        Direct O(N^2 L) evaluation through triangular solves.
        """
        N = self.N
        thetas = (np.arange(L, dtype=np.float64) / L) if points is None else np.asarray(points, np.float64)
        d = index_weights(N)[:, None]
        out = {k: [] for k in (("q", "s", "dq", "d2q", "ds", "d2s") if derivatives else ("q", "s"))}
        for a in range(0, thetas.shape[0], chunk):
            P = steering(N, thetas[a:a + chunk])
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

    # ---- Gohberg-Semencul generators read off the dense factorisation -------
    def gs_generators(self):
        """rho and delta_0..delta_{N-1} of eq. (gohberg-semencul).

        delta_i are the pivots of C = L B L^H (Sec. III-A): with C = G G^H,
        delta_i = |G_ii|^2.  rho is the last column of C^{-1} scaled so that
        rho_{N-1} = 1, and delta_{N-1} = 1 / [C^{-1}]_{N-1,N-1}.
        """
        N = self.N
        e = np.zeros(N, complex)
        e[-1] = 1.0
        z = self.solve(e)
        rho = z / z[-1]
        delta = np.abs(np.diag(self.G)) ** 2
        return rho, delta


def prior_term(K: int, N: int, zeta: float) -> float:
    """sum_k z_k ln zeta + (1 - z_k) ln(1 - zeta) with K of N = K_max active (eq. obj)."""
    a = K * np.log(zeta) if K else 0.0
    b = (N - K) * np.log1p(-zeta) if N - K else 0.0
    return float(a + b)


def derivatives(vec, gamma, N: int):
    """First and second partial derivatives of eq. (obj) in theta_k and gamma_k
    (eqs. derivative, derivative2), from the vectors of eqs. (q)-(x)."""
    q, r, s, t, u, v, x = (vec[k] for k in "qrstuvx")
    g = np.asarray(gamma, dtype=np.float64)
    aq2 = np.abs(q) ** 2
    g_theta = 2.0 * g * np.imag(t - np.conj(q) * r)
    g_gamma = s - aq2
    h_theta = 2.0 * g * np.real(
        x - v + g * (t * t - x * s)
        + g * (x * aq2 + s * np.abs(r) ** 2 - 2.0 * t * r * np.conj(q))
        + (u * np.conj(q) - np.abs(r) ** 2))
    h_gamma = 2.0 * s * aq2 - s * s
    return g_theta, g_gamma, h_theta, h_gamma


# ---- single-component quantities (Sec. II-C4, II-C5) ------------------------

def leave_one_out(q, s, gamma):
    """q_{~k}, s_{~k} from q_k, s_k by Woodbury (Sec. II-C4, after eq. deactivate)."""
    den = 1.0 - np.asarray(gamma) * np.asarray(s)
    return np.asarray(q) / den, np.asarray(s) / den


def log_prior_odds(zeta: float) -> float:
    """ln((1 - zeta) / zeta); +inf when zeta = 0."""
    return np.inf if zeta <= 0.0 else float(np.log1p(-zeta) - np.log(zeta))


def delta_objective(q, s, gamma_bar, zeta: float):
    """Delta L(theta) of eq. (delta_L): change of eq. (obj) when a component with
    variance gamma_bar is activated at a frequency where q_{~k} = q, s_{~k} = s.
    |q|^2 / (gamma^-1 + s) is written gamma |q|^2 / (1 + gamma s)."""
    gb = np.asarray(gamma_bar, dtype=np.float64)
    s = np.asarray(s, dtype=np.float64)
    aq2 = np.abs(q) ** 2
    return np.log1p(gb * s) + log_prior_odds(zeta) - gb * aq2 / (1.0 + gb * s)


def activate_gamma(q, s):
    """Minimiser of the single-component objective over gamma (eq. activate_gamma)."""
    s = np.asarray(s, dtype=np.float64)
    aq2 = np.abs(q) ** 2
    return np.where(aq2 > s, (aq2 - s) / (s * s), 0.0)


def activation_rhs(s, gamma_bar, zeta: float):
    """Right-hand side of eq. (activate_derived) without tau."""
    gs = np.asarray(gamma_bar, dtype=np.float64) * np.asarray(s, dtype=np.float64)
    with np.errstate(divide="ignore"):
        return (1.0 + 1.0 / gs) * (np.log1p(gs) + log_prior_odds(zeta))


def activation_test(q, s, gamma_bar, zeta: float, tau: float = 0.0):
    """Eq. (activate_derived) for tau = 0 and eq. (activate_criterion) for tau > 0."""
    s = np.asarray(s, dtype=np.float64)
    return np.abs(q) ** 2 / s > activation_rhs(s, gamma_bar, zeta) + tau


def deactivation_statistic(q, s, gamma):
    """Left-hand side of eq. (deactivate) with q_{~k}, s_{~k} by Woodbury."""
    qt, st = leave_one_out(q, s, gamma)
    g = np.asarray(gamma, dtype=np.float64)
    return g * np.abs(qt) ** 2 / (1.0 + g * st) - np.log1p(g * st)


def zeta_update(K: int, N: int) -> float:
    """Eq. (zetaUpdate) with K_max = N."""
    return min(0.5, K / N)


def beta_update(ev: DenseEval, s, eps_beta: float) -> float:
    """Eq. (betaUpdate) with the Woodbury forms of Sec. II-C3:
    tr(Sigma A^H A) = sum_k beta s_k gamma_k, and ||y - A mu||^2 written as
    beta^2 ||C^{-1} y||^2 (y - A Gamma A^H C^{-1} y = beta C^{-1} y)."""
    b = ev.beta
    num = b * float(np.sum(np.asarray(s) * ev.gamma)) + b * b * float(np.vdot(ev.x, ev.x).real)
    return max(eps_beta, num / ev.N)
