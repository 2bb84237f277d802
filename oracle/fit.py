"""The superfast-LSE estimator run with dense linear algebra (oracle; test
infrastructure only).

Block-coordinate descent on eq. (obj) in the order of Sec. II-D:
(1) activation (Sec. II-C5; approximate multi-activation of Sec. II-E in the
first iterations), (2) zeta (eq. zetaUpdate), (3) beta (eq. betaUpdate),
(4) repeat { one (theta, gamma) update; deactivation (eq. deactivate) }.

Readings where the paper is silent or leaves a choice (each also listed in the
design notes):

R1  (theta, gamma) update.  One iteration of step 4a is a per-component
    diagonal Newton step: d = -g / h, with g and h from eqs. (derivative),
    (derivative2); a non-positive h is replaced by (50N)^2 for theta and
    gamma_k^-2 for gamma (Sec. II-C1).  The step length starts at 1, is cut
    to 0.99 of the distance at which the first gamma_k would reach zero, and
    is halved (at most 30 times) until the Armijo condition
    f(new) <= f + 1e-4 alpha g.d holds for f = ln|C| + y^H C^{-1} y.  If no
    length is accepted the state is kept.  theta is taken modulo 1.
R2  Step 4 stops after 5 iterations, or after the iteration whose squared
    Newton decrement sum g^2/h is below N 1e-8 (that iteration takes no step
    but still runs the deactivation check).
R3  Deactivation: among the components meeting eq. (deactivate), the one whose
    removal lowers eq. (obj) most is removed; ties go to the earliest
    activated.  Repeat until none qualifies.
R4  gamma-bar (eq. delta_L) is the mean of the active gamma; with no active
    component it is the candidate's own gamma of eq. (activate_gamma).
R5  Exact activation (step 1): argmin of Delta L over the grid (lowest index on
    ties); activate if gamma > 0 and eq. (activate_criterion) holds with
    tau = 5; repeat until nothing is activated.
R6  Approximate activation (Sec. II-E) runs in outer iterations 1..10 while it
    activates something; once a pass activates nothing, that iteration and all
    later ones use exact activation.  Candidates are grid points with
    Delta L(l) < Delta L(l-1) and Delta L(l) <= Delta L(l+1) (cyclic); they are
    visited in ascending Delta L (ties by index) and accepted when
    Delta L <= Delta L_min / 5 with Delta L_min < 0, gamma > 0, eq.
    (activate_derived) holds, and every active frequency (including ones
    accepted earlier in the pass) is at wrap distance >= 0.05/N.  All
    quantities come from the one grid evaluated at the start of the pass.
R7  eps_beta = 1e-12 ||y||^2 / N; eps_L = 2^-52; K_max = N.
R8  Termination: |L_i - L_{i-1}| < N 1e-7 with L_0 the objective of the
    initial state; at most 200 outer iterations (status "not converged").
R9  beta is updated with s, q and C^{-1}y at the current state and the old beta.
R10 Output components are sorted by frequency; alpha = gamma * q at the final
    state (footnote to eq. bmu).
R11 y = 0 is degenerate: the result is K = 0, beta = 0.

With update="lbfgs" step 4a is the paper's own L-BFGS update (Sec. II-C1,
J = 10 saved pairs) instead of R1's diagonal Newton step:
L1  The variables are (theta_k, gamma_k) of the active components; the
    initial inverse Hessian of every iteration is diag(1/h) with h the
    diagonal Hessian of eqs. (derivative2) and its replacements (R1), as
    Sec. II-C1 proposes; the direction is -H g by the two-loop recursion
    (Nocedal and Wright, Numerical Optimization, Alg. 7.4) over the saved
    pairs (s_i, y_i) = (step, gradient change).
L2  The same step rule as R1 (length 1 cut to 0.99 of the distance to the
    first gamma = 0, Armijo backtracking); a pair is saved only when
    s.y > 0; at most J = 10 pairs, the oldest dropped.
L3  The memory is emptied whenever the problem changes under it: at the
    start of step 4 of every outer iteration (beta and possibly the active
    set changed) and after every deactivation (the paper: the Hessian
    estimate is reinitialised when the activation variables change).
L4  The squared Newton decrement of R2 is g.H g with H the L-BFGS inverse
    Hessian (-g.d), against the same N 1e-8 threshold.
With no saved pair the direction is R1's diagonal Newton step.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import dense as dn

EPS_L = 2.0 ** -52


@dataclasses.dataclass
class FitResult:
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
    trace: list  # (block name, objective after the block)

    @property
    def K(self) -> int:
        return int(self.theta.shape[0])


class _State:
    def __init__(self, y, L, tau, trace):
        self.y = np.asarray(y, dtype=np.complex128)
        self.N = self.y.shape[0]
        self.L = int(L)
        self.tau = float(tau)
        yy = float(np.vdot(self.y, self.y).real)
        self.beta = 0.01 * yy / self.N
        self.eps_beta = 1e-12 * yy / self.N
        self.zeta = 0.2
        self.theta = np.zeros(0)
        self.gamma = np.zeros(0)
        self.n_evals = 0
        self.n_grid = 0
        self.trace = trace
        self.ev = self.evaluate()

    @property
    def K(self):
        return self.theta.shape[0]

    def evaluate(self, theta=None, gamma=None):
        self.n_evals += 1
        return dn.DenseEval(self.y, self.theta if theta is None else theta,
                            self.gamma if gamma is None else gamma, self.beta)

    def refresh(self):
        self.ev = self.evaluate()

    def objective(self):
        return self.ev.objective(self.zeta)

    def log(self, name):
        if self.trace is not None:
            self.trace.append((name, self.objective()))

    def grid_delta(self):
        """Grid q, s and Delta L with gamma-bar per R4 (Sec. II-C5)."""
        self.n_grid += 1
        g = self.ev.grid(self.L)
        q, s = g["q"], g["s"]
        gbar = np.mean(self.gamma) if self.K else dn.activate_gamma(q, s)
        dl = dn.delta_objective(q, s, gbar, self.zeta)
        return q, s, gbar, dl

    def add(self, theta, gamma):
        self.theta = np.append(self.theta, theta)
        self.gamma = np.append(self.gamma, gamma)


def _exact_activation(st: _State, first=None):
    """R5: single activations until none qualifies (Sec. II-C5, step 1)."""
    n = 0
    while st.K < st.N and st.zeta > 0.0:
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


def approximate_activation_select(dl, q, s, gbar, zeta: float, theta_active, N: int, L: int, K_room: int):
    """The candidate rules of the approximate multi-activation scheme (Sec. II-E,
    reading R6), on one grid evaluation.

    dl, q, s: Delta L (eq. delta_L), q and s at the grid points l/L; gbar: the
    gamma-bar of that evaluation (a scalar, or one value per grid point when no
    component is active, R4); theta_active: the frequencies active before the
    pass; K_room: how many more components the model may hold (K_max - K).
    A candidate is taken when its eq. (activate_gamma) value is > 0 and eq.
    (activate_derived) holds (no tau); the rest of the rules are those of
    ``select_candidates``.  Returns [(l, gamma_hat)] in the order taken."""
    s = np.asarray(s, dtype=np.float64)
    with np.errstate(divide="ignore", invalid="ignore"):
        ghat = dn.activate_gamma(q, s)
        gb = np.broadcast_to(np.asarray(gbar, dtype=np.float64), s.shape)
        passes = dn.activation_test(q, s, gb, zeta, 0.0)
    return select_candidates(dl, ghat, passes, theta_active, N, L, K_room)


def select_candidates(dl, ghat, passes, theta_active, N: int, L: int, K_room: int):
    """Sec. II-E (reading R6) given, per grid point, the variance a component
    would get there (ghat) and whether the activation test holds (passes).

    Candidates are the cyclic local minima Delta L(l) < Delta L(l-1),
    Delta L(l) <= Delta L(l+1) (a plateau keeps its first point).  With
    Delta L_min the smallest candidate value, nothing happens unless
    Delta L_min < 0; otherwise the candidates are visited in ascending
    Delta L (ties by index) while Delta L <= Delta L_min / 5, and a candidate
    is taken when ghat > 0, the test holds and it lies at wrap distance
    >= 0.05/N from every active frequency, those taken earlier in the same
    pass included.  Returns [(l, gamma_hat)] in the order taken."""
    dl = np.asarray(dl, dtype=np.float64)
    left = np.roll(dl, 1)
    right = np.roll(dl, -1)
    cand = np.nonzero((dl < left) & (dl <= right))[0]
    if cand.size == 0:
        return []
    dlmin = float(np.min(dl[cand]))
    if not dlmin < 0.0:
        return []
    order = cand[np.lexsort((cand, dl[cand]))]
    taken = []
    active = list(np.atleast_1d(np.asarray(theta_active, dtype=np.float64)))
    for l in order:
        if not dl[l] <= dlmin / 5.0:
            break
        if len(taken) >= K_room:
            break
        gh = float(ghat[l])
        if not gh > 0.0:
            continue
        if not bool(passes[l]):
            continue
        th = l / L
        if active and np.min(_wrap(th, np.array(active))) < 0.05 / N:
            continue
        taken.append((int(l), gh))
        active.append(th)
    return taken


def _approximate_activation(st: _State):
    """R6: one pass of the approximate multi-activation scheme (Sec. II-E).
    Returns (number activated, grid data for reuse when nothing changed)."""
    if st.zeta <= 0.0 or st.K >= st.N:
        return 0, None
    grid = st.grid_delta()
    q, s, gbar, dl = grid
    taken = approximate_activation_select(dl, q, s, gbar, st.zeta, st.theta, st.N, st.L, st.N - st.K)
    for l, ghat in taken:
        st.add(l / st.L, ghat)
    if taken:
        st.refresh()
    return len(taken), grid


def _wrap(a, b):
    d = np.abs(np.asarray(a) - np.asarray(b)) % 1.0
    return np.minimum(d, 1.0 - d)


def _newton_iteration(st: _State):
    """R1/R2: one (theta, gamma) update.  Returns (decrement, step taken)."""
    N = st.N
    vec = st.ev.active_vectors()
    gt, gg, ht, hg = dn.derivatives(vec, st.gamma, N)
    ht = np.where(ht > 0.0, ht, (50.0 * N) ** 2)
    hg = np.where(hg > 0.0, hg, 1.0 / st.gamma ** 2)
    dt = -gt / ht
    dg = -gg / hg
    dec = float(np.sum(gt * gt / ht) + np.sum(gg * gg / hg))
    if dec < N * 1e-8:
        return dec, False
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
            return dec, True
        alpha *= 0.5
    return dec, False


def lbfgs_direction(g, h, S, Y):
    """L1: d = -H g for the L-BFGS inverse Hessian H built from the initial
    diag(1/h) and the pairs (S[i], Y[i]) (oldest first), by the two-loop
    recursion."""
    q = np.array(g, dtype=np.float64)
    stack = []
    for s_, y_ in zip(reversed(S), reversed(Y)):
        rho = 1.0 / float(np.dot(y_, s_))
        a = rho * float(np.dot(s_, q))
        q = q - a * y_
        stack.append((rho, a, s_, y_))
    r = q / np.asarray(h, dtype=np.float64)
    for rho, a, s_, y_ in reversed(stack):
        b = rho * float(np.dot(y_, r))
        r = r + (a - b) * s_
    return -r


class LbfgsMemory:
    """L2/L3: the saved pairs and the step waiting for its gradient change."""

    def __init__(self, J: int = 10):
        self.J = J
        self.reset()

    def reset(self):
        self.S, self.Y = [], []
        self.pending = None  # (step s, gradient before the step)

    def absorb(self, g):
        """Turn the pending step into a pair with the gradient g after it."""
        if self.pending is not None:
            s_, g0 = self.pending
            y_ = g - g0
            if float(np.dot(s_, y_)) > 0.0:
                self.S.append(s_)
                self.Y.append(y_)
                if len(self.S) > self.J:
                    self.S.pop(0)
                    self.Y.pop(0)
        self.pending = None


def _lbfgs_iteration(st: _State, mem: LbfgsMemory):
    """L1-L4: one L-BFGS update of (theta, gamma).  Returns (decrement, step taken)."""
    N = st.N
    K = st.K
    vec = st.ev.active_vectors()
    gt, gg, ht, hg = dn.derivatives(vec, st.gamma, N)
    ht = np.where(ht > 0.0, ht, (50.0 * N) ** 2)
    hg = np.where(hg > 0.0, hg, 1.0 / st.gamma ** 2)
    g = np.concatenate([gt, gg])
    mem.absorb(g)
    d = lbfgs_direction(g, np.concatenate([ht, hg]), mem.S, mem.Y)
    dec = float(-np.dot(g, d))
    if dec < N * 1e-8:
        return dec, False
    dt, dg = d[:K], d[K:]
    slope = float(np.dot(g, d))
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
            mem.pending = (alpha * d, g)
            return dec, True
        alpha *= 0.5
    return dec, False


def deactivation_pick(stat, threshold: float):
    """Which component one step of the deactivation of Sec. II-C4 removes
    (reading R3): among those whose eq. (deactivate) statistic is below the
    threshold ln((1 - zeta)/zeta), the one with the smallest statistic, whose
    removal lowers eq. (obj) most (the change is statistic - threshold); ties go
    to the lowest index, i.e. the earliest activated.  None if none qualifies."""
    stat = np.asarray(stat, dtype=np.float64)
    hit = np.nonzero(stat < threshold)[0]
    if hit.size == 0:
        return None
    return int(hit[np.argmin(stat[hit])])


def _deactivation(st: _State):
    """R3: remove components meeting eq. (deactivate) one at a time, re-evaluating
    the model after each removal ("repeated until no more can be deactivated")."""
    n = 0
    while st.K > 0:
        vec = st.ev.active_vectors()
        stat = dn.deactivation_statistic(vec["q"], vec["s"], st.gamma)
        k = deactivation_pick(stat, dn.log_prior_odds(st.zeta))
        if k is None:
            break
        st.theta = np.delete(st.theta, k)
        st.gamma = np.delete(st.gamma, k)
        st.refresh()
        n += 1
    return n


def fit(y, L: int, tau: float = 5.0, max_outer: int = 200, max_inner: int = 5,
        approx_iters: int = 10, trace: bool = False, update: str = "newton") -> FitResult:
    """Run the estimator of Sec. II on y (complete data, K_max = N); update is
    "newton" (R1) or "lbfgs" (L1-L4) for step 4a."""
    y = np.asarray(y, dtype=np.complex128)
    N = y.shape[0]
    tr = [] if trace else None
    if float(np.vdot(y, y).real) == 0.0:  # R11
        return FitResult(np.zeros(0), np.zeros(0), np.zeros(0, complex), 0.0, 0.0, 0.0,
                         0, True, 0, 0, tr or [])
    st = _State(y, L, tau, tr)
    L_prev = st.objective()
    st.log("init")
    approx = approx_iters > 0
    converged = False
    it = 0
    for it in range(1, max_outer + 1):
        # step 1: activation
        if approx and it <= approx_iters:
            n, grid = _approximate_activation(st)
            if n == 0:
                approx = False
                _exact_activation(st, first=grid)
        else:
            _exact_activation(st)
        st.log("activate")
        # step 2: zeta
        st.zeta = dn.zeta_update(st.K, N)
        st.log("zeta")
        # step 3: beta (R9)
        if st.K:
            s = st.ev.active_vectors()["s"]
        else:
            s = np.zeros(0)
        st.beta = dn.beta_update(st.ev, s, st.eps_beta)
        st.refresh()
        st.log("beta")
        # step 4
        mem = LbfgsMemory() if update == "lbfgs" else None
        for _ in range(max_inner):
            if st.K == 0:
                break
            if mem is None:
                dec, _stepped = _newton_iteration(st)
            else:
                dec, _stepped = _lbfgs_iteration(st, mem)
            st.log("theta_gamma")
            if _deactivation(st) and mem is not None:
                mem.reset()
            st.log("deactivate")
            if dec < N * 1e-8:
                break
        L_cur = st.objective()
        if abs(L_cur - L_prev) < N * 1e-7:
            converged = True
            break
        L_prev = L_cur
    K = st.K
    q = st.ev.active_vectors()["q"] if K else np.zeros(0, complex)
    order = np.argsort(st.theta, kind="stable")
    return FitResult(theta=st.theta[order], gamma=st.gamma[order], alpha=(st.gamma * q)[order],
                     beta=st.beta, zeta=st.zeta, objective=st.objective(), iters=it,
                     converged=converged, n_evals=st.n_evals, n_grid_evals=st.n_grid,
                     trace=tr or [])
