"""Pins of the oracle's selection rules: the approximate multi-activation of
Sec. II-E (reading R6) and the deactivation of Sec. II-C4 (reading R3).

The inputs are built by hand so that the answer follows from the rules as the
paper states them: cyclic grid local minima, the Delta L <= Delta L_min / 5
threshold with Delta L_min < 0, the 0.05/N spacing by wrap distance against
every active frequency (including those taken earlier in the same pass),
ascending Delta L order; and for deactivation, removal of the qualifying
component whose removal lowers eq. (obj) most, one at a time with a
re-evaluation in between.  Each case is chosen so that a plausible slip (a
different divisor or spacing, no wrap-around, a non-strict left comparison,
the wrong plateau point, descending order, forgetting components taken in
the same pass, removing every qualifying component at once) gives a
different answer.
"""
import numpy as np
import pytest

from oracle import dense as dn
from oracle import fit as of

N, L = 4, 256          # 0.05/N = 3.2 grid steps of 1/L
ZETA = 0.2             # ln((1 - zeta)/zeta) = ln 4
GBAR = 1.0


def grid(dips, base=1.0, strong=True):
    """Delta L = base everywhere except the given {l: value}; s = 1 and
    |q|^2 = 10 at every point, so gamma-hat = 9 > 0 and eq. (activate_derived)
    holds (10 > (1 + 1)(ln 2 + ln 4) = 4.16) wherever it is asked."""
    dl = np.full(L, base)
    for l, v in dips.items():
        dl[l] = v
    s = np.ones(L)
    q = np.full(L, np.sqrt(10.0) if strong else 1.0, dtype=complex)
    return dl, q, s


def select(dl, q, s, active=(), room=L, gbar=GBAR):
    taken = of.approximate_activation_select(dl, q, s, gbar, ZETA, np.array(active, float), N, L, room)
    return [l for l, _ in taken]


def test_strong_grid_point_passes_activation_test():
    # the premise of the hand-built grids
    assert dn.activation_test(np.sqrt(10.0), 1.0, GBAR, ZETA, 0.0)
    assert float(dn.activate_gamma(np.sqrt(10.0), 1.0)) == pytest.approx(9.0)


def test_threshold_is_one_fifth_of_the_deepest_minimum():
    """-10, -3, -1.5: Delta L_min / 5 = -2 takes the first two only (/2 would
    take one, /10 all three)."""
    dl, q, s = grid({10: -10.0, 50: -3.0, 90: -1.5})
    assert select(dl, q, s) == [10, 50]


def test_nothing_happens_unless_the_deepest_minimum_is_negative():
    dl, q, s = grid({7: 0.5, 70: 0.2}, base=5.0)
    assert select(dl, q, s) == []
    dl, q, s = grid({7: 0.0}, base=5.0)
    assert select(dl, q, s) == []


def test_spacing_is_five_hundredths_of_a_bin_against_active_frequencies():
    """Active theta = 0.5 (grid point 128).  130 is 2 steps away (< 3.2: too
    close), 134 is 6 steps away (kept; 0.5/N = 32 steps would reject it)."""
    dl, q, s = grid({130: -10.0, 134: -9.0})
    assert select(dl, q, s, active=[0.5]) == [134]


def test_spacing_uses_wrap_distance():
    """theta = 0.999 is 1.26 grid steps from grid point 1 across 1 = 0;
    grid point 40 is far from it."""
    dl, q, s = grid({1: -10.0, 40: -9.0})
    assert select(dl, q, s, active=[0.999]) == [40]


def test_local_minima_are_cyclic():
    """Grid point 0 is a minimum through its left neighbour L-1."""
    dl, q, s = grid({0: -10.0, L - 1: -9.0, 1: -9.5})
    assert select(dl, q, s) == [0]


def test_left_neighbour_of_the_first_point_is_the_last():
    """A descent L-1 -> L-4 that continues across the end: grid point 0 is not
    a minimum (its left neighbour L-1 is lower); an edge without the cyclic
    neighbour would take it too (4 steps from L-4)."""
    dl, q, s = grid({L - 4: -10.0, L - 3: -9.8, L - 2: -9.6, L - 1: -9.4, 0: -9.2})
    assert select(dl, q, s) == [L - 4]


def test_right_neighbour_of_the_last_point_is_the_first():
    """A descent L-1 -> 3 across the end: L-1 is not a minimum (its right
    neighbour 0 is lower)."""
    dl, q, s = grid({L - 1: -9.2, 0: -9.4, 1: -9.6, 2: -9.8, 3: -10.0})
    assert select(dl, q, s) == [3]


def test_plateau_keeps_its_first_point():
    """A plateau over 20..24: only 20 is a candidate (strict on the left, not
    on the right).  A non-strict left test would also take 24 (4 steps away);
    keeping the last point would take 24 instead of 20."""
    dl, q, s = grid({20: -10.0, 21: -10.0, 22: -10.0, 23: -10.0, 24: -10.0})
    assert select(dl, q, s) == [20]


def test_visited_in_ascending_delta_L_against_those_taken_in_the_same_pass():
    """Minima at 100 (-8) and 102 (-10), 2 steps apart: 102 is visited first
    and taken, which excludes 100.  Descending order would give [100];
    forgetting what the pass took would give [102, 100]."""
    dl, q, s = grid({100: -8.0, 101: -5.0, 102: -10.0})
    assert select(dl, q, s) == [102]


def test_ties_are_visited_by_index():
    dl, q, s = grid({200: -10.0, 40: -10.0})
    assert select(dl, q, s) == [40, 200]
    assert select(dl, q, s, room=1) == [40]


def test_failed_activation_test_skips_the_candidate_only():
    """The deepest minimum has gamma-hat = 0 (|q|^2 <= s), the next fails eq.
    (activate_derived) (|q|^2 / s = 3 < 4.16): both are skipped and the third
    is still taken."""
    dl, q, s = grid({10: -10.0, 60: -9.0, 120: -8.0})
    q[10] = 1.0
    q[60] = np.sqrt(3.0)
    assert float(dn.activate_gamma(q[60], s[60])) > 0.0
    assert not dn.activation_test(q[60], s[60], GBAR, ZETA, 0.0)
    assert select(dl, q, s) == [120]


def test_per_point_gamma_bar_when_nothing_is_active():
    """With no active component gamma-bar is the point's own gamma-hat (R4):
    the pure function reads it per grid point."""
    dl, q, s = grid({10: -10.0, 60: -9.0})
    gbar = np.full(L, 1.0)
    gbar[60] = 1e-12  # eq. (activate_derived) fails for a vanishing gamma-bar
    assert select(dl, q, s, gbar=gbar) == [10]


# ------------------------------------------------------------ deactivation --

def test_deactivation_pick_smallest_statistic_below_threshold_earliest_on_ties():
    assert of.deactivation_pick([1.0, -0.5, 0.2, -0.5], 0.0) == 1
    assert of.deactivation_pick([0.5, 0.3], 0.4) == 1
    assert of.deactivation_pick([0.5, 0.45], 0.4) is None
    assert of.deactivation_pick([], 0.4) is None


def _state(y, theta, gamma, beta, zeta):
    st = of._State(y, 8 * len(y), 5.0, None)
    st.theta, st.gamma, st.beta, st.zeta = np.array(theta, float), np.array(gamma, float), beta, zeta
    st.refresh()
    return st


def _signal(seed=1, n=32):
    r = np.random.default_rng(seed)
    t = np.arange(n)
    return 3.0 * np.exp(2j * np.pi * t * 0.3) + 0.3 * (r.standard_normal(n) + 1j * r.standard_normal(n)) / np.sqrt(2)


def test_deactivation_removes_the_component_whose_removal_lowers_the_objective_most():
    """The picked component is, among those meeting eq. (deactivate), the one
    whose removal gives the lowest dense objective (eq. obj), and every
    qualifying removal lowers it."""
    y = _signal()
    beta, zeta = 0.09, 0.1
    theta = [0.3, 0.71, 0.12, 0.52]
    gamma = [9.0, 0.02, 0.2, 0.05]
    ev = dn.DenseEval(y, theta, gamma, beta)
    vec = ev.active_vectors()
    stat = dn.deactivation_statistic(vec["q"], vec["s"], np.array(gamma))
    thr = dn.log_prior_odds(zeta)
    hit = [k for k in range(4) if stat[k] < thr]
    assert len(hit) >= 2  # premise: a real choice
    base = ev.objective(zeta)
    after = {k: dn.DenseEval(y, np.delete(theta, k), np.delete(gamma, k), beta).objective(zeta) for k in range(4)}
    for k in range(4):
        assert (after[k] < base) == (k in hit)
    assert of.deactivation_pick(stat, thr) == min(hit, key=lambda k: after[k])


def test_deactivation_removes_one_at_a_time_and_re_evaluates():
    """Two components at the same frequency with equal gamma both meet eq.
    (deactivate) (a tie: the earliest goes); once one is gone the other
    explains the sinusoid and stays.  Removing every qualifying component of
    the first evaluation would remove both."""
    y = _signal()
    st = _state(y, [0.3, 0.3], [9.0, 9.0], 0.09, 0.1)
    vec = st.ev.active_vectors()
    stat = dn.deactivation_statistic(vec["q"], vec["s"], st.gamma)
    assert np.all(stat < dn.log_prior_odds(st.zeta))
    assert of._deactivation(st) == 1
    assert st.K == 1 and st.theta[0] == 0.3


def test_deactivation_repeats_until_nothing_qualifies():
    """Two weak components at noise-only frequencies beside the sinusoid: each
    still qualifies after the other is removed, so both go; the sinusoid
    stays."""
    y = _signal()
    st = _state(y, [0.3, 0.71, 0.52], [9.0, 0.02, 0.05], 0.09, 0.1)
    assert of._deactivation(st) == 2
    assert st.K == 1 and st.theta[0] == 0.3
