"""Pins for the control rules that steer the oracle's restarted PDHG loop.

orc_solve calls orc_restart_rule, orc_pid_update and orc_inner_tol; these tests
feed each one cases whose answers follow by hand from the printed formulas and
the constants of Table practical-defaults:

* eq. practical-restart-rule with (beta_s, beta_n, beta_a) = (0.20, 0.80, 0.36):
  each of its three clauses fires alone, on both sides of its threshold, and
  none fires;
* eqs. pid-error / pid-weight with (beta_I, K_P, K_I, K_D) = (0.30, 0.99, 0.01,
  0.00): a movement ratio ||dy|| = e^c omega ||dx|| gives e_n = c exactly, so
  log omega moves by K_P c + K_I I_n with I_n = beta_I I_{n-1} + c;
* eq. monotone-primal-inner-tol with (gamma_in, eps_min) = (5e-4, 1e-9): the
  min / max structure on cases where each of the three candidates wins.

Each expected value is written out as a number, so a swapped constant, a
flipped comparison or sign, or min in place of max changes at least one answer.
"""
import math

import pytest


# --------------------------------------------------------------------------- restart rule

@pytest.mark.parametrize("E,E0,Eprev,k,ktot,expect", [
    # clause 1 (sufficient decay E <= 0.2 E0) alone: E falls, k small
    (0.19, 1.0, 0.50, 5, 100, True),
    (0.20, 1.0, 0.50, 5, 100, True),          # threshold included
    (0.21, 1.0, 0.50, 5, 100, False),         # just above, still falling, k below 0.36 ktot
    (1.9, 10.0, 5.0, 5, 100, True),           # scale invariance in E0
    # clause 2 (necessary decay E <= 0.8 E0 with a rise E > Eprev) alone
    (0.79, 1.0, 0.70, 5, 100, True),
    (0.80, 1.0, 0.70, 5, 100, True),          # threshold included
    (0.81, 1.0, 0.70, 5, 100, False),         # rise, but above 0.8 E0
    (0.79, 1.0, 0.80, 5, 100, False),         # below 0.8 E0, but no rise
    (0.79, 1.0, 0.79, 5, 100, False),         # equal is not a rise
    (0.50, 1.0, 0.60, 5, 100, False),         # falling between 0.2 and 0.8: nothing fires
    # clause 3 (artificial limit k >= 0.36 ktot) alone: E high and rising
    (0.95, 1.0, 0.90, 36, 100, True),
    (0.95, 1.0, 0.90, 35, 100, False),
    (0.95, 1.0, 0.90, 18, 50, True),          # 18 = 0.36 * 50
    (0.95, 1.0, 0.90, 17, 50, False),
    # nothing restarts at the first iteration of an epoch
    (0.0, 1.0, 1.0, 0, 100, False),
])
def test_restart_rule_clauses(orc, E, E0, Eprev, k, ktot, expect):
    assert orc.restart_rule(E, E0, Eprev, k, ktot) is expect


def test_restart_rule_follows_its_constants(orc):
    # the same case restarts or not as each threshold is moved across it
    assert orc.restart_rule(0.5, 1.0, 0.6, 5, 100, beta_s=0.6)
    assert not orc.restart_rule(0.5, 1.0, 0.4, 5, 100, beta_n=0.45)
    assert orc.restart_rule(0.5, 1.0, 0.4, 5, 100, beta_n=0.5)
    assert orc.restart_rule(0.9, 1.0, 0.95, 5, 100, beta_a=0.05)


# --------------------------------------------------------------------------- PID primal weight

def test_pid_unit_error_step(orc):
    # ||dy|| = e * omega * ||dx||: e_0 = 1, I_0 = 0.3 * 0 + 1 = 1,
    # log omega_1 = log 2 + 0.99 * 1 + 0.01 * 1 + 0 = log 2 + 1
    st = [0.0, 0.0]
    w1 = orc.pid_update(2.0, 0.5, 0.5 * 2.0 * math.e, st)
    assert w1 == pytest.approx(2.0 * math.e, rel=1e-14)
    assert st == pytest.approx([1.0, 1.0], rel=1e-14)
    # second restart at the same ratio relative to the new weight: e_1 = 1,
    # I_1 = 0.3 * 1 + 1 = 1.3, log omega_2 = log omega_1 + 0.99 + 0.013
    w2 = orc.pid_update(w1, 3.0, 3.0 * w1 * math.e, st)
    assert math.log(w2) == pytest.approx(math.log(w1) + 1.003, rel=1e-14)
    assert st == pytest.approx([1.3, 1.0], rel=1e-14)


def test_pid_sign_and_integral(orc):
    # ||dy|| = omega ||dx|| / 4: e = -log 4; I = 0.3 * 2 - log 4 from I_{-1} = 2
    st = [2.0, 0.0]
    w = orc.pid_update(1.5, 2.0, 1.5 * 2.0 / 4.0, st)
    e = -math.log(4.0)
    assert math.log(w) == pytest.approx(math.log(1.5) + 0.99 * e + 0.01 * (0.6 + e), rel=1e-13)
    assert st[0] == pytest.approx(0.6 + e, rel=1e-14)
    assert st[1] == pytest.approx(e, rel=1e-14)


def test_pid_derivative_term(orc):
    # K_D = 0.5 with e_{n-1} = 0.25 and e_n = log 3: the derivative adds 0.5 (log 3 - 0.25)
    st = [0.0, 0.25]
    w = orc.pid_update(1.0, 1.0, 3.0, st, K_D=0.5)
    e = math.log(3.0)
    assert math.log(w) == pytest.approx(0.99 * e + 0.01 * e + 0.5 * (e - 0.25), rel=1e-13)


def test_pid_skips_tiny_movements_and_off_switch(orc):
    st = [0.7, 0.2]
    assert orc.pid_update(3.0, 1e-12, 1.0, st) == 3.0
    assert orc.pid_update(3.0, 1.0, 1e-12, st) == 3.0
    assert orc.pid_update(3.0, 1.0, 10.0, st, pid=0) == 3.0
    assert st == [0.7, 0.2]


def test_pid_balanced_movement_keeps_weight(orc):
    # ||dy|| = omega ||dx||: e = 0, and with I_{-1} = 0 the weight is unchanged
    st = [0.0, 0.0]
    assert orc.pid_update(0.37, 2.0, 0.74, st) == pytest.approx(0.37, rel=1e-15)


# --------------------------------------------------------------------------- inner tolerance

@pytest.mark.parametrize("eps_prev,mov,tau,expect", [
    (1e-3, 1.0, 10.0, 5e-5),      # gamma mov / tau = 5e-5 wins over eps_prev = 1e-3
    (1e-6, 1.0, 10.0, 1e-6),      # monotone: the previous tolerance is never raised
    (1e-3, 0.0, 10.0, 1e-9),      # no movement: the floor eps_min
    (1e-3, 1e-7, 1.0, 1e-9),      # 5e-11 < eps_min: the floor
    (1e-3, 2.0, 0.5, 1e-3),       # 2e-3 > eps_prev: eps_prev stays
])
def test_inner_tolerance(orc, eps_prev, mov, tau, expect):
    assert orc.inner_tol(eps_prev, mov, tau) == pytest.approx(expect, rel=1e-15)
