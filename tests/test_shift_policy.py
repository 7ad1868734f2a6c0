"""Host logic of the shift policies (Prop. 4.2, Algorithm 1's policies),
checked against the oracle's statement of the reuse rule.  No GPU needed:
rsign_shift_can_reuse and rsign_shift_damped are host functions of the
library."""
import math

import numpy as np
import pytest

import oracle
from helpers import lib_or_fail


def _state(rs, m_hat, eps, shift=0.0):
    st = rs.shift_state()
    st.shift = shift
    st.lam_k_est = shift - m_hat
    st.lam_k1_est = shift + m_hat
    st.eps = eps
    st.margin_cert = m_hat - eps
    return st


def test_fresh_state_never_reuses():
    rs = lib_or_fail()
    st = rs.shift_state()
    assert math.isnan(st.shift) and math.isnan(st.margin_cert)
    assert st.refreshes == 0 and st.reuses == 0
    assert not rs.shift_can_reuse(st, 0.0, 0.0)


def test_reuse_rule_matches_prop_4_2():
    rs = lib_or_fail()
    rng = np.random.default_rng(3)
    for _ in range(2000):
        m_hat = rng.uniform(1e-4, 1.0)
        eps = m_hat * rng.uniform(0.0, 1.2)
        drift = m_hat * rng.uniform(0.0, 1.2)
        ok_or, guaranteed = oracle.reuse_admissible(m_hat, eps, drift)
        st = _state(rs, m_hat, eps)
        if m_hat - eps <= 0:
            continue  # a shift with no certified margin is never in a state
        assert rs.shift_can_reuse(st, drift, 0.0) == ok_or
        # with a threshold the certified margin must stay above it
        tau = 0.5 * max(guaranteed, 0.0)
        assert rs.shift_can_reuse(st, drift, tau) == (ok_or and guaranteed > tau)


def test_reuse_rejects_bad_inputs():
    rs = lib_or_fail()
    st = _state(rs, 0.5, 0.1)
    assert rs.shift_can_reuse(st, 0.1, 0.0)
    assert not rs.shift_can_reuse(st, float("nan"), 0.0)
    assert not rs.shift_can_reuse(st, -1.0, 0.0)
    assert not rs.shift_can_reuse(st, float("inf"), 0.0)
    assert not rs.shift_can_reuse(st, 0.1, -1.0)


def test_damped_midpoint():
    rs = lib_or_fail()
    lk, lk1, eps = -0.3, 0.5, 0.05
    mid = oracle.midpoint(lk, lk1)
    # no previous shift: the midpoint
    assert rs.shift_damped(float("nan"), lk, lk1, eps, 0.5) == mid
    # damping 0: the midpoint; inside the interval: the blend
    assert rs.shift_damped(0.2, lk, lk1, eps, 0.0) == pytest.approx(mid)
    assert rs.shift_damped(0.2, lk, lk1, eps, 0.5) == pytest.approx(0.5 * 0.2 + 0.5 * mid)
    # far outside: clipped, and certified by the margin test of Prop. 4.2
    lo, hi = lk + eps, lk1 - eps
    pad = 0.25 * 0.5 * (hi - lo)
    for s_prev in (-5.0, 5.0, lk, lk1):
        s = rs.shift_damped(s_prev, lk, lk1, eps, 0.9)
        assert lo + pad - 1e-15 <= s <= hi - pad + 1e-15
        ok, m_hat, _ = oracle.admissible(s, lk, lk1, eps)
        assert ok and m_hat > eps
    # an empty certified interval falls back to the midpoint (the caller's test then fails)
    assert rs.shift_damped(0.1, -0.01, 0.01, 0.05, 0.5) == 0.0
