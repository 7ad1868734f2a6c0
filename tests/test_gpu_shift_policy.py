"""GPU checks of rsign_shift_update along slowly varying sequences
(Sec. 4.4, Prop. 4.2): the Weyl drift bound, the reuse/refresh decisions
(replayed with the oracle's reuse rule), admissibility of every shift used
against the eigenvalues known by construction, and certified reflectors."""
import numpy as np
import pytest

import oracle
import workloads
from helpers import cuda_or_skip, lib_or_fail

pytestmark = pytest.mark.gpu


def _sequence(d, k, delta, n, eta, seed, rotate=0.0):
    """H_j = Q_j diag(lam + j eta w) Q_j^T: eigenvalue drift eta |w| per step
    (w fixed, |w_i| <= 1), optionally with a small rotation of the basis."""
    sp = workloads.controlled_spectrum(d, k, delta, seed)
    rng = np.random.default_rng(seed + 1)
    w = rng.uniform(-1.0, 1.0, d)
    Q = sp.Q
    out = []
    for j in range(n):
        lam = sp.lam + j * eta * w
        if rotate and j:
            S = rng.standard_normal((d, d)) * rotate / np.sqrt(d)
            K = S - S.T
            Q = Q @ (np.eye(d) + K + 0.5 * K @ K)  # near-orthogonal step
            Q, _ = np.linalg.qr(Q)
        H = (Q * lam) @ Q.T
        out.append((0.5 * (H + H.T), np.sort(lam)))
    return out


def test_drift_bound_and_reuse_decisions_follow_prop_4_2():
    torch = cuda_or_skip()
    rs = lib_or_fail()
    d, k = 300, 5
    seq = _sequence(d, k, 0.05, 8, 4e-3, seed=61, rotate=1e-3)
    st = rs.shift_state()
    H_old = None
    replay_margin = None
    refreshed = []
    for j, (H, lam) in enumerate(seq):
        prev = rs.ShiftState.from_buffer_copy(st)
        status, rep = rs.shift_update(torch.from_numpy(H).cuda(), None if H_old is None else
                                      torch.from_numpy(H_old).cuda(), k, st, rs.ShiftPolicy.REUSE_REFRESH,
                                      threshold=0.02)
        assert status == rs.Status.OK
        refreshed.append(rep.refreshed)
        if H_old is not None:
            true = np.max(np.abs(np.linalg.eigvalsh(H - H_old)))
            assert rep.drift_ub >= true * (1 - 1e-12)
            assert rep.drift_est <= true * (1 + 1e-9)
            # the library's decision is the oracle's rule applied to its state
            ok, guaranteed = oracle.reuse_admissible(prev.margin_cert + prev.eps, prev.eps, rep.drift_ub)
            assert rep.refreshed == (0 if (ok and guaranteed > 0.02) else 1)
        # the shift in use is admissible with at least the certified margin
        s = st.shift
        true_margin = oracle.margin(s, lam[k - 1], lam[k])
        assert true_margin >= st.margin_cert - 1e-12 > 0
        # and the reflector with it certifies
        R, info, st_r = rs.reflector(H, k, s, tol=1e-12, policy=rs.Policy.FP64, check=False)
        assert st_r == rs.Status.OK and info.cert_ok == 1
        H_old = H
    assert refreshed[0] == 1 and 0 in refreshed[1:]  # the first matrix refreshes, some later ones reuse
    assert st.reuses + st.refreshes == len(seq)


def test_refresh_when_the_margin_runs_out():
    torch = cuda_or_skip()
    rs = lib_or_fail()
    d, k = 200, 3
    # large drift relative to the half-gap: the certified margin is used up fast
    seq = _sequence(d, k, 0.05, 6, 2e-2, seed=62)
    st = rs.shift_state()
    H_old = None
    for H, lam in seq:
        status, rep = rs.shift_update(H, H_old, k, st, rs.ShiftPolicy.REUSE_REFRESH, threshold=0.0)
        assert status == rs.Status.OK
        assert oracle.margin(st.shift, lam[k - 1], lam[k]) >= st.margin_cert > 0
        H_old = H
    assert st.refreshes >= 2


@pytest.mark.parametrize("policy", ["MIDPOINT", "DAMPED"])
def test_midpoint_and_damped_policies_refresh_every_matrix(policy):
    torch = cuda_or_skip()
    rs = lib_or_fail()
    d, k = 256, 4
    seq = _sequence(d, k, 0.05, 4, 3e-3, seed=63)
    st = rs.shift_state()
    H_old = None
    for H, lam in seq:
        prev_shift = st.shift
        status, rep = rs.shift_update(H, H_old, k, st, rs.ShiftPolicy[policy], damping=0.6)
        assert status == rs.Status.OK and rep.refreshed == 1
        ok, m_hat, guaranteed = oracle.admissible(st.shift, st.lam_k_est, st.lam_k1_est, st.eps)
        assert ok and st.margin_cert == pytest.approx(guaranteed, rel=1e-12, abs=1e-15)
        if policy == "MIDPOINT":
            assert st.shift == oracle.midpoint(st.lam_k_est, st.lam_k1_est)
        else:
            assert st.shift == rs.shift_damped(prev_shift, st.lam_k_est, st.lam_k1_est, st.eps, 0.6)
        assert lam[k - 1] < st.shift < lam[k]
        H_old = H
    assert st.refreshes == len(seq) and st.reuses == 0


def test_unresolved_gap_is_reported():
    torch = cuda_or_skip()
    rs = lib_or_fail()
    # lam_k and lam_{k+1} equal: no admissible shift
    sp = workloads.controlled_spectrum(128, 4, 0.05, seed=64)
    lam = sp.lam.copy()
    lam[3] = lam[4] = 0.0
    H = (sp.Q * lam) @ sp.Q.T
    H = 0.5 * (H + H.T)
    st = rs.shift_state()
    status, rep = rs.shift_update(H, None, 4, st, rs.ShiftPolicy.MIDPOINT)
    assert status == rs.Status.ERR_GAP
    assert np.isnan(st.shift)
