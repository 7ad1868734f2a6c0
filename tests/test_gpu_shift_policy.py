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


def _eig_drift_sequence(d, k, delta, n, eta, seed):
    """H_j = Q diag(lam + j eta w) Q^T with w fixed, |w_i| <= 1: the step
    H_{j+1} - H_j = eta Q diag(w) Q^T has 2-norm eta max|w| exactly."""
    sp = workloads.controlled_spectrum(d, k, delta, seed)
    w = np.random.default_rng(seed + 1).uniform(-1.0, 1.0, d)
    out = []
    for j in range(n):
        lam = sp.lam + j * eta * w
        H = (sp.Q * lam) @ sp.Q.T
        out.append((0.5 * (H + H.T), np.sort(lam)))
    return out, eta * np.max(np.abs(w))


def _check_state(rs, st, lam, k, H):
    s = st.shift
    assert oracle.margin(s, lam[k - 1], lam[k]) >= st.margin_cert - 1e-12 > 0
    R, info, st_r = rs.reflector(H, k, s, tol=1e-12, policy=rs.Policy.FP64, check=False)
    assert st_r == rs.Status.OK and info.cert_ok == 1


def test_reuse_refresh_decisions_follow_prop_4_2():
    torch = cuda_or_skip()
    rs = lib_or_fail()
    d, k, tau = 300, 5, 0.03
    seq, step = _eig_drift_sequence(d, k, 0.05, 8, 4e-3, seed=61)
    st = rs.shift_state()
    H_old = None
    refreshed = []
    for j, (H, lam) in enumerate(seq):
        prev = rs.ShiftState.from_buffer_copy(st)
        Hd = torch.from_numpy(H).cuda()
        status, rep = rs.shift_update(Hd, None if H_old is None else torch.from_numpy(H_old).cuda(), k, st,
                                      rs.ShiftPolicy.REUSE_REFRESH, threshold=tau,
                                      drift_bound=None if H_old is None else step)
        assert status == rs.Status.OK
        refreshed.append(rep.refreshed)
        if H_old is not None:
            assert rep.drift_ub == step
            # the library's decision is the oracle's rule applied to its state
            ok, guaranteed = oracle.reuse_admissible(prev.margin_cert + prev.eps, prev.eps, step)
            assert rep.refreshed == (0 if (ok and guaranteed > tau) else 1)
            if not rep.refreshed:
                assert st.margin_cert == pytest.approx(guaranteed, rel=1e-12)
        _check_state(rs, st, lam, k, H)
        H_old = H
    assert refreshed[0] == 1 and 0 in refreshed[1:] and 1 in refreshed[1:]
    assert st.reuses + st.refreshes == len(seq)


def test_gpu_drift_bound_is_an_upper_bound():
    torch = cuda_or_skip()
    rs = lib_or_fail()
    d, k = 400, 6
    sp = workloads.controlled_spectrum(d, k, 0.05, seed=65)
    rng = np.random.default_rng(66)
    cases = []
    v = rng.standard_normal(d)
    v /= np.linalg.norm(v)
    cases.append(1e-3 * np.outer(v, v))                   # rank one: the Frobenius bound is tight
    S = rng.standard_normal((d, d))
    cases.append(1e-4 * (S + S.T))                        # spread out: the bound is loose
    cases.append(np.diag(rng.uniform(-1e-3, 1e-3, d)))    # diagonal: (|.|_1 + |.|_inf)/2 is tight
    for D in cases:
        H_new = sp.H + D
        st = rs.shift_state()
        rs.shift_update(sp.H, None, k, st, rs.ShiftPolicy.REUSE_REFRESH)
        status, rep = rs.shift_update(H_new, sp.H, k, st, rs.ShiftPolicy.REUSE_REFRESH)
        assert status == rs.Status.OK
        true = np.max(np.abs(np.linalg.eigvalsh(H_new - sp.H)))
        bound = min(np.linalg.norm(D), 0.5 * (np.abs(D).sum(0).max() + np.abs(D).sum(1).max()))
        assert rep.drift_ub >= true * (1 - 1e-12)
        assert rep.drift_ub == pytest.approx(bound, rel=1e-10)
        assert rep.drift_est <= true * (1 + 1e-9) and rep.drift_est >= 0.5 * true


def test_refresh_when_the_margin_runs_out():
    torch = cuda_or_skip()
    rs = lib_or_fail()
    d, k = 200, 3
    seq, step = _eig_drift_sequence(d, k, 0.05, 6, 5e-3, seed=62)
    st = rs.shift_state()
    H_old = None
    for H, lam in seq:
        status, rep = rs.shift_update(H, H_old, k, st, rs.ShiftPolicy.REUSE_REFRESH, threshold=0.03,
                                      drift_bound=None if H_old is None else step)
        assert status == rs.Status.OK
        _check_state(rs, st, lam, k, H)
        H_old = H
    assert st.refreshes >= 2 and st.reuses >= 1


@pytest.mark.parametrize("policy", ["MIDPOINT", "DAMPED"])
def test_midpoint_and_damped_policies_refresh_every_matrix(policy):
    torch = cuda_or_skip()
    rs = lib_or_fail()
    d, k = 256, 4
    seq, step = _eig_drift_sequence(d, k, 0.05, 4, 3e-3, seed=63)
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
        _check_state(rs, st, lam, k, H)
        H_old = H
    assert st.refreshes == len(seq) and st.reuses == 0


def test_unresolved_gap_is_reported():
    torch = cuda_or_skip()
    rs = lib_or_fail()
    # an interior gap (k = d/2) of 2e-9 among eigenvalues ~1e-3 apart: the
    # Lanczos budget cannot resolve it, so the margin test of Prop. 4.2 fails
    sp = workloads.controlled_spectrum(1024, 512, 1e-9, seed=64)
    st = rs.shift_state()
    status, rep = rs.shift_update(sp.H, None, 512, st, rs.ShiftPolicy.MIDPOINT)
    assert status == rs.Status.ERR_GAP
    assert np.isnan(st.shift) and np.isnan(st.margin_cert)


def test_bad_arguments():
    torch = cuda_or_skip()
    rs = lib_or_fail()
    H = np.eye(64)
    st = rs.shift_state()
    assert rs.shift_update(H, None, 0, st)[0] == rs.Status.ERR_ARG
    assert rs.shift_update(H, None, 3, st, threshold=-1.0)[0] == rs.Status.ERR_ARG
    assert rs.shift_update(H, H, 3, st, drift_bound=-1.0)[0] == rs.Status.ERR_ARG
