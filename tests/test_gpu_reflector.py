"""GPU parity of rsign_reflector / rsign_apply against the CPU oracle.

Each case runs the CUDA path through the C ABI on seeded inputs and compares
with the oracle's definition R = I - 2 Q_k Q_k^T (Jacobi, or the eigenbasis
known by construction) element by element / in the spectral norm.
"""
import math

import numpy as np
import pytest

import oracle
import workloads
from helpers import cuda_or_skip, lib_or_fail, spec_norm_sym

pytestmark = pytest.mark.gpu


def _run(rs, torch, H, k, s, policy, tol=1e-12, **opt):
    Hd = torch.from_numpy(np.ascontiguousarray(H)).cuda()
    o = rs.default_options(**opt)
    R, info, st = rs.reflector(Hd, k, s, tol=tol, policy=policy, options=o, check=False)
    torch.cuda.synchronize()
    return R.cpu().numpy(), info, st


def test_plain_method_fp64_d256():
    # d = 256, k = 4, midpoint shift, Gershgorin alpha, NS to 1e-12 / 80 steps
    torch = cuda_or_skip()
    rs = lib_or_fail()
    spec = workloads.split_spectrum_config(seed=0)
    s = oracle.midpoint(*spec.gap)
    R_or, _ = oracle.reflector(spec.H, spec.k)
    R, info, st = _run(rs, torch, spec.H, spec.k, s, rs.Policy.FP64, tol=1e-12, max_steps=80)
    assert st == rs.Status.OK
    assert spec_norm_sym(R - R_or) <= 1e-12
    assert np.array_equal(R, R.T)
    assert info.cert_ok == 1 and abs(info.trace - 248) < 1e-9
    # iterate-level agreement with the oracle's naive loop: same stopping step
    A = oracle.shifted(spec.H, s)
    alpha = oracle.gershgorin_alpha(A)
    assert info.alpha == pytest.approx(alpha, rel=1e-14)
    X, steps, hist, conv = oracle.newton_schulz(alpha * A, 1e-12, 80)
    assert info.steps_fp64 == steps
    assert np.max(np.abs(R - X)) <= 1e-12


@pytest.mark.parametrize("d,k", [(33, 1), (33, 32), (300, 7), (513, 256)])
def test_fp64_ragged_sizes(d, k):
    torch = cuda_or_skip()
    rs = lib_or_fail()
    spec = workloads.controlled_spectrum(d, k, 0.05, seed=100 + d + k)
    R, info, st = _run(rs, torch, spec.H, k, 0.0, rs.Policy.FP64, tol=1e-12)
    assert st == rs.Status.OK
    R_ex = oracle.reflector_from_basis(spec.Q, k)
    assert spec_norm_sym(R - R_ex) <= 1e-11
    assert abs(info.trace - (d - 2 * k)) < 1e-8


@pytest.mark.parametrize("policy,floor", [("FP16", 2e-2), ("BF16", 2e-1), ("FP32", 1e-4)])
def test_low_precision_stage(policy, floor):
    torch = cuda_or_skip()
    rs = lib_or_fail()
    d, k = 1024, 16
    spec = workloads.controlled_spectrum(d, k, 0.1, seed=7)
    R, info, st = _run(rs, torch, spec.H, k, 0.0, rs.Policy[policy])
    R_ex = oracle.reflector_from_basis(spec.Q, k)
    err = spec_norm_sym(R - R_ex)
    assert st == rs.Status.OK, (st, info.as_dict())
    assert info.steps_low > 5 and info.cert_ok == 1
    assert abs(info.trace - (d - 2 * k)) < 0.5
    assert err < floor, err


def test_low_stage_then_fp64_polish():
    torch = cuda_or_skip()
    rs = lib_or_fail()
    d, k = 768, 10
    spec = workloads.controlled_spectrum(d, k, 0.1, seed=9)
    R, info, st = _run(rs, torch, spec.H, k, 0.0, rs.Policy.FP16_POLISH, polish_steps=2)
    assert st == rs.Status.OK
    assert info.steps_fp64 == 2
    R_ex = oracle.reflector_from_basis(spec.Q, k)
    # the polish restores R^2 = I but keeps the low-precision subspace error
    assert info.resid_fro < 1e-6
    assert spec_norm_sym(R - R_ex) < 2e-2


@pytest.mark.parametrize("policy", ["FP16_POLISH", "BF16_POLISH"])
def test_polish_steps_equal_fp64_newton_schulz_steps(policy):
    # The polish runs FP64-emulating tensor-core products; two of its steps
    # from the low-precision result must agree with two naive FP64 steps of
    # the oracle from the same iterate (polish_steps = 0 returns that iterate).
    torch = cuda_or_skip()
    rs = lib_or_fail()
    d, k = 700, 6
    spec = workloads.controlled_spectrum(d, k, 0.05, seed=21)
    X0, i0, st0 = _run(rs, torch, spec.H, k, 0.0, rs.Policy[policy], polish_steps=0)
    X2, i2, st2 = _run(rs, torch, spec.H, k, 0.0, rs.Policy[policy], polish_steps=2)
    assert i0.steps_low == i2.steps_low and i2.steps_fp64 == 2
    ref = oracle.ns_iterates(X0, 2)
    assert np.max(np.abs(X2 - ref[2])) < 1e-13
    # the reported residual is ||X_2^2 - I||_F of the returned iterate
    res = np.linalg.norm(ref[2] @ ref[2] - np.eye(d))
    assert abs(i2.resid_fro - res) <= 1e-13 + 0.1 * res


def test_host_pointers_roundtrip():
    torch = cuda_or_skip()
    rs = lib_or_fail()
    spec = workloads.controlled_spectrum(64, 3, 0.2, seed=1)
    R, info, st = rs.reflector(np.ascontiguousarray(spec.H), 3, 0.0, tol=1e-12, policy=rs.Policy.FP64)
    assert isinstance(R, np.ndarray) and st == rs.Status.OK
    assert spec_norm_sym(R - oracle.reflector_from_basis(spec.Q, 3)) < 1e-12


@pytest.mark.parametrize("mapped", [0, 1])
def test_pinned_host_buffers_give_the_device_bits(mapped):
    # page-locked host H and R (staged through copies, or read and written in
    # place by the kernels): the same bits as device buffers
    torch = cuda_or_skip()
    rs = lib_or_fail()
    d, k = 700, 9
    spec = workloads.controlled_spectrum(d, k, 5e-2, seed=33)
    Hh = torch.from_numpy(spec.H).pin_memory()
    Rh = torch.empty((d, d), dtype=torch.float64).pin_memory()
    Rd, info_d, st_d = rs.reflector(Hh.cuda(), k, 0.0, tol=1e-6, policy=rs.Policy.FP16_REFINE)
    prev = rs.dbg_set_host_mapped(mapped)
    try:
        _, info_h, st_h = rs.reflector(Hh.numpy(), k, 0.0, tol=1e-6, policy=rs.Policy.FP16_REFINE, out=Rh.numpy())
    finally:
        rs.dbg_set_host_mapped(prev)
    torch.cuda.synchronize()
    assert st_d == rs.Status.OK and st_h == rs.Status.OK
    assert np.array_equal(Rd.cpu().numpy(), Rh.numpy())
    assert spec_norm_sym(Rh.numpy() - oracle.reflector_from_basis(spec.Q, k)) <= 1e-6


@pytest.mark.parametrize("streams", [1, 4])
def test_staged_host_copies_over_several_streams_give_the_device_bits(streams):
    # host H and R of 128 MiB each, copied in and out in parts on several
    # streams that fork from and join the call's stream: the device bits
    torch = cuda_or_skip()
    rs = lib_or_fail()
    d, k = 4096, 16
    H, lam, Q = workloads.controlled_spectrum_torch(d, k, 1e-2, seed=4097)
    Rd, _, st_d = rs.reflector(H, k, 0.0, tol=1e-6, policy=rs.Policy.FP16_REFINE)
    Hh = H.cpu().numpy()
    Rh = np.empty((d, d))
    prev = rs.dbg_set_copy_streams(streams)
    try:
        _, info_h, st_h = rs.reflector(Hh, k, 0.0, tol=1e-6, policy=rs.Policy.FP16_REFINE, out=Rh)
    finally:
        rs.dbg_set_copy_streams(prev)
    torch.cuda.synchronize()
    assert st_d == rs.Status.OK and st_h == rs.Status.OK
    assert np.array_equal(Rd.cpu().numpy(), Rh)


def test_shift_outside_gap_fails_certificate():
    torch = cuda_or_skip()
    rs = lib_or_fail()
    spec = workloads.controlled_spectrum(128, 4, 0.1, seed=3)
    lam = spec.lam
    s_bad = 0.5 * (lam[5] + lam[6])  # admissible for k = 6, not for k = 4
    R, info, st = _run(rs, torch, spec.H, 4, s_bad, rs.Policy.FP64)
    assert st == rs.Status.ERR_CERT
    assert abs(info.trace - (128 - 12)) < 1e-6


def test_nonfinite_input_rejected():
    torch = cuda_or_skip()
    rs = lib_or_fail()
    H = np.eye(40)
    H[3, 7] = np.nan
    R, info, st = _run(rs, torch, H, 2, 0.0, rs.Policy.FP64)
    assert st == rs.Status.ERR_ARG


def test_diagonal_input_exact():
    # Q = I: the reflector is diag(+-1) exactly (Prop. 2.1 proof)
    torch = cuda_or_skip()
    rs = lib_or_fail()
    h = np.linspace(-1.0, 1.0, 50) + 0.01
    k = int((h < 0).sum())
    R, info, st = _run(rs, torch, np.diag(h), k, 0.0, rs.Policy.FP64, tol=1e-14)
    assert st == rs.Status.OK
    assert np.max(np.abs(R - np.diag(np.sign(h)))) < 1e-13


@pytest.mark.parametrize("nv", [1, 3, 16])
def test_apply_matches_the_oracle_product(nv):
    # out = R V (Eq. discrete_step directions) against the oracle's plain FP64
    # triple loop; |error| <= 2 d u sum_k |R_ik V_kj| per entry
    torch = cuda_or_skip()
    rs = lib_or_fail()
    d = 777
    rng = np.random.default_rng(nv)
    Rm = rng.standard_normal((d, d))
    V = rng.standard_normal((d, nv))
    want = oracle.matmul(Rm, V)
    bound = 2.0 * d * np.finfo(np.float64).eps * oracle.matmul(np.abs(Rm), np.abs(V))
    out = rs.apply(torch.from_numpy(Rm).cuda(), torch.from_numpy(V).cuda()).cpu().numpy()
    assert np.all(np.abs(out - want) <= bound)
    out_h = rs.apply(Rm, V)  # host buffers
    assert np.all(np.abs(out_h - want) <= bound)


def test_direction_error_bound():
    # Prop. 3.3: ||R~ g - R g|| <= ||R~ - R||_2 ||g||
    torch = cuda_or_skip()
    rs = lib_or_fail()
    spec = workloads.controlled_spectrum(256, 8, 0.1, seed=4)
    R_lo, _, _ = _run(rs, torch, spec.H, 8, 0.0, rs.Policy.BF16)
    R_ex = oracle.reflector_from_basis(spec.Q, 8)
    g = np.random.default_rng(0).standard_normal(256)
    dt = rs.apply(R_lo, g.reshape(-1, 1)).ravel()
    de = R_ex @ g
    assert np.linalg.norm(dt - de) <= spec_norm_sym(R_lo - R_ex) * np.linalg.norm(g) * (1 + 1e-12)


@pytest.mark.parametrize("policy", ["FP16_REFINE", "BF16_REFINE"])
@pytest.mark.parametrize("d,k,delta", [(1024, 16, 1e-2), (768, 384, 1e-2), (300, 5, 1e-1)])
def test_refine_reaches_1e6(policy, d, k, delta):
    # low-precision steps + commutator refinement: ||R - R_exact||_2 <= 1e-6
    torch = cuda_or_skip()
    rs = lib_or_fail()
    spec = workloads.controlled_spectrum(d, k, delta, seed=40 + d + k)
    R, info, st = _run(rs, torch, spec.H, k, 0.0, rs.Policy[policy], tol=1e-6)
    R_ex = oracle.reflector_from_basis(spec.Q, k)
    err = spec_norm_sym(R - R_ex)
    assert st == rs.Status.OK, (st, info.as_dict())
    assert info.sweeps_refine >= 1 and info.cert_ok == 1
    assert abs(info.trace - (d - 2 * k)) < 1e-6
    assert err <= 1e-6, (err, info.as_dict())
    # the returned R is an involution and symmetric to working accuracy
    assert np.linalg.norm(R @ R - np.eye(d)) < 1e-6
    assert np.array_equal(R, R.T)
    assert info.resid_fro < 1e-3  # measured before the last polish step
    assert info.err_est <= 1e-6


def test_auto_shift_plain_method_d256():
    # s = NaN: Lanczos endpoints, midpoint (Prop. 4.1), margin test (Prop. 4.2)
    torch = cuda_or_skip()
    rs = lib_or_fail()
    spec = workloads.split_spectrum_config(seed=0)
    R_or, lam = oracle.reflector(spec.H, spec.k)
    R, info, st = _run(rs, torch, spec.H, spec.k, float("nan"), rs.Policy.FP64, tol=1e-12)
    assert st == rs.Status.OK
    assert spec_norm_sym(R - R_or) <= 1e-12
    lk, lk1 = lam[spec.k - 1], lam[spec.k]
    assert lk < info.shift < lk1
    # each estimate lies within its bound of the true endpoint, and the certified
    # margin is a true lower bound (Prop. 4.2)
    assert abs(info.lam_k_est - lk) <= info.shift_eps + 1e-12
    assert abs(info.lam_k1_est - lk1) <= info.shift_eps + 1e-12
    assert 0 < info.margin_lb <= oracle.margin(info.shift, lk, lk1) + 1e-12
    assert info.lanczos_iters > 0 and info.steps_pred > 0


@pytest.mark.parametrize("d,k,delta,policy,tol", [(256, 4, None, "FP64", 1e-12), (512, 3, 2e-2, "FP16_REFINE", 1e-7),
                                                   (1000, 990, 5e-2, "FP64", 1e-10)])
def test_auto_shift_step_prediction_matches_the_oracle(d, k, delta, policy, tol):
    # Prop. 3.6 / Eq. pm: the predicted depth m* = min m with eps_m(gamma_hat) <= tol,
    # gamma_hat = alpha (m_hat - eps) from the certified margin, equals the
    # oracle's scalar recurrence at the reported gamma_hat; and since the
    # certified margin is a lower bound of the true one (Prop. 4.2), the true
    # gamma needs no more steps than predicted
    torch = cuda_or_skip()
    rs = lib_or_fail()
    if delta is None:
        spec = workloads.split_spectrum_config(seed=0)
    else:
        spec = workloads.controlled_spectrum(d, k, delta, seed=910 + d + k)
    R, info, st = _run(rs, torch, spec.H, k, float("nan"), rs.Policy[policy], tol=tol)
    assert st == rs.Status.OK and info.cert_ok == 1, (st, info.as_dict())
    assert info.gamma_est == pytest.approx(info.alpha * info.margin_lb, rel=1e-15)
    assert info.steps_pred == oracle.ns_steps(info.gamma_est, tol)
    assert oracle.eps_m(info.gamma_est, info.steps_pred) <= tol < oracle.eps_m(info.gamma_est, info.steps_pred - 1)
    true_gamma = info.alpha * oracle.margin(info.shift, *spec.gap)
    assert info.gamma_est <= true_gamma
    assert oracle.ns_steps(true_gamma, tol) <= info.steps_pred


@pytest.mark.parametrize("d,k,delta", [(300, 290, 5e-2), (512, 3, 2e-2)])
def test_auto_shift_both_spectrum_ends(d, k, delta):
    torch = cuda_or_skip()
    rs = lib_or_fail()
    spec = workloads.controlled_spectrum(d, k, delta, seed=60 + d)
    R, info, st = _run(rs, torch, spec.H, k, float("nan"), rs.Policy.FP16_REFINE, tol=1e-7)
    assert st == rs.Status.OK, (st, info.as_dict())
    assert -delta < info.shift < delta
    assert spec_norm_sym(R - oracle.reflector_from_basis(spec.Q, k)) <= 1e-7


def test_auto_shift_unresolved_gap_is_reported():
    # lam_k == lam_{k+1}: no admissible shift exists (Prop. 2.1 needs lam_k < s < lam_{k+1})
    torch = cuda_or_skip()
    rs = lib_or_fail()
    d, k = 128, 3
    rng = np.random.default_rng(1)
    Q = workloads.haar_orthogonal(d, rng)
    lam = np.sort(np.concatenate([[-1.0, -0.8, 0.3, 0.3], rng.uniform(0.5, 1.0, d - 4)]))
    H = (Q * lam) @ Q.T
    H = 0.5 * (H + H.T)
    R, info, st = _run(rs, torch, H, k, float("nan"), rs.Policy.FP64)
    # either the margin test fails (GAP) or, when the Krylov space held only one
    # copy of the double eigenvalue, the trace certificate rejects the shift
    assert st in (rs.Status.ERR_GAP, rs.Status.ERR_CERT)
    if st == rs.Status.ERR_CERT:
        assert abs(info.trace - (d - 2 * k)) >= 0.5


def test_power_alpha_enlarges_margin_and_saves_steps():
    # Sec. 4.3: alpha near 1/||H - sI||_2 gives a larger scaled margin than the
    # infinity-norm bound, hence fewer steps (Prop. 3.6), with the same reflector
    torch = cuda_or_skip()
    rs = lib_or_fail()
    d, k = 1024, 16
    spec = workloads.controlled_spectrum(d, k, 1e-2, seed=5)
    R_ex = oracle.reflector_from_basis(spec.Q, k)
    out = {}
    for mode in (rs.AlphaMode.INF, rs.AlphaMode.POWER):
        R, info, st = _run(rs, torch, spec.H, k, 0.0, rs.Policy.FP16_REFINE, tol=1e-6, alpha_mode=int(mode))
        assert st == rs.Status.OK
        assert spec_norm_sym(R - R_ex) <= 1e-6
        out[mode] = info
    a_inf, a_pow = out[rs.AlphaMode.INF].alpha, out[rs.AlphaMode.POWER].alpha
    rho = np.abs(spec.lam).max()
    assert a_inf * rho <= 1.0 and 1.0 / 1.02 * 0.9 <= a_pow * rho < np.sqrt(3.0)
    assert a_pow > 5 * a_inf
    assert out[rs.AlphaMode.POWER].steps_low < out[rs.AlphaMode.INF].steps_low


def test_power_alpha_fp64_matches_oracle_definition():
    torch = cuda_or_skip()
    rs = lib_or_fail()
    spec = workloads.split_spectrum_config(seed=0)
    s = oracle.midpoint(*spec.gap)
    R_or, _ = oracle.reflector(spec.H, spec.k)
    R, info, st = _run(rs, torch, spec.H, spec.k, s, rs.Policy.FP64, tol=1e-12, alpha_mode=int(rs.AlphaMode.POWER))
    assert st == rs.Status.OK
    assert spec_norm_sym(R - R_or) <= 1e-12


@pytest.mark.parametrize("theta", [0.1, 0.9])
def test_refine_off_midpoint_shift_same_reflector(theta):
    # Prop. 2.1 on the GPU path: shifts inside the gap give the same R
    torch = cuda_or_skip()
    rs = lib_or_fail()
    spec = workloads.controlled_spectrum(512, 12, 5e-2, seed=77)
    s = workloads.shift_in_gap(spec, theta)
    R, info, st = _run(rs, torch, spec.H, 12, s, rs.Policy.FP16_REFINE, tol=1e-7)
    assert st == rs.Status.OK
    assert spec_norm_sym(R - oracle.reflector_from_basis(spec.Q, 12)) <= 1e-7


def test_scaled_steps_fp64_match_the_oracle_iterates():
    # plain-method workload with the scaled step (margin = half-gap of the midpoint shift)
    torch = cuda_or_skip()
    rs = lib_or_fail()
    spec = workloads.split_spectrum_config(seed=0)
    s = oracle.midpoint(*spec.gap)
    margin = oracle.margin(s, *spec.gap)
    R_or, _ = oracle.reflector(spec.H, spec.k)
    R, info, st = _run(rs, torch, spec.H, spec.k, s, rs.Policy.FP64, tol=1e-12, ns_scaling=1, margin=margin)
    _, info_p, _ = _run(rs, torch, spec.H, spec.k, s, rs.Policy.FP64, tol=1e-12)
    assert st == rs.Status.OK and info.cert_ok == 1
    assert spec_norm_sym(R - R_or) <= 1e-12
    A = oracle.shifted(spec.H, s)
    alpha = oracle.gershgorin_alpha(A)
    coef = oracle.scaled_ns_coeffs(alpha * margin)
    assert info.ns_scaled_steps == len(coef)
    assert info.steps_fp64 < info_p.steps_fp64
    its = oracle.scaled_ns_iterates(alpha * A, coef, info.steps_fp64)
    assert np.max(np.abs(R - its[-1])) <= 1e-12


@pytest.mark.parametrize("policy", ["FP16_REFINE", "BF16_REFINE"])
def test_scaled_steps_refine_reach_1e6_with_fewer_steps(policy):
    torch = cuda_or_skip()
    rs = lib_or_fail()
    d, k, delta = 1024, 16, 1e-2
    spec = workloads.controlled_spectrum(d, k, delta, seed=40 + d + k)
    R, info, st = _run(rs, torch, spec.H, k, 0.0, rs.Policy[policy], tol=1e-6, ns_scaling=1, margin=delta)
    _, info_p, _ = _run(rs, torch, spec.H, k, 0.0, rs.Policy[policy], tol=1e-6)
    err = spec_norm_sym(R - oracle.reflector_from_basis(spec.Q, k))
    assert st == rs.Status.OK and info.cert_ok == 1, info.as_dict()
    assert err <= 1e-6, (err, info.as_dict())
    assert info.err_est <= 1e-6
    assert info.steps_low < info_p.steps_low
    assert info.ns_scaled_steps > 0


@pytest.mark.parametrize("factor", [0.1, 10.0])
def test_scaled_steps_with_a_wrong_margin_stay_correct(factor):
    # an underestimated margin only slows the scaled steps down; an
    # overestimated one leaves eigenvalues below l behind (they still grow),
    # the stop rule waits for them and the result is the same reflector
    torch = cuda_or_skip()
    rs = lib_or_fail()
    d, k, delta = 512, 7, 2e-2
    spec = workloads.controlled_spectrum(d, k, delta, seed=77)
    R, info, st = _run(rs, torch, spec.H, k, 0.0, rs.Policy.FP64, tol=1e-12, ns_scaling=1,
                       margin=factor * delta)
    assert st == rs.Status.OK and info.cert_ok == 1
    assert spec_norm_sym(R - oracle.reflector_from_basis(spec.Q, k)) <= 1e-11


def test_scaled_steps_with_power_alpha_and_auto_shift():
    torch = cuda_or_skip()
    rs = lib_or_fail()
    d, k = 768, 12
    spec = workloads.controlled_spectrum(d, k, 3e-2, seed=78)
    R, info, st = _run(rs, torch, spec.H, k, float("nan"), rs.Policy.FP16_REFINE, tol=1e-6, ns_scaling=1,
                       alpha_mode=int(rs.AlphaMode.POWER))
    assert st == rs.Status.OK and info.cert_ok == 1
    assert info.ns_scaled_steps > 0  # the automatic shift's certified margin drives the scaling
    assert spec_norm_sym(R - oracle.reflector_from_basis(spec.Q, k)) <= 1e-6


def test_refine_stop_on_bound_certifies_a_controlled_spectrum():
    # with the margin known and the bound as the stop test the returned R is
    # certified: ||R - R_exact||_2 <= err_bound <= tol.  (The bound needs the
    # rounding noise of R small against the margin: d = 4096, half-gap 5e-2.)
    torch = cuda_or_skip()
    rs = lib_or_fail()
    d, k, delta = 4096, 16, 5e-2
    H, lam, Q = workloads.controlled_spectrum_torch(d, k, delta, seed=92)
    R, info, st = rs.reflector(H, k, 0.0, tol=1e-6, policy=rs.Policy.FP16_REFINE, check=False,
                               options=rs.default_options(ns_scaling=1, margin=delta,
                                                          refine_stop=int(rs.RefineStop.BOUND)))
    Qk = Q[:, :k]
    D = R - (torch.eye(d, dtype=torch.float64, device=R.device) - 2.0 * Qk @ Qk.T)
    err = float(torch.linalg.eigvalsh(0.5 * (D + D.T)).abs().max())
    assert st == rs.Status.OK and info.cert_ok == 1, (st, info.as_dict())
    assert info.err_bound <= 1e-6 and err <= info.err_bound, (err, info.as_dict())


def test_refine_largest_order_d16384():
    # the largest supported order: d = 16384 (FP64-emulating digit width 5,
    # 11 planes in the polish tables; 2 GiB per FP64 matrix)
    torch = cuda_or_skip()
    rs = lib_or_fail()
    d, k, delta = 16384, 16, 1e-2
    H, lam, Q = workloads.controlled_spectrum_torch(d, k, delta, seed=93)
    R, info, st = rs.reflector(H, k, 0.0, tol=1e-6, policy=rs.Policy.FP16_REFINE, check=False,
                               options=rs.default_options(ns_scaling=1, margin=delta,
                                                          alpha_mode=int(rs.AlphaMode.POWER)))
    assert st == rs.Status.OK and info.cert_ok == 1, (st, info.as_dict())
    Qk = Q[:, :k]
    D = R - (torch.eye(d, dtype=torch.float64, device=R.device) - 2.0 * Qk @ Qk.T)
    del H, Q
    # ||D||_2 by power steps on the symmetric D (converging from below), and
    # the Frobenius norm as a loose upper bound
    v = torch.ones(d, dtype=torch.float64, device=R.device)
    for _ in range(60):
        v = D @ (D @ v)
        v = v / v.norm()
    err = float((D @ v).norm())
    assert err <= 1e-6, (err, info.as_dict())
    assert float(D.norm()) <= 1e-4
    assert abs(info.trace - (d - 2 * k)) < 1e-6


@pytest.mark.parametrize("policy,tol,bound", [("FP64", 1e-12, 1e-12), ("FP16_POLISH", 1e-12, 2e-2),
                                              ("FP16_REFINE", 1e-6, 1e-6)])
@pytest.mark.parametrize("d,k", [(2, 1), (3, 1), (3, 2)])
def test_smallest_orders(policy, tol, bound, d, k):
    # the degenerate orders: one 256-wide padded tile holding a 2 x 2 or 3 x 3
    # problem (eigenvalues -delta, +delta pinned, the rest spread)
    torch = cuda_or_skip()
    rs = lib_or_fail()
    spec = workloads.controlled_spectrum(d, k, 0.05, seed=700 + d + k)
    R, info, st = _run(rs, torch, spec.H, k, 0.0, rs.Policy[policy], tol=tol)
    assert st == rs.Status.OK and info.cert_ok == 1, (st, info.as_dict())
    assert spec_norm_sym(R - oracle.reflector_from_basis(spec.Q, k)) <= bound
    assert abs(info.trace - (d - 2 * k)) < 1e-6


def test_timed_workload_sampled_entries_match_the_oracle():
    # the timed workload at full size and in its launch configuration: d = 8192,
    # k = 16, half-gap 1e-2, shift at the middle of the gap, FP16_REFINE to
    # 1e-6, power-step alpha, scaled steps from the margin.  The whole diagonal,
    # the last row and 4096 seeded entries against the oracle's entries of
    # I - 2 Q_k Q_k^T (|entry error| <= ||R - R_exact||_2 <= 1e-6).
    torch = cuda_or_skip()
    rs = lib_or_fail()
    d, k, delta = 8192, 16, 1e-2
    H, lam, Q = workloads.controlled_spectrum_torch(d, k, delta, workloads.controlled_seed(d, 1, 1))
    lam_h = lam.cpu().numpy()
    s = float(lam_h[k - 1] + 0.5 * (lam_h[k] - lam_h[k - 1]))
    margin = float(min(s - lam_h[k - 1], lam_h[k] - s))
    opt = rs.default_options(alpha_mode=int(rs.AlphaMode.POWER), ns_scaling=1, margin=margin)
    R, info, st = rs.reflector(H, k, s, tol=1e-6, policy=rs.Policy.FP16_REFINE, options=opt, check=False)
    torch.cuda.synchronize()
    assert st == rs.Status.OK and info.cert_ok == 1, (st, info.as_dict())
    assert abs(info.trace - (d - 2 * k)) < 1e-6
    Qk = Q[:, :k].cpu().numpy()
    del H, Q
    rng = np.random.default_rng(8192)
    rows = np.concatenate([np.arange(d), np.full(d, d - 1), rng.integers(0, d, 4096)])
    cols = np.concatenate([np.arange(d), np.arange(d), rng.integers(0, d, 4096)])
    got = R[torch.from_numpy(rows).to(R.device), torch.from_numpy(cols).to(R.device)].cpu().numpy()
    want = np.array([oracle.reflector_entry(Qk, k, int(i), int(j)) for i, j in zip(rows, cols)])
    assert np.max(np.abs(got - want)) <= 1e-6
    # symmetric to the bit on the sampled entries
    assert np.array_equal(got, R[torch.from_numpy(cols).to(R.device), torch.from_numpy(rows).to(R.device)].cpu().numpy())


@pytest.mark.parametrize("policy,tol,bound", [("FP64", 1e-12, 1e-11), ("FP16_REFINE", 1e-6, 1e-6)])
def test_nonsymmetric_input_uses_the_symmetric_part(policy, tol, bound):
    # only 1/2 (H + H^T) enters (the boundary's contract): an antisymmetric
    # part of size 1 added to H leaves the reflector of the symmetric part
    torch = cuda_or_skip()
    rs = lib_or_fail()
    d, k = 640, 9
    spec = workloads.controlled_spectrum(d, k, 5e-2, seed=801)
    K = np.random.default_rng(802).standard_normal((d, d))
    H = spec.H + (K - K.T) / np.linalg.norm(K - K.T, 2)
    assert not np.array_equal(H, H.T)
    R, info, st = _run(rs, torch, H, k, 0.0, rs.Policy[policy], tol=tol)
    assert st == rs.Status.OK and info.cert_ok == 1, (st, info.as_dict())
    assert spec_norm_sym(R - oracle.reflector_from_basis(spec.Q, k)) <= bound
    assert np.array_equal(R, R.T)


@pytest.mark.parametrize("policy", ["FP64", "FP16_POLISH", "FP16_REFINE"])
@pytest.mark.parametrize("e", [-300, 300])
def test_power_of_two_scaling_gives_the_same_bits(policy, e):
    # sign(c (H - sI)) = sign(H - sI) for c > 0.  With c = 2^e every FP64
    # operation before the normalisation by alpha scales exactly, alpha
    # scales by 1/c, and X_0 = alpha A is the same bits, so are the steps and
    # the result.  REFINE handles the commutator of the unnormalised A and
    # must stay in range at both ends (the margin option is in the units of
    # H and scales with it); d = 700 has padding rows, whose digit-split row
    # scale once entered the refinement's level rule and made it depend on
    # the scale of H.
    torch = cuda_or_skip()
    rs = lib_or_fail()
    d, k = 700, 11
    spec = workloads.controlled_spectrum(d, k, 5e-2, seed=901)
    s = workloads.shift_in_gap(spec, 0.3)
    mu = oracle.margin(s, *spec.gap)
    refine = policy.endswith("REFINE")
    tol = 1e-6 if refine else 1e-12
    c = 2.0 ** e

    def opts(scale):
        if not refine:
            return {}
        return dict(alpha_mode=int(rs.AlphaMode.POWER), ns_scaling=1, margin=mu * scale)

    R0, i0, st0 = _run(rs, torch, spec.H, k, s, rs.Policy[policy], tol=tol, **opts(1.0))
    R1, i1, st1 = _run(rs, torch, spec.H * c, k, s * c, rs.Policy[policy], tol=tol, **opts(c))
    assert st0 == rs.Status.OK and st1 == rs.Status.OK, (st0, st1, i1.as_dict())
    assert (i1.steps_low, i1.steps_fp64, i1.sweeps_refine) == (i0.steps_low, i0.steps_fp64, i0.sweeps_refine)
    assert i1.alpha == i0.alpha / c
    assert i1.refine_levels == i0.refine_levels
    # every policy, the refinement included, gives the same bits at either scale
    assert np.array_equal(R0, R1)
    if refine:
        R_ex = oracle.reflector_from_basis(spec.Q, k)
        assert spec_norm_sym(R0 - R_ex) <= tol


def test_apply_full_size_sampled_rows():
    # out = R V at d = 8192, nv = 16 (device buffers): 64 seeded rows against
    # the oracle's triple-loop product of those rows
    torch = cuda_or_skip()
    rs = lib_or_fail()
    d, nv = 8192, 16
    g = torch.Generator(device="cuda").manual_seed(8193)
    Rm = torch.randn((d, d), generator=g, device="cuda", dtype=torch.float64)
    V = torch.randn((d, nv), generator=g, device="cuda", dtype=torch.float64)
    out = rs.apply(Rm, V)
    torch.cuda.synchronize()
    rows = np.random.default_rng(8193).choice(d, 64, replace=False)
    Rh = Rm[torch.from_numpy(rows).cuda()].cpu().numpy()
    Vh = V.cpu().numpy()
    got = out[torch.from_numpy(rows).cuda()].cpu().numpy()
    want = oracle.matmul(Rh, Vh)
    bound = 2.0 * d * np.finfo(np.float64).eps * oracle.matmul(np.abs(Rh), np.abs(Vh))
    assert np.all(np.abs(got - want) <= bound)
