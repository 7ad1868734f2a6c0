"""GPU parity at full size and at the corners of the controlled-spectrum sweep.

The reflector of each case is compared with the oracle's definition
R = I - 2 Q_k Q_k^T (Eq. Pk), computed by the oracle's C routine from the
eigenbasis that the seeded construction knows, over the WHOLE matrix:
every entry, the spectral norm of the difference (Lanczos on the symmetric
difference, converged to 1e-10 relative) and its Frobenius norm.

Cases: the timed workload (d = 8192, k = 16, half-gap 1e-2, midpoint shift,
FP16_REFINE to 1e-6, power-step alpha, scaled steps) in its launch
configuration, and the corners of the sweep that the timed workload does not
reach: half-gap 1e-3 (d = 2048, 8192), k = 1 and k = d/2 (d = 4096), shifts
at 10 % and 90 % of the gap (d = 8192), under FP16_REFINE and BF16_REFINE.
Also: two identical REFINE calls give identical bits.
"""
import functools

import numpy as np
import pytest

import oracle
import workloads
from helpers import cuda_or_skip, lib_or_fail

pytestmark = pytest.mark.gpu

_K_IDX = {"1": 0, "16": 1, "half": 2}
_DELTA_IDX = {1e-1: 0, 1e-2: 1, 1e-3: 2}


def _k_of(d, kname):
    return d // 2 if kname == "half" else int(kname)


def _problem(torch, d, kname, delta):
    """(H on the GPU, lam, Q on the GPU) of one sweep point, seeded by (d, k, delta)."""
    k = _k_of(d, kname)
    seed = workloads.controlled_seed(d, _K_IDX[kname], _DELTA_IDX[delta])
    return workloads.controlled_spectrum_torch(d, k, delta, seed)


@functools.lru_cache(maxsize=3)
def _exact(d, kname, delta):
    """The oracle's reflector of one sweep point (host FP64, d x d)."""
    torch = cuda_or_skip()
    H, lam, Q = _problem(torch, d, kname, delta)
    k = _k_of(d, kname)
    Qh = Q.cpu().numpy()
    lam_h = lam.cpu().numpy()
    del H, Q
    torch.cuda.empty_cache()
    return oracle.reflector_from_basis(Qh, k), lam_h


def _spectral_norm_sym(D):
    """||D||_2 of a symmetric D by Lanczos (largest |eigenvalue|, converged)."""
    from scipy.sparse.linalg import eigsh
    vals = eigsh(D, k=1, which="LM", tol=1e-10, return_eigenvectors=False, maxiter=5000)
    return float(np.abs(vals).max())


def _call(rs, torch, d, kname, delta, theta, policy, tol=1e-6, with_margin=True):
    H, lam, _ = _problem(torch, d, kname, delta)
    k = _k_of(d, kname)
    lam_h = lam.cpu().numpy()
    s = float(lam_h[k - 1] + theta * (lam_h[k] - lam_h[k - 1]))
    margin = float(min(s - lam_h[k - 1], lam_h[k] - s))
    kw = dict(alpha_mode=int(rs.AlphaMode.POWER))
    if with_margin:
        kw.update(ns_scaling=1, margin=margin)
    opt = rs.default_options(**kw)
    R, info, st = rs.reflector(H, k, s, tol=tol, policy=rs.Policy[policy], options=opt, check=False)
    torch.cuda.synchronize()
    Rh = R.cpu().numpy()
    del H, R
    torch.cuda.empty_cache()
    return Rh, info, st, k


def _check_against_oracle(R, R_ex, tol):
    D = R - R_ex
    err_max = float(np.abs(D).max())
    err_2 = _spectral_norm_sym(0.5 * (D + D.T))
    err_fro = float(np.linalg.norm(D))
    assert np.array_equal(R, R.T)
    assert err_max <= tol and err_2 <= tol, (err_max, err_2, err_fro)
    return err_2, err_fro


def test_timed_workload_every_entry_matches_the_oracle():
    # the bench's call: d = 8192, k = 16, half-gap 1e-2, midpoint shift,
    # FP16_REFINE to 1e-6, power-step alpha, scaled steps from the margin
    torch = cuda_or_skip()
    rs = lib_or_fail()
    R, info, st, k = _call(rs, torch, 8192, "16", 1e-2, 0.5, "FP16_REFINE")
    assert st == rs.Status.OK and info.cert_ok == 1, (st, info.as_dict())
    assert abs(info.trace - (8192 - 2 * k)) < 1e-6
    R_ex, _ = _exact(8192, "16", 1e-2)
    err_2, err_fro = _check_against_oracle(R, R_ex, 1e-6)
    # the library's own error estimate (with its safety factor) is not below
    # the true error
    assert info.err_est >= err_2, (info.err_est, err_2)
    # the whole difference, not only its largest direction: the Frobenius
    # norm bounds every singular value at once
    assert err_fro <= 4e-6, err_fro


@pytest.mark.parametrize("policy", ["FP16_REFINE", "BF16_REFINE"])
@pytest.mark.parametrize("d,kname,delta,theta", [
    (2048, "16", 1e-3, 0.5),
    (8192, "16", 1e-3, 0.5),
    (4096, "1", 1e-2, 0.5),
    (4096, "half", 1e-2, 0.5),
    (8192, "16", 1e-2, 0.1),
    (8192, "16", 1e-2, 0.9),
])
def test_sweep_corners_reach_1e6_with_the_certificate(policy, d, kname, delta, theta):
    torch = cuda_or_skip()
    rs = lib_or_fail()
    R, info, st, k = _call(rs, torch, d, kname, delta, theta, policy)
    assert st == rs.Status.OK and info.cert_ok == 1, (st, info.as_dict())
    assert abs(info.trace - (d - 2 * k)) < 1e-6
    R_ex, _ = _exact(d, kname, delta)
    _check_against_oracle(R, R_ex, 1e-6)


@pytest.mark.parametrize("d,kname,delta", [(2048, "16", 1e-3), (4096, "1", 1e-2)])
def test_margin_free_refine_reaches_1e6(d, kname, delta):
    # no margin supplied: plain Newton-Schulz steps, the refinement's first
    # digit levels from the stage-1 step count
    torch = cuda_or_skip()
    rs = lib_or_fail()
    R, info, st, k = _call(rs, torch, d, kname, delta, 0.5, "FP16_REFINE", with_margin=False)
    assert st == rs.Status.OK and info.cert_ok == 1, (st, info.as_dict())
    assert info.ns_scaled_steps == 0
    R_ex, _ = _exact(d, kname, delta)
    _check_against_oracle(R, R_ex, 1e-6)


@pytest.mark.parametrize("d,kname,delta", [(768, "16", 1e-2), (8192, "16", 1e-2)])
def test_refine_calls_repeat_bit_for_bit(d, kname, delta):
    # the refinement runs its norm estimates on a side stream beside the
    # tensor-core products: two identical calls must still give the same bits
    torch = cuda_or_skip()
    rs = lib_or_fail()
    R0, i0, st0, _ = _call(rs, torch, d, kname, delta, 0.5, "FP16_REFINE")
    R1, i1, st1, _ = _call(rs, torch, d, kname, delta, 0.5, "FP16_REFINE")
    assert st0 == rs.Status.OK and st1 == rs.Status.OK
    assert (i0.steps_low, i0.sweeps_refine, i0.steps_fp64) == (i1.steps_low, i1.sweeps_refine, i1.steps_fp64)
    assert i0.err_est == i1.err_est and i0.commutator_norm == i1.commutator_norm
    assert np.array_equal(R0, R1)
