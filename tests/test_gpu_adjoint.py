"""GPU checks of rsign_reflector_backward (adjoint of the Newton-Schulz map with
s and alpha held fixed) against the oracle's FP64 Daleckii-Krein gradient and
against central finite differences of the converged forward reflector.

Loss as in the adjoint workload: L = <G, sign(H - sI)> + g^T R g, so
dL/dR = G_sym + g g^T.
"""
import numpy as np
import pytest

import oracle
import workloads
from helpers import cuda_or_skip, lib_or_fail

pytestmark = pytest.mark.gpu


def _loss_seed(d, seed):
    rng = np.random.default_rng(seed)
    G = rng.standard_normal((d, d))
    G = 0.5 * (G + G.T)
    g = rng.standard_normal(d)
    return G + np.outer(g, g)


def _dk_gradient(spec, s, Rbar):
    # gradient of <Rbar, sign(A)> w.r.t. A = H - sI: L_sign(A, sym(Rbar)) (self-adjoint)
    W = 0.5 * (Rbar + Rbar.T)
    return oracle.daleckii_krein(spec.lam - s, spec.Q, W)


@pytest.mark.parametrize("ckpt", [1, 4, 7])
def test_backward_fp64_matches_daleckii_krein(ckpt):
    torch = cuda_or_skip()
    rs = lib_or_fail()
    d, k = 256, 8
    spec = workloads.controlled_spectrum(d, k, 5e-2, seed=501)
    Rbar = _loss_seed(d, 3)
    Hd = torch.from_numpy(spec.H).cuda()
    Hbar = rs.reflector_backward(Hd, k, 0.0, torch.from_numpy(Rbar).cuda(), policy=rs.Policy.FP64,
                                 ckpt_every=ckpt).cpu().numpy()
    dk = _dk_gradient(spec, 0.0, Rbar)
    rel = np.linalg.norm(Hbar - dk) / np.linalg.norm(dk)
    assert rel < 1e-8, rel
    assert np.max(np.abs(Hbar - Hbar.T)) < 1e-12 * np.abs(Hbar).max()


def test_backward_fp64_matches_finite_differences():
    torch = cuda_or_skip()
    rs = lib_or_fail()
    d, k = 192, 5
    spec = workloads.controlled_spectrum(d, k, 1e-1, seed=502)
    Rbar = _loss_seed(d, 4)
    Hbar = rs.reflector_backward(np.ascontiguousarray(spec.H), k, 0.0, Rbar, policy=rs.Policy.FP64)
    rng = np.random.default_rng(5)
    for _ in range(3):
        W = rng.standard_normal((d, d))
        W = 0.5 * (W + W.T)
        h = 1e-5
        Rp, _, sp = rs.reflector(spec.H + h * W, k, 0.0, tol=1e-14, policy=rs.Policy.FP64, check=False)
        Rm, _, sm = rs.reflector(spec.H - h * W, k, 0.0, tol=1e-14, policy=rs.Policy.FP64, check=False)
        fd = (np.sum(Rbar * Rp) - np.sum(Rbar * Rm)) / (2 * h)
        an = np.sum(Hbar * W)
        assert abs(fd - an) <= 1e-5 * max(1.0, abs(an)), (fd, an)


@pytest.mark.parametrize("policy,tol", [("FP16_REFINE", 2e-2), ("BF16_REFINE", 1e-1), ("FP16", 1e-1),
                                        ("FP16_POLISH", 1e-1), ("BF16_POLISH", 2e-1), ("FP32", 2e-2)])
def test_backward_low_precision_close_to_daleckii_krein(policy, tol):
    torch = cuda_or_skip()
    rs = lib_or_fail()
    d, k = 512, 8
    spec = workloads.controlled_spectrum(d, k, 1e-2 * 5, seed=503)
    Rbar = _loss_seed(d, 6)
    Hbar = rs.reflector_backward(torch.from_numpy(spec.H).cuda(), k, 0.0, torch.from_numpy(Rbar).cuda(),
                                 policy=rs.Policy[policy]).cpu().numpy()
    dk = _dk_gradient(spec, 0.0, Rbar)
    rel = np.linalg.norm(Hbar - dk) / np.linalg.norm(dk)
    assert rel < tol, rel


def test_backward_rejects_bad_arguments():
    torch = cuda_or_skip()
    rs = lib_or_fail()
    H = torch.eye(8, dtype=torch.float64, device="cuda")
    with pytest.raises(rs.RsignError):
        rs.reflector_backward(H, 0, 0.0, H)
    with pytest.raises(rs.RsignError):
        rs.reflector_backward(H, 2, float("nan"), H)


def test_autograd_function_matches_backward_and_daleckii_krein():
    # the adjoint workload's loss L = <G, R> + g^T R g through torch.autograd
    torch = cuda_or_skip()
    rs = lib_or_fail()
    d, k = 256, 6
    spec = workloads.controlled_spectrum(d, k, 5e-2, seed=505)
    rng = np.random.default_rng(8)
    Gm = rng.standard_normal((d, d))
    Gm = 0.5 * (Gm + Gm.T)
    g = rng.standard_normal(d)
    H = torch.from_numpy(spec.H).cuda().requires_grad_(True)
    R = rs.sign_reflector(H, k, 0.0, policy=rs.Policy.FP64)
    Gt, gt = torch.from_numpy(Gm).cuda(), torch.from_numpy(g).cuda()
    loss = (Gt * R).sum() + gt @ R @ gt
    loss.backward()
    Rbar = Gm + np.outer(g, g)
    direct = rs.reflector_backward(spec.H, k, 0.0, Rbar, policy=rs.Policy.FP64)
    assert np.max(np.abs(H.grad.cpu().numpy() - direct)) <= 1e-12 * np.abs(direct).max()
    dk = _dk_gradient(spec, 0.0, Rbar)
    assert np.linalg.norm(H.grad.cpu().numpy() - dk) / np.linalg.norm(dk) < 1e-8
    # the forward value is the reflector itself
    assert np.max(np.abs(R.detach().cpu().numpy() - oracle.reflector_from_basis(spec.Q, k))) < 1e-10


@pytest.mark.parametrize("policy,tol", [("FP32", 2e-2), ("BF16_POLISH", 3e-1), ("FP64", 1e-8)])
def test_backward_adjoint_workload_d2048(policy, tol):
    # the adjoint workload: d = 2048 controlled spectrum, k = 8, half-gap 1e-2,
    # checkpoints every 4 iterates; against the oracle's Daleckii-Krein gradient
    torch = cuda_or_skip()
    rs = lib_or_fail()
    d, k = 2048, 8
    spec = workloads.controlled_spectrum(d, k, 1e-2, seed=504)
    Rbar = _loss_seed(d, 9)
    Hbar = rs.reflector_backward(torch.from_numpy(spec.H).cuda(), k, 0.0, torch.from_numpy(Rbar).cuda(),
                                 policy=rs.Policy[policy], ckpt_every=4).cpu().numpy()
    dk = _dk_gradient(spec, 0.0, Rbar)
    rel = np.linalg.norm(Hbar - dk) / np.linalg.norm(dk)
    assert rel < tol, rel
    if policy == "FP64":
        # central finite differences of the FP64 forward, step 1e-6
        rng = np.random.default_rng(10)
        W = rng.standard_normal((d, d))
        W = 0.5 * (W + W.T) / np.linalg.norm(W)
        h = 1e-6
        Hd = torch.from_numpy(spec.H).cuda()
        Wd = torch.from_numpy(W).cuda()
        Rp, _, _ = rs.reflector(Hd + h * Wd, k, 0.0, tol=1e-14, policy=rs.Policy.FP64, check=False)
        Rm, _, _ = rs.reflector(Hd - h * Wd, k, 0.0, tol=1e-14, policy=rs.Policy.FP64, check=False)
        Rb = torch.from_numpy(Rbar).cuda()
        fd = float(((Rp - Rm) * Rb).sum()) / (2 * h)
        an = float(np.sum(Hbar * W))
        assert abs(fd - an) <= 1e-4 * max(1.0, abs(an)), (fd, an)
