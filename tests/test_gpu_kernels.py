"""Kernel-level GPU tests: the tcgen05 tensor-core product and the FP64 product
against plain PyTorch references of the same operation."""
import pytest

from helpers import cuda_or_skip, lib_or_fail

pytestmark = pytest.mark.gpu


def _rand(torch, n, dtype, seed, sym=False):
    g = torch.Generator(device="cuda").manual_seed(seed)
    A = torch.randn((n, n), generator=g, device="cuda", dtype=torch.float32)
    if sym:
        A = 0.5 * (A + A.T)
    return A.to(dtype)


def _check_fp32_accumulation(torch, out, ref, ref_abs, K):
    # products of FP16/BF16 values are exact in FP32; the sum of K of them carries
    # a rounding error of order sqrt(K) u_32 sum|a_k b_k| (u_32 = 2^-24 ~ 6e-8)
    bound = 1e-6 * (K ** 0.5) * ref_abs + 1e-6
    excess = ((out - ref).abs() - bound).max().item()
    assert excess <= 0.0, excess


@pytest.mark.parametrize("dp,fmt", [(256, 0), (256, 1), (512, 0), (1024, 1), (4096, 0)])
def test_tc_gemm_full_matches_torch(dp, fmt):
    torch = cuda_or_skip()
    rs = lib_or_fail()
    dt = torch.float16 if fmt == 0 else torch.bfloat16
    A = _rand(torch, dp, dt, 1 + dp)
    B = _rand(torch, dp, dt, 2 + dp)
    out, status = rs.dbg_tc_gemm(A, B, fmt=fmt, sym=0)
    ref = A.float() @ B.float().T
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    _check_fp32_accumulation(torch, out, ref, A.float().abs() @ B.float().abs().T, dp)


@pytest.mark.parametrize("dp,fmt", [(256, 0), (768, 1), (2048, 0)])
def test_tc_gemm_symmetric_schedule(dp, fmt):
    torch = cuda_or_skip()
    rs = lib_or_fail()
    dt = torch.float16 if fmt == 0 else torch.bfloat16
    X = _rand(torch, dp, dt, 7 + dp, sym=True)
    out, status = rs.dbg_tc_gemm(X, X, fmt=fmt, sym=1)
    ref = X.float() @ X.float()
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    assert (out - out.T).abs().max().item() == 0.0  # mirrored exactly
    _check_fp32_accumulation(torch, out, ref, X.float().abs() @ X.float().abs(), dp)


@pytest.mark.parametrize("dp,sym", [(64, 0), (128, 1), (320, 0), (512, 1)])
def test_f64_gemm_matches_torch(dp, sym):
    torch = cuda_or_skip()
    rs = lib_or_fail()
    g = torch.Generator(device="cuda").manual_seed(dp)
    A = torch.randn((dp, dp), generator=g, device="cuda", dtype=torch.float64)
    if sym:
        A = 0.5 * (A + A.T)
        B = A
    else:
        B = torch.randn((dp, dp), generator=g, device="cuda", dtype=torch.float64)
    out = rs.dbg_f64_gemm(A, B, sym=sym)
    ref = A @ B
    torch.cuda.synchronize()
    assert (out - ref).abs().max().item() <= 1e-13 * dp
