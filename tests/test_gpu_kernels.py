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


@pytest.mark.parametrize("dp,sym", [(512, 0), (1536, 1), (4096, 0), (4096, 1)])
def test_tc_gemm_repeats_bit_for_bit(dp, sym):
    # the persistent schedule is static: two launches on the same operands
    # give identical bits (and match FP32 accumulation)
    torch = cuda_or_skip()
    rs = lib_or_fail()
    X = _rand(torch, dp, torch.float16, 99 + dp, sym=bool(sym))
    Y = X if sym else _rand(torch, dp, torch.float16, 98 + dp)
    out, status = rs.dbg_tc_gemm(X, Y, fmt=0, sym=sym)
    out2, status2 = rs.dbg_tc_gemm(X, Y, fmt=0, sym=sym)
    torch.cuda.synchronize()
    assert int(status.item()) == 0 and int(status2.item()) == 0
    assert torch.equal(out, out2)
    ref = X.float() @ Y.float().T
    _check_fp32_accumulation(torch, out, ref, X.float().abs() @ Y.float().abs().T, dp)


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


@pytest.mark.parametrize("dp,d_real,sym", [(256, 256, 0), (512, 300, 1), (1024, 1024, 0), (2048, 2048, 1)])
def test_fp64grade_product_matches_fp64(dp, d_real, sym):
    # digit-plane product on the FP16 tensor cores vs an FP64 matmul
    torch = cuda_or_skip()
    rs = lib_or_fail()
    g = torch.Generator(device="cuda").manual_seed(dp + d_real)
    A = torch.zeros((dp, dp), device="cuda", dtype=torch.float64)
    B = torch.zeros((dp, dp), device="cuda", dtype=torch.float64)
    a = torch.randn((d_real, d_real), generator=g, device="cuda", dtype=torch.float64)
    A[:d_real, :d_real] = 0.5 * (a + a.T) * torch.logspace(-3, 0, d_real, device="cuda", dtype=torch.float64)
    A = 0.5 * (A + A.T)
    if sym:
        B = A
    else:
        b = torch.randn((d_real, d_real), generator=g, device="cuda", dtype=torch.float64)
        B[:d_real, :d_real] = 0.5 * (b + b.T)
    out = rs.dbg_fp64grade_gemm(A, B, d_real=d_real, sym=sym)
    ref = A @ B
    torch.cuda.synchronize()
    # 35 bits per operand relative to the row maxima, exact integer accumulation
    rmax = A.abs().amax(dim=1, keepdim=True)
    cmax = B.abs().amax(dim=1, keepdim=True).T
    bound = 1e-9 * (d_real ** 0.5) * rmax * cmax + 1e-13 * (A.abs() @ B.abs())
    assert ((out - ref).abs() - bound).max().item() <= 0.0
    if sym:
        assert (out - out.T).abs().max().item() == 0.0


@pytest.mark.parametrize("dp,d_real,sym,kind", [(256, 200, 1, "random"), (1024, 1000, 0, "random"),
                                                (2048, 2048, 1, "coherent"), (4096, 4096, 0, "random"),
                                                (8192, 8192, 1, "coherent"), (8192, 8192, 0, "random"),
                                                (16384, 16384, 1, "coherent")])
def test_fp8_digit_planes_give_the_fp16_bits(dp, d_real, sym, kind):
    # The 5-bit balanced digits (|d| <= 16) are exact in E4M3 and each level
    # group sums to an integer below 2^24, so the kind::f8f6f4 product must
    # reproduce the kind::f16 product bit for bit.  "coherent" operands have
    # every off-diagonal entry in [1.5, 2) (leading digits 12..16, all of one
    # sign): each level sum comes near its 2^24 bound, where an accumulator
    # narrower than 24 bits would drop bits.
    torch = cuda_or_skip()
    rs = lib_or_fail()
    g = torch.Generator(device="cuda").manual_seed(11 * dp + d_real)
    A = torch.zeros((dp, dp), device="cuda", dtype=torch.float64)
    if kind == "coherent":
        a = 1.5 + 0.5 * torch.rand((d_real, d_real), generator=g, device="cuda", dtype=torch.float64)
    else:
        a = torch.randn((d_real, d_real), generator=g, device="cuda", dtype=torch.float64)
    A[:d_real, :d_real] = 0.5 * (a + a.T)
    A.diagonal()[:d_real] += 3.0
    if sym:
        B = A
    else:
        B = torch.zeros_like(A)
        b = torch.randn((d_real, d_real), generator=g, device="cuda", dtype=torch.float64)
        B[:d_real, :d_real] = 0.5 * (b + b.T)
    prev = rs.dbg_set_digit_fp8(0)
    try:
        out16 = rs.dbg_fp64grade_gemm(A, B, d_real=d_real, sym=sym)
        rs.dbg_set_digit_fp8(1)
        out8 = rs.dbg_fp64grade_gemm(A, B, d_real=d_real, sym=sym)
    finally:
        rs.dbg_set_digit_fp8(prev)
    torch.cuda.synchronize()
    assert torch.equal(out8, out16)
    ref = A @ B
    rmax = (A - torch.diag(torch.diagonal(A))).abs().amax(dim=1, keepdim=True)
    cmax = (B - torch.diag(torch.diagonal(B))).abs().amax(dim=1, keepdim=True).T
    bound = 1e-9 * (d_real ** 0.5) * rmax * cmax + 1e-13 * (A.abs() @ B.abs())
    assert ((out8 - ref).abs() - bound).max().item() <= 0.0


@pytest.mark.parametrize("d,k", [(1024, 16), (3000, 40), (8192, 16)])
def test_refinement_with_fp8_digits_gives_the_same_reflector(d, k):
    # the whole FP16_REFINE call with FP8 and with FP16 digit planes: the same bits
    torch = cuda_or_skip()
    rs = lib_or_fail()
    import workloads
    H, lam, Q = workloads.controlled_spectrum_torch(d, k, 1e-2, seed=3 * d + k)
    outs = []
    prev = rs.dbg_set_digit_fp8(0)
    try:
        for f8 in (0, 1):
            rs.dbg_set_digit_fp8(f8)
            R, info, st = rs.reflector(H, k, 0.0, tol=1e-6, policy=rs.Policy.FP16_REFINE, check=False)
            assert st == rs.Status.OK, (st, info.as_dict())
            outs.append(R.clone())
    finally:
        rs.dbg_set_digit_fp8(prev)
    torch.cuda.synchronize()
    assert torch.equal(outs[0], outs[1])


@pytest.mark.parametrize("dp,d_real,sym", [(256, 200, 1), (512, 512, 0), (1024, 1000, 1), (8192, 8192, 1)])
def test_fp64e_product_is_fp64_accurate(dp, d_real, sym):
    # FP64-emulating digit-plane product (>= 54 bits per operand): within a
    # few FP64 roundings of the exact product, like a native FP64 GEMM
    torch = cuda_or_skip()
    rs = lib_or_fail()
    g = torch.Generator(device="cuda").manual_seed(7 * dp + d_real)
    A = torch.zeros((dp, dp), device="cuda", dtype=torch.float64)
    a = torch.randn((d_real, d_real), generator=g, device="cuda", dtype=torch.float64)
    A[:d_real, :d_real] = 0.5 * (a + a.T) * torch.logspace(-4, 0, d_real, device="cuda", dtype=torch.float64)
    A = 0.5 * (A + A.T)
    A.diagonal()[:d_real] += 3.0  # a heavy exact diagonal, as in a near-involution
    if sym:
        B = A
    else:
        B = torch.zeros_like(A)
        b = torch.randn((d_real, d_real), generator=g, device="cuda", dtype=torch.float64)
        B[:d_real, :d_real] = 0.5 * (b + b.T)
    out = rs.dbg_fp64e_gemm(A, B, d_real=d_real, sym=sym)
    # reference: A = hi + lo (hi the FP32 rounding), each part multiplied in
    # FP64, so the reference itself is within ~u K |A||B| of the exact product
    hi = A.float().double()
    ref = hi @ B + (A - hi) @ B
    torch.cuda.synchronize()
    bound = 8 * 2.0 ** -53 * (A.abs() @ B.abs()) * (d_real ** 0.5)
    assert ((out - ref).abs() - bound).max().item() <= 0.0
    if sym:
        assert (out - out.T).abs().max().item() == 0.0


@pytest.mark.parametrize("dp,scale_spread", [(256, 0), (768, 2), (1024, 8), (8192, 4)])
def test_gemv_df_is_fp64_accurate(dp, scale_spread):
    # double-float GEMV of the refinement check: per term ~2^-46 relative, so
    # |y - y_exact| <= 2^-44 sum_j |m_ij x_j| (checked against FP64 torch,
    # whose own error is below 2^-50 sqrt(K) sum |m x| here)
    torch = cuda_or_skip()
    rs = lib_or_fail()
    g = torch.Generator(device="cuda").manual_seed(11 + dp)
    M = torch.randn((dp, dp), generator=g, device="cuda", dtype=torch.float64)
    if scale_spread:  # rows and columns over 2^(+-spread): a wide dynamic range
        e = torch.randint(-scale_spread, scale_spread + 1, (dp,), generator=g, device="cuda").double()
        M = M * torch.pow(2.0, e)[:, None] * torch.pow(2.0, -e)[None, :]
    x = torch.randn(dp, generator=g, device="cuda", dtype=torch.float64)
    y = rs.dbg_gemv_df(M, x)
    ref = M @ x
    scale = M.abs() @ x.abs()
    assert float(((y - ref).abs() - 2.0 ** -44 * scale).max()) <= 0.0


@pytest.mark.parametrize("dp,scale_spread", [(256, 0), (768, 2), (1024, 8), (8192, 4)])
def test_symmetric_gemv_df_reads_the_upper_triangle_only(dp, scale_spread):
    # the check's symmetric form: the same bound as the row kernel, with every
    # 128 x 128 tile below the diagonal tiles set to NaN (never read; the
    # diagonal tiles are read whole)
    torch = cuda_or_skip()
    rs = lib_or_fail()
    g = torch.Generator(device="cuda").manual_seed(23 + dp)
    M = torch.randn((dp, dp), generator=g, device="cuda", dtype=torch.float64)
    M = 0.5 * (M + M.T)
    if scale_spread:  # symmetric scaling D M D over 2^(+-spread)
        e = torch.randint(-scale_spread, scale_spread + 1, (dp,), generator=g, device="cuda").double()
        M = M * torch.pow(2.0, e)[:, None] * torch.pow(2.0, e)[None, :]
    x = torch.randn(dp, generator=g, device="cuda", dtype=torch.float64)
    ref = M @ x
    scale = M.abs() @ x.abs()
    Mu = M.clone()
    blk = torch.arange(dp, device="cuda") // 128
    Mu[blk[:, None] > blk[None, :]] = float("nan")
    y = rs.dbg_gemv_df_sym(Mu, x)
    assert bool(torch.isfinite(y).all())
    assert float(((y - ref).abs() - 2.0 ** -44 * scale).max()) <= 0.0
    y_row = rs.dbg_gemv_df(M, x)
    assert float(((y - y_row).abs() - 2.0 ** -43 * scale).max()) <= 0.0


@pytest.mark.parametrize("d,dp", [(512, 512), (700, 768), (1000, 1024)])
def test_commutator_check_matches_fp64_power_steps(d, dp):
    # the matrix-free check against the same power steps in FP64 (torch), on a
    # reflector perturbed by 1e-7: ||C v||/2 and ||N z|| to the cancellation's
    # accuracy (C and N are 1e-7 of the products, so their directions, and the
    # Rayleigh-Ritz entries taken on them, agree to ~1e-7 relative)
    torch = cuda_or_skip()
    rs = lib_or_fail()
    g = torch.Generator(device="cuda").manual_seed(d)
    Q, _ = torch.linalg.qr(torch.randn((d, d), generator=g, device="cuda", dtype=torch.float64))
    lam = torch.cat([-torch.linspace(1.0, 0.05, 8, device="cuda", dtype=torch.float64),
                     torch.linspace(0.05, 1.0, d - 8, device="cuda", dtype=torch.float64)])
    A = (Q * lam) @ Q.T
    R = torch.eye(d, device="cuda", dtype=torch.float64) - 2.0 * Q[:, :8] @ Q[:, :8].T
    P = torch.randn((d, d), generator=g, device="cuda", dtype=torch.float64)
    R = R + 1e-7 * (P + P.T)
    Ap = torch.zeros((dp, dp), device="cuda", dtype=torch.float64)
    Rp = torch.zeros((dp, dp), device="cuda", dtype=torch.float64)
    Ap[:d, :d] = A
    Rp[:d, :d] = R
    iters = 12
    g2, rho, (a11, a12, a22) = rs.dbg_commutator_check(Ap, Rp, d=d, iters=iters)
    # the same steps in FP64
    i = torch.arange(d, device="cuda", dtype=torch.float64)
    v = 1.0 + torch.remainder(i, 7.0) * 0.125
    v = v / v.norm()
    z = v.clone()
    for _ in range(iters):
        v_prev = v
        Av = A @ v
        w = R @ Av - A @ (R @ v)
        c_norm = float(w.norm())
        v = w / w.norm()
        w3 = R @ (R @ z) - z
        n_norm = float(w3.norm())
        z = w3 / w3.norm()
    assert g2 == pytest.approx(0.5 * c_norm, rel=1e-5)
    assert rho == pytest.approx(n_norm, rel=1e-5)
    assert a11 == pytest.approx(float(v_prev @ (A @ v_prev)), rel=1e-6, abs=1e-9)
    assert a12 == pytest.approx(float(v @ (A @ v_prev)), rel=1e-6, abs=1e-9)
    assert a22 == pytest.approx(float(v @ (A @ v)), rel=1e-6, abs=1e-9)


@pytest.mark.parametrize("d,k", [(1024, 16), (1280, 640)])
def test_refinement_products_same_bits_on_both_tile_widths(d, k):
    # the FP64-grade products are exact integer level sums converted once, so
    # the 128-wide (int64 sums in TMEM) and 256-wide (sums in
    # global memory) launches give the same reflector bit for bit
    torch = cuda_or_skip()
    rs = lib_or_fail()
    import workloads
    H, lam, Q = workloads.controlled_spectrum_torch(d, k, 1e-2, seed=d + k)
    outs = []
    prev = rs.dbg_set_ozaki_tile(256)
    try:
        for bn in (256, 128):
            rs.dbg_set_ozaki_tile(bn)
            R, info, st = rs.reflector(H, k, 0.0, tol=1e-6, policy=rs.Policy.FP16_REFINE, check=False)
            assert st == rs.Status.OK
            outs.append(R.clone())
    finally:
        rs.dbg_set_ozaki_tile(prev)
    assert torch.equal(outs[0], outs[1])


@pytest.mark.parametrize("d", [768, 2048])
def test_polish_products_same_bits_on_both_tile_widths(d):
    # the FP64-emulating polish products are exact integer level sums as
    # well: 128-wide (TMEM sums) and 256-wide launches give the same bits
    torch = cuda_or_skip()
    rs = lib_or_fail()
    import workloads
    H, lam, Q = workloads.controlled_spectrum_torch(d, 8, 5e-2, seed=d + 3)
    outs = []
    prev = rs.dbg_set_ozaki_tile(256)
    try:
        for bn in (256, 128):
            rs.dbg_set_ozaki_tile(bn)
            R, info, st = rs.reflector(H, 8, 0.0, tol=1e-12, policy=rs.Policy.FP16_POLISH, check=False)
            assert st == rs.Status.OK and info.steps_fp64 == 2
            outs.append(R.clone())
    finally:
        rs.dbg_set_ozaki_tile(prev)
    assert torch.equal(outs[0], outs[1])


def test_digit_sum_conversion_matches_128_bit_rounding_and_numpy():
    # The digit-plane products turn each exact int64 level sum v into
    # v 2^e in FP64 (round to nearest, ties to even).  The epilogue does it with
    # one correctly rounded conversion and an exponent shift; the 128-bit
    # integer path rounds the significand itself.  Both must give numpy's
    # ldexp(float64(v), e) bit for bit: normal results, ties at 2^53 + 1 and
    # beyond, the full int64 range, and exponents that underflow or overflow.
    import numpy as np
    torch = cuda_or_skip()
    rs = lib_or_fail()
    rng = np.random.default_rng(11)
    vals = []
    for bits in range(64):
        lo, hi = (0, 1) if bits == 0 else (1 << (bits - 1), (1 << bits) - 1)
        vals.extend(int(x) for x in rng.integers(lo, hi, size=40, endpoint=True, dtype=np.uint64))
    special = [0, 1, 2 ** 53, 2 ** 53 + 1, 2 ** 53 + 3, 2 ** 54 + 2, 2 ** 54 + 6, 2 ** 62 + 2 ** 9,
               2 ** 62 + 2 ** 9 + 1, 2 ** 63 - 1, 2 ** 63 - 2 ** 10, 2 ** 63 - 2 ** 10 - 1]
    vals = [v for v in vals if v < 2 ** 63] + special
    vals = vals + [-v for v in vals] + [-(2 ** 63)]
    v = np.array(vals, dtype=np.int64)
    e = rng.integers(-80, 80, size=v.size).astype(np.int32)
    e[::17] = -1100   # deep underflow: subnormal or zero
    e[5::17] = -1040  # around the subnormal boundary
    e[9::17] = 1000   # overflow for the larger v
    a, b = rs.dbg_oz_convert(torch.from_numpy(v).cuda(), torch.from_numpy(e).cuda())
    with np.errstate(over="ignore", under="ignore"):
        ref = np.ldexp(v.astype(np.float64), e)
    a, b = a.cpu().numpy(), b.cpu().numpy()
    assert np.array_equal(a.view(np.int64), ref.view(np.int64))
    assert np.array_equal(b.view(np.int64), ref.view(np.int64))


@pytest.mark.parametrize("dp", [256, 512, 768])
def test_power_steps_in_one_launch_give_the_per_step_bits(dp):
    # up to order 512 the power steps of the alpha rule and of the
    # refinement's norms run in one launch: the same arithmetic in the same
    # order as one GEMV and one normalisation launch per step, so the same
    # bits; above 512 both settings take the per-step path.  The estimate
    # itself approaches ||M||_2 from below.
    torch = cuda_or_skip()
    rs = lib_or_fail()
    g = torch.Generator(device="cuda").manual_seed(5 + dp)
    Q, _ = torch.linalg.qr(torch.randn((dp, dp), generator=g, device="cuda", dtype=torch.float64))
    lam = torch.linspace(-0.5, 1.0, dp, device="cuda", dtype=torch.float64)
    M = (Q * lam) @ Q.T
    M = 0.5 * (M + M.T)
    for iters in (1, 2, 20):
        a = rs.dbg_spectral_norm(M, iters)
        b = rs.dbg_spectral_norm(M, iters, per_step=True)
        assert a == b, (iters, a, b)
    est = rs.dbg_spectral_norm(M, 200)
    assert 0.98 <= est <= 1.0 + 1e-5, est
