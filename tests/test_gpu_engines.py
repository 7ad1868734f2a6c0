"""GPU parity of the quintic Newton-Schulz engine (RSIGN_ENGINE_NS5,
X <- 1/8 X (15I - 10X^2 + 3X^4)) against the oracle's iterates of the same
filter, and its argument rules."""
import numpy as np
import pytest

import oracle
import workloads
from helpers import cuda_or_skip, lib_or_fail, spec_norm_sym

pytestmark = pytest.mark.gpu


def _run(rs, torch, H, k, s, policy, tol=1e-12, **opt):
    Hd = torch.from_numpy(np.ascontiguousarray(H)).cuda()
    R, info, st = rs.reflector(Hd, k, s, tol=tol, policy=policy, options=rs.default_options(**opt), check=False)
    torch.cuda.synchronize()
    return R.cpu().numpy(), info, st


def test_ns5_fp64_matches_the_oracle_iterates():
    # plain-method workload (d = 256, k = 4, Gershgorin alpha): the same
    # stopping step as the oracle's quintic iterates and the same reflector
    torch = cuda_or_skip()
    rs = lib_or_fail()
    spec = workloads.split_spectrum_config(seed=0)
    s = oracle.midpoint(*spec.gap)
    R, info, st = _run(rs, torch, spec.H, spec.k, s, rs.Policy.FP64, tol=1e-12, max_steps=80,
                       engine=int(rs.Engine.NS5))
    assert st == rs.Status.OK and info.cert_ok == 1
    A = oracle.shifted(spec.H, s)
    alpha = oracle.gershgorin_alpha(A)
    its = oracle.ns5_iterates(alpha * A, 40)
    d = spec.H.shape[0]
    tol_fro = max(1e-12, 16 * d * np.finfo(np.float64).eps)
    res = [np.linalg.norm(X @ X - np.eye(d)) for X in its]
    m_or = next(m for m, r in enumerate(res) if r < tol_fro)
    assert info.steps_fp64 == m_or
    assert np.max(np.abs(R - its[m_or])) <= 1e-12
    R_or, _ = oracle.reflector(spec.H, spec.k)
    assert spec_norm_sym(R - R_or) <= 1e-12
    # fewer steps than Eq. NS (three products each instead of two)
    _, info3, _ = _run(rs, torch, spec.H, spec.k, s, rs.Policy.FP64, tol=1e-12, max_steps=80)
    assert info.steps_fp64 < info3.steps_fp64


@pytest.mark.parametrize("d,k", [(300, 7), (513, 256)])
def test_ns5_fp64_ragged_sizes(d, k):
    torch = cuda_or_skip()
    rs = lib_or_fail()
    spec = workloads.controlled_spectrum(d, k, 0.05, seed=200 + d + k)
    R, info, st = _run(rs, torch, spec.H, k, 0.0, rs.Policy.FP64, engine=int(rs.Engine.NS5))
    assert st == rs.Status.OK and info.cert_ok == 1
    assert spec_norm_sym(R - oracle.reflector_from_basis(spec.Q, k)) <= 1e-11


@pytest.mark.parametrize("policy,floor", [("FP16", 2e-2), ("BF16", 2e-1), ("FP32", 1e-4),
                                          ("FP16_POLISH", 2e-2), ("BF16_POLISH", 2e-1)])
def test_ns5_low_precision_within_floors(policy, floor):
    torch = cuda_or_skip()
    rs = lib_or_fail()
    d, k = 768, 12
    spec = workloads.controlled_spectrum(d, k, 1e-1, seed=301)
    R, info, st = _run(rs, torch, spec.H, k, 0.0, rs.Policy[policy], engine=int(rs.Engine.NS5))
    assert st == rs.Status.OK and info.cert_ok == 1, (st, info.as_dict())
    assert spec_norm_sym(R - oracle.reflector_from_basis(spec.Q, k)) <= floor
    assert info.flops_low == pytest.approx(float(d) ** 3 * (3 * info.steps_low + 1))


def test_ns5_argument_rules():
    torch = cuda_or_skip()
    rs = lib_or_fail()
    spec = workloads.controlled_spectrum(256, 4, 5e-2, seed=302)
    Hd = torch.from_numpy(spec.H).cuda()
    for pol in (rs.Policy.FP16_REFINE, rs.Policy.BF16_REFINE):
        _, _, st = rs.reflector(Hd, 4, 0.0, tol=1e-6, policy=pol, check=False,
                                options=rs.default_options(engine=int(rs.Engine.NS5)))
        assert st == rs.Status.ERR_ARG
    _, _, st = rs.reflector(Hd, 4, 0.0, tol=1e-6, policy=rs.Policy.FP64, check=False,
                            options=rs.default_options(engine=7))
    assert st == rs.Status.ERR_ARG
    _, _, st = rs.reflector_batched([Hd, Hd], [4, 4], [0.0, 0.0], tol=1e-12, policy=rs.Policy.FP64,
                                    options=rs.default_options(engine=int(rs.Engine.NS5)))
    assert st == rs.Status.ERR_ARG
