"""Failure detection on the GPU without a GPU fault.

Every pipeline wait of the tcgen05 kernels is bounded: after a wall-clock
limit it records RSIGN_ERR_TIMEOUT in the call's device status word and the
kernel returns, so the context stays usable.  Here one such wait runs with a
short limit on a barrier that nothing completes (the failure is made on
purpose, by withholding the one arrival), and the host reads the status.
"""
import numpy as np
import pytest

import oracle
import workloads
from helpers import cuda_or_skip, lib_or_fail, spec_norm_sym

pytestmark = pytest.mark.gpu


def test_bounded_wait_gives_up_and_reports_the_timeout():
    torch = cuda_or_skip()
    rs = lib_or_fail()
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    # with its arrival the wait completes and the status stays 0
    assert rs.dbg_bounded_wait(1, 50_000_000, status) == rs.Status.OK
    assert int(status.item()) == 0
    # without it the wait runs out after 50 ms and reports the timeout
    assert rs.dbg_bounded_wait(0, 50_000_000, status) == rs.Status.OK
    assert int(status.item()) == int(rs.Status.ERR_TIMEOUT)
    # a limit outside (0, 2 s] is refused before any launch
    assert rs.dbg_bounded_wait(0, 0, status) == rs.Status.ERR_ARG
    assert rs.dbg_bounded_wait(0, 3_000_000_000, status) == rs.Status.ERR_ARG


def test_context_stays_usable_after_a_timeout():
    torch = cuda_or_skip()
    rs = lib_or_fail()
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    assert rs.dbg_bounded_wait(0, 20_000_000, status) == rs.Status.OK
    assert int(status.item()) == int(rs.Status.ERR_TIMEOUT)
    # the next library call runs normally on the same context
    spec = workloads.controlled_spectrum(300, 7, 5e-2, seed=21)
    H = torch.from_numpy(spec.H).cuda()
    R, info, st = rs.reflector(H, 7, 0.0, tol=1e-6, policy=rs.Policy.FP16_REFINE, check=False)
    torch.cuda.synchronize()
    assert st == rs.Status.OK
    assert spec_norm_sym(R.cpu().numpy() - oracle.reflector_from_basis(spec.Q, 7)) <= 1e-6
