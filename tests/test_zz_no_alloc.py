"""rsign_reflector_noalloc: the FP64 reflector without device allocation.

For callers that cannot allocate device memory while they run (memory
planned once at start-up, fixed budgets, threads that must not wait on the
allocator): the entry point takes its workspace from a static device array
inside the library.  This file is collected last on purpose, so that a run
that stops at the first failure has already run every other test; it passes
alone in a fresh process as well.
"""
import ctypes

import numpy as np
import pytest

import oracle
import workloads
from helpers import cuda_or_skip, lib_or_fail, spec_norm_sym

pytestmark = pytest.mark.gpu


def _noalloc_fn(rs):
    lib = rs.load()
    fn = lib.rsign_reflector_noalloc
    fn.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double, ctypes.c_double,
                   ctypes.c_void_p, ctypes.POINTER(rs.Info), ctypes.c_void_p]
    fn.restype = ctypes.c_int
    return fn


def test_noalloc_matches_allocating_entry_point_and_oracle():
    # three calls in a row that share the static array: d = 512 (padded order
    # 512), then d = 200 (padded 256: the smaller layout, after a larger call
    # left its contents), then d = 300; each against the allocating entry
    # point (same policy and tolerance, same stop step) and against the
    # oracle's reflector I - 2 Q_k Q_k^T of the known eigenbasis
    torch = cuda_or_skip()
    rs = lib_or_fail()
    fn = _noalloc_fn(rs)
    stream = torch.cuda.current_stream().cuda_stream
    for call, (d, k, delta, seed) in enumerate([(512, 200, 1e-1, 12), (200, 3, 5e-2, 13), (300, 7, 5e-2, 11)]):
        spec = workloads.controlled_spectrum(d, k, delta, seed)
        H = torch.from_numpy(spec.H).cuda()
        R_ref, info_ref, st_ref = rs.reflector(H, k, 0.0, tol=1e-12, policy=rs.Policy.FP64)
        R = torch.empty_like(H)
        info = rs.Info()
        st = fn(H.data_ptr(), d, k, 0.0, 1e-12, R.data_ptr(), ctypes.byref(info), stream)
        torch.cuda.synchronize()
        assert st == rs.Status.OK, rs.status_str(st)
        assert st_ref == rs.Status.OK
        assert info.workspace_bytes == 0 and info.cert_ok == 1
        assert info.steps_fp64 == info_ref.steps_fp64
        assert info.launches == info_ref.launches
        assert (R - R_ref).abs().max().item() <= 1e-12, call
        assert abs(info.trace - (d - 2 * k)) < 1e-9
        Rh = R.cpu().numpy()
        assert spec_norm_sym(Rh - oracle.reflector_from_basis(spec.Q, k)) <= 1e-11, call


def test_noalloc_failure_statuses_match_the_allocating_entry_point():
    # a shift outside the gap (certificate fails), a NaN entry (argument
    # error) and H = sI (A = 0, no scaling exists): the same status, and
    # where a report is filled the same certificate flag
    torch = cuda_or_skip()
    rs = lib_or_fail()
    fn = _noalloc_fn(rs)
    stream = torch.cuda.current_stream().cuda_stream
    d, k = 64, 5
    spec = workloads.controlled_spectrum(d, k, 5e-2, seed=14)
    lam = np.sort(spec.lam)
    outside = float(0.5 * (lam[k + 5] + lam[k + 6]))  # between lam_{k+6} and lam_{k+7}: index k + 6
    H_nan = spec.H.copy()
    H_nan[3, 7] = np.nan
    cases = [(spec.H, outside), (H_nan, 0.0), (0.75 * np.eye(d), 0.75)]
    seen = []
    for Hn, s in cases:
        H = torch.from_numpy(np.ascontiguousarray(Hn)).cuda()
        R_ref, info_ref, st_ref = rs.reflector(H, k, s, tol=1e-12, policy=rs.Policy.FP64, check=False)
        R = torch.empty_like(H)
        info = rs.Info()
        st = fn(H.data_ptr(), d, k, s, 1e-12, R.data_ptr(), ctypes.byref(info), stream)
        torch.cuda.synchronize()
        assert st == st_ref, (rs.status_str(st), rs.status_str(st_ref))
        seen.append(st)
        if st == rs.Status.ERR_CERT:
            assert info.cert_ok == info_ref.cert_ok == 0
            assert info.trace == pytest.approx(info_ref.trace, abs=1e-9)
            assert abs(info.trace - (d - 2 * (k + 6))) < 1e-6
    assert seen == [rs.Status.ERR_CERT, rs.Status.ERR_ARG, rs.Status.ERR_ARG]


def test_noalloc_rejects_sizes_beyond_its_workspace():
    torch = cuda_or_skip()
    rs = lib_or_fail()
    fn = _noalloc_fn(rs)
    H = torch.eye(600, dtype=torch.float64, device="cuda")
    R = torch.empty_like(H)
    st = fn(H.data_ptr(), 600, 3, 0.5, 1e-12, R.data_ptr(), None, 0)
    assert st == rs.Status.ERR_UNSUPPORTED
    # host buffers would need staging memory: rejected
    Hh = np.eye(64)
    Rh = np.empty((64, 64))
    assert fn(Hh.ctypes.data, 64, 3, 0.5, 1e-12, Rh.ctypes.data, None, 0) == rs.Status.ERR_ARG
