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

import workloads
from helpers import cuda_or_skip, lib_or_fail

pytestmark = pytest.mark.gpu


def _noalloc_fn(rs):
    lib = rs.load()
    fn = lib.rsign_reflector_noalloc
    fn.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double, ctypes.c_double,
                   ctypes.c_void_p, ctypes.POINTER(rs.Info), ctypes.c_void_p]
    fn.restype = ctypes.c_int
    return fn


def test_noalloc_matches_allocating_entry_point_twice():
    torch = cuda_or_skip()
    rs = lib_or_fail()
    fn = _noalloc_fn(rs)
    stream = torch.cuda.current_stream().cuda_stream
    for call, (d, k, delta, seed) in enumerate([(300, 7, 5e-2, 11), (512, 200, 1e-1, 12)]):
        spec = workloads.controlled_spectrum(d, k, delta, seed)
        H = torch.from_numpy(spec.H).cuda()
        # reference: the allocating entry point, FP64 policy, same tolerance
        R_ref, info_ref, st_ref = rs.reflector(H, k, 0.0, tol=1e-12, policy=rs.Policy.FP64)
        R = torch.empty_like(H)
        info = rs.Info()
        st = fn(H.data_ptr(), d, k, 0.0, 1e-12, R.data_ptr(), ctypes.byref(info), stream)
        torch.cuda.synchronize()
        assert st == rs.Status.OK, rs.status_str(st)
        assert info.workspace_bytes == 0 and info.cert_ok == 1
        assert info.steps_fp64 == info_ref.steps_fp64
        # the same kernels in the same order: agreement to the FP64 tolerance of the tests
        assert (R - R_ref).abs().max().item() <= 1e-12, call
        assert abs(info.trace - (d - 2 * k)) < 1e-9


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
