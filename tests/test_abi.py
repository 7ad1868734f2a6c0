"""CPU-side checks of the C ABI: the library builds, loads and exports every
function that include/*.h declares; host logic of the binding.  No GPU calls."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def rs():
    import paper_2605_24840_gb300 as rs
    rs.build()
    return rs


def test_library_exports_every_header_function(rs):
    names = rs.header_functions()
    assert "rsign_reflector" in names and "rsign_apply" in names
    assert "rsign_reflector_batched" in names and "rsign_reflector_backward" in names
    lib = rs.load()
    for n in names:
        assert hasattr(lib, n), "librsign.so does not export %s" % n
    # and nothing exported is undeclared (C symbols of the ABI)
    out = subprocess.run(["nm", "-D", "--defined-only", rs.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (rsign_\w+)$", out, flags=re.M))
    assert exported == set(names)


def test_header_is_plain_c(tmp_path):
    # the headers compile as C99 with no CUDA or torch types
    src = tmp_path / "t.c"
    src.write_text('#include "rsign.h"\n#include "rsign_debug.h"\nint main(void){rsign_options o;'
                   'rsign_options_default(&o);return (int)sizeof(rsign_info);}\n')
    r = subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-fsyntax-only", "-I",
                        os.path.join(ROOT, "include"), str(src)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_struct_layouts_match_header(rs, tmp_path):
    src = tmp_path / "s.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "rsign.h"\nint main(void){'
                   'printf("%zu %zu %zu %zu\\n", sizeof(rsign_info), offsetof(rsign_info, launches),'
                   'sizeof(rsign_options), offsetof(rsign_info, ms_total));return 0;}\n')
    exe = tmp_path / "s"
    subprocess.check_call(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    sz, off_l, osz, off_ms = map(int, subprocess.check_output([str(exe)]).split())
    assert sz == ctypes.sizeof(rs.Info)
    assert off_l == rs.Info.launches.offset
    assert off_ms == rs.Info.ms_total.offset
    assert osz == ctypes.sizeof(rs.Options)


def test_status_strings_and_defaults(rs):
    for st in rs.Status:
        assert isinstance(rs.status_str(st), str) and rs.status_str(st)
    o = rs.default_options()
    assert o.max_steps == 100 and o.polish_steps == 2 and o.timing == 1
    assert o.power_steps == 20 and o.alpha_mode == rs.AlphaMode.INF and o.low_split == 1
    assert "sm_103a" in rs.version()


def test_argument_errors_need_no_gpu(rs):
    # validation happens before any device work, so these run on a CPU-only host
    H = np.eye(4)
    R = np.empty((4, 4))
    lib = rs.load()
    info = rs.Info()
    bad = [
        (H.ctypes.data, 4, 0, 0.0, 1e-12, 0),    # k < 1
        (H.ctypes.data, 4, 4, 0.0, 1e-12, 0),    # k > d-1
        (H.ctypes.data, 1, 1, 0.0, 1e-12, 0),    # d < 2
        (H.ctypes.data, 4, 1, 0.0, -1.0, 0),     # tol <= 0
        (H.ctypes.data, 4, 1, 0.0, 1e-12, 99),   # policy
        (None, 4, 1, 0.0, 1e-12, 0),             # NULL H
        (H.ctypes.data, 4, 1, float("inf"), 1e-12, 0),  # infinite shift
    ]
    for (hp, d, k, s, tol, pol) in bad:
        st = lib.rsign_reflector(hp, d, k, s, tol, pol, R.ctypes.data, ctypes.byref(info), None)
        assert st == rs.Status.ERR_ARG, (d, k, s, tol, pol, st)
    assert lib.rsign_apply(None, 4, H.ctypes.data, 1, R.ctypes.data, None) == rs.Status.ERR_ARG
    # stopping the refinement on the bound needs a margin (or the automatic shift)
    o = rs.default_options(refine_stop=int(rs.RefineStop.BOUND))
    st = lib.rsign_reflector_ex(H.ctypes.data, 4, 1, 0.0, 1e-6, int(rs.Policy.FP16_REFINE), ctypes.byref(o),
                                R.ctypes.data, ctypes.byref(info), None)
    assert st == rs.Status.ERR_ARG
    o.refine_stop = 2
    st = lib.rsign_reflector_ex(H.ctypes.data, 4, 1, 0.0, 1e-6, int(rs.Policy.FP64), ctypes.byref(o),
                                R.ctypes.data, ctypes.byref(info), None)
    assert st == rs.Status.ERR_ARG


def test_empty_batch_is_a_no_op(rs):
    # n = 0 is valid and returns before any device work (no GPU needed)
    lib = rs.load()
    st = lib.rsign_reflector_batched_ex(0, None, None, None, None, 1e-12, 0, None, None, None, None)
    assert st == rs.Status.OK
    outs, infos, st = rs.reflector_batched([], [], [])
    assert st == rs.Status.OK and outs == [] and infos == []
    # a negative count is an argument error
    assert lib.rsign_reflector_batched_ex(-1, None, None, None, None, 1e-12, 0, None, None, None, None) \
        == rs.Status.ERR_ARG


@pytest.mark.parametrize("m,seed", [(1, 0), (2, 1), (7, 2), (60, 3), (200, 4)])
def test_tridiagonal_ritz_solver_matches_scipy(rs, m, seed):
    # host part of the automatic shift: eigenvalues (Sturm bisection) and the last
    # eigenvector components (inverse iteration) of a symmetric tridiagonal
    scipy_linalg = pytest.importorskip("scipy.linalg")
    rng = np.random.default_rng(seed)
    a = rng.standard_normal(m)
    b = rng.uniform(0.05, 1.0, max(m - 1, 0))
    if m > 1:
        w, V = scipy_linalg.eigh_tridiagonal(a, b)
    else:
        w, V = a.copy(), np.ones((1, 1))
    for j in sorted({0, m // 2, m - 1}):
        th, last = rs.dbg_tridiag_ritz(a, b if m > 1 else np.zeros(1), j)
        assert th == pytest.approx(w[j], abs=1e-12 * max(1.0, np.abs(w).max()))
        assert abs(last) == pytest.approx(abs(V[-1, j]), abs=1e-8)


def test_binding_rejects_wrong_dtype(rs):
    with pytest.raises(TypeError):
        rs.reflector(np.eye(4, dtype=np.float32), 1, 0.0)
    with pytest.raises(ValueError):
        rs.reflector(np.eye(4), 1, 0.0, out=np.empty((3, 3)))


def test_missing_library_fails_loudly(rs, monkeypatch, tmp_path):
    import paper_2605_24840_gb300 as pkg
    monkeypatch.setattr(pkg, "_lib", None)
    monkeypatch.setattr(pkg, "LIB_PATH", str(tmp_path / "nope.so"))
    with pytest.raises(ImportError):
        pkg.load()


@pytest.mark.parametrize("dp", [256, 512, 1280, 4096, 8192])
@pytest.mark.parametrize("sym", [0, 1])
@pytest.mark.parametrize("cluster", [1, 2])
def test_tile_order_is_a_permutation_of_the_needed_tiles(rs, dp, sym, cluster):
    # the blocked visiting order of the persistent GEMM covers every needed
    # 128 x 256 output tile exactly once (host computation, no GPU)
    if cluster == 2 and (dp // 128) % 2:
        pytest.skip("cluster pairs need an even number of 128-row tiles")
    bm, bn = rs.dbg_tile_order(dp, sym, cluster)
    nbm, nbn = dp // 128, dp // 256
    want = {(r, c) for r in range(nbm) for c in range(nbn) if not sym or c * 256 + 255 >= r * 128}
    got = list(zip(bm.tolist(), bn.tolist()))
    assert len(got) == len(set(got)) == len(want)
    assert set(got) == want
    if cluster == 2:  # the two ranks of a unit share the B panel
        assert np.all(bn[0::2] == bn[1::2]) and np.all(bm[1::2] == bm[0::2] + 1)
    # blocked: the first ~150 units touch few distinct row and column panels
    head = got[: min(len(got), 152)]
    assert len({c for _, c in head}) <= 16 and len({r for r, _ in head}) <= 40


@pytest.mark.parametrize("l0,u0", [(1e-4, 1.0), (3e-3, 1.0), (1e-2, 1.04), (0.3, 1.0), (0.9, 1.04), (2.0, 1.0),
                                   (2.0, 1.04)])
def test_scaled_step_coefficients_match_the_oracle(rs, oracle_mod, l0, u0):
    # the host routine behind rsign_options.ns_scaling against the oracle's
    # step scalings (Sec. 3.5 reading), same interval and stop rule
    got = rs.dbg_scaled_coeffs(l0, u0)
    want = oracle_mod.scaled_ns_coeffs(min(1.0, l0), u0)
    assert len(got) == len(want)
    np.testing.assert_allclose(got, want, rtol=1e-15, atol=0)
    if l0 >= 1.0 and u0 == 1.0:
        assert got == []  # an involution needs no scaled step


@pytest.mark.parametrize("m", [0, 1, 5, 12, 30])
def test_margin_bound_from_steps_is_the_root_of_p_m(rs, oracle_mod, m):
    # gamma with p_m(gamma) = 0.9 (Eq. pm), from the oracle's polynomial
    g = rs.dbg_gamma_from_steps(m)
    assert 0.0 < g <= 0.9
    assert float(oracle_mod.p_m(g, m)) >= 0.9 - 1e-12
    assert float(oracle_mod.p_m(g * (1.0 - 1e-9), m)) < 0.9
    if m == 0:
        assert g == pytest.approx(0.9, abs=1e-15)


def test_host_routines_reject_bad_arguments(rs):
    lib = rs.load()
    n = ctypes.c_int32()
    buf = (ctypes.c_double * 4)()
    assert lib.rsign_dbg_scaled_coeffs(0.0, 1.0, 4, buf, ctypes.byref(n)) == rs.Status.ERR_ARG
    assert lib.rsign_dbg_scaled_coeffs(0.1, 0.5, 4, buf, ctypes.byref(n)) == rs.Status.ERR_ARG
    g = ctypes.c_double()
    assert lib.rsign_dbg_gamma_from_steps(-1, ctypes.byref(g)) == rs.Status.ERR_ARG
