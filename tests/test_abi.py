"""CPU-side checks of the C ABI: the library builds, loads and exports every
function that include/*.h declares; host logic of the binding.  No GPU calls."""
import ctypes
import math
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
def test_tile_order_is_a_permutation_of_the_needed_tiles(rs, dp, sym):
    # the blocked visiting order of the persistent GEMM covers every needed
    # 128 x 256 output tile exactly once (host computation, no GPU)
    bm, bn = rs.dbg_tile_order(dp, sym)
    nbm, nbn = dp // 128, dp // 256
    want = {(r, c) for r in range(nbm) for c in range(nbn) if not sym or c * 256 + 255 >= r * 128}
    got = list(zip(bm.tolist(), bn.tolist()))
    assert len(got) == len(set(got)) == len(want)
    assert set(got) == want
    # blocked: the first ~150 units touch few distinct row and column panels
    head = got[: min(len(got), 152)]
    assert len({c for _, c in head}) <= 16 and len({r for r, _ in head}) <= 40


@pytest.mark.parametrize("dp", [256, 768, 1024, 8192, 16384])
def test_symmetric_check_tiles_fill_every_slot_once(rs, dp):
    # the check's symmetric GEMV: block t handles upper-triangle tile (I, J);
    # its row sums fill slot J of block I's rows and, off the diagonal, its
    # column sums slot I of block J's rows.  Every (block, slot) pair must be
    # written exactly once, so that the slot-order sum of a row sees each
    # 128-column block of the matrix once (host computation, no GPU)
    I, J = rs.dbg_sym_gemv_tiles(dp)
    nb = dp // 128
    assert len(I) == nb * (nb + 1) // 2
    assert all(0 <= i <= j < nb for i, j in zip(I.tolist(), J.tolist()))
    writes = {}
    for i, j in zip(I.tolist(), J.tolist()):
        writes[(i, j)] = writes.get((i, j), 0) + 1      # rows of block i, slot j
        if i != j:
            writes[(j, i)] = writes.get((j, i), 0) + 1  # rows of block j, slot i
    assert writes == {(a, b): 1 for a in range(nb) for b in range(nb)}
    with pytest.raises(Exception):
        rs.dbg_sym_gemv_tiles(300)


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


@pytest.mark.parametrize("l0,u0", [(1e-2, 1.04), (2e-3, 1.0), (0.2, 1.04), (0.7, 1.0)])
def test_refine_stage_plan_follows_the_oracle_iterates(rs, oracle_mod, l0, u0):
    # the lower end of the spectrum that the REFINE stage plan tracks: the
    # oracle's scaled iterates of a diagonal X_0 (eigenvalues from l0 to u0)
    # have smallest |entry| equal to the library's l_m for m >= 1 (l_0 is
    # normalised by u0); hi/lo pairs until l_m >= 1/2, tangent steps until
    # l_m >= 1 - 1e-3 (Sec. 3.5 reading of the scaled steps)
    steps = 40
    le, n_split, m_tan = rs.dbg_stage_plan(l0, u0, scaled=True, max_steps=steps, steps_low=steps)
    coef = oracle_mod.scaled_ns_coeffs(min(1.0, l0), u0)
    X0 = np.diag(np.array([l0, -l0, 0.5 * (l0 + u0), -u0, u0]))
    its = oracle_mod.scaled_ns_iterates(X0, coef, steps)
    assert le[0] * u0 == pytest.approx(min(1.0, l0), rel=1e-15)
    for m in range(1, 12):
        assert le[m] == pytest.approx(np.abs(np.diag(its[m])).min(), rel=1e-11, abs=1e-15)
    assert n_split == next(m for m in range(steps + 1) if le[m] >= 0.5)
    assert all(le[m] < 0.5 for m in range(n_split))
    first_conv = next(m for m in range(steps) if le[m] >= 1.0 - 1e-3)
    assert m_tan == max(1, first_conv)
    # a stage that stopped before the cut runs every tangent step
    _, _, m_short = rs.dbg_stage_plan(l0, u0, scaled=True, max_steps=steps, steps_low=min(first_conv, 3))
    assert m_short == min(first_conv, 3)
    # plain steps (no scaling): l_m = p_m(l0 / u0) (Eq. pm), the conservative end
    le_p, n_p, _ = rs.dbg_stage_plan(l0, u0, scaled=False, max_steps=steps, steps_low=steps)
    for m in range(0, 20):
        assert le_p[m] == pytest.approx(float(oracle_mod.p_m(min(1.0, l0) / u0, m)), rel=1e-11, abs=1e-15)
    assert n_p >= n_split


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


_K_EXTENTS = [1, 255, 256, 700, 1024, 3072, 4096, 8191, 8192, 12288, 16384]


def _check_fp64e_plan(plan, n_planes, beta, levels, k_extent):
    L = min(levels, n_planes)
    groups = plan["groups"]
    # every pair of planes (p, q) with p + q < L appears exactly once
    pairs = [pq for g in groups for pq in g[0]]
    want = sorted((p, t - p) for t in range(L) for p in range(t + 1) if p < n_planes and t - p < n_planes)
    assert sorted(pairs) == want and plan["n_pairs"] == len(pairs)
    two = plan["n_sg"] == 2
    assert plan["n_sg"] in (0, 2)
    for g, (gp, shift, sg) in enumerate(groups):
        levels_g = {p + q for p, q in gp}
        assert len(levels_g) == 1  # one digit level per group
        t = levels_g.pop()
        # FP32 exactness: |digit| <= 2^(beta - 1), so a group sums to at most
        # n 2^(2 beta - 2) K, which must stay within 2^24
        assert len(gp) * 2 ** (2 * beta - 2) * k_extent <= 2 ** 24
        # the group's weight reproduces the digit expansion: pair (p, q) of
        # M_ik = sigma_i sum_p d_p 2^(-beta (p + 1)) weighs 2^(-beta (t + 2))
        w = shift + plan["unit_exp"] + (plan["sh01"] if (two and sg == 0) else 0)
        assert w == -beta * (t + 2), (g, t, shift, sg)
        assert shift >= 0
    # the int64 sums cannot overflow: 2^24 per group at its shift, per sum
    for s in ((0, 1) if two else (0,)):
        assert sum(2 ** (24 + sh) for gp, sh, sg in groups if sg == s) < 2 ** 62
    # execution order: super-group 0 before 1, top level first within each
    key = [(sg, -(gp[0][0] + gp[0][1])) for gp, sh, sg in groups]
    assert key == sorted(key)
    if two:
        top0 = max(p + q for gp, sh, sg in groups if sg == 0 for p, q in gp)
        low1 = min(p + q for gp, sh, sg in groups if sg == 1 for p, q in gp)
        assert top0 < low1


@pytest.mark.parametrize("k_extent", _K_EXTENTS)
@pytest.mark.parametrize("levels", [1, 3, 5, 6, 7])
def test_refinement_product_plans_are_exact(rs, k_extent, levels):
    # the refinement's products: 7 planes of 5-bit digits, 5..7 levels
    plan = rs.dbg_fp64e_plan(7, 5, levels, k_extent)
    _check_fp64e_plan(plan, 7, 5, levels, k_extent)


@pytest.mark.parametrize("k_extent", _K_EXTENTS)
def test_fp64_emulating_plans_are_exact(rs, k_extent):
    # the polish products: the widest digit with one exact pair product, all
    # levels of ceil(54 / beta) planes (at least 54 bits)
    beta = rs.dbg_fp64e_beta(k_extent)
    assert beta in (5, 6, 7)
    assert 2 ** (2 * beta - 2) * k_extent <= 2 ** 24
    if beta < 7:  # a wider digit would not fit (exactness or the kernel's limits)
        wider = 2 ** (2 * beta) * k_extent > 2 ** 24
        assert wider or rs.dbg_fp64e_beta(max(1, k_extent // 4)) > beta
    P = -(-54 // beta)
    assert P * beta >= 54
    plan = rs.dbg_fp64e_plan(P, beta, P, k_extent)
    _check_fp64e_plan(plan, P, beta, P, k_extent)


def test_fp64e_digit_width_shrinks_with_the_extent(rs):
    widths = [rs.dbg_fp64e_beta(k) for k in _K_EXTENTS]
    assert widths == sorted(widths, reverse=True)
    assert rs.dbg_fp64e_beta(0) == 0 and rs.dbg_fp64e_beta(16385) == 0


@pytest.mark.parametrize("bn", [128, 256])
@pytest.mark.parametrize("sym", [0, 1])
@pytest.mark.parametrize("order", [0, 1])
def test_batch_tile_tables_cover_every_tile_once(rs, bn, sym, order):
    # ragged padded orders (multiples of bn); each needed tile of each matrix
    # appears once, its slot inside the matrix's own slot range
    rng = np.random.default_rng(bn + 2 * sym + order)
    dps = [bn * int(x) for x in rng.integers(1, 1024 // bn + 1, 37)]
    units, sb = rs.dbg_batch_units(dps, bn, sym, order)
    want = set()
    for m, dp in enumerate(dps):
        for r in range(dp // 128):
            for c in range(dp // bn):
                if not sym or (c + 1) * bn > r * 128:  # the tile meets the upper triangle
                    want.add((m, r, c))
    got = [(m, r, c) for m, r, c, _ in units]
    assert len(got) == len(set(got)) and set(got) == want
    assert sb[0] == 0 and sb[-1] == len(units) and all(a <= b for a, b in zip(sb, sb[1:]))
    slots = sorted(s for *_, s in units)
    assert slots == list(range(len(units)))
    for m, r, c, s in units:
        assert sb[m] <= s < sb[m + 1]
    if order == 0:  # largest matrices first
        sizes = [dps[m] for m, *_ in units]
        assert sizes == sorted(sizes, reverse=True)
    else:
        assert [m for m, *_ in units] == sorted(m for m, *_ in units)


def test_batch_tile_table_rejects_bad_orders(rs):
    with pytest.raises(rs.RsignError):
        rs.dbg_batch_units([256, 300], 128)
    assert rs.dbg_batch_units([], 128) == ([], [0])


def test_refinement_level_rule(rs):
    # the first sweep's levels: the smallest L in 5..6 whose truncation model
    # 2^(-5L) s_A s_R sqrt(d) stays within tol mu / 2, else 7
    for tol in (1e-4, 1e-6, 1e-8, 1e-10):
        for mu in (1e-1, 1e-2, 1e-3, 1e-4):
            for d in (256, 4096, 16384):
                L, _ = rs.dbg_refine_levels(tol, 2.0, 4.0, d, mu, 16)
                model = [2.0 ** (-5 * l) * 8.0 * math.sqrt(d) <= 0.5 * tol * mu for l in (5, 6)]
                assert L == (5 if model[0] else 6 if model[1] else 7)
    # monotone: a smaller margin or a tighter tolerance never takes fewer levels
    Ls = [rs.dbg_refine_levels(1e-6, 1.0, 1.0, 8192, mu, 16)[0] for mu in (1.0, 1e-1, 1e-2, 1e-3, 1e-4, 1e-5)]
    assert Ls == sorted(Ls)
    # polish: five levels for a small index at tol >= 1e-6, else six
    assert rs.dbg_refine_levels(1e-6, 1, 1, 8192, 1e-2, 16)[1] == 5
    assert rs.dbg_refine_levels(1e-6, 1, 1, 768, 1e-2, 384)[1] == 6
    assert rs.dbg_refine_levels(1e-8, 1, 1, 8192, 1e-2, 16)[1] == 6
    with pytest.raises(rs.RsignError):
        rs.dbg_refine_levels(0.0, 1, 1, 8192, 1e-2, 16)
