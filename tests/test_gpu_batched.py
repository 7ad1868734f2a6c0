"""GPU checks of rsign_reflector_batched: grouped launches over a slab of
matrices of uneven order (the batched regime of Sec. 4.5).

Every matrix of a batch is compared with (a) the construction-known reflector
I - 2 Q_k Q_k^T of its controlled spectrum (the oracle's definition of R_k,
Prop. 2.1) and (b) its own one-matrix rsign_reflector call with the same
policy and Gershgorin alpha, which the grouped path must reproduce.
"""
import numpy as np
import pytest

import oracle
import workloads
from helpers import cuda_or_skip, lib_or_fail

pytestmark = pytest.mark.gpu


def _batch(count, d_choices, delta_range, seed):
    return workloads.batched_workload(count, d_choices=d_choices, delta_range=delta_range, seed=seed)


def _exact(sp):
    return oracle.reflector_from_basis(sp.Q, sp.k)


def _run(rs, torch, items, policy, tol=1e-12, **opt):
    Hs = [torch.from_numpy(sp.H).cuda() for sp, _ in items]
    ks = [sp.k for sp, _ in items]
    ss = [s for _, s in items]
    options = rs.default_options(**opt) if opt else None
    outs, infos, st = rs.reflector_batched(Hs, ks, ss, tol=tol, policy=policy, options=options)
    torch.cuda.synchronize()
    return [o.cpu().numpy() for o in outs], infos, st


# ragged orders: multiples of 32 and odd sizes, several 128-row tiles, one matrix above 256
RAGGED = (32, 37, 64, 100, 128, 160, 250, 256, 300, 384)


@pytest.mark.parametrize("policy,err_tol", [("FP64", 1e-9), ("FP16_POLISH", 2e-2), ("BF16_POLISH", 1e-1),
                                            ("FP16", 2e-2)])
def test_batched_matches_exact_and_single_calls(policy, err_tol):
    torch = cuda_or_skip()
    rs = lib_or_fail()
    items = _batch(20, RAGGED, (1e-2, 1e-1), seed=11)
    pol = rs.Policy[policy]
    Rb, infos, st = _run(rs, torch, items, pol)
    assert st == rs.Status.OK, st
    for (sp, s), R, inf in zip(items, Rb, infos):
        assert inf.batch_grouped == 1
        assert inf.cert_ok == 1
        assert abs(inf.trace - (sp.d - 2 * sp.k)) < 0.5
        err = np.linalg.norm(R - _exact(sp), 2)
        assert err <= err_tol, (sp.d, sp.k, err)
        # the one-matrix path with the same policy and alpha rule
        R1, inf1, st1 = rs.reflector(sp.H, sp.k, s, tol=1e-12, policy=pol, check=False)
        assert st1 == rs.Status.OK
        assert inf1.alpha == inf.alpha
        if inf1.steps_low == inf.steps_low and inf1.steps_fp64 == inf.steps_fp64:
            np.testing.assert_allclose(R, R1, rtol=0, atol=1e-13)
        else:  # a stop test decided one step apart (partials summed in another order)
            assert abs(inf1.steps_low - inf.steps_low) + abs(inf1.steps_fp64 - inf.steps_fp64) <= 1
            assert np.max(np.abs(R - R1)) <= 4 * err_tol


@pytest.mark.parametrize("policy", ["FP16", "BF16_POLISH"])
def test_tile_widths_orders_and_graphs_agree_bitwise(policy):
    torch = cuda_or_skip()
    rs = lib_or_fail()
    items = _batch(12, RAGGED, (1e-2, 1e-1), seed=12)
    pol = rs.Policy[policy]
    ref, ref_inf, st = _run(rs, torch, items, pol, batch_tile=128, batch_graphs=0)
    assert st == rs.Status.OK
    assert all(i.batch_tile == 128 for i in ref_inf)
    for opt in (dict(batch_tile=256, batch_graphs=0), dict(batch_tile=128, batch_graphs=1),
                dict(batch_tile=256, batch_graphs=1), dict(batch_tile=0)):
        Rb, infos, st = _run(rs, torch, items, pol, **opt)
        assert st == rs.Status.OK
        for a, b, ia, ib in zip(ref, Rb, ref_inf, infos):
            assert ia.steps_low == ib.steps_low
            assert np.array_equal(a, b), opt
        if opt.get("batch_tile", 0):
            assert all(i.batch_tile == opt["batch_tile"] for i in infos)
        else:
            assert all(i.batch_tile in (128, 256) for i in infos)


def test_fp64_batched_matches_single_bitwise_and_iterates():
    torch = cuda_or_skip()
    rs = lib_or_fail()
    items = _batch(8, (64, 96, 200, 256), (5e-2, 1e-1), seed=13)
    Rb, infos, st = _run(rs, torch, items, rs.Policy.FP64)
    assert st == rs.Status.OK
    for (sp, s), R, inf in zip(items, Rb, infos):
        R1, inf1, _ = rs.reflector(sp.H, sp.k, s, tol=1e-12, policy=rs.Policy.FP64, check=False)
        assert inf.steps_fp64 == inf1.steps_fp64
        assert np.array_equal(R, R1)
        # the oracle's naive FP64 loop takes the same number of steps
        A = oracle.shifted(sp.H, s)
        its = oracle.ns_iterates(oracle.gershgorin_alpha(A) * A, inf.steps_fp64)
        assert np.max(np.abs(its[-1] - R)) < 1e-11


def test_mixed_batch_with_fallback_entries_and_host_pointers():
    torch = cuda_or_skip()
    rs = lib_or_fail()
    items = _batch(5, (64, 128, 192), (2e-2, 1e-1), seed=14)
    big = workloads.controlled_spectrum(1100, 3, 5e-2, seed=15)  # above the grouped limit
    Hs = [sp.H for sp, _ in items] + [big.H]
    ks = [sp.k for sp, _ in items] + [big.k]
    ss = [s for _, s in items] + [0.0]
    ss[1] = None  # automatic shift: one-matrix path
    outs, infos, st = rs.reflector_batched(Hs, ks, ss, tol=1e-12, policy=rs.Policy.FP64)
    assert st == rs.Status.OK, st
    grouped = [i.batch_grouped for i in infos]
    assert grouped == [1, 0, 1, 1, 1, 0]
    for j, (sp, _) in enumerate(items):
        assert np.linalg.norm(outs[j] - _exact(sp), 2) < 1e-9
    assert np.linalg.norm(outs[-1] - _exact(big), 2) < 1e-9


def test_bad_entries_are_reported_and_the_rest_computed():
    torch = cuda_or_skip()
    rs = lib_or_fail()
    items = _batch(3, (64, 96), (5e-2, 1e-1), seed=16)
    Hs = [torch.from_numpy(sp.H).cuda() for sp, _ in items]
    ks = [sp.k for sp, _ in items]
    ks[1] = Hs[1].shape[0]  # k = d: outside [1, d-1]
    ss = [s for _, s in items]
    outs, infos, st = rs.reflector_batched(Hs, ks, ss, tol=1e-12, policy=rs.Policy.FP64)
    assert st == rs.Status.ERR_ARG
    for j in (0, 2):
        assert infos[j].cert_ok == 1
        assert np.linalg.norm(outs[j].cpu().numpy() - _exact(items[j][0]), 2) < 1e-9
    # an empty batch is a no-op
    _, _, st0 = rs.reflector_batched([], [], [], policy=rs.Policy.FP64)
    assert st0 == rs.Status.OK


def test_nonfinite_matrix_is_rejected_alone():
    torch = cuda_or_skip()
    rs = lib_or_fail()
    items = _batch(3, (64, 128), (5e-2, 1e-1), seed=17)
    Hs = [sp.H.copy() for sp, _ in items]
    Hs[2][3, 5] = np.nan
    outs, infos, st = rs.reflector_batched(Hs, [sp.k for sp, _ in items], [s for _, s in items],
                                           tol=1e-12, policy=rs.Policy.FP16_POLISH)
    assert st == rs.Status.ERR_ARG
    assert infos[0].cert_ok == 1 and infos[1].cert_ok == 1
    assert np.linalg.norm(outs[0] - _exact(items[0][0]), 2) < 2e-2


def test_full_batched_workload_certifies_and_samples_match():
    """512 matrices, d in {32, ..., 512}, k in 1..8, delta log-uniform in
    [1e-3, 1e-1], own midpoint shifts: FP16 steps + FP64 polish, every
    certificate checked, every 16th matrix compared with its exact reflector."""
    torch = cuda_or_skip()
    rs = lib_or_fail()
    items = workloads.batched_workload(512)
    Rb, infos, st = _run(rs, torch, items, rs.Policy.FP16_POLISH)
    certified = sum(i.cert_ok for i in infos)
    assert certified == 512, (certified, st)
    for j in range(0, 512, 16):
        sp, _ = items[j]
        lam = np.sort(np.abs(sp.lam - items[j][1]))
        err = np.linalg.norm(Rb[j] - _exact(sp), 2)
        # FP16 floor: a few u_fp16 over the scaled margin
        assert err <= 2e-3 / (lam[0] / np.max(np.abs(sp.lam - items[j][1]))) + 1e-6, (j, err)


@pytest.mark.parametrize("policy", ["BF16_REFINE", "FP16_REFINE"])
def test_full_batched_workload_refined_to_1e6(policy):
    """The 512-matrix workload with a REFINE policy to tol 1e-6: the matrices
    take one-matrix calls run concurrently on worker streams; every matrix is
    certified and within 1e-6 of its exact reflector (the oracle's I - 2 Q_k
    Q_k^T), and a sample equals its lone one-matrix call bit for bit."""
    torch = cuda_or_skip()
    rs = lib_or_fail()
    items = workloads.batched_workload(512)
    pol = rs.Policy[policy]
    Rb, infos, st = _run(rs, torch, items, pol, tol=1e-6)
    assert st == rs.Status.OK, st
    assert sum(i.cert_ok for i in infos) == 512
    worst = 0.0
    for (sp, s), R in zip(items, Rb):
        D = R - _exact(sp)
        worst = max(worst, float(np.abs(np.linalg.eigvalsh(0.5 * (D + D.T))).max()))
    assert worst <= 1e-6, worst
    for j in range(0, 512, 64):
        sp, s = items[j]
        R1, inf1, st1 = rs.reflector(torch.from_numpy(sp.H).cuda(), sp.k, s, tol=1e-6, policy=pol, check=False)
        torch.cuda.synchronize()
        assert st1 == rs.Status.OK
        assert np.array_equal(R1.cpu().numpy(), Rb[j]), j


def test_sharded_batch_on_one_rank_equals_the_batched_call():
    # the multi-GPU batched path at world size 1: its share is the whole batch
    # and its outputs are those of one batched call, bit for bit
    torch = cuda_or_skip()
    rs = lib_or_fail()
    from paper_2605_24840_gb300 import shard
    items = _batch(6, (64, 128, 256), (2e-2, 1e-1), seed=31)
    Hs = [torch.from_numpy(sp.H).cuda() for sp, _ in items]
    ks = [sp.k for sp, _ in items]
    ss = [s for _, s in items]
    mine, outs, reports = shard.reflectors_sharded(Hs, ks, ss, 1e-12, rs.Policy.FP16_POLISH, 0, 1)
    ref, infos, st = rs.reflector_batched(Hs, ks, ss, tol=1e-12, policy=rs.Policy.FP16_POLISH)
    assert st == rs.Status.OK and mine == list(range(6))
    for a, b in zip(outs, ref):
        assert torch.equal(a, b)
    assert [r["cert_ok"] for r in reports] == [1] * 6
