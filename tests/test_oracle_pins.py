"""Pins of the CPU oracle against facts the paper and the mathematics fix.

None of these compares the oracle with itself: each check uses a closed form,
a hand-derived golden value, an invariant, a library routine (LAPACK eigh,
numpy products) or brute force on tiny inputs.  A dropped term, a wrong sign
or index, or a transposed operand in ``oracle/`` fails at least one of them.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rand_sym(d, seed, scale=1.0):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((d, d)) * scale
    return 0.5 * (A + A.T)


def _spec_norm_sym(M):
    return float(np.abs(np.linalg.eigvalsh(0.5 * (M + M.T))).max())


# ----------------------------------------------------------------------------
# Spectral definition: Jacobi + R = I - 2 Q_k Q_k^T   (Sec. 2.1, Prop. 2.1)
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("d", [1, 2, 3, 5, 8, 17, 40])
def test_jacobi_eigenvalues_match_lapack(oracle_mod, d):
    H = _rand_sym(d, 100 + d)
    lam, V, _ = oracle_mod.jacobi_eigh(H)
    ref = np.linalg.eigvalsh(H)
    assert np.all(np.diff(lam) >= 0)
    assert np.max(np.abs(lam - ref)) <= 1e-13 * max(1.0, np.abs(ref).max())
    # orthonormal eigenvectors, H V = V diag(lam)
    assert np.max(np.abs(V.T @ V - np.eye(d))) < 1e-13
    assert np.max(np.abs(H @ V - V * lam)) < 1e-12


def test_jacobi_nonsymmetric_input_uses_symmetric_part(oracle_mod):
    rng = np.random.default_rng(3)
    A = rng.standard_normal((9, 9))
    lam, _, _ = oracle_mod.jacobi_eigh(A)
    assert np.allclose(lam, np.linalg.eigvalsh(0.5 * (A + A.T)), atol=1e-13)


def test_reflector_2x2_golden(oracle_mod):
    rows = {}
    with open(os.path.join(GOLDEN, "reflector_2x2.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            tok = line.split()
            rows[tok[0]] = [float(x) for x in tok[1:]]
    H = np.array(rows["H"]).reshape(2, 2)
    Rg = np.array(rows["R_over_inv_sqrt2"]).reshape(2, 2) / math.sqrt(2.0)
    k = int(rows["k"][0])
    R, lam = oracle_mod.reflector(H, k)
    assert np.allclose(lam, [1 - math.sqrt(2), 1 + math.sqrt(2)], atol=1e-15)
    assert np.max(np.abs(R - Rg)) < 1e-15


@pytest.mark.parametrize("seed", range(6))
def test_reflector_2x2_closed_form(oracle_mod, seed):
    # any 2x2 symmetric H: at the midpoint m = tr/2, A = H - mI has A^2 = r^2 I,
    # so sign(A) = A / r with r = sqrt(((a - c)/2)^2 + b^2)
    rng = np.random.default_rng(seed)
    a, b, c = rng.standard_normal(3)
    H = np.array([[a, b], [b, c]])
    r = math.hypot(0.5 * (a - c), b)
    R, _ = oracle_mod.reflector(H, 1)
    assert np.max(np.abs(R - (H - 0.5 * (a + c) * np.eye(2)) / r)) < 1e-14


def test_two_level_spectrum_closed_form(oracle_mod):
    # H with eigenvalues lo (k times) and hi (d-k times): sign(H - mI) = (H - mI)/r
    d, k, lo, hi = 24, 7, -0.3, 0.9
    rng = np.random.default_rng(11)
    Q = workloads.haar_orthogonal(d, rng)
    lam = np.array([lo] * k + [hi] * (d - k))
    H = (Q * lam) @ Q.T
    H = 0.5 * (H + H.T)
    m, r = 0.5 * (lo + hi), 0.5 * (hi - lo)
    R, _ = oracle_mod.reflector(H, k)
    assert np.max(np.abs(R - (H - m * np.eye(d)) / r)) < 1e-13


def test_diagonal_gives_exact_sign(oracle_mod):
    # Q = I in the proof of Prop. 2.1: R = diag(+-1) exactly
    h = np.array([0.7, -0.2, 3.0, -1.5, 0.1, 2.2, -0.9])
    H = np.diag(h)
    k = int((h < 0).sum())
    R, _ = oracle_mod.reflector(H, k)
    assert np.array_equal(R, np.diag(np.where(h < 0, -1.0, 1.0)))


@pytest.mark.parametrize("d,k", [(3, 1), (5, 2), (8, 4), (8, 7)])
def test_brute_force_tiny_against_eigh(oracle_mod, d, k):
    H = _rand_sym(d, 7 * d + k)
    R, _ = oracle_mod.reflector(H, k)
    w, V = np.linalg.eigh(H)
    P = V[:, :k] @ V[:, :k].T
    assert np.max(np.abs(R - (np.eye(d) - 2 * P))) < 1e-12
    # sign by the eigenvalue signs of H - sI with s in the gap
    s = 0.5 * (w[k - 1] + w[k])
    S = (V * np.sign(w - s)) @ V.T
    assert np.max(np.abs(R - S)) < 1e-12


@pytest.mark.parametrize("d,k", [(16, 1), (33, 5), (64, 32)])
def test_reflector_invariants(oracle_mod, d, k):
    H = _rand_sym(d, 1000 + d)
    R, lam = oracle_mod.reflector(H, k)
    assert np.array_equal(R, R.T)
    assert np.max(np.abs(R @ R - np.eye(d))) < 1e-12
    assert abs(np.trace(R) - (d - 2 * k)) < 1e-12
    # R is a spectral function of H: it commutes with H
    assert np.max(np.abs(R @ H - H @ R)) < 1e-12 * np.abs(lam).max() * d


@pytest.mark.parametrize("d,k,delta", [(48, 3, 1e-1), (96, 16, 1e-2), (128, 64, 1e-3)])
def test_jacobi_reflector_matches_construction(oracle_mod, d, k, delta):
    spec = workloads.controlled_spectrum(d, k, delta, seed=5 + d)
    R_jac, lam = oracle_mod.reflector(spec.H, k)
    R_con = oracle_mod.reflector_from_basis(spec.Q, k)
    assert np.allclose(lam, spec.lam, atol=1e-13)
    # subspace perturbation from rounding H is ~ u ||H|| / gap
    assert _spec_norm_sym(R_jac - R_con) < 1e-12 / delta


def test_reflector_eigh_route_matches_jacobi(oracle_mod):
    H = _rand_sym(50, 4)
    R1, _ = oracle_mod.reflector(H, 20)
    R2, _ = oracle_mod.reflector_eigh(H, 20)
    assert np.max(np.abs(R1 - R2)) < 1e-12


def test_reflector_entry(oracle_mod):
    spec = workloads.controlled_spectrum(20, 3, 0.1, seed=2)
    R = oracle_mod.reflector_from_basis(spec.Q, 3)
    for (i, j) in [(0, 0), (3, 7), (19, 2)]:
        assert abs(oracle_mod.reflector_entry(spec.Q, 3, i, j) - R[i, j]) < 1e-15


def test_unresolved_gap_rejected(oracle_mod):
    H = np.diag([-1.0, 0.5, 0.5, 2.0])
    with pytest.raises(ValueError):
        oracle_mod.reflector(H, 2)


# ----------------------------------------------------------------------------
# Scaling (Sec. 4.3, Cor. 3.5)
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("d", [1, 7, 64])
def test_inf_norm_and_gershgorin(oracle_mod, d):
    A = _rand_sym(d, 50 + d)
    assert abs(oracle_mod.inf_norm(A) - np.linalg.norm(A, np.inf)) < 1e-12 * d
    alpha = oracle_mod.gershgorin_alpha(A)
    rho = np.abs(np.linalg.eigvalsh(A)).max()
    assert alpha * rho <= 1.0 + 1e-15


def test_shifted_matrix(oracle_mod):
    rng = np.random.default_rng(0)
    H = rng.standard_normal((5, 5))
    A = oracle_mod.shifted(H, 0.25)
    assert np.allclose(A, 0.5 * (H + H.T) - 0.25 * np.eye(5), atol=0)


# ----------------------------------------------------------------------------
# Scalar Newton-Schulz (Eq. pm, Lemma 3.4, Prop. 3.6)
# ----------------------------------------------------------------------------
def test_scalar_golden_gamma_half(oracle_mod):
    with open(os.path.join(GOLDEN, "ns_scalar_gamma_half.txt")) as f:
        rows = [list(map(int, l.split())) for l in f if l.strip() and not l.startswith("#")]
    for m, pn, pd, en, ed in rows:
        assert float(oracle_mod.p_m(0.5, m)) == pytest.approx(pn / pd, abs=1e-16)
        assert oracle_mod.eps_m(0.5, m) == pytest.approx(en / ed, abs=1e-16)


def test_scalar_closed_form_p1_p2(oracle_mod):
    t = np.linspace(-1, 1, 101)
    p1 = 1.5 * t - 0.5 * t ** 3
    assert np.max(np.abs(oracle_mod.p_m(t, 1) - p1)) < 1e-15
    # p_2 expanded: 1/2 p1 (3 - p1^2) with p1 = (3t - t^3)/2
    p2 = 0.75 * (3 * t - t ** 3) - (3 * t - t ** 3) ** 3 / 16.0
    assert np.max(np.abs(oracle_mod.p_m(t, 2) - p2)) < 1e-15


def test_eps_recurrence_two_routes(oracle_mod):
    # eps_m by the Prop. 3.6 recurrence equals 1 - p_m(gamma) by Eq. pm; the two
    # routes round differently and the map amplifies rounding by up to 1.5x per
    # step in the near-linear phase, hence the 1e-12 allowance
    for g in [1e-3, 0.01, 0.2, 0.5, 0.9, 1.0]:
        for m in range(0, 25):
            assert oracle_mod.eps_m(g, m) == pytest.approx(1.0 - float(oracle_mod.p_m(g, m)), abs=1e-12)


def test_eps_recurrence_bound_and_exact_fraction(oracle_mod):
    # eps_{m+1} <= 3/2 eps_m^2; exact rational check of one step at eps = 3/7
    for g in [0.05, 0.3, 0.7]:
        for m in range(12):
            e, e1 = oracle_mod.eps_m(g, m), oracle_mod.eps_m(g, m + 1)
            assert e1 <= 1.5 * e * e + 1e-18
    e = Fraction(3, 7)
    e1 = e * e * (3 - e) / 2  # = 9/49 * 18/7 / 2 = 81/343
    assert e1 == Fraction(81, 343)
    assert oracle_mod.eps_m(1 - 3 / 7, 1) == pytest.approx(81 / 343, abs=1e-16)


def test_lemma_sign_preservation(oracle_mod):
    t = np.concatenate([np.linspace(-1, -1e-6, 500), np.linspace(1e-6, 1, 500)])
    for m in range(0, 30, 3):
        p = oracle_mod.p_m(t, m)
        assert np.all(np.sign(p) == np.sign(t))
        pos = p[t > 0]
        assert np.all((pos > 0) & (pos <= 1.0))
        # increasing on [0, 1] (Prop. 3.6), up to one rounding of values near 1
        assert np.all(np.diff(pos) >= -2 * np.finfo(float).eps)


def test_ns_steps_predictor(oracle_mod):
    for g in [1e-3, 1e-2, 0.3]:
        for tol in [1e-3, 1e-8, 1e-14]:
            m = oracle_mod.ns_steps(g, tol)
            assert oracle_mod.eps_m(g, m) <= tol
            assert m == 0 or oracle_mod.eps_m(g, m - 1) > tol
    # small gamma: near-linear phase p ~ 1.5^m gamma (Sec. 3.3 discussion)
    assert oracle_mod.ns_steps(1e-4, 1e-6) > oracle_mod.ns_steps(1e-2, 1e-6) + 10


# ----------------------------------------------------------------------------
# Matrix Newton-Schulz (Eq. NS) against the spectral error formula
# ----------------------------------------------------------------------------
def test_matmul_matches_numpy(oracle_mod):
    rng = np.random.default_rng(9)
    A, B = rng.standard_normal((13, 7)), rng.standard_normal((7, 11))
    assert np.max(np.abs(oracle_mod.matmul(A, B) - A @ B)) < 1e-13


def test_ns_iterates_follow_scalar_polynomials(oracle_mod):
    # Prop. 3.2: ||X_m - sign(A)||_2 = max_i |p_m(mu_i) - sign(mu_i)|, with
    # mu = alpha (lam - s); Prop. 3.6: <= eps_m(gamma)
    spec = workloads.controlled_spectrum(64, 5, 0.05, seed=21)
    s = workloads.shift_in_gap(spec, 0.5)
    A = oracle_mod.shifted(spec.H, s)
    alpha = oracle_mod.gershgorin_alpha(A)
    mu = alpha * (spec.lam - s)
    gamma = np.abs(mu).min()
    R = oracle_mod.reflector_from_basis(spec.Q, spec.k)
    its = oracle_mod.ns_iterates(alpha * A, 30)
    for m, X in enumerate(its):
        err = _spec_norm_sym(X - R)
        pred = np.abs(oracle_mod.p_m(mu, m) - np.sign(mu)).max()
        assert err == pytest.approx(pred, abs=1e-12)
        assert err <= oracle_mod.eps_m(gamma, m) + 1e-12


def test_ns_step_rows_equals_matrix_formula(oracle_mod):
    X = _rand_sym(20, 8, scale=0.1)
    Xn, r2 = oracle_mod.ns_step_rows(X, 0, 20)
    assert np.max(np.abs(Xn - 0.5 * X @ (3 * np.eye(20) - X @ X))) < 1e-14
    assert r2 == pytest.approx(np.linalg.norm(X @ X - np.eye(20)) ** 2, rel=1e-13)
    part, _ = oracle_mod.ns_step_rows(X, 5, 9)
    assert np.array_equal(part, Xn[5:9])


def test_ns_plain_method_256(oracle_mod):
    # d = 256, k = 4, midpoint shift, Gershgorin alpha, NS to 1e-12 / 80 steps
    spec = workloads.split_spectrum_config(seed=0)
    s = oracle_mod.midpoint(*spec.gap)
    A = oracle_mod.shifted(spec.H, s)
    X, steps, hist, conv = oracle_mod.newton_schulz(oracle_mod.gershgorin_alpha(A) * A, 1e-12, 80)
    assert conv and steps < 80
    assert hist[-1] < 1e-12 and hist[-2] >= 1e-12
    R, _ = oracle_mod.reflector(spec.H, spec.k)
    assert _spec_norm_sym(X - R) < 1e-12
    assert abs(np.trace(X) - (256 - 8)) < 1e-10


def test_ns_stop_rule_and_max_steps(oracle_mod):
    X0 = np.diag([0.5, -0.25, 0.75])
    X, steps, hist, conv = oracle_mod.newton_schulz(X0, 1e-30, 3)
    assert not conv and steps == 3 and len(hist) == 4
    assert np.allclose(np.diag(X), oracle_mod.p_m(np.array([0.5, -0.25, 0.75]), 3), atol=1e-16)


@pytest.mark.parametrize("theta", [0.1, 0.9])
def test_shift_invariance_of_limit(oracle_mod, theta):
    # Prop. 2.1: every admissible shift gives the same reflector
    spec = workloads.controlled_spectrum(48, 6, 0.1, seed=31)
    Rs = []
    for th in (0.5, theta):
        s = workloads.shift_in_gap(spec, th)
        A = oracle_mod.shifted(spec.H, s)
        X, _, _, conv = oracle_mod.newton_schulz(oracle_mod.gershgorin_alpha(A) * A, 1e-13, 200)
        assert conv
        Rs.append(X)
    assert _spec_norm_sym(Rs[0] - Rs[1]) < 1e-12


def test_midpoint_minimises_finite_step_error(oracle_mod):
    # Prop. 4.1 + Prop. 3.6: at fixed depth the midpoint error is the smallest
    spec = workloads.controlled_spectrum(48, 6, 0.05, seed=12)
    R = oracle_mod.reflector_from_basis(spec.Q, spec.k)
    errs = {}
    for th in (0.1, 0.5, 0.9):
        s = workloads.shift_in_gap(spec, th)
        A = oracle_mod.shifted(spec.H, s)
        X = oracle_mod.ns_iterates(oracle_mod.gershgorin_alpha(A) * A, 14)[-1]
        errs[th] = _spec_norm_sym(X - R)
    assert errs[0.5] < errs[0.1] and errs[0.5] < errs[0.9]
    assert oracle_mod.margin(workloads.shift_in_gap(spec, 0.5), *spec.gap) == pytest.approx(0.05)


def test_midpoint_and_margin(oracle_mod):
    assert oracle_mod.midpoint(-0.2, 0.6) == pytest.approx(0.2)
    ss = np.linspace(-0.19, 0.59, 79)
    m = [oracle_mod.margin(s, -0.2, 0.6) for s in ss]
    assert ss[int(np.argmax(m))] == pytest.approx(0.2, abs=0.006)
    assert max(m) <= 0.4 + 1e-15


def test_prop42_certificate(oracle_mod):
    lam_k, lam_k1 = -0.01, 0.03
    rng = np.random.default_rng(0)
    for _ in range(200):
        eps = rng.uniform(0, 0.02)
        lk = lam_k + rng.uniform(-eps, eps)
        lk1 = lam_k1 + rng.uniform(-eps, eps)
        s = rng.uniform(-0.05, 0.07)
        ok, m_hat, guaranteed = oracle_mod.admissible(s, lk, lk1, eps)
        if ok:  # certified shifts are admissible with at least the stated margin
            assert lam_k < s < lam_k1
            assert oracle_mod.margin(s, lam_k, lam_k1) >= guaranteed - 1e-15
    # estimated midpoint with eps < gap/2 is admissible (last statement of Prop. 4.2)
    eps = 0.019
    s = oracle_mod.midpoint(lam_k + eps, lam_k1 - eps)
    assert lam_k < s < lam_k1
    ok, _ = oracle_mod.reuse_admissible(0.015, 0.005, 0.004)
    assert ok
    ok, _ = oracle_mod.reuse_admissible(0.015, 0.005, 0.011)
    assert not ok


# ----------------------------------------------------------------------------
# Daleckii-Krein derivative of sign (used for the adjoint)
# ----------------------------------------------------------------------------
def test_daleckii_krein_matches_finite_differences(oracle_mod):
    spec = workloads.controlled_spectrum(24, 5, 0.2, seed=17)
    A = spec.H
    W = _rand_sym(24, 99)

    def sgn(M):
        w, V = np.linalg.eigh(M)
        return (V * np.sign(w)) @ V.T

    h = 1e-6
    fd = (sgn(A + h * W) - sgn(A - h * W)) / (2 * h)
    dk = oracle_mod.daleckii_krein(spec.lam, spec.Q, W)
    assert np.max(np.abs(fd - dk)) < 1e-7
    # the derivative of an involution anticommutes with it: S L + L S = 0
    S = sgn(A)
    assert np.max(np.abs(S @ dk + dk @ S)) < 1e-12


# ----------------------------------------------------------------------------
# Workload construction sanity (inputs the oracle and the GPU path share)
# ----------------------------------------------------------------------------
def test_allen_cahn_hessian_structure(oracle_mod):
    n, eps = 8, 0.04
    H, u = workloads.allen_cahn_hessian(n=n, eps=eps, seed=1)
    d = n * n
    assert np.array_equal(H, H.T)
    # the Laplacian part annihilates constants: H 1 = 3u^2 - 1
    assert np.allclose(H @ np.ones(d), (3 * u ** 2 - 1).ravel(), atol=1e-12)
    lam, _, _ = oracle_mod.jacobi_eigh(H)
    assert np.allclose(lam, np.linalg.eigvalsh(H), atol=1e-12 * np.abs(lam).max())
    c = eps * eps * n * n
    assert lam[-1] <= 8 * c + 2 + 1e-12 and lam[0] >= -1 - 1e-12


# ---------------------------------------------------------------------------
# Scaled Newton-Schulz steps (the step scalings of the cited stable scaling)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("l", [1e-4, 3e-3, 1e-2, 0.1, 0.3, 0.7, 0.95])
def test_scaled_step_equioscillates_on_its_interval(oracle_mod, l):
    oracle = oracle_mod
    a = oracle.scaled_ns_coeffs(l)[0]
    g = lambda x: oracle.scaled_ns_map(x, a)
    # equal values at both ends of [l, 1] and the maximum 1 inside
    assert abs(float(g(l)) - float(g(1.0))) <= 4e-15  # 3 - a^2 cancels near a^2 = 3
    xs = np.linspace(l, 1.0, 20001)
    gx = g(xs)
    assert gx.max() <= 1.0 + 4e-16
    assert abs(float(g(1.0 / a)) - 1.0) <= 4e-16 and l <= 1.0 / a <= 1.0
    # so the next interval is [g(l), 1], strictly larger at the bottom, signs kept
    assert gx.min() >= float(g(l)) - 4e-15 and float(g(l)) > l
    assert np.all(g(-xs) == -gx)


def test_scaled_steps_reach_one_and_beat_the_plain_steps(oracle_mod):
    oracle = oracle_mod
    for l0 in (1e-3, 1e-2, 0.1):
        c = oracle.scaled_ns_coeffs(l0)
        l = l0
        for a in c:
            l = float(oracle.scaled_ns_map(l, a))
        assert 1.0 - l <= 1e-13
        # the plain recurrence needs more steps for the same bottom end
        plain = oracle.ns_steps(l0, 1e-13)
        assert len(c) < plain
        assert all(1.0 <= a <= math.sqrt(3.0) for a in c)
    assert oracle.scaled_ns_coeffs(1.0) == []  # an involution needs no scaled step


def test_scaled_first_step_normalises_by_the_upper_bound(oracle_mod):
    oracle = oracle_mod
    # with |eigenvalues| up to u0 > 1 the first factor absorbs 1/u0 and no sign flips
    l0, u0 = 2e-2, 1.05
    c = oracle.scaled_ns_coeffs(l0, u0)
    xs = np.linspace(l0, u0, 5001)
    y = oracle.scaled_ns_map(xs, c[0])
    assert np.all(y > 0) and y.max() <= 1.0 + 1e-15
    # without the normalisation the same interval would flip the top eigenvalues
    bad = oracle.scaled_ns_map(xs, oracle.scaled_ns_coeffs(l0)[0])
    assert bad.min() < 0


def test_scaled_iteration_on_a_diagonal_is_the_scalar_map(oracle_mod):
    oracle = oracle_mod
    d = np.array([-0.9, -0.02, 0.015, 0.4, 1.0])
    c = oracle.scaled_ns_coeffs(0.015)
    its = oracle.scaled_ns_iterates(np.diag(d), c, len(c) + 2)
    x = d.copy()
    for m in range(len(c) + 2):
        x = oracle.scaled_ns_map(x, c[m] if m < len(c) else 1.0)
        np.testing.assert_allclose(np.diag(its[m + 1]), x, rtol=0, atol=2e-15)
        assert np.count_nonzero(its[m + 1] - np.diag(np.diag(its[m + 1]))) == 0
    np.testing.assert_allclose(np.diag(its[-1]), np.sign(d), atol=1e-14)


def test_scaled_iteration_reaches_the_reflector_brute_force(oracle_mod):
    oracle = oracle_mod
    rng = np.random.default_rng(11)
    for d in (4, 6, 8):
        Q, _ = np.linalg.qr(rng.standard_normal((d, d)))
        lam = np.sort(np.concatenate([rng.uniform(-1, -0.05, 2), rng.uniform(0.05, 1, d - 2)]))
        H = (Q * lam) @ Q.T
        H = 0.5 * (H + H.T)
        A = oracle.shifted(H, 0.0)
        alpha = oracle.gershgorin_alpha(A)
        l0 = alpha * np.min(np.abs(lam))
        c = oracle.scaled_ns_coeffs(l0)
        X = oracle.scaled_ns_iterates(alpha * A, c, len(c) + 3)[-1]
        w, V = np.linalg.eigh(H)
        R = V @ np.diag(np.sign(w)) @ V.T
        assert np.max(np.abs(X - R)) < 1e-13


# ---------------------------------------------------------------------------
# commutator error bound of a refined reflector (Sylvester argument)
# ---------------------------------------------------------------------------
def _expm_antisym(K):
    # exp of an antisymmetric matrix through the eigen-decomposition of the
    # Hermitian matrix iK (an orthogonal result)
    w, U = np.linalg.eigh(1j * K)
    return np.real((U * np.exp(-1j * w)) @ U.conj().T)


@pytest.mark.parametrize("seed", range(6))
def test_commutator_bound_holds_brute_force(oracle_mod, seed):
    # random spectra with a known margin, reflectors rotated away from sign(A)
    # (exact involutions) and scaled off the involution set: the true error
    # never exceeds the bound
    rng = np.random.default_rng(100 + seed)
    d = 24
    mu = 10.0 ** rng.uniform(-3, -1)
    k = int(rng.integers(1, d))
    lam = np.concatenate([-mu - rng.exponential(0.5, k), mu + rng.exponential(0.5, d - k)])
    lam[0], lam[-1] = -mu, mu  # the margin is attained on both sides
    V, _ = np.linalg.qr(rng.standard_normal((d, d)))
    A = (V * lam) @ V.T
    S = (V * np.sign(lam)) @ V.T
    for eps in (1e-8, 1e-5, 1e-3):
        K = rng.standard_normal((d, d))
        Q = _expm_antisym(eps * (K - K.T))
        R = Q @ S @ Q.T
        eta = rng.uniform(-eps, eps, d)
        R = R + eps * 0.1 * ((V * eta) @ V.T)  # leaves the involution set
        R = 0.5 * (R + R.T)
        comm = np.linalg.norm(R @ A - A @ R, 2)
        rho = np.linalg.norm(R @ R - np.eye(d), 2)
        err = np.linalg.norm(R - S, 2)
        b = oracle_mod.commutator_error_bound(comm, mu, rho)
        assert err <= b * (1 + 1e-9) + 1e-14, (eps, err, b)


def test_commutator_bound_is_tight_on_a_two_by_two_rotation(oracle_mod):
    # A = diag(-mu, mu), R = the reflector S rotated by theta: ||R - S|| =
    # 2 sin theta and ||R A - A R|| = 2 mu sin 2 theta, so the bound is
    # sin 2 theta + O(theta^2): the ratio tends to 1 (a bound with mu in place
    # of 2 mu would tend to 2)
    mu = 0.3
    A = np.diag([-mu, mu])
    S = np.diag([-1.0, 1.0])
    for th in (1e-3, 1e-5):
        c, s = math.cos(th), math.sin(th)
        Q = np.array([[c, -s], [s, c]])
        R = Q @ S @ Q.T
        comm = np.linalg.norm(R @ A - A @ R, 2)
        assert comm == pytest.approx(2 * mu * math.sin(2 * th), rel=1e-9)
        err = np.linalg.norm(R - S, 2)
        b = oracle_mod.commutator_error_bound(comm, mu, 0.0)
        assert err <= b and b / err < 1 + 2 * th


def test_commutator_bound_residual_term_is_tight_for_commuting_errors(oracle_mod):
    # R = S (1 + eta) commutes with A: C = 0, ||R - S|| = eta and ||R^2 - I|| =
    # 2 eta + eta^2, so the bound is eta + O(eta^2)
    mu = 0.1
    for eta in (1e-9, 1e-6):
        S = np.diag([-1.0, -1.0, 1.0])
        R = S * (1 + eta)
        rho = np.linalg.norm(R @ R - np.eye(3), 2)
        b = oracle_mod.commutator_error_bound(0.0, mu, rho)
        assert eta * (1 - 1e-6) <= b <= eta * (1 + 4 * eta) + 1e-15
    assert oracle_mod.commutator_error_bound(1.0, 1.0, 0.0) == math.inf


# ---------------------------------------------------------------------------
# quintic Newton-Schulz filter (the higher-degree engine)
# ---------------------------------------------------------------------------
def test_ns5_map_closed_forms(oracle_mod):
    x = np.linspace(-1.2, 1.2, 2401)
    q = oracle_mod.ns5_map(x)
    # odd, fixes 0 and +-1, derivative 15/8 (1 - x^2)^2 by central differences
    assert np.allclose(q, -oracle_mod.ns5_map(-x), atol=1e-15)
    assert oracle_mod.ns5_map(1.0) == 1.0 and oracle_mod.ns5_map(-1.0) == -1.0 and oracle_mod.ns5_map(0.0) == 0.0
    h = 1e-6
    dq = (oracle_mod.ns5_map(x + h) - oracle_mod.ns5_map(x - h)) / (2 * h)
    assert np.allclose(dq, 15.0 / 8.0 * (1 - x * x) ** 2, atol=1e-8)
    # cubic convergence at 1: 1 - q(1 - e) = 5/2 e^3 + O(e^4)
    for e in (1e-2, 1e-3):
        assert (1.0 - oracle_mod.ns5_map(1.0 - e)) / e ** 3 == pytest.approx(2.5, rel=10 * e)
    # the update form X + 1/2 X W, W = E + 3/4 E^2, E = 1 - x^2 (the GPU's form)
    E = 1.0 - x * x
    assert np.allclose(x + 0.5 * x * (E + 0.75 * E * E), q, atol=1e-14)


def test_ns5_iterates_on_a_diagonal_are_the_scalar_map(oracle_mod):
    d = np.array([-0.9, -0.3, -0.02, 0.05, 0.4, 1.0])
    it = oracle_mod.ns5_iterates(np.diag(d), 4)
    y = d.copy()
    for m in range(1, 5):
        y = oracle_mod.ns5_map(y)
        assert np.allclose(np.diag(it[m]), y, atol=1e-15)
        assert np.allclose(it[m] - np.diag(np.diag(it[m])), 0.0)


def test_ns5_iterates_reach_the_reflector_brute_force(oracle_mod):
    rng = np.random.default_rng(21)
    for d, k in ((6, 2), (9, 4)):
        Q, _ = np.linalg.qr(rng.standard_normal((d, d)))
        lam = np.concatenate([-rng.uniform(0.05, 1.0, k), rng.uniform(0.05, 1.0, d - k)])
        H = (Q * lam) @ Q.T
        X0 = H / np.abs(lam).max()
        it = oracle_mod.ns5_iterates(X0, 14)
        R = np.eye(d) - 2 * Q[:, :k] @ Q[:, :k].T
        assert np.abs(it[-1] - R).max() < 1e-12
        # fewer steps than Eq. NS from the same start
        m3 = next(m for m, X in enumerate(oracle_mod.ns_iterates(X0, 40)) if np.abs(X - R).max() < 1e-10)
        m5 = next(m for m, X in enumerate(it) if np.abs(X - R).max() < 1e-10)
        assert m5 < m3
