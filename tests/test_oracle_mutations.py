"""Planted mistakes in the oracle must fail its pins.

Each case below plants one plausible slip in the oracle: a sign, a factor, a
transposed index, a dropped term or an off-by-one. The slip goes either into
a copy of the C source, which is compiled into a temporary library, or into
one Python function, which is replaced for the duration of the test. Each
case then runs the pins of ``test_oracle_pins.py`` until one of them fails.

The oracle in the tree is never modified. A baseline case runs the same
harness on the unmodified oracle, and every pin must pass there.
"""
import itertools
import math

import numpy as np
import pytest

import test_oracle_pins as pins

# pins that take a second or more run last: most slips fail a fast pin first
_SLOW = ("test_ns_plain_method_256", "test_ns5_iterates_reach_the_reflector_brute_force")


def _pin_cases():
    cases = []
    for name, fn in list(vars(pins).items()):
        if not (name.startswith("test_") and callable(fn)):
            continue
        grids = []
        for mark in getattr(fn, "pytestmark", []):
            if mark.name != "parametrize":
                continue
            names = [s.strip() for s in mark.args[0].split(",")]
            grid = []
            for vals in mark.args[1]:
                vals = vals if len(names) > 1 else (vals,)
                grid.append(dict(zip(names, vals)))
            grids.append(grid)
        for combo in itertools.product(*grids) if grids else [()]:
            kw = {}
            for part in combo:
                kw.update(part)
            cases.append((name, fn, kw))
    cases.sort(key=lambda c: c[0] in _SLOW)
    return cases


CASES = _pin_cases()
CAUGHT = (AssertionError, RuntimeError, ValueError, pytest.fail.Exception)


def _first_failing_pin(oracle):
    for name, fn, kw in CASES:
        try:
            fn(oracle, **kw)
        except CAUGHT:
            return name
    return None


def _plant_c(monkeypatch, tmp_path, oracle, old, new):
    with open(oracle._SRC) as f:
        src = f.read()
    assert src.count(old) == 1, old
    path = tmp_path / "rsign_oracle_planted.c"
    path.write_text(src.replace(old, new))
    monkeypatch.setattr(oracle, "_SRC", str(path))
    monkeypatch.setattr(oracle, "_BUILD", str(tmp_path / "build"))
    monkeypatch.setattr(oracle, "_LIB", str(tmp_path / "build" / "liboracle.so"))
    monkeypatch.setattr(oracle, "_lib", None)


def test_unmodified_oracle_passes_every_pin(oracle_mod):
    assert len(CASES) > 60
    assert _first_failing_pin(oracle_mod) is None


# (what the slip is, text in rsign_oracle.c, its replacement)
C_SLIPS = [
    ("Jacobi: rotation tangent with the wrong sign",
     "if (theta < 0.0) t = -t;", "if (theta > 0.0) t = -t;"),
    ("Jacobi: theta from the transposed diagonal difference",
     "const double theta = (aqq - app) / (2.0 * apq);", "const double theta = (app - aqq) / (2.0 * apq);"),
    ("Jacobi: accumulated rotation with a flipped sign",
     "W[r * d + p] = c * wrp - s * wrq;", "W[r * d + p] = c * wrp + s * wrq;"),
    ("Jacobi: eigenvectors stored as rows instead of columns",
     "V[r * d + i] = W[r * d + ord[i]];", "V[i * d + r] = W[r * d + ord[i]];"),
    ("Jacobi: eigenvalues sorted descending",
     "A[ord[j] * d + ord[j]] > A[key * d + key]", "A[ord[j] * d + ord[j]] < A[key * d + key]"),
    ("reflector: I + 2 Q_k Q_k^T",
     "R[i * d + j] = (i == j ? 1.0 : 0.0) - 2.0 * p;", "R[i * d + j] = (i == j ? 1.0 : 0.0) + 2.0 * p;"),
    ("reflector: transposed operand Q_k Q^T_k -> Q_k Q_k (rows for columns)",
     "p += V[i * d + l] * V[j * d + l];", "p += V[i * d + l] * V[l * d + j];"),
    ("reflector: k + 1 columns (off by one)",
     "for (int64_t l = 0; l < k; ++l)", "for (int64_t l = 0; l <= k; ++l)"),
    ("infinity norm without the absolute value",
     "s += fabs(A[i * d + j]);", "s += A[i * d + j];"),
    ("Newton-Schulz: factor 3 replaced by 2",
     "Xn[i * d + j] = 0.5 * (3.0 * X[i * d + j] - T[j]);", "Xn[i * d + j] = 0.5 * (2.0 * X[i * d + j] - T[j]);"),
    ("Newton-Schulz: residual without the identity",
     "const double e = Z[j] - (i == j ? 1.0 : 0.0);", "const double e = Z[j];"),
    ("Newton-Schulz: X^2 X replaced by X^2 X^2 (second product on Z)",
     "const double a = Z[k];\n      for (int64_t j = 0; j < d; ++j) T[j] += a * X[k * d + j];",
     "const double a = Z[k];\n      for (int64_t j = 0; j < d; ++j) T[j] += a * Z[j] * X[k * d + j];"),
    ("Newton-Schulz: one update too few at the step limit",
     "if (m == max_steps) break;", "if (m == max_steps - 1) break;"),
    ("product: transposed B operand",
     "C[i * m + j] += a * B[k * m + j];", "C[i * m + j] += a * B[j * m + k];"),
    ("Daleckii-Krein: divided difference with the wrong sign",
     "(si - sj) / (mu[i] - mu[j]);", "(si - sj) / (mu[j] - mu[i]);"),
    ("Daleckii-Krein: V^T W V formed as V W V",
     "rsign_oracle_matmul(d, d, d, Vt, W, T); /* V^T W */", "rsign_oracle_matmul(d, d, d, V, W, T); /* V^T W */"),
]


@pytest.mark.parametrize("what,old,new", C_SLIPS, ids=[c[0] for c in C_SLIPS])
def test_planted_c_slip_fails_a_pin(oracle_mod, monkeypatch, tmp_path, what, old, new):
    _plant_c(monkeypatch, tmp_path, oracle_mod, old, new)
    assert _first_failing_pin(oracle_mod) is not None, what


# Python-level slips: (what, attribute, replacement built from the oracle module)
def _py_slips():
    def p_m_dropped_square(t, m):
        p = np.asarray(t, dtype=np.float64)
        for _ in range(m):
            p = 0.5 * p * (3.0 - p)
        return p

    def eps_m_dropped_factor(gamma, m):
        e = 1.0 - float(gamma)
        for _ in range(m):
            e = 0.5 * e * e
        return e

    def eps_m_wrong_start(gamma, m):
        e = float(gamma)
        for _ in range(m):
            e = 0.5 * e * e * (3.0 - e)
        return e

    def midpoint_wrong_sign(lam_k, lam_k1):
        return 0.5 * (lam_k1 - lam_k)

    def margin_max(s, lam_k, lam_k1):
        return max(s - lam_k, lam_k1 - s)

    def admissible_wrong_guarantee(s, lk, lk1, eps):
        m_hat = min(s - lk, lk1 - s)
        return (m_hat > eps), m_hat, m_hat + eps

    def reuse_ignores_eps(m_hat, eps, drift):
        return (drift < m_hat), m_hat - drift

    def shifted_plus(H, s):
        A = 0.5 * (H + H.T)
        A[np.diag_indices_from(A)] += s
        return A

    def shifted_no_sym(H, s):
        A = np.array(H, dtype=np.float64)
        A[np.diag_indices_from(A)] -= s
        return A

    def gershgorin_max_entry(A):
        return 1.0 / float(np.abs(A).max())

    def bound_margin_not_doubled(comm2, margin_, rho=0.0):
        c = comm2 / margin_ + 0.5 * rho
        return math.inf if not (2.0 * c < 1.0) else 2.0 * c / (1.0 + math.sqrt(1.0 - 2.0 * c))

    def bound_without_rho(comm2, margin_, rho=0.0):
        c = comm2 / (2.0 * margin_)
        return math.inf if not (2.0 * c < 1.0) else 2.0 * c / (1.0 + math.sqrt(1.0 - 2.0 * c))

    def scaled_coeffs_dropped_term(l0, u0=1.0, tol=1e-15, max_steps=200):
        l = float(l0) / float(u0)
        out = []
        for m in range(max_steps):
            a = math.sqrt(3.0 / (1.0 + l * l))
            if abs(a - 1.0) <= tol:
                break
            out.append(a / u0 if m == 0 else a)
            l = 0.5 * a * l * (3.0 - a * a * l * l)
        return out

    def scaled_map_unsquared(x, a):
        x = np.asarray(x, dtype=np.float64)
        return 0.5 * a * x * (3.0 - a * x * x)

    def ns5_wrong_coefficient(x):
        x = np.asarray(x, dtype=np.float64)
        x2 = x * x
        return x * (15.0 - 9.0 * x2 + 3.0 * x2 * x2) / 8.0

    def entry_plus(Q, k, i, j):
        return (1.0 if i == j else 0.0) + 2.0 * float(np.dot(Q[i, :k], Q[j, :k]))

    def ns_steps_one_short(gamma, tol, max_steps=1000):
        e, m = 1.0 - float(gamma), 0
        while 0.5 * e * e * (3.0 - e) > tol:
            e = 0.5 * e * e * (3.0 - e)
            m += 1
        return m

    return [
        ("p_m without the square", "p_m", p_m_dropped_square),
        ("eps recurrence without the factor (3 - eps)", "eps_m", eps_m_dropped_factor),
        ("eps recurrence started at gamma", "eps_m", eps_m_wrong_start),
        ("midpoint with a wrong sign", "midpoint", midpoint_wrong_sign),
        ("margin as the max of the two distances", "margin", margin_max),
        ("Prop. 4.2 guarantee m_hat + eps", "admissible", admissible_wrong_guarantee),
        ("reuse rule without eps", "reuse_admissible", reuse_ignores_eps),
        ("A = H + sI", "shifted", shifted_plus),
        ("A without the symmetric part", "shifted", shifted_no_sym),
        ("alpha from the largest entry", "gershgorin_alpha", gershgorin_max_entry),
        ("commutator bound with mu for 2 mu", "commutator_error_bound", bound_margin_not_doubled),
        ("commutator bound without the residual term", "commutator_error_bound", bound_without_rho),
        ("scaled-step coefficient without the l term", "scaled_ns_coeffs", scaled_coeffs_dropped_term),
        ("scaled step with a for a^2", "scaled_ns_map", scaled_map_unsquared),
        ("quintic filter with 9 for 10", "ns5_map", ns5_wrong_coefficient),
        ("reflector entry I + 2 Q Q^T", "reflector_entry", entry_plus),
        ("step predictor one short", "ns_steps", ns_steps_one_short),
    ]


PY_SLIPS = _py_slips()


@pytest.mark.parametrize("what,attr,fn", PY_SLIPS, ids=[c[0] for c in PY_SLIPS])
def test_planted_python_slip_fails_a_pin(oracle_mod, monkeypatch, what, attr, fn):
    assert hasattr(oracle_mod, attr)
    monkeypatch.setattr(oracle_mod, attr, fn)
    assert _first_failing_pin(oracle_mod) is not None, what
