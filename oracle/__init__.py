"""CPU oracle for the shifted matrix-sign reflector (FP64, plain and slow).

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this package.  It shares no code with
the CUDA library ``paper_2605_24840_gb300`` and never imports it.

The heavy loops (cyclic Jacobi, naive Newton-Schulz, dense products) live in
``rsign_oracle.c`` (plain C, FP64, OpenMP over rows); this module loads it
with ctypes and adds the scalar pieces of the method, each citing the
passage of the paper it restates:

  * R_k = I - 2 Q_k Q_k^T from an eigen-decomposition (Eq. Pk / Rk_intro,
    Prop. 2.1 sign(H - sI) = I - 2 P_k for s in (lam_k, lam_{k+1}));
  * the scalar Newton-Schulz polynomials p_m (Eq. pm) and the error
    recurrence eps_{m+1} = 1/2 eps_m^2 (3 - eps_m) (Prop. 3.6);
  * the midpoint shift (Prop. 4.1) and the inexact-shift admissibility
    margin (Prop. 4.2);
  * alpha = 1/||A||_inf (Sec. 4.3 scaling discussion);
  * the Daleckii-Krein derivative of sign (used to check the adjoint);
  * the commutator error bound of a refined reflector (Sylvester argument);
  * the quintic Newton-Schulz filter and its iterates (Sec. 5.4 reading).

Pins: every function here is checked in ``tests/test_oracle_pins.py`` against
closed forms, library routines, brute force on tiny inputs and hand-derived
golden values (``tests/golden``).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rsign_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)


def build(force: bool = False) -> str:
    """Compile rsign_oracle.c into oracle/_build/liboracle.so with gcc."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".%d.tmp" % os.getpid()
        cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-std=c11", "-o", tmp, _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i64, c_int, c_double = ctypes.c_int64, ctypes.c_int, ctypes.c_double
            lib.rsign_oracle_jacobi.argtypes = [i64, _dp, _dp, _dp, c_int, c_double]
            lib.rsign_oracle_jacobi.restype = c_int
            lib.rsign_oracle_reflector_from_basis.argtypes = [i64, i64, _dp, _dp]
            lib.rsign_oracle_inf_norm.argtypes = [i64, _dp]
            lib.rsign_oracle_inf_norm.restype = c_double
            lib.rsign_oracle_ns_step_rows.argtypes = [i64, _dp, _dp, i64, i64]
            lib.rsign_oracle_ns_step_rows.restype = c_double
            lib.rsign_oracle_newton_schulz.argtypes = [i64, _dp, _dp, c_double, c_int, _dp,
                                                       ctypes.POINTER(c_int)]
            lib.rsign_oracle_newton_schulz.restype = c_int
            lib.rsign_oracle_matmul.argtypes = [i64, i64, i64, _dp, _dp, _dp]
            lib.rsign_oracle_daleckii_krein.argtypes = [i64, _dp, _dp, _dp, _dp]
            lib.rsign_oracle_num_threads.restype = c_int
            _lib = lib
    return _lib


def _c(a: np.ndarray) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _p(a: np.ndarray):
    return a.ctypes.data_as(_dp)


def num_threads() -> int:
    """OpenMP threads the oracle's parallel loops use."""
    return int(_load().rsign_oracle_num_threads())


# --------------------------------------------------------------------------
# Spectral definition (Sec. 2.1, Prop. 2.1)
# --------------------------------------------------------------------------
def jacobi_eigh(H: np.ndarray, max_sweeps: int = 30, tol: float = 1e-14):
    """Cyclic-Jacobi eigen-decomposition of sym(H); returns (lam ascending, V, sweeps)."""
    H = _c(H)
    d = H.shape[0]
    lam = np.empty(d)
    V = np.empty((d, d))
    sweeps = _load().rsign_oracle_jacobi(d, _p(H), _p(lam), _p(V), max_sweeps, tol)
    if sweeps < 0:
        raise RuntimeError("Jacobi did not converge in %d sweeps" % max_sweeps)
    return lam, V, sweeps


def reflector_from_basis(V: np.ndarray, k: int) -> np.ndarray:
    """R_k = I - 2 V_k V_k^T with V_k the first k columns (Eq. Pk, Eq. Rk_intro)."""
    V = _c(V)
    d = V.shape[0]
    R = np.empty((d, d))
    _load().rsign_oracle_reflector_from_basis(d, int(k), _p(V), _p(R))
    return R


def gap_resolved(lam: np.ndarray, k: int, H_scale: float) -> bool:
    """The reflector is defined only for lam_k < lam_{k+1} (Prop. 2.1); a gap
    below 64 u ||H|| is not resolved in FP64 and is reported as such."""
    return float(lam[k] - lam[k - 1]) > 64.0 * np.finfo(np.float64).eps * H_scale


def reflector(H: np.ndarray, k: int):
    """Exact reflector sign(H - sI) = I - 2 P_k of sym(H) via cyclic Jacobi.

    Returns (R, lam).  Raises if the gap (lam_k, lam_{k+1}) is not resolved.
    """
    lam, V, _ = jacobi_eigh(H)
    if not gap_resolved(lam, k, float(np.abs(lam).max())):
        raise ValueError("gap (lam_k, lam_k+1) not resolved in FP64")
    return reflector_from_basis(V, k), lam


def reflector_eigh(H: np.ndarray, k: int):
    """Same definition with LAPACK ``eigh`` as the eigen-decomposition step.

    Used where Jacobi is too slow (d in the thousands); pinned against
    ``reflector`` on small inputs.  Returns (R, lam).
    """
    Hs = 0.5 * (H + H.T)
    lam, V = np.linalg.eigh(Hs)
    if not gap_resolved(lam, k, float(np.abs(lam).max())):
        raise ValueError("gap (lam_k, lam_k+1) not resolved in FP64")
    Vk = V[:, :k]
    R = np.eye(H.shape[0]) - 2.0 * (Vk @ Vk.T)
    return 0.5 * (R + R.T), lam


def reflector_entry(Q: np.ndarray, k: int, i: int, j: int) -> float:
    """One entry of R_k = I - 2 Q_k Q_k^T, from an eigenbasis known by construction."""
    return (1.0 if i == j else 0.0) - 2.0 * float(np.dot(Q[i, :k], Q[j, :k]))


# --------------------------------------------------------------------------
# Scaling (Sec. 4.3): alpha = 1/||A||_inf, the Gershgorin bound on rho(A)
# --------------------------------------------------------------------------
def inf_norm(A: np.ndarray) -> float:
    A = _c(A)
    return float(_load().rsign_oracle_inf_norm(A.shape[0], _p(A)))


def shifted(H: np.ndarray, s: float) -> np.ndarray:
    """A = sym(H) - s I, the matrix whose sign is the reflector (Prop. 2.1)."""
    A = 0.5 * (H + H.T)
    A[np.diag_indices_from(A)] -= s
    return A


def gershgorin_alpha(A: np.ndarray) -> float:
    """alpha = 1/||A||_inf <= 1/rho(A) (Cor. 3.5 admits any alpha <= 1/rho)."""
    return 1.0 / inf_norm(A)


# --------------------------------------------------------------------------
# Newton-Schulz (Eq. NS) and its scalar polynomials (Eq. pm, Prop. 3.6)
# --------------------------------------------------------------------------
def newton_schulz(X0: np.ndarray, tol: float, max_steps: int):
    """Naive FP64 NS from X0 = alpha A.

    Returns (X, steps, resid_hist, converged): steps = number of updates
    applied, resid_hist[m] = ||X_m^2 - I||_F for m = 0..steps.
    """
    X0 = _c(X0)
    d = X0.shape[0]
    X = np.empty_like(X0)
    hist = np.full(max_steps + 1, np.nan)
    conv = ctypes.c_int(0)
    m = _load().rsign_oracle_newton_schulz(d, _p(X0), _p(X), float(tol), int(max_steps), _p(hist),
                                            ctypes.byref(conv))
    return X, int(m), hist[: m + 1], bool(conv.value)


def ns_step_rows(X: np.ndarray, row0: int, row1: int):
    """Rows [row0, row1) of one NS update; returns (Xn rows, residual^2 contribution)."""
    X = _c(X)
    d = X.shape[0]
    Xn = np.zeros_like(X)
    r2 = _load().rsign_oracle_ns_step_rows(d, _p(X), _p(Xn), int(row0), int(row1))
    return Xn[row0:row1], float(r2)


def ns_iterates(X0: np.ndarray, steps: int):
    """X_0..X_steps of Eq. NS (no stopping test); a list of FP64 arrays."""
    out = [_c(X0).copy()]
    X = out[0]
    for _ in range(steps):
        Xn, _ = ns_step_rows(X, 0, X.shape[0])
        X = Xn
        out.append(X)
    return out


def p_m(t, m: int):
    """Scalar NS polynomial p_m(t): p_0 = t, p_{m+1} = 1/2 p_m (3 - p_m^2) (Eq. pm)."""
    p = np.asarray(t, dtype=np.float64)
    for _ in range(m):
        p = 0.5 * p * (3.0 - p * p)
    return p


def eps_m(gamma: float, m: int) -> float:
    """eps_m(gamma) = 1 - p_m(gamma) through the recurrence of Prop. 3.6:
    eps_0 = 1 - gamma, eps_{m+1} = 1/2 eps_m^2 (3 - eps_m)."""
    e = 1.0 - float(gamma)
    for _ in range(m):
        e = 0.5 * e * e * (3.0 - e)
    return e


def ns_steps(gamma: float, tol: float, max_steps: int = 1000) -> int:
    """Smallest m with eps_m(gamma) <= tol (the depth condition of Sec. 3.3 discussion)."""
    e = 1.0 - float(gamma)
    m = 0
    while e > tol:
        if m >= max_steps:
            return -1
        e = 0.5 * e * e * (3.0 - e)
        m += 1
    return m


def scaled_ns_coeffs(l0: float, u0: float = 1.0, tol: float = 1e-15, max_steps: int = 200):
    """Step scalings of the scaled Newton-Schulz sign iteration (Chen and Chow's
    stable scaling, cited by the paper for GPU implementations, Sec. 3.5):
    for a spectrum in [-1, -l] U [l, 1] the step X <- 1/2 a X (3I - a^2 X^2)
    with a = sqrt(3 / (1 + l + l^2)) maps [l, 1] into [l', 1],
    l' = 1/2 a l (3 - a^2 l^2) (the scaled cubic takes equal values at l and 1
    and its maximum 1 at 1/a).  u0 >= the largest |eigenvalue| of X_0: the
    interval is first normalised to [l0/u0, 1] and the first factor divided
    by u0.  Returns [a_0, a_1, ...] up to the first a with |a - 1| <= tol
    (after which the plain step, a = 1, is the scaled one)."""
    l = float(l0) / float(u0)
    out = []
    for m in range(max_steps):
        a = math.sqrt(3.0 / (1.0 + l + l * l))
        if abs(a - 1.0) <= tol:
            break
        out.append(a / u0 if m == 0 else a)
        l = 0.5 * a * l * (3.0 - a * a * l * l)
    return out


def scaled_ns_map(x, a: float):
    """The scalar scaled step g(x) = 1/2 a x (3 - a^2 x^2)."""
    x = np.asarray(x, dtype=np.float64)
    return 0.5 * a * x * (3.0 - a * a * x * x)


def ns5_map(x):
    """The quintic odd filter q(x) = x (15 - 10 x^2 + 3 x^4) / 8: the degree-5
    member of the Newton-Schulz family (a higher-degree odd polynomial filter
    of the kind Sec. 5.4 points to).  q(1) = 1, q'(x) = 15/8 (1 - x^2)^2, so
    q is increasing on [0, 1], fixes +-1 with q'(1) = q''(1) = 0 (cubic
    convergence), and grows small x by 15/8."""
    x = np.asarray(x, dtype=np.float64)
    x2 = x * x
    return x * (15.0 - 10.0 * x2 + 3.0 * x2 * x2) / 8.0


def ns5_iterates(X0: np.ndarray, steps: int):
    """X_0..X_steps of X <- 1/8 X (15I - 10X^2 + 3X^4), formed as written
    (matrix products by the oracle's plain triple loop)."""
    X = _c(X0).copy()
    out = [X]
    d = X.shape[0]
    eye = np.eye(d)
    for _ in range(steps):
        X2 = matmul(X, X)
        X4 = matmul(X2, X2)
        X = matmul(X, 15.0 * eye - 10.0 * X2 + 3.0 * X4) / 8.0
        out.append(X)
    return out


def scaled_ns_iterates(X0: np.ndarray, coeffs, steps: int):
    """X_0..X_steps of the scaled iteration: step m applies the plain map of
    Eq. NS to a_m X_m (a_m = 1 once the coefficient list is exhausted)."""
    out = [_c(X0).copy()]
    X = out[0]
    for m in range(steps):
        a = coeffs[m] if m < len(coeffs) else 1.0
        Xn, _ = ns_step_rows(a * X, 0, X.shape[0])
        X = Xn
        out.append(X)
    return out


# --------------------------------------------------------------------------
# Shift placement (Prop. 4.1, Prop. 4.2)
# --------------------------------------------------------------------------
def midpoint(lam_k: float, lam_k1: float) -> float:
    """s* = (lam_k + lam_{k+1})/2, the maximiser of delta(s) (Prop. 4.1)."""
    return 0.5 * (lam_k + lam_k1)


def margin(s: float, lam_k: float, lam_k1: float) -> float:
    """delta(s) = min(s - lam_k, lam_{k+1} - s) (Prop. 4.1)."""
    return min(s - lam_k, lam_k1 - s)


def admissible(s: float, lam_k_hat: float, lam_k1_hat: float, eps: float):
    """Prop. 4.2: with endpoint estimates accurate to eps, s is admissible if the
    estimated margin m_hat exceeds eps; the true margin is then >= m_hat - eps.
    Returns (certified, m_hat, guaranteed margin)."""
    m_hat = margin(s, lam_k_hat, lam_k1_hat)
    return (m_hat > eps), m_hat, m_hat - eps


def reuse_admissible(m_hat: float, eps: float, drift: float):
    """Prop. 4.2 reuse rule: a shift stays admissible at the next iterate when the
    endpoint drift (bounded by ||H_{n+1} - H_n||_2 via Weyl) is below m_hat - eps.
    Returns (certified, guaranteed margin)."""
    return (drift < m_hat - eps), m_hat - eps - drift


def commutator_error_bound(comm2: float, margin_: float, rho: float = 0.0) -> float:
    """A-posteriori bound of ||R - sign(A)||_2 for a symmetric R from the
    commutator C = R A - A R, the margin mu = min |lam_i(A)| and rho = ||R^2 - I||_2.

    Not printed in the paper; it is the standard Sylvester-equation argument
    (Bhatia-Davis-McIntosh) for the refined reflector of the commutator
    refinement.  With S = sign(A) and F = R - S, split F in the eigenbasis of A
    into the blocks between the negative and positive eigenspaces (F_off) and
    within them (F_same).  F_off solves F_off A_+ - A_- F_off = C_off with
    A_- <= -mu and A_+ >= mu, so ||F_off|| <= ||C||/(2 mu); R^2 - I = S F + F S
    + F^2 gives ||F_same|| <= (rho + ||F||^2)/2.  Hence f = ||F|| satisfies
    f <= c + f^2/2, c = ||C||/(2 mu) + rho/2, and on the branch connected to S
    (f < 1): f <= 1 - sqrt(1 - 2c).  Returns inf when 2c >= 1."""
    c = comm2 / (2.0 * margin_) + 0.5 * rho
    if not (2.0 * c < 1.0):
        return math.inf
    return 2.0 * c / (1.0 + math.sqrt(1.0 - 2.0 * c))


# --------------------------------------------------------------------------
# Frechet derivative of sign (Daleckii-Krein), for gradient checks
# --------------------------------------------------------------------------
def daleckii_krein(mu: np.ndarray, V: np.ndarray, W: np.ndarray) -> np.ndarray:
    """V (F o V^T W V) V^T with F_ij = (sign mu_i - sign mu_j)/(mu_i - mu_j)."""
    mu, V, W = _c(mu), _c(V), _c(W)
    d = V.shape[0]
    out = np.empty((d, d))
    _load().rsign_oracle_daleckii_krein(d, _p(mu), _p(V), _p(W), _p(out))
    return out


def matmul(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """Plain triple-loop FP64 product (used by the pins as an independent route)."""
    A, B = _c(A), _c(B)
    C = np.empty((A.shape[0], B.shape[1]))
    _load().rsign_oracle_matmul(A.shape[0], A.shape[1], B.shape[1], _p(A), _p(B), _p(C))
    return C
