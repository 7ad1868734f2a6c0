"""Seeded synthetic inputs for the shifted matrix-sign reflector.

This module only builds inputs: symmetric matrices with a prescribed
spectrum (H = Q diag(lam) Q^T), the Allen-Cahn-shaped Hessian of the paper's
stiff-spectrum experiment (Sec. 5.4), and the batched size mix.  It holds no
arithmetic of the method itself (no sign, no Newton-Schulz, no reflector, no
shift or scaling rule); both the CPU oracle and the CUDA path consume what it
returns.

Every generator is deterministic in its seed (numpy ``default_rng``).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Spectrum",
    "haar_orthogonal",
    "controlled_spectrum",
    "split_spectrum_config",
    "allen_cahn_hessian",
    "batched_sizes",
    "shift_in_gap",
    "controlled_seed",
]


@dataclass
class Spectrum:
    """A symmetric test matrix together with the data it was built from.

    ``H`` is d x d float64, symmetric to the last bit.  ``lam`` holds the
    prescribed eigenvalues in ascending order and ``Q`` the orthogonal basis
    (column i belongs to lam[i]), so that H = Q diag(lam) Q^T up to rounding.
    ``k`` is the target index; the gap is (lam[k-1], lam[k]).
    """

    H: np.ndarray
    lam: np.ndarray
    Q: np.ndarray | None
    k: int
    meta: dict = field(default_factory=dict)

    @property
    def d(self) -> int:
        return self.H.shape[0]

    @property
    def gap(self) -> tuple[float, float]:
        return float(self.lam[self.k - 1]), float(self.lam[self.k])


def controlled_seed(d: int, k_idx: int, delta_idx: int) -> int:
    """Seed of one controlled-spectrum sweep point: 1000*log2(d) + 10*k_idx + delta_idx."""
    return 1000 * int(round(math.log2(d))) + 10 * k_idx + delta_idx


def haar_orthogonal(d: int, rng: np.random.Generator) -> np.ndarray:
    """Orthogonal Q from the QR factorisation of a d x d standard Gaussian.

    The columns are sign-fixed (Q <- Q diag(sign(diag R))) so that the result
    is unique for a given Gaussian draw.
    """
    G = rng.standard_normal((d, d))
    Q, Rf = np.linalg.qr(G)
    sgn = np.sign(np.diag(Rf))
    sgn[sgn == 0] = 1.0
    return Q * sgn


def _assemble(Q: np.ndarray, lam: np.ndarray) -> np.ndarray:
    H = (Q * lam) @ Q.T
    return 0.5 * (H + H.T)


def controlled_spectrum(d: int, k: int, delta: float, seed: int) -> Spectrum:
    """Controlled spectrum split at index k with half-gap ``delta`` around 0.

    lam_k = -delta and lam_{k+1} = +delta exactly; the other k-1 eigenvalues
    are uniform in [-1, -delta] and the remaining d-k-1 uniform in [delta, 1].
    The gap is centred at 0, so its midpoint is s = 0.
    """
    if not (1 <= k <= d - 1):
        raise ValueError("k must lie in [1, d-1]")
    rng = np.random.default_rng(seed)
    Q = haar_orthogonal(d, rng)
    lo = -rng.uniform(delta, 1.0, size=k - 1)
    hi = rng.uniform(delta, 1.0, size=d - k - 1)
    lam = np.sort(np.concatenate([lo, [-delta, delta], hi]))
    # the two pinned endpoints keep positions k-1 and k after sorting
    assert lam[k - 1] == -delta and lam[k] == delta
    return Spectrum(_assemble(Q, lam), lam, Q, k,
                    dict(kind="controlled", d=d, k=k, delta=delta, seed=seed))


def split_spectrum_config(d: int = 256, k: int = 4, lo=(-1.0, -0.1), hi=(0.1, 1.0),
                          seed: int = 0) -> Spectrum:
    """Spectrum with lam_1..lam_k uniform in ``lo`` and the rest uniform in ``hi``.

    This is the d=256, k=4 plain-method workload (no endpoint pinning).
    """
    rng = np.random.default_rng(seed)
    Q = haar_orthogonal(d, rng)
    lam = np.sort(np.concatenate([rng.uniform(lo[0], lo[1], size=k),
                                  rng.uniform(hi[0], hi[1], size=d - k)]))
    return Spectrum(_assemble(Q, lam), lam, Q, k,
                    dict(kind="split", d=d, k=k, lo=lo, hi=hi, seed=seed))


def shift_in_gap(spec: Spectrum, theta: float) -> float:
    """Shift placed at fraction theta of the target gap: lam_k + theta (lam_{k+1} - lam_k).

    This is the parametrisation of the shift sweep of the controlled spectral
    tests (Sec. 5.1); theta = 0.5 is the gap midpoint.
    """
    a, b = spec.gap
    return a + theta * (b - a)


def allen_cahn_hessian(n: int = 64, eps: float = 0.04, n_modes: int = 8,
                       max_wavenumber: int = 4, seed: int = 1):
    """Allen-Cahn-shaped Hessian on an n x n periodic grid (d = n*n).

    H = eps^2 L + diag(3 u^2 - 1), with L the positive semidefinite 5-point
    operator (4 u_ij - sum of the four neighbours) / h^2, h = 1/n, periodic;
    unknowns ordered row-major (i*n + j).  u = tanh(phi / (sqrt(2) eps)) where
    phi is a sum of ``n_modes`` Fourier modes with distinct integer wavevectors
    (kx, ky), 0 < kx^2 + ky^2 <= max_wavenumber^2, drawn without replacement,
    unit-normal amplitudes and uniform phases, normalised to max|phi| = 1.

    Returns (H, u).  The eigen-decomposition is not known by construction.
    """
    rng = np.random.default_rng(seed)
    h = 1.0 / n
    cand = [(kx, ky) for kx in range(-max_wavenumber, max_wavenumber + 1)
            for ky in range(-max_wavenumber, max_wavenumber + 1)
            if 0 < kx * kx + ky * ky <= max_wavenumber * max_wavenumber]
    pick = rng.choice(len(cand), size=n_modes, replace=False)
    amp = rng.standard_normal(n_modes)
    phase = rng.uniform(0.0, 2.0 * math.pi, size=n_modes)
    x = np.arange(n) * h
    X, Y = np.meshgrid(x, x, indexing="ij")
    phi = np.zeros((n, n))
    for m, c in enumerate(pick):
        kx, ky = cand[c]
        phi += amp[m] * np.cos(2.0 * math.pi * (kx * X + ky * Y) + phase[m])
    phi /= np.abs(phi).max()
    u = np.tanh(phi / (math.sqrt(2.0) * eps))
    d = n * n
    H = np.zeros((d, d))
    c = eps * eps / (h * h)
    idx = np.arange(d).reshape(n, n)
    for i in range(n):
        for j in range(n):
            r = idx[i, j]
            H[r, r] += 4.0 * c + 3.0 * u[i, j] ** 2 - 1.0
            for (a, b) in ((i + 1, j), (i - 1, j), (i, j + 1), (i, j - 1)):
                H[r, idx[a % n, b % n]] -= c
    return H, u


def batched_sizes(count: int = 512, d_choices=tuple(range(32, 513, 32)), k_max: int = 8,
                  delta_range=(1e-3, 1e-1), seed: int = 7):
    """Size mix of the batched workload: (d_i, k_i, delta_i) for ``count`` matrices.

    d uniform over ``d_choices``, k uniform in 1..k_max, delta log-uniform.
    """
    rng = np.random.default_rng(seed)
    d = rng.choice(np.asarray(d_choices), size=count)
    k = rng.integers(1, k_max + 1, size=count)
    logd = rng.uniform(math.log(delta_range[0]), math.log(delta_range[1]), size=count)
    return [(int(d[i]), int(min(k[i], d[i] - 1)), float(math.exp(logd[i]))) for i in range(count)]


def batched_workload(count: int = 512, d_choices=tuple(range(32, 513, 32)), k_max: int = 8,
                     delta_range=(1e-3, 1e-1), offset: float = 0.5, seed: int = 7):
    """The batched workload: ``count`` controlled spectra of uneven order.

    (d_i, k_i, delta_i) come from ``batched_sizes``; matrix i is the controlled
    spectrum of that size with seed ``seed * 100003 + i``, moved by a seeded
    offset c_i uniform in [-offset, offset] (H_i + c_i I, eigenvalues lam + c_i),
    so every matrix has its own gap midpoint s_i = c_i while its reflector
    I - 2 Q_k Q_k^T is unchanged.  Returns a list of (Spectrum, s_i).
    """
    sizes = batched_sizes(count, d_choices, k_max, delta_range, seed)
    rng = np.random.default_rng(seed + 1)
    c = rng.uniform(-offset, offset, size=count)
    out = []
    for i, (d, k, delta) in enumerate(sizes):
        sp = controlled_spectrum(d, k, delta, seed * 100003 + i)
        H = sp.H + c[i] * np.eye(d)
        meta = dict(sp.meta, offset=float(c[i]))
        out.append((Spectrum(H, sp.lam + c[i], sp.Q, k, meta), float(c[i])))
    return out


def controlled_spectrum_torch(d: int, k: int, delta: float, seed: int, device="cuda"):
    """Same recipe as ``controlled_spectrum`` built with torch on ``device``.

    Used where the numpy construction is too slow (d in the thousands on the
    host).  The random stream is torch's, so the matrix differs from the numpy
    one with the same seed; the spectrum distribution and the structure are
    the same.  Returns (H, lam, Q) as float64 tensors on ``device``.
    """
    import torch
    g = torch.Generator(device=device).manual_seed(seed)
    G = torch.randn((d, d), generator=g, device=device, dtype=torch.float64)
    Q, Rf = torch.linalg.qr(G)
    sgn = torch.sign(torch.diagonal(Rf))
    sgn[sgn == 0] = 1.0
    Q = Q * sgn
    del G, Rf
    lo = -(delta + (1.0 - delta) * torch.rand(k - 1, generator=g, device=device, dtype=torch.float64))
    hi = delta + (1.0 - delta) * torch.rand(d - k - 1, generator=g, device=device, dtype=torch.float64)
    pin = torch.tensor([-delta, delta], device=device, dtype=torch.float64)
    lam, _ = torch.sort(torch.cat([lo, pin, hi]))
    H = (Q * lam) @ Q.T
    H = 0.5 * (H + H.T)
    return H.contiguous(), lam, Q
