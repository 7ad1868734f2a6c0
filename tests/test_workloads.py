"""The seeded input generators follow their stated recipes.

The generators feed both the oracle and the CUDA path. These CPU checks pin
the shapes and structures that the parity cases and the benchmark rely on.
"""
import math

import numpy as np
import pytest

import workloads


@pytest.mark.parametrize("d,k,delta", [(2, 1, 0.05), (40, 1, 1e-2), (64, 63, 1e-3), (200, 16, 0.1)])
def test_controlled_spectrum_recipe(d, k, delta):
    sp = workloads.controlled_spectrum(d, k, delta, seed=3 + d)
    lam = sp.lam
    assert lam.shape == (d,) and np.all(np.diff(lam) >= 0)
    assert lam[k - 1] == -delta and lam[k] == delta  # pinned half-gap around 0
    assert np.all(lam[: k - 1] >= -1.0) and np.all(lam[: k - 1] <= -delta)
    assert np.all(lam[k + 1:] >= delta) and np.all(lam[k + 1:] <= 1.0)
    Q = sp.Q
    assert np.max(np.abs(Q.T @ Q - np.eye(d))) < 1e-13
    assert np.array_equal(sp.H, sp.H.T)
    assert np.max(np.abs(sp.H - (Q * lam) @ Q.T)) < 1e-14 * d
    assert workloads.shift_in_gap(sp, 0.5) == 0.0


def test_haar_orthogonal_sign_convention():
    # Q diag(sign(diag R)) makes R's diagonal positive: the factorisation is unique
    rng = np.random.default_rng(5)
    G = np.random.default_rng(5).standard_normal((30, 30))
    Q = workloads.haar_orthogonal(30, rng)
    Rf = Q.T @ G
    assert np.all(np.diag(Rf) > 0)
    assert np.max(np.abs(np.tril(Rf, -1))) < 1e-12


def test_split_spectrum_config_recipe():
    sp = workloads.split_spectrum_config(seed=0)
    assert sp.H.shape == (256, 256) and sp.k == 4
    assert np.all((sp.lam[:4] >= -1.0) & (sp.lam[:4] <= -0.1))
    assert np.all((sp.lam[4:] >= 0.1) & (sp.lam[4:] <= 1.0))


def test_controlled_seed_formula():
    assert workloads.controlled_seed(8192, 1, 1) == 13011
    assert workloads.controlled_seed(256, 0, 2) == 8002


def test_batched_workload_recipe():
    items = workloads.batched_workload(64)
    assert len(items) == 64
    for sp, s in items:
        d = sp.H.shape[0]
        assert d in range(32, 513, 32) and 1 <= sp.k <= min(8, d - 1)
        delta = sp.meta["delta"]
        assert 1e-3 <= delta <= 1e-1 and abs(s) <= 0.5
        # the offset moves the spectrum, the gap midpoint is s, the reflector is unchanged
        assert sp.lam[sp.k - 1] == pytest.approx(s - delta, abs=1e-15)
        assert sp.lam[sp.k] == pytest.approx(s + delta, abs=1e-15)
    ds = [sp.H.shape[0] for sp, _ in workloads.batched_workload(512)]
    assert len(set(ds)) == 16  # every order of the mix occurs


def test_controlled_spectrum_torch_recipe_on_cpu():
    torch = pytest.importorskip("torch")
    d, k, delta = 96, 5, 2e-2
    H, lam, Q = workloads.controlled_spectrum_torch(d, k, delta, seed=9, device="cpu")
    lam = lam.numpy()
    Q = Q.numpy()
    H = H.numpy()
    assert lam[k - 1] == -delta and lam[k] == delta and np.all(np.diff(lam) >= 0)
    assert np.max(np.abs(Q.T @ Q - np.eye(d))) < 1e-13
    assert np.array_equal(H, H.T)
    w = np.linalg.eigvalsh(H)
    assert np.max(np.abs(w - lam)) < 1e-13
    # the eigenvalues of the gap pair belong to columns k-1 and k of Q
    assert np.linalg.norm(H @ Q[:, k - 1] + delta * Q[:, k - 1]) < 1e-13
    assert math.isclose(float(Q[:, k] @ H @ Q[:, k]), delta, abs_tol=1e-14)
