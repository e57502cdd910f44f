"""Pins of the oracle's tables against what the mathematics fixes:
lattice isotropy, equilibrium moments, force-split moments (Sec. 2.1), GLL
quadrature and differentiation exactness (Sec. 2.2), filter properties (Sec. 2.4)."""
import itertools
import os

import numpy as np
import pytest

from oracle import gll
from oracle.lattice import CS2, equilibrium, force_split, lattice

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.mark.parametrize("name,Q", [("D2Q9", 9), ("D3Q19", 19), ("D3Q27", 27)])
def test_lattice_isotropy(name, Q):
    """sum t = 1, sum t e = 0, sum t e e = cs2 I, sum t e e e e = cs2^2 (d d + d d + d d)."""
    e, t, opp = lattice(name)
    assert len(t) == Q
    d = e.shape[1]
    ef = e.astype(float)
    assert abs(t.sum() - 1.0) < 1e-15
    assert np.abs(t @ ef).max() < 1e-15
    assert np.abs(np.einsum("a,ai,aj->ij", t, ef, ef) - CS2 * np.eye(d)).max() < 1e-15
    m4 = np.einsum("a,ai,aj,ak,al->ijkl", t, ef, ef, ef, ef)
    I = np.eye(d)
    ref = CS2 ** 2 * (np.einsum("ij,kl->ijkl", I, I) + np.einsum("ik,jl->ijkl", I, I) + np.einsum("il,jk->ijkl", I, I))
    assert np.abs(m4 - ref).max() < 1e-15
    assert np.all(e[opp] == -e)
    assert np.all(e[0] == 0)


def test_lattice_order_rule():
    """Speed class first, then ternary code ascending."""
    e, _, _ = lattice("D2Q9")
    assert e.tolist() == [[0, 0], [0, -1], [-1, 0], [1, 0], [0, 1], [-1, -1], [1, -1], [-1, 1], [1, 1]]
    e27, _, _ = lattice("D3Q27")
    e19, _, _ = lattice("D3Q19")
    assert np.all(e27[:19] == e19)


@pytest.mark.parametrize("name", ["D2Q9", "D3Q19", "D3Q27"])
def test_equilibrium_moments(name):
    """Moments 0-2 of f^eq: rho, rho u, rho cs2 I + rho u u (textbook LBM equilibrium)."""
    e, t, _ = lattice(name)
    d = e.shape[1]
    rng = np.random.default_rng(0)
    rho = 1 + 0.1 * rng.standard_normal(7)
    u = 0.05 * rng.standard_normal((7, d))
    f = equilibrium(e, t, rho, u)
    ef = e.astype(float)
    assert np.abs(f.sum(0) - rho).max() < 1e-14
    assert np.abs(ef.T @ f - (rho[:, None] * u).T).max() < 1e-14
    P = np.einsum("ai,aj,an->nij", ef, ef, f)
    ref = rho[:, None, None] * (CS2 * np.eye(d)[None] + np.einsum("ni,nj->nij", u, u))
    assert np.abs(P - ref).max() < 1e-14


@pytest.mark.parametrize("name", ["D2Q9", "D3Q19", "D3Q27"])
def test_force_split_moments(name):
    """sum F** = sum e F** = 0 (Sec. 2.2, force splitting); sum F* = 0, sum e F* = F;
    F* + F** equals the full forcing term F_alpha of Sec. 2.1."""
    e, t, _ = lattice(name)
    d = e.shape[1]
    rng = np.random.default_rng(1)
    u = 0.05 * rng.standard_normal((5, d))
    F = 1e-3 * rng.standard_normal((5, d))
    Fs, Fss = force_split(e, t, u, F)
    ef = e.astype(float)
    assert np.abs(Fss.sum(0)).max() < 1e-17
    assert np.abs(ef.T @ Fss).max() < 1e-17
    assert np.abs(Fs.sum(0)).max() < 1e-17
    assert np.abs(ef.T @ Fs - F.T).max() < 1e-17
    full = np.stack([t[a] * (((ef[a][None] - u) / CS2 + (u @ ef[a])[:, None] * ef[a][None] / CS2 ** 2) * F).sum(1)
                     for a in range(len(t))])
    assert np.abs(full - (Fs + Fss)).max() < 1e-17


def test_gll_golden_n4():
    ref = np.loadtxt(os.path.join(GOLDEN, "gll_n4.txt"))
    xi = gll.gll_nodes(4)
    assert np.abs(xi - ref[:, 0]).max() < 1e-15
    assert np.abs(gll.gll_weights(4, xi) - ref[:, 1]).max() < 1e-15


@pytest.mark.parametrize("N", [2, 3, 4, 5, 6, 7, 8, 10, 12, 14])
def test_gll_exactness(N):
    """D_hat differentiates x^m exactly for m <= N; GLL quadrature is exact to degree 2N-1 (P2)."""
    xi = gll.gll_nodes(N)
    w = gll.gll_weights(N, xi)
    D = gll.derivative_matrix(xi)
    for m in range(N + 1):
        deriv = m * xi ** (m - 1) if m > 0 else np.zeros_like(xi)
        assert np.abs(D @ xi ** m - deriv).max() < 1e-11 * max(1, N ** 2)
    for m in range(2 * N):
        exact = 0.0 if m % 2 else 2.0 / (m + 1)
        assert abs(w @ xi ** m - exact) < 1e-14
    exact = 2.0 / (2 * N + 1)
    assert abs(w @ xi ** (2 * N) - exact) > 1e-9        # first inexact degree
    assert np.all(np.diff(xi) > 0)


@pytest.mark.parametrize("N,kc,gamma,shape", [(7, 5, 0.1, 0), (8, 6, 0.1, 1), (4, 2, 0.3, 0), (7, 3.4, 0.2, 1)])
def test_filter_properties(N, kc, gamma, shape):
    """P4: degree <= kc polynomials pass unchanged, sigma_N = 1 - gamma, boundary
    rows are identity rows, reversal symmetry, GLL integral preserved for kc >= 2."""
    xi = gll.gll_nodes(N)
    w = gll.gll_weights(N, xi)
    sig = gll.filter_sigma(N, shape, gamma, kc)
    F = gll.filter_matrix(N, xi, sig)
    assert abs(sig[N] - (1 - gamma)) < 1e-15
    for m in range(int(np.floor(kc)) + 1):
        assert np.abs(F @ xi ** m - xi ** m).max() < 1e-13
    # the top mode is damped by exactly sigma_N
    phiN = gll.legendre(N, xi) - gll.legendre(N - 2, xi)
    assert np.abs(F @ phiN - sig[N] * phiN).max() < 1e-13
    assert np.abs(F[0] - np.eye(N + 1)[0]).max() < 1e-13
    assert np.abs(F[N] - np.eye(N + 1)[N]).max() < 1e-13
    Jr = np.eye(N + 1)[::-1]
    assert np.abs(Jr @ F @ Jr - F).max() < 1e-13
    rng = np.random.default_rng(2)
    v = rng.standard_normal(N + 1)
    assert abs(w @ (F @ v) - w @ v) < 1e-13


def test_filter_identity_and_shapes():
    N = 6
    xi = gll.gll_nodes(N)
    F = gll.filter_matrix(N, xi, gll.filter_sigma(N, 0, 0.0, 2))
    assert np.abs(F - np.eye(N + 1)).max() < 1e-13
    q = gll.filter_sigma(N, 0, 0.2, 2)
    assert np.allclose(q[:3], 1.0)
    assert abs(q[4] - (1 - 0.2 * 0.25)) < 1e-15        # r = 1/2 -> 1 - gamma/4
    x = gll.filter_sigma(N, 1, 0.2, 2, p=8)
    assert abs(x[4] - 0.8 ** (0.5 ** 8)) < 1e-15
