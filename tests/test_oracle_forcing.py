"""Pins of the per-node acceleration field (Sec. 4, pipe: the divergence-free perturbation
force of the first three eddy turnover times) and of the oracle's handling of it.

The field is pinned by what the paper states about it, not by retyping its formulas:
it is divergence-free, it vanishes outside the band l0 <= R - r <= l0 + l, and the
weighting kappa moves it between the r-z and theta-z planes.  Its use in the step is
pinned by the uniform special case (identical to a body force) and by the discrete
momentum budget of a periodic mesh.
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle.selbm import OracleSELBM


def band_points(n, seed, R=1.0, L=10.0, l0=0.2, l=0.4):
    rng = np.random.default_rng(seed)
    r = rng.uniform(R - l0 - l + 0.01, R - l0 - 0.01, n)
    th = rng.uniform(0.0, 2.0 * np.pi, n)
    z = rng.uniform(0.0, L, n)
    return np.stack([r * np.cos(th), r * np.sin(th), z], 1)


def divergence(f, x, h=1e-4):
    d = np.zeros(x.shape[0])
    for k in range(3):
        e = np.zeros(3)
        e[k] = h
        d += (f(x + e)[:, k] - f(x - e)[:, k]) / (2 * h)
    return d


@pytest.mark.parametrize("kappa,kz,kt", [(0.5, 3, 4), (0.0, 3, 4), (1.0, 3, 4), (0.3, 2, 1)])
def test_peng_field_divergence_free(kappa, kz, kt):
    f = W.peng_forcing(1.0, kz=kz, ktheta=kt, kappa=kappa)
    x = band_points(300, 1)
    F = f(x)
    scale = np.abs(F).max() * 2 * np.pi / 0.4                 # steepest gradient: the radial band
    assert scale > 0
    assert np.abs(divergence(f, x)).max() < 1e-6 * scale


def test_peng_field_support_and_continuity():
    f = W.peng_forcing(1.0)
    rng = np.random.default_rng(2)
    th = rng.uniform(0, 2 * np.pi, 200)
    z = rng.uniform(0, 10, 200)
    for r in (0.05, 0.3, 0.39, 0.81, 0.9, 0.999):              # outside 0.4 <= r <= 0.8
        x = np.stack([r * np.cos(th), r * np.sin(th), z], 1)
        assert np.abs(f(x)).max() == 0.0, r
    x = band_points(200, 3)
    assert np.abs(f(x)).max() > 1.0                           # g B0 = 50: O(10) inside
    # continuous at both band edges: |F| <= g B0 (R / r) (2 pi / l) delta at distance delta
    for edge, sgn in ((0.4, 1.0), (0.8, -1.0)):
        for delta in (1e-5, 1e-7):
            r = edge + sgn * delta
            x = np.stack([r * np.cos(th), r * np.sin(th), z], 1)
            assert np.abs(f(x)).max() <= 50.0 * (1.0 / 0.4) * (2 * np.pi / 0.4) * delta * 1.01, (edge, delta)


def test_peng_field_kappa_split():
    """kappa = 1: no azimuthal component; kappa = 0: no radial component."""
    x = band_points(200, 4)
    r = np.hypot(x[:, 0], x[:, 1])
    er = np.stack([x[:, 0] / r, x[:, 1] / r], 1)
    et = np.stack([-x[:, 1] / r, x[:, 0] / r], 1)
    F1 = W.peng_forcing(1.0, kappa=1.0)(x)
    F0 = W.peng_forcing(1.0, kappa=0.0)(x)
    assert np.abs((F1[:, :2] * et).sum(1)).max() < 1e-12 * np.abs(F1).max()
    assert np.abs((F0[:, :2] * er).sum(1)).max() < 1e-12 * np.abs(F0).max()
    assert np.abs((F1[:, :2] * er).sum(1)).max() > 0.1 and np.abs((F0[:, :2] * et).sum(1)).max() > 0.1


def test_uniform_field_is_a_body_force():
    """A constant field with A = 1 is the body force g: identical steps."""
    mesh = W.box_mesh((2, 2), (0, 0), (1, 1), (True, True))
    g = np.array([2e-4, -1e-4])
    filt = {"shape": 0, "gamma": 0.1, "kc": 2.0}
    a = OracleSELBM(mesh, "D2Q9", 4, nu=0.01, body_accel=g, filt=filt)
    b = OracleSELBM(mesh, "D2Q9", 4, nu=0.01, filt=filt)
    b.set_force_field(np.tile(g, (b.G, 1)), period=0.0, t_end=math.inf)
    init = W.shear_layer_init(U0=0.02, kappa=5.0)
    fa, fb = a.initial_state_from(init), b.initial_state_from(init)
    assert np.array_equal(fa, fb)
    for _ in range(3):
        fa, fb = a.step(fa), b.step(fb)
    assert np.array_equal(fa, fb)


def test_field_momentum_budget_and_schedule():
    """Periodic affine mesh: each step adds dt sum_g M_g rho_g (g + A(t_n) S_g) of momentum,
    with A(t_n) = sin(2 pi t_n / P) at the step's start time and 0 from t_end on."""
    mesh = W.box_mesh((2, 2), (0, 0), (1, 1), (True, True))
    g = np.array([1e-4, 0.0])
    o = OracleSELBM(mesh, "D2Q9", 4, nu=0.01, body_accel=g, filt={"shape": 0, "gamma": 0.1, "kc": 2.0})
    X = o.Xg
    S = 3e-3 * np.stack([np.sin(2 * np.pi * X[:, 1]), np.cos(2 * np.pi * X[:, 0]) + 0.5], 1)
    P = 8 * o.dt
    o.set_force_field(S, period=P, t_end=4.5 * o.dt)
    f = o.initial_state_from(W.shear_layer_init(U0=0.02, kappa=5.0))
    amps = []
    for n in range(7):
        _, mom0, _ = o.integrals(f)
        rho, _ = o.moments(f)
        A = math.sin(2 * math.pi * n * o.dt / P) if n <= 4 else 0.0
        amps.append(o.amplitude(o.time))
        expect = o.dt * ((o.mass * rho)[:, None] * (g[None, :] + A * S)).sum(0)
        f = o.step(f)
        _, mom1, _ = o.integrals(f)
        assert np.abs(mom1 - mom0 - expect).max() < 1e-15, n
    assert amps[0] == 0.0 and amps[2] == pytest.approx(1.0) and amps[5] == 0.0 and amps[6] == 0.0
    assert o.time == pytest.approx(7 * o.dt)
