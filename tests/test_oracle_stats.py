"""Pins of the oracle's pipe-flow statistics (Sec. 4): wall shear stress and radially binned mean
velocity, against closed forms and exact quadrature identities; the log-law profile."""
import math

import numpy as np

import workloads as W
from oracle.selbm import OracleSELBM


def _state(o, u):
    return o.initial_state(np.ones(o.G), u)


def test_wall_stress_channel_poiseuille_exact():
    """u_x = 4 U y (1 - y) between walls y = 0, 1: -mu n.grad u_x = 4 mu U on both walls (the
    parabola is exact in the GLL basis for N >= 2, on affine elements)."""
    for dim, N in ((2, 4), (3, 3)):
        if dim == 2:
            mesh = W.box_mesh((3, 2), (0, 0), (1.5, 1.0), (True, False), walls={2: 1, 3: 1})
            lat = "D2Q9"
        else:
            mesh = W.box_mesh((2, 2, 2), (0, 0, 0), (1.0, 1.0, 1.0), (True, False, True), walls={2: 1, 3: 1})
            lat = "D3Q19"
        nu, U = 0.01, 0.02
        o = OracleSELBM(mesh, lat, N, nu)
        u = np.zeros((o.G, dim))
        y = o.Xg[:, 1]
        u[:, 0] = 4 * U * y * (1 - y)
        tau = o.wall_stress(_state(o, u), [1.0, 0.0, 0.0][:dim])
        assert abs(tau - 4 * nu * U) <= 1e-12 * 4 * nu * U, tau
        # a flow along the walls' normal carries no stress along x
        assert abs(o.wall_stress(_state(o, u), [0.0, 1.0, 0.0][:dim])) <= 1e-15


def test_wall_stress_pipe_poiseuille():
    """u_z = U (1 - r^2 / R^2) in the butterfly pipe: tau_w = 2 mu U / R, up to the isoparametric
    approximation of the circle."""
    mesh = W.pipe_mesh(n_core=2, n_radial=2, n_axial=1, length=1.0)
    nu, U = 1e-3, 0.03
    o = OracleSELBM(mesh, "D3Q19", 5, nu)
    u = np.zeros((o.G, 3))
    u[:, 2] = U * (1 - (o.Xg[:, 0] ** 2 + o.Xg[:, 1] ** 2))
    tau = o.wall_stress(_state(o, u), [0, 0, 1])
    assert abs(tau - 2 * nu * U) <= 1e-3 * 2 * nu * U, tau


def test_radial_profile_identities_box():
    """Bins partition the unique nodes: their masses sum to the volume and their mass-weighted
    means to the quadrature integral (exact for the quadratic u_z = 1 - x^2 - y^2)."""
    mesh = W.box_mesh((2, 2, 2), (-1, -1, 0), (1, 1, 1), (False, False, True))
    o = OracleSELBM(mesh, "D3Q19", 4, 1e-3)
    u = np.zeros((o.G, 3))
    u[:, 2] = 1 - o.Xg[:, 0] ** 2 - o.Xg[:, 1] ** 2
    mean, mass = o.radial_profile(_state(o, u), [0, 0, 0], [0, 0, 1], math.sqrt(2), 7)
    assert abs(mass.sum() - 4.0) <= 1e-12
    assert abs((mean * mass).sum() - 4.0 / 3.0) <= 1e-12


def test_radial_profile_pipe_bounds():
    """In the pipe, each bin's mean of 1 - r^2 lies between its values at the bin edges."""
    mesh = W.pipe_mesh(n_core=2, n_radial=2, n_axial=1, length=1.0)
    o = OracleSELBM(mesh, "D3Q19", 4, 1e-3)
    u = np.zeros((o.G, 3))
    u[:, 2] = 1 - (o.Xg[:, 0] ** 2 + o.Xg[:, 1] ** 2)
    nb = 8
    mean, mass = o.radial_profile(_state(o, u), [0, 0, 0], [0, 0, 1], 1.0, nb)
    edges = np.linspace(0, 1, nb + 1)
    for b in range(nb):
        if mass[b] > 0:
            lo, hi = 1 - edges[b + 1] ** 2 - 1e-9, 1 - edges[b] ** 2 + 1e-9
            assert lo <= mean[b] <= hi, (b, mean[b])
    assert abs(mass.sum() - math.pi) <= 2e-3 * math.pi          # pipe volume, isoparametric circle


def test_loglaw_profile():
    """u+ = y+ below the crossing of the two branches, (1/kappa) ln y+ + C+ above; continuous."""
    y = np.array([0.5, 5.0, 30.0, 180.0])
    up = W.loglaw_uplus(y)
    assert np.allclose(up[:2], y[:2])
    assert np.allclose(up[2:], np.log(y[2:]) / 0.41 + 5.0)
    grid = np.linspace(0, 30, 3000)
    assert np.abs(np.diff(W.loglaw_uplus(grid))).max() < 0.02
    assert W.loglaw_uplus(0.0) == 0.0 and W.loglaw_uplus(1e-3) == 1e-3       # no-slip wall, viscous sublayer
