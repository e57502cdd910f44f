"""Pins of the oracle's mesh processing: metrics of affine elements, areas and
volumes of curved pipe meshes, wall normals and surface weights (Nanson),
global numbering counts on periodic meshes."""
import math

import numpy as np
import pytest

import workloads as W
from oracle import geometry as geo
from oracle import gll


def _geom(mesh, N):
    xi = gll.gll_nodes(N)
    w = gll.gll_weights(N, xi)
    D = gll.derivative_matrix(xi)
    X = geo.element_nodes(mesh, xi)
    dxdr, J, drdx, wJ = geo.metrics(X, D, N, mesh.dim, w)
    return xi, w, D, X, dxdr, J, drdx, wJ


def test_box_metrics_affine():
    mesh = W.box_mesh((3, 2, 2), (0.0, 0.0, 0.0), (1.5, 1.0, 2.0), (True, False, True))
    N = 4
    _, _, _, X, dxdr, J, drdx, wJ = _geom(mesh, N)
    h = np.array([0.5, 0.5, 1.0])
    assert np.abs(J - np.prod(h / 2)).max() < 1e-14
    assert np.abs(drdx - np.diag(2 / h)[None, None]).max() < 1e-12
    assert abs(wJ.sum() - 1.5 * 1.0 * 2.0) < 1e-13


def test_global_numbering_counts():
    N = 5
    xi = gll.gll_nodes(N)
    # fully periodic 2D: (nx N)(ny N) unique nodes
    m = W.box_mesh((4, 3), (0, 0), (1, 1), (True, True))
    X = geo.element_nodes(m, xi)
    glo = geo.global_numbering(X, m)
    assert glo.max() + 1 == (4 * N) * (3 * N)
    # periodic in x only (Couette): (nx N)(ny N + 1)
    m = W.box_mesh((4, 3), (0, 0), (1, 1), (True, False))
    glo = geo.global_numbering(geo.element_nodes(m, xi), m)
    assert glo.max() + 1 == (4 * N) * (3 * N + 1)
    # copies of one global node share coordinates (modulo the period)
    X = geo.element_nodes(m, xi).reshape(-1, 2)
    g = glo.ravel()
    for gid in range(0, glo.max() + 1, 7):
        P = X[g == gid]
        dx = np.mod(P[:, 0] - P[0, 0] + 0.5, 1.0) - 0.5
        assert np.abs(dx).max() < 1e-12 and np.abs(P[:, 1] - P[0, 1]).max() < 1e-12


def test_pipe_volume_and_wall_area():
    """One axial layer of the butterfly pipe: volume pi R^2 L, wall area 2 pi R L,
    outward unit normals radial, closed-surface sum of n w_s J_s zero along x, y."""
    L = 0.5
    mesh = W.pipe_mesh(n_core=4, n_radial=3, n_axial=1, length=L)
    N = 6
    _, w, _, X, dxdr, J, drdx, wJ = _geom(mesh, N)
    assert np.all(J > 0)
    assert abs(wJ.sum() - math.pi * L) < 1e-6
    walls = geo.wall_faces(mesh, drdx, J, w, N)
    area = sum(float(ws.sum()) for (_, _, _, ws, _) in walls)
    assert abs(area - 2 * math.pi * L) < 1e-6
    for (e, nodes, n, ws, wid) in walls:
        P = X[e, nodes]
        radial = P[:, :2] / np.linalg.norm(P[:, :2], axis=1)[:, None]
        assert np.abs(n[:, :2] - radial).max() < 1e-5
        assert np.abs(n[:, 2]).max() < 1e-12
        assert np.abs(np.linalg.norm(P[:, :2], axis=1) - 1.0).max() < 1e-12
    tot = sum((n * ws[:, None]).sum(0) for (_, _, n, ws, _) in walls)
    assert np.abs(tot).max() < 1e-6


def test_pipe_numbering_and_periodicity():
    mesh = W.pipe_mesh(n_core=2, n_radial=2, n_axial=3, length=1.5)
    N = 3
    xi = gll.gll_nodes(N)
    X = geo.element_nodes(mesh, xi)
    glo = geo.global_numbering(X, mesh)
    # 2D cross-section unique nodes x (axial N * n_axial) layers (periodic)
    m2 = W.pipe_mesh(n_core=2, n_radial=2, n_axial=1, length=1.0)
    X2 = geo.element_nodes(m2, xi)
    sec = X2[:, :, :2][X2[:, :, 2] == 0.0]
    # count unique cross-section points
    r = np.round(sec, 9)
    nsec = len({tuple(p) for p in r})
    assert glo.max() + 1 == nsec * N * 3


def test_box_wall_faces():
    mesh = W.box_mesh((2, 2), (0, 0), (1, 1), (True, False), walls={2: 1, 3: 2},
                      wall_velocity=[[0, 0], [0.1, 0]])
    N = 4
    _, w, _, X, dxdr, J, drdx, wJ = _geom(mesh, N)
    walls = geo.wall_faces(mesh, drdx, J, w, N)
    assert len(walls) == 4
    for (e, nodes, n, ws, wid) in walls:
        y = X[e, nodes, 1]
        if wid == 1:
            assert np.allclose(y, 0.0) and np.allclose(n, [0, -1])
        else:
            assert np.allclose(y, 1.0) and np.allclose(n, [0, 1])
        assert abs(ws.sum() - 0.5) < 1e-14           # edge length of one element


def test_min_spacing_box():
    mesh = W.box_mesh((8, 4), (0, 0), (1, 1), (True, False))
    N = 4
    xi = gll.gll_nodes(N)
    X = geo.element_nodes(mesh, xi)
    assert abs(geo.min_node_spacing(X, N, 2) - (xi[1] - xi[0]) * (1 / 8) / 2) < 1e-15
