"""Pins of the oracle's node form of the mesh (Sec. 2.2: curved isoparametric elements given by
the GLL node coordinates of their maps, joined through face connectivity), and host-side
checks of the library's node-form setup against it.

* the element map interpolated from the given nodes is exact for maps of degree <= the
  given order (a polynomial deformation of a box);
* the numbering from face connectivity alone equals the numbering by coincident coordinates
  (periods included), with element frames turned so that non-zero orientation codes occur;
* turning element frames changes nothing physical: the oracle's step on the node form equals
  its step on the corner form node by node;
* the library's setup of the node form has the oracle's unique nodes and measure, and rejects
  inconsistent connectivity.
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import geometry as geo
from oracle import gll
from oracle.selbm import OracleSELBM


def test_map_interpolation_exact_for_polynomial_maps():
    Ng, N = 4, 7
    box = W.box_mesh((2, 1, 2), (0, 0, 0), (1.0, 0.5, 1.2), (False, False, False))
    deform = lambda x: x + 0.01 * np.stack([x[:, 1] ** 2 * x[:, 2], x[:, 0] ** 3, x[:, 0] * x[:, 1] ** 2], 1)
    nm = W.node_mesh(box, gll.gll_nodes(Ng), deform=deform)
    xi = gll.gll_nodes(N)
    X = geo.element_nodes_from_map(nm, xi)
    Xd = geo.element_nodes(box, xi)
    ref = deform(Xd.reshape(-1, 3)).reshape(Xd.shape)
    assert np.abs(X - ref).max() < 1e-14
    # degree N_g + 1 is not reproduced: the pin can fail
    deform5 = lambda x: x + 0.01 * np.stack([x[:, 1] ** 5, 0 * x[:, 0], 0 * x[:, 0]], 1)
    nm5 = W.node_mesh(box, gll.gll_nodes(Ng), deform=deform5)
    X5 = geo.element_nodes_from_map(nm5, xi)
    assert np.abs(X5 - deform5(Xd.reshape(-1, 3)).reshape(Xd.shape)).max() > 1e-8


@pytest.mark.parametrize("case", ["periodic3d", "walls2d", "periodic_single"])
def test_connectivity_numbering_equals_coordinate_numbering(case):
    if case == "periodic3d":
        mesh = W.box_mesh((2, 3, 2), (0, 0, 0), (1, 1.5, 1), (True, True, True))
        rot, Ng, N = [1, 4, 7, 10], 3, 5
    elif case == "walls2d":
        mesh = W.box_mesh((3, 2), (0, 0), (1, 1), (True, False), walls={2: 1, 3: 2},
                          wall_velocity=[[0, 0], [0.01, 0]])
        rot, Ng, N = [0, 4], 2, 6
    else:                          # one element periodic in x: it is its own neighbour
        mesh = W.box_mesh((1, 2, 2), (0, 0, 0), (1, 1, 1), (True, True, False))
        rot, Ng, N = [2], 2, 4
    nm = W.node_mesh(mesh, gll.gll_nodes(Ng), rotate=rot)
    if mesh.dim == 3:
        assert np.any(nm.face_orient != 0)
    X = geo.element_nodes_from_map(nm, gll.gll_nodes(N))
    glo_c = geo.global_numbering_connectivity(nm, N)
    glo_x = geo.global_numbering(X, mesh)
    assert np.array_equal(glo_c, glo_x)


def test_rotated_frames_give_the_same_step():
    """D3Q27 N=5, quadratic filter, random state: the node form with turned element frames and
    the corner form take the same step at every unique node (matched by coordinates)."""
    L = 2 * math.pi
    mesh = W.box_mesh((2, 2, 2), (0, 0, 0), (L, L, L), (True, True, True))
    N = 5
    nm = W.node_mesh(mesh, gll.gll_nodes(N), rotate=[0, 3, 5])
    filt = {"shape": 0, "gamma": 0.1, "kc": 3.0}
    oc = OracleSELBM(mesh, "D3Q27", N, 1e-3, filt=filt)
    on = OracleSELBM(nm, "D3Q27", N, 1e-3, filt=filt)
    assert oc.G == on.G and abs(oc.dt - on.dt) < 1e-15
    # node j of the node form <-> node perm[j] of the corner form (same coordinates)
    from scipy.spatial import cKDTree
    d, perm = cKDTree(oc.Xg).query(on.Xg)
    assert d.max() < 1e-12 and len(set(perm)) == oc.G
    init = W.tgv3d_init(0.05)
    fc = oc.initial_state_from(init)
    fn = on.initial_state_from(init)
    assert np.abs(fn - fc[:, perm]).max() < 1e-15
    for _ in range(2):
        fc, fn = oc.step(fc), on.step(fn)
    assert np.abs(fn - fc[:, perm]).max() < 1e-13 * np.abs(fc).max()


@pytest.fixture(scope="module")
def P():
    from paper_2509_19171_gb300 import build
    build.build()
    import paper_2509_19171_gb300 as pkg
    return pkg


def _deformed(periodic=True):
    mesh = W.box_mesh((2, 2, 2), (0, 0, 0), (1, 1, 1), (periodic,) * 3)
    deform = lambda x: x + np.stack([0.03 * np.sin(2 * np.pi * x[:, 1]), 0.02 * np.sin(2 * np.pi * x[:, 2]),
                                      0.025 * np.sin(2 * np.pi * x[:, 0])], 1)
    return mesh, W.node_mesh(mesh, gll.gll_nodes(4), deform=deform, rotate=[2, 5])


def test_library_setup_matches_oracle(P):
    _, nm = _deformed()
    for lat, N in (("D3Q27", 5), ("D3Q19", 7)):
        info = P.mesh_check(nm, lat, N)
        o = OracleSELBM(nm, lat, N, 1e-3)
        assert info["G"] == o.G and not info["affine"]
        assert abs(info["measure"] - o.mass.sum()) < 1e-12 * o.mass.sum()
        assert abs(info["min_spacing"] - geo.min_node_spacing(o.X, N, 3)) < 1e-12


def test_library_rejects_inconsistent_connectivity(P):
    import copy
    _, nm = _deformed()
    bad = copy.deepcopy(nm)
    f = int(np.nonzero(bad.face_nbr[0] >= 0)[0][0])
    bad.face_orient[0, f] = (int(bad.face_orient[0, f]) + 3) % 8          # orientation that does not fit
    with pytest.raises(P.SelbmError) as ei:
        P.mesh_check(bad, "D3Q27", 5)
    assert ei.value.code == -2
    bad = copy.deepcopy(nm)
    bad.face_nbr[0, f] = (int(bad.face_nbr[0, f]) + 1) % nm.nelem          # not mutual
    with pytest.raises(P.SelbmError):
        P.mesh_check(bad, "D3Q27", 5)
    bad = copy.deepcopy(nm)
    bad.bc[0, f] = 1                                                        # wall with a neighbour
    bad.wall_velocity = np.zeros((1, 3))
    with pytest.raises(P.SelbmError):
        P.mesh_check(bad, "D3Q27", 5)
