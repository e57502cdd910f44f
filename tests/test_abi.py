"""C-ABI checks that need no GPU: the library builds/loads, exports every
function declared in include/selbm.h, its host-side setup agrees with the
oracle's (unique-node count, assembled mass, wall surface), and bad meshes
or arguments are rejected before any device work."""
import os
import re

import numpy as np
import pytest

import workloads as W
from oracle.selbm import OracleSELBM

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def P():
    from paper_2509_19171_gb300 import build
    build.build()
    import paper_2509_19171_gb300 as pkg
    pkg.load_library()
    return pkg


def _declared(header):
    src = open(os.path.join(ROOT, "include", header)).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(selbm_\w+)\s*\(", src)))


def test_exports_every_declared_symbol(P):
    lib = P.load_library()
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            names += _declared(h)
    assert "selbm_create" in names and "selbm_step" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    assert set(P.EXPORTS) <= set(names)


@pytest.mark.parametrize("case,lat,N", [
    ("couette", "D2Q9", 4),
    ("box3", "D3Q27", 5),
    ("pipe", "D3Q19", 4),
    ("box_walls", "D3Q19", 3),
])
def test_setup_matches_oracle(P, case, lat, N):
    if case == "couette":
        mesh = W.couette_case().mesh
    elif case == "box3":
        mesh = W.box_mesh((3, 2, 2), (0, 0, 0), (1.5, 1, 1), (True, True, True))
    elif case == "pipe":
        mesh = W.pipe_mesh(n_core=2, n_radial=2, n_axial=2, length=1.0)
    else:
        mesh = W.box_mesh((2, 2, 2), (0, 0, 0), (1, 1, 1), (False, False, False),
                          walls={0: 1, 1: 1, 2: 1, 3: 1, 4: 1, 5: 2}, wall_velocity=[[0, 0, 0], [0.01, 0, 0]])
    info = P.mesh_check(mesh, lat, N)
    o = OracleSELBM(mesh, lat, N, nu=0.01)
    assert info["G"] == o.G
    assert info["Np"] == o.Np and info["Q"] == o.Q and info["E"] == o.E
    assert abs(info["measure"] - o.mass.sum()) < 1e-12 * o.mass.sum()
    assert abs(info["min_spacing"] * 0.5 - o.dt) < 1e-14
    area = sum(float(ws.sum()) for (_, _, _, ws, _) in o.walls)
    assert abs(info["wall_area"] - area) < 1e-12 * max(area, 1.0)
    assert info["wall_nodes"] == sum(len(nodes) for (_, nodes, _, _, _) in o.walls)
    assert info["affine"] == (case != "pipe")


def test_rejects_bad_meshes(P):
    mesh = W.box_mesh((2, 2), (0, 0), (1, 1), (True, True))
    bad = W.MeshSpec(**{**mesh.__dict__})
    bad.verts = mesh.verts[:, [1, 0, 3, 2], :].copy()          # mirrored corners -> J < 0
    with pytest.raises(P.SelbmError) as ei:
        P.mesh_check(bad, "D2Q9", 4)
    assert ei.value.code == -2
    with pytest.raises(P.SelbmError) as ei:
        P.mesh_check(mesh, "D3Q19", 4)                          # lattice/mesh dimension mismatch
    assert ei.value.code == -1
    with pytest.raises(P.SelbmError) as ei:
        P.mesh_check(mesh, "D2Q9", 15)                          # order out of range (2 <= N <= 14)
    assert ei.value.code == -1
    walls = W.box_mesh((2, 2), (0, 0), (1, 1), (True, False), walls={2: 3})
    walls.wall_velocity = np.zeros((1, 2))                      # wall id 3 > nwalls
    with pytest.raises(P.SelbmError) as ei:
        P.mesh_check(walls, "D2Q9", 4)
    assert ei.value.code == -2
    # selbm_create fails on the mesh before touching any device
    with pytest.raises(P.SelbmError) as ei:
        P.SELBM(bad, "D2Q9", 4, nu=0.01, stream=0)
    assert ei.value.code == -2


def test_single_element_periodic(P):
    """Degenerate mesh: one periodic element, every boundary node is its own neighbour."""
    mesh = W.box_mesh((1, 1), (0, 0), (1, 1), (True, True))
    info = P.mesh_check(mesh, "D2Q9", 5)
    assert info["G"] == 25
    o = OracleSELBM(mesh, "D2Q9", 5, nu=0.01)
    assert o.G == 25


def test_binding_constants_match_header(P):
    """The binding's copies of the header's size limits are the header's values."""
    src = open(os.path.join(ROOT, "include", "selbm.h")).read()
    defines = dict(re.findall(r"#define\s+(SELBM_\w+)\s+(\d+)", src))
    assert int(defines["SELBM_NOALLOC_MAX_ELEMS"]) == P.NOALLOC_MAX_ELEMS
    assert int(defines["SELBM_TIMER_KINDS"]) == P.TIMER_KINDS
