"""GPU parity of the node form of the mesh (selbm_create_nodes: GLL node coordinates of curved
isoparametric element maps + face connectivity with orientation codes, Sec. 2.2) against the
FP64 oracle on the same node mesh: curved elements that the corner form cannot express
(a smooth periodic deformation of a box, given at order-4 nodes), with element frames turned so
that non-zero orientation codes occur.  Tolerances as for the corner form: FP64 1e-12 after
one step and 1e-11 after five; FP32 deviations 1e-6 per step."""
import math

import numpy as np
import pytest

import workloads as W
from oracle import gll
from oracle.selbm import OracleSELBM

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_19171_gb300 import build
    build.build()
    import paper_2509_19171_gb300 as pkg
    return pkg


def rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def deformed_box(dim=3, walls=False):
    if dim == 3:
        mesh = W.box_mesh((2, 2, 2), (0, 0, 0), (1, 1, 1), (True, True, True))
        deform = lambda x: x + np.stack([0.03 * np.sin(2 * np.pi * x[:, 1]), 0.02 * np.sin(2 * np.pi * x[:, 2]),
                                          0.025 * np.sin(2 * np.pi * x[:, 0])], 1)
        rot = [2, 5]
    else:
        mesh = W.box_mesh((3, 2), (0, 0), (1, 1), (True, False), walls={2: 1, 3: 2},
                          wall_velocity=[[0, 0], [0.02, 0]])
        # periodic in x, the walls stay flat (the deformation vanishes at y = 0, 1)
        deform = lambda x: x + np.stack([0.04 * np.sin(np.pi * x[:, 1]) * np.cos(2 * np.pi * x[:, 0]),
                                          0.03 * np.sin(np.pi * x[:, 1]) * np.sin(2 * np.pi * x[:, 0])], 1)
        rot = [1, 4]
    return W.node_mesh(mesh, gll.gll_nodes(4), deform=deform, rotate=rot)


def random_state(o, amp, seed):
    rng = np.random.default_rng(seed)
    rho = 1 + 0.01 * rng.standard_normal(o.G)
    u = amp * rng.standard_normal((o.G, o.dim))
    return o.initial_state(rho, u) + 1e-3 * o.t[:, None] * rng.standard_normal((o.Q, o.G))


@pytest.mark.parametrize("lat,N", [("D3Q27", 5), ("D3Q19", 7)])
def test_nodes_curved_fp64(P, lat, N):
    nm = deformed_box()
    filt = {"shape": 0, "gamma": 0.1, "kc": float(N - 2)}
    o = OracleSELBM(nm, lat, N, 2e-3, filt=filt, body_accel=(0.0, 0.0, 1e-4))
    s = P.SELBM(nm, lat, N, 2e-3, filt=filt, body_accel=(0.0, 0.0, 1e-4))
    assert s.G == o.G and abs(s.dt - o.dt) < 1e-15
    f = random_state(o, 0.02, 3)
    s.set_state(np.ascontiguousarray(o.to_local(f)))
    f = o.step(f)
    s.step(1)
    assert rel(s.get_state(), o.to_local(f)) <= 1e-12
    f = o.run(f, 4)
    s.step(4)
    assert rel(s.get_state(), o.to_local(f)) <= 1e-11
    # the node coordinates the library interpolated are the oracle's
    assert np.abs(s.node_coords().reshape(o.E, o.Np, 3) - o.X).max() < 1e-13


@pytest.mark.parametrize("lat", ["D3Q19", "D3Q27"])
def test_nodes_curved_fp32_split(P, lat):
    """FP32 deviations, N = 7: the population-split step on curved elements (groups of 10 / 9
    populations with the per-node metric planes)."""
    nm = deformed_box()
    filt = {"shape": 0, "gamma": 0.1, "kc": 5.0}
    o = OracleSELBM(nm, lat, 7, 2e-3, filt=filt)
    s = P.SELBM(nm, lat, 7, 2e-3, precision=P.FP32DEV, filt=filt)
    assert s.split
    f = random_state(o, 0.02, 4)
    s.set_state(np.ascontiguousarray(o.to_local(f)))
    for _ in range(2):
        f = o.step(f)
        s.step(1)
        assert rel(s.get_state(), o.to_local(f)) <= 1e-6


def test_nodes_2d_walls_moving_lid(P):
    nm = deformed_box(dim=2)
    o = OracleSELBM(nm, "D2Q9", 6, 5e-3, filt={"shape": 1, "gamma": 0.1, "kc": 4.0})
    s = P.SELBM(nm, "D2Q9", 6, 5e-3, filt={"shape": 1, "gamma": 0.1, "kc": 4.0})
    f = random_state(o, 0.01, 5)
    s.set_state(np.ascontiguousarray(o.to_local(f)))
    for k in range(3):
        f = o.step(f)
        s.step(1)
        assert rel(s.get_state(), o.to_local(f)) <= 1e-12, k
