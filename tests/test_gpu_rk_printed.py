"""GPU parity of the printed four-stage time scheme (Sec. 2.2.2, selbm_set_time_scheme(h, 1))
against the FP64 oracle: whole-element and population-split FP64 steps on the curved pipe
with walls, body force and filter; FP32 split steps on curved and affine hexahedra; graph
replays against eager launches; switching back to the Shu-Osher scheme.
"""
import math

import numpy as np
import pytest

import workloads as W
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


def random_continuous_state(o, amp, seed):
    rng = np.random.default_rng(seed)
    rho = 1 + 0.01 * rng.standard_normal(o.G)
    u = amp * rng.standard_normal((o.G, o.dim))
    f = o.initial_state(rho, u)
    return f + 1e-3 * o.t[:, None] * rng.standard_normal((o.Q, o.G))


def pipe_pair(P, monkeypatch, N, precision, split):
    monkeypatch.setenv("SELBM_SPLIT", "1" if split else "0")
    mesh = W.pipe_mesh(n_core=2, n_radial=2, n_axial=2 if N == 4 else 1, length=1.0)
    filt = {"shape": 0, "gamma": 0.1, "kc": float(N - 2)}
    g = (0.0, 0.0, 2e-4)
    o = OracleSELBM(mesh, "D3Q19", N, 2e-3, filt=filt, body_accel=g)
    s = P.SELBM(mesh, "D3Q19", N, 2e-3, precision=precision, filt=filt, body_accel=g)
    o.set_time_scheme(1)
    s.set_time_scheme(1)
    f = random_continuous_state(o, 0.02, 21)
    s.set_state(np.ascontiguousarray(o.to_local(f)))
    return o, s, f


@pytest.mark.parametrize("split", [False, True])
def test_printed_fp64_parity(P, monkeypatch, split):
    o, s, f = pipe_pair(P, monkeypatch, 4, 0, split)
    assert s.split == split
    f = o.step(f)
    s.step(1)
    assert rel(s.get_state(), o.to_local(f)) <= 1e-12
    f = o.run(f, 4)
    s.step(4)
    assert rel(s.get_state(), o.to_local(f)) <= 1e-11


@pytest.mark.parametrize("N", [4, 7])
def test_printed_fp32_split_curved(P, monkeypatch, N):
    o, s, f = pipe_pair(P, monkeypatch, N, P.FP32DEV, True)
    for _ in range(2):
        f = o.step(f)
        s.step(1)
        assert rel(s.get_state(), o.to_local(f)) <= 1e-6


def test_printed_fp32_split_affine_and_back(P):
    """Affine hexahedra N = 7 (the paired-axis passes with per-element coefficients); after
    two printed steps the handle and the oracle both go back to the Shu-Osher scheme."""
    L = 2 * math.pi
    mesh = W.box_mesh((2, 2, 2), (0, 0, 0), (L, L, L), (True, True, True))
    filt = {"shape": 0, "gamma": 0.1, "kc": 5.0}
    o = OracleSELBM(mesh, "D3Q27", 7, 1e-3, filt=filt)
    s = P.SELBM(mesh, "D3Q27", 7, 1e-3, precision=P.FP32DEV, filt=filt)
    o.set_time_scheme(1)
    s.set_time_scheme(1)
    f = random_continuous_state(o, 0.03, 22)
    s.set_state(np.ascontiguousarray(o.to_local(f)))
    for _ in range(2):
        f = o.step(f)
        s.step(1)
        assert rel(s.get_state(), o.to_local(f)) <= 1e-6
    o.set_time_scheme(0)
    s.set_time_scheme(0)
    f = o.step(f)
    s.step(1)
    assert rel(s.get_state(), o.to_local(f)) <= 1e-6


def test_printed_graph_matches_eager(P, monkeypatch):
    def run(no_graph):
        if no_graph:
            monkeypatch.setenv("SELBM_NO_GRAPH", "1")
        else:
            monkeypatch.delenv("SELBM_NO_GRAPH", raising=False)
        _, s, _ = pipe_pair(P, monkeypatch, 4, P.FP32DEV, True)
        s.step(6)
        return s.get_state()
    assert np.array_equal(run(False), run(True))


@pytest.mark.parametrize("split,precision,tol", [(False, 0, 1e-11), (True, 0, 1e-11), (True, 1, 1e-6)])
def test_weighted_scheme_moving_lid_box(P, monkeypatch, split, precision, tol):
    """Time scheme 2 (sources kept for the state arguments only) on a closed box with a moving
    lid and a body force: the difference stages run without F* and with the walls at rest."""
    monkeypatch.setenv("SELBM_SPLIT", "1" if split else "0")
    mesh = W.box_mesh((2, 3, 2), (0, 0, 0), (1, 1.5, 1), (False, False, False),
                      walls={0: 1, 1: 1, 2: 1, 3: 2, 4: 1, 5: 1}, wall_velocity=[[0, 0, 0], [0.02, 0, 0.01]])
    g = (1e-4, 0.0, -2e-4)
    o = OracleSELBM(mesh, "D3Q27", 5, 1e-2, body_accel=g)
    s = P.SELBM(mesh, "D3Q27", 5, 1e-2, precision=precision, body_accel=g)
    assert s.split == split
    o.set_time_scheme(2)
    s.set_time_scheme(2)
    f = random_continuous_state(o, 0.01, 23)
    s.set_state(np.ascontiguousarray(o.to_local(f)))
    for k in range(3):
        f = o.step(f)
        s.step(1)
        assert rel(s.get_state(), o.to_local(f)) <= tol, k
