"""GPU parity of the per-node acceleration field (Sec. 4, pipe: the perturbation force
added to the body force for the first eddy turnover times) against the FP64 oracle:
the whole-element and population-split FP64 steps, the FP32 split step, the initial
state, the time schedule across graph replays, and removing the field.
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


def pipe_setup(P, monkeypatch, N, precision, split):
    """Curved pipe, walls, body force and the banded perturbation field (B0 = 5)."""
    monkeypatch.setenv("SELBM_SPLIT", "1" if split else "0")
    mesh = W.pipe_mesh(n_core=2, n_radial=2, n_axial=2, length=1.0)
    filt = {"shape": 0, "gamma": 0.1, "kc": float(N - 2)}
    g = (0.0, 0.0, 2e-4)
    o = OracleSELBM(mesh, "D3Q19", N, 2e-3, filt=filt, body_accel=g)
    s = P.SELBM(mesh, "D3Q19", N, 2e-3, precision=precision, filt=filt, body_accel=g)
    field = W.peng_forcing(2e-4, radius=1.0, length=1.0, kz=1, ktheta=2, B0=5.0)
    period, t_end = 8 * o.dt, 5.5 * o.dt
    o.set_force_field(field(o.Xg), period, t_end)
    s.set_force_field(field, period, t_end)
    rng = np.random.default_rng(11)
    rho = 1 + 0.01 * rng.standard_normal(o.G)
    u = 0.02 * rng.standard_normal((o.G, 3))
    f = o.initial_state(rho, u) + 1e-3 * o.t[:, None] * rng.standard_normal((o.Q, o.G))
    s.set_state(np.ascontiguousarray(o.to_local(f)))
    return o, s, f


@pytest.mark.parametrize("N,split", [(4, False), (4, True), (7, True)])
def test_field_fp64_parity(P, monkeypatch, N, split):
    o, s, f = pipe_setup(P, monkeypatch, N, 0, split)
    assert s.split == split
    for k in range(8):                   # the field rises, peaks, is cut off at t_end
        f = o.step(f)
        s.step(1)
        assert rel(s.get_state(), o.to_local(f)) <= 1e-11, k


def test_field_fp32_split_parity(P, monkeypatch):
    o, s, f = pipe_setup(P, monkeypatch, 4, P.FP32DEV, True)
    for k in range(8):
        f = o.step(f)
        s.step(1)
        assert rel(s.get_state(), o.to_local(f)) <= 1e-6, k


def test_field_changes_the_flow_and_can_be_removed(P, monkeypatch):
    """Without the field the pipe run differs (the field acts); after removing it both
    sides continue without it."""
    o, s, f = pipe_setup(P, monkeypatch, 4, 0, False)
    o_plain = OracleSELBM(o.mesh, "D3Q19", 4, 2e-3, filt=o.filt, body_accel=o.g)
    f_plain = f.copy()
    for _ in range(3):
        f = o.step(f)
        f_plain = o_plain.step(f_plain)
    s.step(3)
    assert rel(o.to_local(f), o.to_local(f_plain)) > 1e-9
    o.fS = None
    s.clear_force_field()
    for _ in range(3):
        f = o.step(f)
    s.step(3)
    assert rel(s.get_state(), o.to_local(f)) <= 1e-11


def test_field_in_initial_state(P, monkeypatch):
    """selbm_init takes the field at t = 0 (A = 1 for a constant field): a uniform field
    gives the same initial state and steps as the same body force."""
    monkeypatch.setenv("SELBM_SPLIT", "0")
    L = 2 * math.pi
    mesh = W.box_mesh((2, 2, 2), (0, 0, 0), (L, L, L), (True, True, True))
    g = np.array([3e-4, -1e-4, 2e-4])
    a = P.SELBM(mesh, "D3Q27", 4, 1e-3, body_accel=g)
    b = P.SELBM(mesh, "D3Q27", 4, 1e-3)
    b.set_force_field(lambda x: np.tile(g, (x.shape[0], 1)), 0.0, math.inf)
    init = W.tgv3d_init(0.05)
    a.init_from(init)
    b.init_from(init)
    assert rel(b.get_state(), a.get_state()) <= 1e-15
    a.step(3)
    b.step(3)
    assert rel(b.get_state(), a.get_state()) <= 1e-15
    o = OracleSELBM(mesh, "D3Q27", 4, 1e-3)
    o.set_force_field(np.tile(g, (o.G, 1)), 0.0, math.inf)
    f = o.run(o.initial_state_from(init), 3)
    assert rel(b.get_state(), o.to_local(f)) <= 1e-11


def test_field_schedule_graph_matches_eager(P, monkeypatch):
    """The time factor is computed on the device each step, so replays of the captured step
    follow the schedule: 12 steps as one call equal 12 eager steps bit for bit."""
    def run(no_graph):
        if no_graph:
            monkeypatch.setenv("SELBM_NO_GRAPH", "1")
        else:
            monkeypatch.delenv("SELBM_NO_GRAPH", raising=False)
        o, s, _ = pipe_setup(P, monkeypatch, 4, P.FP32DEV, True)
        s.step(12)
        return s.get_state()
    assert np.array_equal(run(False), run(True))
