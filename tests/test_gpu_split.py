"""GPU parity of the population-split step (per-element prologue + split advection
stages) against the FP64 oracle.  The split form is the default for FP32 hexahedral
meshes; SELBM_SPLIT=1 selects it for FP64 as well, where the plain path's tolerances
(1e-12 after one step) apply to it unchanged.
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import learned as Lr
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


def split_pair(P, monkeypatch, mesh, lat, N, nu, precision=0, filt=None, g=(0.0, 0.0, 0.0)):
    monkeypatch.setenv("SELBM_SPLIT", "1")
    o = OracleSELBM(mesh, lat, N, nu, filt=filt, body_accel=g)
    s = P.SELBM(mesh, lat, N, nu, precision=precision, filt=filt, body_accel=g)
    assert s.split
    return o, s


@pytest.mark.parametrize("lat,N", [("D3Q19", 7), ("D3Q27", 5), ("D3Q27", 7)])
def test_split_tgv_filtered(P, monkeypatch, lat, N):
    L = 2 * math.pi
    mesh = W.box_mesh((3, 2, 2) if N == 5 else (2, 2, 2), (0, 0, 0), (L, L, L), (True, True, True))
    filt = {"shape": 0, "gamma": 0.1, "kc": float(N - 2)}
    o, s = split_pair(P, monkeypatch, mesh, lat, N, 0.05 / 1600, filt=filt)
    init = W.tgv3d_init(0.05)
    f = o.initial_state_from(init)
    s.init_from(init)
    f = o.step(f)
    s.step(1)
    assert rel(s.get_state(), o.to_local(f)) <= 1e-12
    f = o.run(f, 9)
    s.step(9)
    assert rel(s.get_state(), o.to_local(f)) <= 1e-11


@pytest.mark.parametrize("N", [4, 7])
def test_split_pipe_curved_walls_force(P, monkeypatch, N):
    """Curved elements, flux bounce-back (opposite population from the unique array), body force."""
    mesh = W.pipe_mesh(n_core=2, n_radial=2, n_axial=2 if N == 4 else 1, length=1.0)
    o, s = split_pair(P, monkeypatch, mesh, "D3Q19", N, 2e-3, filt={"shape": 0, "gamma": 0.1, "kc": float(N - 2)},
                      g=(0.0, 0.0, 2e-4))
    f = random_continuous_state(o, 0.02, 2)
    s.set_state(np.ascontiguousarray(o.to_local(f)))
    f = o.step(f)
    s.step(1)
    assert rel(s.get_state(), o.to_local(f)) <= 1e-12
    f = o.run(f, 4)
    s.step(4)
    assert rel(s.get_state(), o.to_local(f)) <= 1e-11


def test_split_unfiltered_closed_box(P, monkeypatch):
    """No filter (collision on unique nodes), walls on every face, moving lid."""
    mesh = W.box_mesh((2, 3, 2), (0, 0, 0), (1, 1.5, 1), (False, False, False),
                      walls={0: 1, 1: 1, 2: 1, 3: 2, 4: 1, 5: 1}, wall_velocity=[[0, 0, 0], [0.02, 0, 0.01]])
    o, s = split_pair(P, monkeypatch, mesh, "D3Q27", 5, 1e-2)
    f = random_continuous_state(o, 0.01, 3)
    s.set_state(np.ascontiguousarray(o.to_local(f)))
    for k in range(3):
        f = o.step(f)
        s.step(1)
        assert rel(s.get_state(), o.to_local(f)) <= 1e-12, k


@pytest.mark.parametrize("lat,N", [("D3Q27", 7), ("D3Q27", 5), ("D3Q19", 7), ("D3Q19", 4)])
def test_split_fp32_default_and_accuracy(P, lat, N):
    """FP32 hexahedral handles take the split form by default at every compiled order; each
    step within 1e-6 of the FP64 oracle."""
    L = 2 * math.pi
    mesh = W.box_mesh((2, 2, 2), (0, 0, 0), (L, L, L), (True, True, True))
    filt = {"shape": 0, "gamma": 0.1, "kc": float(N - 2)}
    o = OracleSELBM(mesh, lat, N, 1e-3, filt=filt)
    s = P.SELBM(mesh, lat, N, 1e-3, precision=P.FP32DEV, filt=filt)
    assert s.split
    f = random_continuous_state(o, 0.03, 8)
    s.set_state(np.ascontiguousarray(o.to_local(f)))
    for _ in range(2):
        f = o.step(f)
        s.step(1)
        assert rel(s.get_state(), o.to_local(f)) <= 1e-6


def test_split_graph_matches_eager(P, monkeypatch):
    L = 2 * math.pi
    mesh = W.box_mesh((2, 2, 2), (0, 0, 0), (L, L, L), (True, True, True))
    filt = {"shape": 0, "gamma": 0.1, "kc": 5.0}
    init = W.tgv3d_init(0.05)
    a = P.SELBM(mesh, "D3Q27", 7, 1e-3, precision=P.FP32DEV, filt=filt)
    monkeypatch.setenv("SELBM_NO_GRAPH", "1")
    b = P.SELBM(mesh, "D3Q27", 7, 1e-3, precision=P.FP32DEV, filt=filt)
    for h in (a, b):
        h.init_from(init)
        h.step(12)
    assert np.array_equal(a.get_state(), b.get_state())


def _smooth_state(o, seed):
    rng = np.random.default_rng(seed)
    X = o.Xg
    k = rng.integers(1, 3, (3, o.dim))
    u = np.stack([0.03 * np.sin(X @ k[c] + c) for c in range(o.dim)], 1) + 1e-4 * rng.standard_normal((o.G, o.dim))
    rho = 1 + 1e-3 * np.cos(X @ k[0]) + 1e-5 * rng.standard_normal(o.G)
    return o.initial_state(rho, u)


def test_split_learned_parity_and_fallback(P, monkeypatch):
    """Learned control inside the prologue (features, network, per-element filter, collision
    of interior nodes; assembly + collision of shared nodes), then the drift fallback."""
    mesh = W.box_mesh((2, 2, 2), (0, 0, 0), (2 * math.pi,) * 3, (True, True, True))
    N = 5
    filt = {"shape": 0, "gamma": 0.1, "kc": float(N - 2)}
    o, s = split_pair(P, monkeypatch, mesh, "D3Q27", N, 1e-3, filt=filt)
    f = _smooth_state(o, 6)
    rho, u = o.moments(f)
    x = Lr.features(rho[o.glo], u[o.glo], 1.0, N, o.dim)
    lo, hi = np.full(x.shape[1], -35.0), np.full(x.shape[1], 5.0)
    params = np.float64(np.float32(Lr.init_params(x.shape[1], seed=11) * 1.5))
    s.set_learned_filter(params, lo, hi, mass_bound=1.0, ke_bound=1.0)
    s.set_state(np.ascontiguousarray(o.to_local(f)))
    for k in range(3):
        f = o.step_learned(f, params, lo, hi)
        s.step(1)
        assert rel(s.get_state(), o.to_local(f)) <= 1e-10, k
    assert s.learned_status()["fixed_element_steps"] == 0
    # drift fallback: a negative bound trips at the first comparison (learned filters in the
    # first two steps, the fixed filter afterwards)
    o2, s2 = split_pair(P, monkeypatch, mesh, "D3Q27", N, 1e-3, filt=filt)
    s2.set_learned_filter(params, lo, hi, mass_bound=-1.0, ke_bound=1.0)
    g = _smooth_state(o2, 6)
    s2.set_state(np.ascontiguousarray(o2.to_local(g)))
    g = o2.step_learned(g, params, lo, hi)
    g = o2.step_learned(g, params, lo, hi)
    g = o2.step(o2.step(g))
    s2.step(4)
    assert rel(s2.get_state(), o2.to_local(g)) <= 1e-10
    assert s2.learned_status()["fallback_flag"] == 1


def test_split_fp32_walls_every_face(P):
    """FP32 N = 7 on an affine box with walls on every face (moving lid): the register-blocked
    split stage path plus flux bounce-back, within 1e-6 of the FP64 oracle per step."""
    mesh = W.box_mesh((2, 2, 2), (0, 0, 0), (1, 1, 1), (False, False, False),
                      walls={0: 1, 1: 1, 2: 1, 3: 2, 4: 1, 5: 1}, wall_velocity=[[0, 0, 0], [0.02, 0, 0.01]])
    filt = {"shape": 0, "gamma": 0.1, "kc": 5.0}
    o = OracleSELBM(mesh, "D3Q27", 7, 1e-2, filt=filt)
    s = P.SELBM(mesh, "D3Q27", 7, 1e-2, precision=P.FP32DEV, filt=filt)
    assert s.split
    f = random_continuous_state(o, 0.01, 5)
    s.set_state(np.ascontiguousarray(o.to_local(f)))
    for _ in range(3):
        f = o.step(f)
        s.step(1)
        assert rel(s.get_state(), o.to_local(f)) <= 1e-6


@pytest.mark.parametrize("N", [4, 7])
def test_split_fp32_curved_pipe(P, N):
    """FP32 curved elements (per-node metrics), flux bounce-back and body force in the
    split form, D3Q19 N = 4 and 7 (the paired-axis passes with metric planes), within 1e-6
    of the FP64 oracle over two steps."""
    mesh = W.pipe_mesh(n_core=2, n_radial=2, n_axial=2 if N == 4 else 1, length=1.0)
    filt = {"shape": 0, "gamma": 0.1, "kc": float(N - 2)}
    g = (0.0, 0.0, 2e-4)
    o = OracleSELBM(mesh, "D3Q19", N, 2e-3, filt=filt, body_accel=g)
    s = P.SELBM(mesh, "D3Q19", N, 2e-3, precision=P.FP32DEV, filt=filt, body_accel=g)
    assert s.split
    f = random_continuous_state(o, 0.02, 9)
    s.set_state(np.ascontiguousarray(o.to_local(f)))
    for _ in range(2):
        f = o.step(f)
        s.step(1)
        assert rel(s.get_state(), o.to_local(f)) <= 1e-6
