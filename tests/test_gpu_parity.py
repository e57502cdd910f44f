"""GPU (CUDA, sm_103a) parity against the FP64 oracle, through the C ABI.

Tolerances: FP64 path <= 1e-12 relative max-norm on the state after one step
and <= 1e-9 on rho and u after 1000 steps; FP32-deviation path within the
FP32 bound stated in each test.
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


def pair(P, mesh, lat, N, nu, precision=0, filt=None, g=(0.0, 0.0, 0.0), cfl=0.5, init=None):
    o = OracleSELBM(mesh, lat, N, nu, cfl=cfl, filt=filt, body_accel=g)
    s = P.SELBM(mesh, lat, N, nu, cfl=cfl, precision=precision, filt=filt, body_accel=g)
    assert abs(s.dt - o.dt) < 1e-15 and s.G == o.G
    e, t, _ = s.lattice_table()
    assert np.array_equal(e, o.e) and np.allclose(t, o.t, rtol=0, atol=1e-17)
    if init is not None:
        f = o.initial_state_from(init)
        s.init_from(init)
    return o, s


def rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def random_continuous_state(o, amp, seed):
    """Equilibrium at random (rho, u) plus a random non-equilibrium part, on unique nodes."""
    rng = np.random.default_rng(seed)
    rho = 1 + 0.01 * rng.standard_normal(o.G)
    u = amp * rng.standard_normal((o.G, o.dim))
    f = o.initial_state(rho, u)
    return f + 1e-3 * o.t[:, None] * rng.standard_normal((o.Q, o.G))


def check_one_step(P, o, s, f, tol):
    s.set_state(np.ascontiguousarray(o.to_local(f)))
    s.step(1)
    fo = o.step(f)
    fg = s.get_state()
    err = rel(fg, o.to_local(fo))
    assert err <= tol, err
    return fo


def test_couette_one_step_and_1000(P):
    c = W.couette_case()
    o, s = pair(P, c.mesh, c.lattice, c.order, c.nu, filt=c.filt, init=c.init)
    f = o.initial_state_from(c.init)
    f = o.step(f)
    s.step(1)
    assert rel(s.get_state(), o.to_local(f)) <= 1e-12
    f = o.run(f, 999)
    s.step(999)
    rho_o, u_o = o.moments(f)
    rho_g, u_g = s.moments()
    assert float(np.abs(rho_g - rho_o[o.glo]).max() / np.abs(rho_o).max()) <= 1e-9
    assert float(np.abs(u_g - u_o[o.glo]).max()) <= 1e-9 * c.U0


def test_shear_layer_filtered_random_state(P):
    """Periodic D2Q9, N=8, exponential filter (double shear layer geometry, 5x3 ragged)."""
    mesh = W.box_mesh((5, 3), (0, 0), (1, 1), (True, True))
    filt = {"shape": 1, "gamma": 0.1, "kc": 6.0, "p": 8.0}
    o, s = pair(P, mesh, "D2Q9", 8, 4e-6 * 100, filt=filt)
    f = random_continuous_state(o, 0.04, 1)
    f = check_one_step(P, o, s, f, 1e-12)
    # the filter of the last step is applied before the next collision: second step
    fo = o.step(f)
    s.step(1)
    assert rel(s.get_state(), o.to_local(fo)) <= 1e-12


def test_shear_layer_100_steps(P):
    mesh = W.box_mesh((4, 4), (0, 0), (1, 1), (True, True))
    case = W.shear_layer_case(n=4, order=8)
    o, s = pair(P, mesh, "D2Q9", 8, case.nu, filt=case.filt, init=case.init)
    f = o.run(o.initial_state_from(case.init), 100)
    s.step(100)
    rho_o, u_o = o.moments(f)
    rho_g, u_g = s.moments()
    assert float(np.abs(rho_g - rho_o[o.glo]).max()) <= 1e-9
    assert float(np.abs(u_g - u_o[o.glo]).max()) <= 1e-9 * case.U0
    d = s.diagnostics()
    m, mom, ke = o.integrals(f)
    assert abs(d[0] - m) <= 1e-12 * m and abs(d[4] - ke) <= 1e-9 * ke
    eps = o.dissipation(f)
    assert abs(d[5] - eps) <= 1e-9 * abs(eps)


@pytest.mark.parametrize("lat,N", [("D3Q19", 5), ("D3Q27", 5), ("D3Q27", 7), ("D3Q19", 7)])
def test_tgv3d_box_quadratic_filter(P, lat, N):
    L = 2 * math.pi
    shape = (3, 2, 2) if N == 5 else (2, 2, 2)
    mesh = W.box_mesh(shape, (0, 0, 0), (L, L, L), (True, True, True))
    filt = {"shape": 0, "gamma": 0.1, "kc": float(N - 2)}
    init = W.tgv3d_init(0.05)
    o, s = pair(P, mesh, lat, N, 0.05 / 1600, filt=filt, init=init)
    f = o.initial_state_from(init)
    f = o.step(f)
    s.step(1)
    assert rel(s.get_state(), o.to_local(f)) <= 1e-12
    f = o.run(f, 9)
    s.step(9)
    assert rel(s.get_state(), o.to_local(f)) <= 1e-11
    d = s.diagnostics()
    assert abs(d[5] - o.dissipation(f)) <= 1e-9 * abs(o.dissipation(f))


@pytest.mark.parametrize("N,prec", [(4, 0), (7, 0), (7, 1)])
def test_pipe_curved_walls_force(P, N, prec):
    """Curved isoparametric wall faces, flux bounce-back, body force (general metrics path);
    FP32 deviations (prec 1) within 1e-6 relative after one step."""
    mesh = W.pipe_mesh(n_core=2, n_radial=2, n_axial=2 if N == 4 else 1, length=1.0)
    g = (0.0, 0.0, 2e-4)
    o, s = pair(P, mesh, "D3Q19", N, 2e-3, precision=prec, filt={"shape": 0, "gamma": 0.1, "kc": float(N - 2)}, g=g)
    if prec == 1:
        f = random_continuous_state(o, 0.02, 2)
        check_one_step(P, o, s, f, 1e-6)
        return
    f = random_continuous_state(o, 0.02, 2)
    f = check_one_step(P, o, s, f, 1e-12)
    for _ in range(4):
        f = o.step(f)
    s.step(4)
    assert rel(s.get_state(), o.to_local(f)) <= 1e-11


def test_box_walls_on_all_faces(P):
    """Nodes on two and three wall faces (edges and corners of a closed box), moving lid."""
    mesh = W.box_mesh((2, 3, 2), (0, 0, 0), (1, 1.5, 1), (False, False, False),
                      walls={0: 1, 1: 1, 2: 1, 3: 2, 4: 1, 5: 1}, wall_velocity=[[0, 0, 0], [0.02, 0, 0.01]])
    o, s = pair(P, mesh, "D3Q27", 3, 1e-2)
    f = random_continuous_state(o, 0.01, 3)
    check_one_step(P, o, s, f, 1e-12)


def test_single_periodic_element(P):
    mesh = W.box_mesh((1, 1), (0, 0), (1, 1), (True, True))
    o, s = pair(P, mesh, "D2Q9", 6, 1e-2, filt={"shape": 0, "gamma": 0.2, "kc": 3.5})
    f = random_continuous_state(o, 0.02, 4)
    f = check_one_step(P, o, s, f, 1e-12)
    check_one_step(P, o, s, f, 1e-12)


@pytest.mark.parametrize("N", [2, 12, 14])
def test_extreme_orders(P, N):
    mesh = W.box_mesh((3, 2), (0, 0), (1, 1), (True, False), walls={2: 1, 3: 2},
                      wall_velocity=[[0, 0], [0.01, 0]])
    filt = {"shape": 0, "gamma": 0.1, "kc": 1.0} if N == 2 else {"shape": 1, "gamma": 0.1, "kc": float(N - 2)}
    o, s = pair(P, mesh, "D2Q9", N, 1e-2, filt=filt)
    f = random_continuous_state(o, 0.02, 5)
    f = check_one_step(P, o, s, f, 1e-12)
    check_one_step(P, o, s, f, 1e-12)


def test_zero_steps_roundtrip(P):
    mesh = W.box_mesh((2, 2), (0, 0), (1, 1), (True, True))
    o, s = pair(P, mesh, "D2Q9", 4, 1e-2, filt={"shape": 0, "gamma": 0.1, "kc": 2.0})
    f = random_continuous_state(o, 0.02, 6)
    s.set_state(np.ascontiguousarray(o.to_local(f)))
    s.step(0)
    assert rel(s.get_state(), o.to_local(f)) <= 1e-15


def test_generic_kernel_matches_oracle(P, monkeypatch):
    """The generic (runtime-order) stage kernel at an order that also has a register-blocked kernel."""
    monkeypatch.setenv("SELBM_GENERIC_KERNEL", "1")
    L = 2 * math.pi
    mesh = W.box_mesh((2, 2, 2), (0, 0, 0), (L, L, L), (True, True, True))
    o, s = pair(P, mesh, "D3Q27", 7, 1e-3, filt={"shape": 0, "gamma": 0.1, "kc": 5.0})
    f = random_continuous_state(o, 0.03, 8)
    f = check_one_step(P, o, s, f, 1e-12)
    check_one_step(P, o, s, f, 1e-12)


def test_graph_launch_matches_eager(P, monkeypatch):
    """Captured steps (CUDA graphs) give bit-identical states to eager launches."""
    mesh = W.box_mesh((3, 2), (0, 0), (1, 1), (True, False), walls={2: 1, 3: 2}, wall_velocity=[[0, 0], [0.01, 0]])
    filt = {"shape": 0, "gamma": 0.1, "kc": 6.0}
    init = W.shear_layer_init(U0=0.02, kappa=5.0)
    a = P.SELBM(mesh, "D2Q9", 8, 1e-3, filt=filt)
    monkeypatch.setenv("SELBM_NO_GRAPH", "1")
    b = P.SELBM(mesh, "D2Q9", 8, 1e-3, filt=filt)
    for h in (a, b):
        h.init_from(init)
        h.step(25)
    assert np.array_equal(a.get_state(), b.get_state())


def test_fp32_deviation_form(P):
    """FP32 deviations: f within 1e-6 relative after one step; rho, u within FP32 bounds after 100."""
    mesh = W.box_mesh((4, 4), (0, 0), (1, 1), (True, True))
    case = W.shear_layer_case(n=4, order=8)
    o, s = pair(P, mesh, "D2Q9", 8, case.nu, precision=P.FP32DEV, filt=case.filt, init=case.init)
    f = o.initial_state_from(case.init)
    f1 = o.step(f)
    s.step(1)
    assert rel(s.get_state(), o.to_local(f1)) <= 1e-6
    f = o.run(f1, 99)
    s.step(99)
    rho_o, u_o = o.moments(f)
    rho_g, u_g = s.moments()
    assert float(np.abs(rho_g - rho_o[o.glo]).max()) <= 1e-6
    assert float(np.abs(u_g - u_o[o.glo]).max()) <= 1e-4 * case.U0


@pytest.mark.parametrize("tau", [0.1, 0.4])
def test_poiseuille_walls_body_force(P, tau):
    """Planar Poiseuille of the slip study (Sec. 3.3): 4 x 4 quads, N = 8, flux bounce-back
    walls at y = 0, 1, body force G; the relaxation time tau = lambda / dt sets nu at the
    CFL-0.5 step.  Started on the parabola, 100 steps: FP64 state within 1e-11 of the oracle,
    and the wall slip the same on both sides."""
    mesh = W.box_mesh((4, 4), (0, 0), (1, 1), (True, False), walls={2: 1, 3: 1}, wall_velocity=[[0, 0]])
    probe = OracleSELBM(mesh, "D2Q9", 8, nu=1.0, cfl=0.5)
    nu = tau * probe.dt / 3.0
    umax = 0.1 / 3.0
    G = 8 * nu * umax
    init = W.poiseuille_init(G, nu)
    o, s = pair(P, mesh, "D2Q9", 8, nu, g=(G, 0.0, 0.0), init=init)
    f = o.run(o.initial_state_from(init), 100)
    s.step(100)
    assert rel(s.get_state(), o.to_local(f)) <= 1e-11
    _, u = o.moments(f)
    wall = np.abs(o.Xg[:, 1]) < 1e-12
    _, ug = s.moments()
    yl = s.node_coords()[..., 1].reshape(-1)
    slip_o = np.abs(u[wall, 0]).max() / umax
    slip_g = np.abs(ug.reshape(-1, 2)[np.abs(yl) < 1e-12, 0]).max() / umax
    assert slip_o > 0 and abs(slip_g - slip_o) <= 1e-9 * max(slip_o, 1e-3)


def test_stress_matches_oracle(P):
    """selbm_stress on a state set from the oracle (planar Poiseuille with walls and body force,
    100 steps from the parabola): the non-equilibrium second moment within 1e-9 of the oracle."""
    mesh = W.box_mesh((4, 4), (0, 0), (1, 1), (True, False), walls={2: 1, 3: 1}, wall_velocity=[[0, 0]])
    probe = OracleSELBM(mesh, "D2Q9", 8, nu=1.0, cfl=0.5)
    nu = 0.2 * probe.dt / 3.0
    G = 8 * nu * (0.1 / 3.0)
    init = W.poiseuille_init(G, nu)
    o, s = pair(P, mesh, "D2Q9", 8, nu, g=(G, 0.0, 0.0), init=init)
    f = o.run(o.initial_state_from(init), 100)
    s.set_state(np.ascontiguousarray(o.to_local(f)))
    pi_o = o.stress(f)[o.glo]
    pi_g = s.stress()
    assert rel(pi_g, pi_o) <= 1e-9


@pytest.mark.parametrize("prec", [0, 1])
def test_stress_with_force_field_mid_schedule(P, prec):
    """selbm_stress with a per-node acceleration field on top of the body force, read at a time
    where the field's factor A(t) = sin(2 pi t / period) is neither 0 nor 1 (t = 3 dt, period
    8 dt: A = 0.707), so the field enters the collision target f_bar^eq = f^eq - dt/2 F** of the
    stress with its current weight.  FP64 within 1e-9 of the oracle; FP32 deviations within
    1e-4 of max |Pi| (the storage rounding of g, ~1e-9, against Pi ~ 5e-5)."""
    mesh = W.box_mesh((4, 4), (0, 0), (1, 1), (True, False), walls={2: 1, 3: 1}, wall_velocity=[[0, 0]])
    probe = OracleSELBM(mesh, "D2Q9", 8, nu=1.0, cfl=0.5)
    nu = 0.2 * probe.dt / 3.0
    G = 8 * nu * (0.1 / 3.0)
    init = W.poiseuille_init(G, nu)
    o, s = pair(P, mesh, "D2Q9", 8, nu, precision=prec, g=(G, 0.0, 0.0), init=init)
    field = lambda x: np.stack([1e-2 * np.sin(2 * np.pi * x[:, 1]), 5e-3 * np.cos(2 * np.pi * x[:, 0])], 1)
    period = 8 * o.dt
    o.set_force_field(field(o.Xg), period, 1.0)
    s.set_force_field(field, period, 1.0)
    f = o.run(o.initial_state_from(init), 3)
    s.init_from(init)
    s.step(3)
    assert abs(o.amplitude(o.time) - math.sqrt(0.5)) < 1e-9
    s.set_state(np.ascontiguousarray(o.to_local(f)))
    pi_o = o.stress(f)[o.glo]
    pi_g = s.stress()
    # the field's part of the collision target is a visible part of Pi (5e-3 of it: a factor
    # A = 1 in place of 0.707 would be off by 1.6e-3, over both tolerances)
    o2 = OracleSELBM(mesh, "D2Q9", 8, nu=nu, body_accel=(G, 0.0))
    o2.time = o.time
    assert rel(o2.stress(f)[o2.glo], pi_o) > 3e-3
    assert rel(pi_g, pi_o) <= (1e-9 if prec == 0 else 1e-4)
