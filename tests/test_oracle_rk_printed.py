"""Pins of the printed four-stage time scheme (Sec. 2.2.2, taken literally).

For a linear operator L (periodic mesh, no force, no walls) the printed stages equal the
fourth-order Taylor polynomial of exp(dt L) applied to f0, which is checked against repeated
applications of L; on pure advection the scheme converges in time at fourth order.  With a
force the printed combinations apply F* once per stage (the literal reading), which differs
from the Taylor polynomial; the step still conserves mass.
"""
import math

import numpy as np

import workloads as W
from oracle.selbm import OracleSELBM


def periodic_oracle(N=6, nu=0.01, g=None):
    L = 2 * np.pi
    mesh = W.box_mesh((2, 2), (0, 0), (L, L), (True, True))
    return OracleSELBM(mesh, "D2Q9", N, nu=nu, body_accel=g)


def test_printed_stages_are_the_fourth_order_taylor_polynomial():
    o = periodic_oracle()
    rng = np.random.default_rng(1)
    f0 = rng.standard_normal((o.Q, o.G))
    z = np.zeros_like(f0)
    terms, t = [f0], f0
    for k in range(1, 5):
        t = o.dt * o.rhs(t, z) / k
        terms.append(t)
    taylor = sum(terms)
    out = o.rk_printed(f0, z)
    assert np.abs(out - taylor).max() < 1e-13 * np.abs(f0).max()
    # and it is not the Shu-Osher step (which stops at the cubic term)
    assert np.abs(out - o.ssprk3(f0, z)).max() > 1e3 * 1e-13 * np.abs(f0).max()


def test_printed_scheme_fourth_order_in_time():
    L = 2 * np.pi
    mesh = W.box_mesh((2, 2), (0, 0), (L, L), (True, True))
    o = OracleSELBM(mesh, "D2Q9", 8, nu=0.01)
    f0 = np.tile(np.sin(o.Xg[:, 0] + 0.1)[None] * np.cos(o.Xg[:, 1])[None], (o.Q, 1))
    z = np.zeros_like(f0)
    T = 0.4

    def run(n):
        dt_save = o.dt
        o.dt = T / n
        f = f0.copy()
        for _ in range(n):
            f = o.rk_printed(f, z)
        o.dt = dt_save
        return f

    ref = run(256)
    errs = [np.abs(run(n) - ref).max() for n in (8, 16, 32)]
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(3.7 < r < 4.3 for r in rates), rates


def test_printed_scheme_step_conserves_mass_with_force():
    o = periodic_oracle(N=4, g=[2e-4, -1e-4])
    o.set_time_scheme(1)
    f = o.initial_state_from(W.shear_layer_init(U0=0.02, kappa=5.0))
    m0, _, _ = o.integrals(f)
    for _ in range(3):
        f = o.step(f)
    m1, _, _ = o.integrals(f)
    assert abs(m1 - m0) < 1e-13 * m0


def test_printed_stages_cancel_a_constant_source():
    """A uniform state under a uniform F*: every application of L returns F* (nothing to
    advect), and the printed stage weights 1/3 - 3/4 + 2/3 - 1/4 sum to zero, so the printed
    stages leave the state unchanged, while the Shu-Osher stages add dt F*."""
    o = periodic_oracle(N=4)
    f0 = np.tile(o.t[:, None], (1, o.G))
    Fs = np.tile((o.t * (o.e.astype(float) @ np.array([3e-4, -2e-4])) * 3.0)[:, None], (1, o.G))
    assert np.abs(o.rk_printed(f0, Fs) - f0).max() < 1e-15
    assert np.abs(o.ssprk3(f0, Fs) - (f0 + o.dt * Fs)).max() < 1e-15


def test_weighted_reading_fourth_order_with_source_and_steady_states():
    """Time scheme 2: the printed stages with L's source terms kept for the state arguments
    (f0, f0 - f1 + f2) and dropped for the differences.  Without sources it is the printed
    scheme; with a constant source it is fourth order in time; a steady state of L with a
    moving wall and a force is kept exactly (the literal reading moves it)."""
    o = periodic_oracle(N=8)
    rng = np.random.default_rng(4)
    f = rng.standard_normal((o.Q, o.G))
    z = np.zeros_like(f)
    assert np.array_equal(o.rk_printed(f, z, weighted=True), o.rk_printed(f, z))
    f0 = np.tile(np.sin(o.Xg[:, 0] + 0.1)[None] * np.cos(o.Xg[:, 1])[None], (o.Q, 1))
    b = 0.3 * np.tile((np.cos(o.Xg[:, 1]) + 0.2)[None], (o.Q, 1)) * o.t[:, None]
    T = 0.4

    def run(n):
        dt_save = o.dt
        o.dt = T / n
        g = f0.copy()
        for _ in range(n):
            g = o.rk_printed(g, b, weighted=True)
        o.dt = dt_save
        return g

    ref = run(256)
    errs = [np.abs(run(n) - ref).max() for n in (8, 16, 32)]
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(3.7 < r < 4.3 for r in rates), rates
    # steady state of L on a box with a moving lid
    c = W.couette_case()
    q = OracleSELBM(c.mesh, c.lattice, c.order, c.nu, cfl=c.cfl)
    fs = q.initial_state_from(c.init) + 1e-3 * q.t[:, None] * rng.standard_normal((q.Q, q.G))
    Fs = -q.rhs(fs, np.zeros_like(fs))
    assert np.array_equal(q.rk_printed(fs, Fs, weighted=True), fs)
    assert np.abs(q.rk_printed(fs, Fs) - fs).max() > 1e-6 * np.abs(fs).max()
