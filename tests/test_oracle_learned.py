"""Pins of the learned-filter oracle: backprop against central finite differences,
the first Adam step's closed form, bfloat16 rounding, modal shell energies of single
modes, interpolation exactness for polynomials, element errors by direct quadrature."""
import numpy as np
import pytest

from oracle import geometry as geo
from oracle import gll
from oracle import learned as Lr


def test_backprop_matches_finite_differences():
    N, nin = 7, 16
    rng = np.random.default_rng(0)
    p = Lr.init_params(nin, seed=1) + 0.05 * rng.standard_normal(Lr.n_params(nin))
    s = rng.uniform(-1, 1, (13, nin))
    y = np.stack([rng.uniform(0, 0.5, 13), rng.uniform(2, N - 1, 13)], 1)
    loss, g = Lr.loss_and_grad(p, s, y, N)
    assert len(g) == Lr.n_params(nin) == 5378
    idx = rng.choice(len(p), 60, replace=False)
    h = 1e-6
    for i in idx:
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (Lr.loss_and_grad(pp, s, y, N)[0] - Lr.loss_and_grad(pm, s, y, N)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 + 1e-5 * abs(fd), (i, fd, g[i])


def test_adam_first_step_closed_form():
    """With m = v = 0 the bias-corrected first step is -lr * g / (|g| + eps)."""
    rng = np.random.default_rng(1)
    p = rng.standard_normal(50)
    g = rng.standard_normal(50)
    p1, m, v = Lr.adam_step(p, np.zeros(50), np.zeros(50), g, 1, 1e-3)
    assert np.allclose(p1, p - 1e-3 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_bf16_rounding():
    x = np.array([1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -9, -2.5, 3.0e-5, 0.0])
    r = Lr.bf16_round(x)
    assert r[0] == 1.0 and r[1] == 1.0                 # tie -> even
    assert r[2] == 1.0 + 2.0 ** -7                     # above the tie -> up
    assert r[3] == -2.5 and r[5] == 0.0
    rng = np.random.default_rng(2)
    z = rng.standard_normal(1000) * 10.0 ** rng.uniform(-4, 4, 1000)
    assert np.all(np.abs(Lr.bf16_round(z) - z) <= 2.0 ** -8 * np.abs(z) * (1 + 1e-6))   # 8 significant bits


@pytest.mark.parametrize("dim", [2, 3])
def test_shell_energy_of_single_modes(dim):
    N = 6
    xi = gll.gll_nodes(N)
    V = gll.modal_basis(N, xi)
    ijk = geo.node_index_grid(N, dim)
    for modes in ([3, 0, 0], [1, 5, 2], [0, 0, 6], [2, 2, 0]):
        modes = modes[:dim]
        q = np.prod([V[ijk[:, l], modes[l]] for l in range(dim)], axis=0)[None] * 0.7
        E = Lr.shell_energies(q, N, dim)[0]
        k = max(modes)
        assert abs(E[k] - 0.49) < 1e-12
        assert np.abs(np.delete(E, k)).max() < 1e-20


def test_interpolation_exact_for_polynomials():
    N, Nr, dim = 5, 9, 3
    rng = np.random.default_rng(3)
    c = rng.standard_normal((Nr + 1, 3))
    def poly(x):   # separable polynomial of degree Nr in each direction
        return np.prod([np.polyval(c[:, l], x[:, l]) for l in range(3)], axis=0)
    ijk_r = geo.node_index_grid(Nr, dim)
    xr = gll.gll_nodes(Nr)[ijk_r]
    ijk = geo.node_index_grid(N, dim)
    x = gll.gll_nodes(N)[ijk]
    q = poly(xr)[None]
    qi = Lr.interpolate_elements(q, Nr, N, dim)
    assert np.abs(qi[0] - poly(x)).max() < 1e-10 * np.abs(poly(x)).max()


def test_element_errors_quadrature():
    N, Nr, dim, E = 4, 8, 2, 3
    rng = np.random.default_rng(4)
    wJ = rng.uniform(0.5, 1.5, (E, (N + 1) ** 2))
    rho_r = rng.standard_normal((E, (Nr + 1) ** 2))
    u_r = rng.standard_normal((E, (Nr + 1) ** 2, 2))
    rho = Lr.interpolate_elements(rho_r, Nr, N, dim)
    u = np.stack([Lr.interpolate_elements(u_r[..., k], Nr, N, dim) for k in range(2)], -1)
    assert np.abs(Lr.element_errors(rho, u, rho_r, u_r, wJ, N, Nr, dim)).max() < 1e-24
    err = Lr.element_errors(rho + 0.1, u, rho_r, u_r, wJ, N, Nr, dim)
    assert np.allclose(err, 0.01 * wJ.sum(1), rtol=1e-12)


def test_outputs_to_filter_ranges():
    o = np.array([[-50.0, -50.0], [0.0, 0.0], [50.0, 50.0]])
    g, kc = Lr.outputs_to_filter(o, 7)
    assert np.all((g >= 0) & (g <= 0.5)) and abs(g[1] - 0.25) < 1e-15
    assert np.all((kc >= 2) & (kc <= 6)) and abs(kc[1] - 4.0) < 1e-15


def test_per_element_filters_conserve_mass():
    """Element-dependent transfer functions (kc >= 2) with the mass-weighted reconciliation of
    shared nodes keep the total mass and momentum on a periodic affine mesh (Sec. 2.4: filtering
    the distributions preserves the conserved moments); a plain mean of the copies would not."""
    import workloads as W
    from oracle.selbm import OracleSELBM
    mesh = W.box_mesh((3, 2), (0, 0), (1.5, 1), (True, True))
    o = OracleSELBM(mesh, "D2Q9", 6, 1e-3)
    rng = np.random.default_rng(7)
    f = o.initial_state(1 + 0.01 * rng.standard_normal(o.G), 0.03 * rng.standard_normal((o.G, 2)))
    f = f + 1e-3 * o.t[:, None] * rng.standard_normal((o.Q, o.G))
    sig = np.array([gll.filter_sigma(6, 0, g, k) for g, k in zip(rng.uniform(0.05, 0.5, o.E), rng.uniform(2, 5, o.E))])
    ff = o.apply_filter_elements(f, sig)
    m0, mom0, _ = o.integrals(f)
    m1, mom1, _ = o.integrals(ff)
    assert abs(m1 - m0) < 1e-14 * m0 and np.abs(mom1 - mom0).max() < 1e-15
    assert np.abs(ff - f).max() > 1e-6                     # the filters did act
