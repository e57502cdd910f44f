"""GPU parity of the pipe-flow statistics (Sec. 4) against the FP64 oracle, through the C ABI:
wall shear stress (selbm_wall_stress) and the radially binned mean velocity
(selbm_radial_profile), on straight and curved walls, FP64 and FP32 states."""
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


def _random_state(o, seed):
    rng = np.random.default_rng(seed)
    rho = 1 + 0.01 * rng.standard_normal(o.G)
    u = 0.02 * rng.standard_normal((o.G, o.dim))
    return o.initial_state(rho, u) + 1e-4 * o.t[:, None] * rng.standard_normal((o.Q, o.G))


CASES = {
    "channel": (lambda: W.box_mesh((2, 3, 2), (0, 0, 0), (1.0, 1.5, 1.0), (True, False, True), walls={2: 1, 3: 2},
                                   wall_velocity=[[0, 0, 0], [0.01, 0, 0]]), "D3Q27", 5),
    "pipe": (lambda: W.pipe_mesh(n_core=2, n_radial=2, n_axial=2, length=1.0), "D3Q19", 4),
}


@pytest.mark.parametrize("name", ["channel", "pipe"])
@pytest.mark.parametrize("prec", [0, 1])
def test_wall_stress_and_profile_match_oracle(P, name, prec):
    mk, lat, N = CASES[name]
    mesh = mk()
    o = OracleSELBM(mesh, lat, N, 2e-3)
    s = P.SELBM(mesh, lat, N, 2e-3, precision=prec)
    f = _random_state(o, 3)
    s.set_state(np.ascontiguousarray(o.to_local(f)))
    tol = 1e-12 if prec == 0 else 2e-5
    for d in ([1, 0, 0], [0, 0, 1], [1, 2, 3]):
        ref = o.wall_stress(f, d)
        got = s.wall_stress(d)
        assert abs(got - ref) <= tol * max(abs(ref), 1e-3 * 2e-3 * 0.02), (d, got, ref)
    origin, axis, radius, nb = ([0, 0, 0], [0, 0, 1], 1.0, 6) if name == "pipe" else ([0.5, 0.75, 0], [0, 0, 1], 0.9, 5)
    mean_o, mass_o = o.radial_profile(f, origin, axis, radius, nb)
    mean_g, mass_g = s.radial_profile(origin, axis, radius, nb)
    assert np.abs(mass_g - mass_o).max() <= 1e-13 * mass_o.sum()
    assert np.abs(mean_g - mean_o).max() <= tol * max(np.abs(mean_o).max(), 1e-3)


def test_stats_without_walls_and_bad_args(P):
    mesh = W.box_mesh((2, 2, 2), (0, 0, 0), (1, 1, 1), (True, True, True))
    s = P.SELBM(mesh, "D3Q19", 4, 1e-3)
    s.init_from(W.tgv3d_init(0.01))
    assert s.wall_stress([0, 0, 1]) == 0.0
    with pytest.raises(P.SelbmError):
        s.wall_stress([0, 0, 0])
    with pytest.raises(P.SelbmError):
        s.radial_profile([0, 0, 0], [0, 0, 1], 1.0, 0)
    with pytest.raises(P.SelbmError):
        s.radial_profile([0, 0, 0], [0, 0, 1], -1.0, 4)
