"""GPU test of selbm_integrals_noalloc, the entry point for callers that cannot
let the library allocate device memory (an application whose memory pool has
already reserved the GPU, or a per-step monitoring hook in a time loop where
cudaMalloc/cudaFree would synchronise the device).  It must agree with the
handle-based selbm_diagnostics on the same state, on two calls in a row, and
reject element counts beyond its fixed scratch.

This file is named to be collected last, so a run that stops at the first
failure has already run every other test; it also passes on its own in a
fresh process (the first call on the device does the scratch address lookup).
"""
import ctypes as C
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
    lib = pkg.load_library()
    lib.selbm_integrals_noalloc.argtypes = [C.c_int32, C.c_int32, C.c_int32, C.c_void_p, C.c_void_p,
                                            C.c_double, C.c_void_p, C.c_void_p]
    lib.selbm_integrals_noalloc.restype = C.c_int
    return pkg


def _noalloc(P, torch, lat, s, f_dev, w_dev, out_dev):
    lib = P.load_library()
    stream = torch.cuda.current_stream().cuda_stream
    rc = lib.selbm_integrals_noalloc(lat, s.E, s.Np, C.c_void_p(f_dev.data_ptr()), C.c_void_p(w_dev.data_ptr()),
                                     1.0, C.c_void_p(out_dev.data_ptr()), C.c_void_p(stream))
    assert rc == 0
    torch.cuda.synchronize()
    return out_dev.cpu().numpy().copy()


def _compare(got, diag, tol):
    mass = diag[0]
    assert abs(got[0] - mass) <= tol * abs(mass)
    assert np.abs(got[1:4] - diag[1:4]).max() <= tol * abs(mass)
    assert abs(got[4] - diag[4]) <= tol * max(abs(diag[4]), 1e-300) + 1e-18 * abs(mass)
    assert got[5] == 0.0


@pytest.mark.parametrize("lattice,lat_id", [("D3Q27", 2), ("D2Q9", 0)])
def test_noalloc_matches_diagnostics_twice(P, lattice, lat_id):
    import torch
    if lattice == "D3Q27":
        L = 2 * math.pi
        mesh = W.box_mesh((3, 2, 2), (0, 0, 0), (L, L, L), (True, True, True))
        init, N, filt = W.tgv3d_init(0.05), 5, {"shape": 0, "gamma": 0.1, "kc": 3.0}
    else:
        mesh = W.box_mesh((4, 3), (0, 0), (1, 1), (True, False), walls={2: 1, 3: 2},
                          wall_velocity=[[0, 0], [0.01, 0]])
        init, N, filt = W.shear_layer_init(U0=0.02, kappa=5.0), 6, {"shape": 1, "gamma": 0.1, "kc": 4.0}
    s = P.SELBM(mesh, lattice, N, 1e-3, filt=filt)
    s.init_from(init)
    w = torch.from_numpy(OracleSELBM(mesh, lattice, N, 1e-3).wJ).cuda()   # quadrature weight per local node
    f = torch.empty((s.Q, s.E, s.Np), dtype=torch.float64, device="cuda")
    out = torch.full((6,), float("nan"), dtype=torch.float64, device="cuda")
    for call in range(2):
        s.step(3 + call)
        s.get_state(f)
        got = _noalloc(P, torch, lat_id, s, f, w, out)
        _compare(got, s.diagnostics(), 1e-12)


def test_noalloc_accepts_maximum(P):
    """nelem == SELBM_NOALLOC_MAX_ELEMS is the largest size the scratch holds: accepted, and
    the integrals of a state at rest (f = t_a rho, rho = 1 + 1e-3 k) with random weights
    equal their direct sums, on two calls in a row."""
    import torch
    lib = P.load_library()
    nelem, np_, Q = P.NOALLOC_MAX_ELEMS, 1, 9
    rng = np.random.default_rng(3)
    w = rng.uniform(0.5, 1.5, (nelem, np_))
    t = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
    for call in range(2):
        rho = 1 + 1e-3 * (call + 1) * rng.standard_normal((nelem, np_))
        f = torch.from_numpy(np.ascontiguousarray(t[:, None, None] * rho[None])).cuda()
        wd = torch.from_numpy(np.ascontiguousarray(w)).cuda()
        out = torch.full((6,), float("nan"), dtype=torch.float64, device="cuda")
        rc = lib.selbm_integrals_noalloc(0, nelem, np_, C.c_void_p(f.data_ptr()), C.c_void_p(wd.data_ptr()), 1.0,
                                         C.c_void_p(out.data_ptr()), C.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert rc == 0
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        mass = float((w * rho).sum())
        assert abs(got[0] - mass) <= 1e-12 * mass
        assert np.abs(got[1:5]).max() <= 1e-12 * mass and got[5] == 0.0


def test_noalloc_rejects_oversize(P):
    import torch
    lib = P.load_library()
    buf = torch.zeros(16, dtype=torch.float64, device="cuda")
    p = C.c_void_p(buf.data_ptr())
    too_many = P.NOALLOC_MAX_ELEMS + 1
    assert lib.selbm_integrals_noalloc(2, too_many, 1, p, p, 1.0, p, None) == -1
    assert lib.selbm_integrals_noalloc(2, 0, 1, p, p, 1.0, p, None) == -1
    assert lib.selbm_integrals_noalloc(7, 1, 1, p, p, 1.0, p, None) == -1
