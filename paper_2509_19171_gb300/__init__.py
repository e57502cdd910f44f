"""Python binding of libselbm.so (include/selbm.h): the filtered spectral-element
lattice Boltzmann method with flux bounce-back walls on one GB300 GPU.

Argument marshalling only: every step of the method runs in the CUDA library.
PyTorch supplies device memory and the CUDA stream.  There is no CPU fallback:
if ``libselbm.so`` is missing this module raises on import of the library
(build it with ``python -m paper_2509_19171_gb300.build``).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libselbm.so")

D2Q9, D3Q19, D3Q27 = 0, 1, 2
LATTICES = {"D2Q9": D2Q9, "D3Q19": D3Q19, "D3Q27": D3Q27}
FP64, FP32DEV = 0, 1
TIMER_KINDS = 5
NOALLOC_MAX_ELEMS = 65536          # SELBM_NOALLOC_MAX_ELEMS of include/selbm.h
TIMER_NAMES = ["stage1", "stage23", "assembly", "learned", "prologue"]
OK_FALLBACK = 1                   # positive status: OK, the learned control's drift fallback is engaged
ERRORS = {1: "OK_FALLBACK", 0: "OK", -1: "ERR_ARG", -2: "ERR_MESH", -3: "ERR_CUDA", -4: "ERR_NONFINITE", -5: "ERR_TIMEOUT", -6: "ERR_STATE"}

# functions declared in include/selbm.h (checked by the ABI test)
EXPORTS = ["selbm_create", "selbm_create_nodes", "selbm_mesh_check_nodes", "selbm_destroy", "selbm_last_error", "selbm_info", "selbm_lattice_table",
           "selbm_node_coords", "selbm_init", "selbm_set_state", "selbm_get_state", "selbm_step",
           "selbm_moments", "selbm_stress", "selbm_set_filter", "selbm_set_body_force", "selbm_set_force_field", "selbm_set_time_scheme",
           "selbm_diagnostics", "selbm_sync",
           "selbm_wall_stress", "selbm_radial_profile",
           "selbm_mesh_check", "selbm_timers", "selbm_timers_read", "selbm_set_learned_filter",
           "selbm_clear_learned_filter", "selbm_learned_status", "selbm_element_sigma", "selbm_features",
           "selbm_element_errors", "selbm_mlp_nparams", "selbm_mlp_grad", "selbm_mlp_forward", "selbm_mlp_train"]


class SelbmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class MeshC(C.Structure):
    _fields_ = [("dim", C.c_int32), ("nelem", C.c_int32), ("verts", C.POINTER(C.c_double)),
                ("curved", C.POINTER(C.c_int32)), ("face_bc", C.POINTER(C.c_int32)),
                ("period", C.POINTER(C.c_double)), ("origin", C.POINTER(C.c_double)),
                ("nwalls", C.c_int32), ("wall_velocity", C.POINTER(C.c_double)), ("radius", C.c_double)]


class MeshNodesC(C.Structure):
    _fields_ = [("dim", C.c_int32), ("nelem", C.c_int32), ("order", C.c_int32), ("xyz", C.POINTER(C.c_double)),
                ("face_nbr", C.POINTER(C.c_int32)), ("face_nbr_face", C.POINTER(C.c_int8)),
                ("face_orient", C.POINTER(C.c_int8)), ("face_bc", C.POINTER(C.c_int32)), ("nwalls", C.c_int32),
                ("wall_velocity", C.POINTER(C.c_double))]


class FilterC(C.Structure):
    _fields_ = [("shape", C.c_int32), ("gamma", C.c_double), ("kc", C.c_double), ("p", C.c_double)]


class ParamsC(C.Structure):
    _fields_ = [("lattice", C.c_int32), ("order", C.c_int32), ("nu", C.c_double), ("dt", C.c_double),
                ("cfl", C.c_double), ("rho0", C.c_double), ("precision", C.c_int32), ("filter", FilterC),
                ("body_accel", C.c_double * 3)]


_lib = None


def load_library(path: str = LIB_PATH):
    """Load libselbm.so (raises if it is absent: no fallback path exists)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with `python -m paper_2509_19171_gb300.build`")
    lib = C.CDLL(path)
    P, I, D, I64 = C.c_void_p, C.c_int, C.POINTER(C.c_double), C.c_int64
    lib.selbm_create.argtypes = [C.POINTER(MeshC), C.POINTER(ParamsC), P, C.POINTER(P)]
    lib.selbm_create_nodes.argtypes = [C.POINTER(MeshNodesC), C.POINTER(ParamsC), P, C.POINTER(P)]
    lib.selbm_mesh_check_nodes.argtypes = [C.POINTER(MeshNodesC), C.c_int32, C.c_int32, C.POINTER(C.c_int64), D]
    lib.selbm_destroy.argtypes = [P]
    lib.selbm_destroy.restype = None
    lib.selbm_last_error.argtypes = [P]
    lib.selbm_last_error.restype = C.c_char_p
    lib.selbm_info.argtypes = [P, C.POINTER(C.c_int64), D]
    lib.selbm_lattice_table.argtypes = [P, C.POINTER(C.c_int32), D, C.POINTER(C.c_int32)]
    lib.selbm_node_coords.argtypes = [P, D]
    lib.selbm_init.argtypes = [P, P, P, I]
    lib.selbm_set_state.argtypes = [P, P, I]
    lib.selbm_get_state.argtypes = [P, P, I]
    lib.selbm_step.argtypes = [P, I64]
    lib.selbm_moments.argtypes = [P, P, P, I]
    lib.selbm_stress.argtypes = [P, P, I]
    lib.selbm_set_filter.argtypes = [P, C.POINTER(FilterC)]
    lib.selbm_set_body_force.argtypes = [P, D]
    lib.selbm_set_force_field.argtypes = [P, P, C.c_double, C.c_double]
    lib.selbm_set_time_scheme.argtypes = [P, I]
    lib.selbm_diagnostics.argtypes = [P, D]
    lib.selbm_wall_stress.argtypes = [P, D, D]
    lib.selbm_radial_profile.argtypes = [P, D, D, C.c_double, I, D, D]
    lib.selbm_sync.argtypes = [P]
    F = C.POINTER(C.c_float)
    lib.selbm_set_learned_filter.argtypes = [P, F, F, F, C.c_double, C.c_double]
    lib.selbm_clear_learned_filter.argtypes = [P]
    lib.selbm_learned_status.argtypes = [P, C.POINTER(C.c_int64)]
    lib.selbm_element_sigma.argtypes = [P, D]
    lib.selbm_features.argtypes = [P, P]
    lib.selbm_element_errors.argtypes = [P, P, P]
    lib.selbm_mlp_nparams.argtypes = [C.c_int32]
    lib.selbm_mlp_grad.argtypes = [P, C.c_int32, C.c_int32, P, P, C.c_int64, P, P, P]
    lib.selbm_mlp_forward.argtypes = [P, C.c_int32, C.c_int32, P, C.c_int64, C.c_int32, P, P]
    lib.selbm_mlp_train.argtypes = [P, P, P, C.c_int32, C.c_int32, P, P, C.c_int64, C.c_int32, C.c_int32,
                                    C.c_float, C.c_uint64, C.POINTER(C.c_int64), F, P]
    lib.selbm_timers.argtypes = [P, I]
    lib.selbm_timers_read.argtypes = [P, D, C.POINTER(C.c_int64)]
    lib.selbm_mesh_check.argtypes = [C.POINTER(MeshC), C.c_int32, C.c_int32, C.POINTER(C.c_int64), D]
    for name in EXPORTS:
        if name not in ("selbm_destroy", "selbm_last_error"):
            getattr(lib, name).restype = C.c_int
    _lib = lib
    return lib


def _dptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _ptr_of(x):
    """(pointer, on_device) for a numpy array (host) or a torch tensor (host or CUDA)."""
    if isinstance(x, np.ndarray):
        assert x.dtype == np.float64 and x.flags["C_CONTIGUOUS"]
        return C.c_void_p(x.ctypes.data), 0
    import torch
    assert isinstance(x, torch.Tensor) and x.dtype == torch.float64 and x.is_contiguous()
    return C.c_void_p(x.data_ptr()), int(x.is_cuda)


def filter_struct(f) -> FilterC:
    f = f or {}
    return FilterC(int(f.get("shape", 0)), float(f.get("gamma", 0.0)), float(f.get("kc", 1.0)), float(f.get("p", 8.0)))


def mesh_struct(mesh):
    """(MeshC, keep-alive list) for a workloads.MeshSpec-like object."""
    dim = int(mesh.dim)
    keep = [np.ascontiguousarray(mesh.verts, np.float64),
            np.ascontiguousarray(mesh.curved, np.int32),
            np.ascontiguousarray(mesh.bc, np.int32),
            np.ascontiguousarray(mesh.period, np.float64),
            np.ascontiguousarray(mesh.origin, np.float64),
            np.ascontiguousarray(np.asarray(mesh.wall_velocity, np.float64).reshape(-1, dim))]
    v, cu, bc, per, org, wv = keep
    m = MeshC(dim, int(v.shape[0]), _dptr(v), cu.ctypes.data_as(C.POINTER(C.c_int32)),
              bc.ctypes.data_as(C.POINTER(C.c_int32)), _dptr(per), _dptr(org), int(wv.shape[0]),
              _dptr(wv) if wv.size else None, float(getattr(mesh, "radius", 0.0)))
    return m, keep


def mesh_nodes_struct(mesh):
    """(MeshNodesC, keep-alive list) for a workloads.NodeMeshSpec-like object."""
    dim = int(mesh.dim)
    keep = [np.ascontiguousarray(mesh.xyz, np.float64), np.ascontiguousarray(mesh.face_nbr, np.int32),
            np.ascontiguousarray(mesh.face_nbr_face, np.int8), np.ascontiguousarray(mesh.face_orient, np.int8),
            np.ascontiguousarray(mesh.bc, np.int32),
            np.ascontiguousarray(np.asarray(mesh.wall_velocity, np.float64).reshape(-1, dim))]
    x, nb, nf, no, bc, wv = keep
    m = MeshNodesC(dim, int(x.shape[0]), int(mesh.order), _dptr(x), nb.ctypes.data_as(C.POINTER(C.c_int32)),
                   nf.ctypes.data_as(C.POINTER(C.c_int8)), no.ctypes.data_as(C.POINTER(C.c_int8)),
                   bc.ctypes.data_as(C.POINTER(C.c_int32)), int(wv.shape[0]), _dptr(wv) if wv.size else None)
    return m, keep


def _is_node_mesh(mesh):
    return hasattr(mesh, "xyz") and hasattr(mesh, "face_nbr")


def mesh_check(mesh, lattice, order):
    """Host-only dry run of the setup: dict of sizes and integrals (no GPU needed).  ``mesh`` is
    a corner mesh (workloads.MeshSpec) or a node mesh (workloads.NodeMeshSpec)."""
    lib = load_library()
    node = _is_node_mesh(mesh)
    m, keep = mesh_nodes_struct(mesh) if node else mesh_struct(mesh)
    ii = (C.c_int64 * 6)()
    dd = (C.c_double * 4)()
    lat = LATTICES[lattice] if isinstance(lattice, str) else int(lattice)
    check = lib.selbm_mesh_check_nodes if node else lib.selbm_mesh_check
    rc = check(C.byref(m), lat, int(order), ii, dd)
    if rc != 0:
        raise SelbmError(rc, lib.selbm_last_error(None).decode())
    del keep
    return {"E": ii[0], "Np": ii[1], "Q": ii[2], "G": ii[3], "Gb": ii[4], "affine": bool(ii[5]),
            "min_spacing": dd[0], "measure": dd[1], "wall_nodes": int(dd[2]), "wall_area": dd[3]}


class SELBM:
    """One simulation handle.  ``mesh`` is a ``workloads.MeshSpec``-like object
    (dim, verts, curved, bc, period, origin, wall_velocity, radius) or a
    ``workloads.NodeMeshSpec``-like one (dim, order, xyz, face_nbr, face_nbr_face,
    face_orient, bc, wall_velocity)."""

    def __init__(self, mesh, lattice, order, nu, cfl=0.5, dt=0.0, rho0=1.0, precision=FP64,
                 filt=None, body_accel=(0.0, 0.0, 0.0), stream=None):
        self.lib = load_library()
        dim = int(mesh.dim)
        node = _is_node_mesh(mesh)
        m, self._keep = mesh_nodes_struct(mesh) if node else mesh_struct(mesh)
        g = list(body_accel) + [0.0] * (3 - len(body_accel))
        lat = LATTICES[lattice] if isinstance(lattice, str) else int(lattice)
        p = ParamsC(lat, int(order), float(nu), float(dt), float(cfl), float(rho0), int(precision),
                    filter_struct(filt), (C.c_double * 3)(*g[:3]))
        if stream is None:
            try:
                import torch
                stream = torch.cuda.current_stream().cuda_stream if torch.cuda.is_available() else 0
            except ImportError:
                stream = 0
        self.stream = stream
        h = C.c_void_p()
        create = self.lib.selbm_create_nodes if node else self.lib.selbm_create
        rc = create(C.byref(m), C.byref(p), C.c_void_p(stream), C.byref(h))
        if rc != 0:
            raise SelbmError(rc, self.lib.selbm_last_error(None).decode())
        self.h = h
        self.dim = dim
        self._info()

    def _check(self, rc):
        """Raise on a negative status; 0 and the positive OK_FALLBACK pass through."""
        if rc < 0:
            raise SelbmError(rc, self.lib.selbm_last_error(self.h).decode())
        return rc

    def _info(self):
        ii = (C.c_int64 * 9)()
        dd = (C.c_double * 4)()
        self._check(self.lib.selbm_info(self.h, ii, dd))
        self.E, self.Np, self.Q, self.G, _, self.N, self.precision, self.steps, split = [int(x) for x in ii]
        self.split = bool(split)
        self.dt, self.tau, self.lam, self.time = [float(x) for x in dd]
        return self

    def close(self):
        if getattr(self, "h", None):
            self.lib.selbm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ----------------------------------------------------------------- tables
    def lattice_table(self):
        e = np.zeros((self.Q, 3), np.int32)
        t = np.zeros(self.Q)
        o = np.zeros(self.Q, np.int32)
        self._check(self.lib.selbm_lattice_table(self.h, e.ctypes.data_as(C.POINTER(C.c_int32)), _dptr(t),
                                                 o.ctypes.data_as(C.POINTER(C.c_int32))))
        return e[:, : self.dim], t, o

    def node_coords(self):
        x = np.zeros((self.E, self.Np, self.dim))
        self._check(self.lib.selbm_node_coords(self.h, _dptr(x)))
        return x

    # ------------------------------------------------------------------ state
    def init(self, rho, u):
        pr, dev = _ptr_of(rho)
        pu, _ = _ptr_of(u)
        self._check(self.lib.selbm_init(self.h, pr, pu, dev))

    def init_from(self, fn):
        """Evaluate a closed-form initial field fn(x[n, dim]) -> (rho, u) at the nodes."""
        x = self.node_coords().reshape(-1, self.dim)
        rho, u = fn(x)
        self.init(np.ascontiguousarray(rho, np.float64), np.ascontiguousarray(u[:, : self.dim], np.float64))

    def set_state(self, f):
        pf, dev = _ptr_of(f)
        self._check(self.lib.selbm_set_state(self.h, pf, dev))

    def get_state(self, out=None):
        if out is None:
            out = np.zeros((self.Q, self.E, self.Np))
        pf, dev = _ptr_of(out)
        self._check(self.lib.selbm_get_state(self.h, pf, dev))
        return out

    def step(self, n=1):
        self._check(self.lib.selbm_step(self.h, int(n)))
        self._info()

    def moments(self, rho=None, u=None):
        if rho is None:
            rho = np.zeros((self.E, self.Np))
            u = np.zeros((self.E, self.Np, self.dim))
        pr, dev = _ptr_of(rho)
        pu, _ = _ptr_of(u)
        self._check(self.lib.selbm_moments(self.h, pr, pu, dev))
        return rho, u

    def stress(self):
        """Non-equilibrium second moment Pi [E, Np, dim, dim] (selbm_stress)."""
        pi = np.zeros((self.E, self.Np, self.dim, self.dim))
        self._check(self.lib.selbm_stress(self.h, _dptr(pi), 0))
        return pi

    def set_filter(self, f):
        fs = filter_struct(f)
        self._check(self.lib.selbm_set_filter(self.h, C.byref(fs)))

    def set_body_force(self, g):
        a = np.zeros(3)
        a[: len(g)] = g
        self._check(self.lib.selbm_set_body_force(self.h, _dptr(a)))

    def set_force_field(self, S, period, t_end):
        """Per-node acceleration A(t) S added to g (selbm_set_force_field).  S is an array
        [E, Np, dim] or a function of the node coordinates x[n, dim] -> [n, dim]."""
        if callable(S):
            S = S(self.node_coords().reshape(-1, self.dim))
        a = np.ascontiguousarray(np.asarray(S, np.float64).reshape(self.E, self.Np, -1)[..., : self.dim])
        self._check(self.lib.selbm_set_force_field(self.h, _dptr(a), float(period), float(t_end)))

    def set_time_scheme(self, scheme):
        """0: Shu-Osher SSPRK3 (default); 1: the four stages as printed; 2: the printed stages with
        the source terms kept for state arguments only (selbm_set_time_scheme)."""
        self._check(self.lib.selbm_set_time_scheme(self.h, int(scheme)))

    def clear_force_field(self):
        self._check(self.lib.selbm_set_force_field(self.h, None, 0.0, 0.0))

    def diagnostics(self):
        """[mass, momentum x3, KE, dissipation, dt, t]; self.fallback_engaged records whether the
        call returned OK_FALLBACK."""
        out = np.zeros(8)
        self.fallback_engaged = self._check(self.lib.selbm_diagnostics(self.h, _dptr(out))) == OK_FALLBACK
        return out

    def wall_stress(self, direction):
        """Surface-weighted mean wall shear stress along `direction` (selbm_wall_stress)."""
        d = np.ascontiguousarray(np.resize(np.asarray(direction, np.float64), 3))
        out = np.zeros(1)
        self._check(self.lib.selbm_wall_stress(self.h, _dptr(d), _dptr(out)))
        return float(out[0])

    def radial_profile(self, origin, axis, radius, nbins):
        """(mean of u.axis, lumped mass) per radial bin (selbm_radial_profile)."""
        o = np.ascontiguousarray(np.resize(np.asarray(origin, np.float64), 3))
        a = np.ascontiguousarray(np.resize(np.asarray(axis, np.float64), 3))
        mean, mass = np.zeros(nbins), np.zeros(nbins)
        self._check(self.lib.selbm_radial_profile(self.h, _dptr(o), _dptr(a), float(radius), int(nbins),
                                                  _dptr(mean), _dptr(mass)))
        return mean, mass

    def timers(self, enable=True):
        self._check(self.lib.selbm_timers(self.h, int(enable)))

    def timers_read(self):
        """{kind: (ms, launches)} for kinds stage1, stage23, assembly, learned, prologue."""
        ms = np.zeros(TIMER_KINDS)
        n = np.zeros(TIMER_KINDS, np.int64)
        self._check(self.lib.selbm_timers_read(self.h, _dptr(ms), n.ctypes.data_as(C.POINTER(C.c_int64))))
        return {k: (float(ms[i]), int(n[i])) for i, k in enumerate(TIMER_NAMES)}

    def sync(self):
        """Wait for the handle's stream; returns OK (0) or OK_FALLBACK (1)."""
        return self._check(self.lib.selbm_sync(self.h))

    # ------------------------------------------------------- learned control
    def set_learned_filter(self, params, lo, hi, mass_bound=1e-6, ke_bound=0.0):
        p = np.ascontiguousarray(params, np.float32)
        l = np.ascontiguousarray(lo, np.float32)
        u = np.ascontiguousarray(hi, np.float32)
        F = C.POINTER(C.c_float)
        self._check(self.lib.selbm_set_learned_filter(self.h, p.ctypes.data_as(F), l.ctypes.data_as(F),
                                                      u.ctypes.data_as(F), float(mass_bound), float(ke_bound)))

    def clear_learned_filter(self):
        self._check(self.lib.selbm_clear_learned_filter(self.h))

    def learned_status(self):
        out = np.zeros(4, np.int64)
        self._check(self.lib.selbm_learned_status(self.h, out.ctypes.data_as(C.POINTER(C.c_int64))))
        return {"fallback_flag": int(out[0]), "fixed_element_steps": int(out[1]), "enabled": bool(out[2])}

    def element_sigma(self):
        out = np.zeros((self.E, self.N + 1))
        self._check(self.lib.selbm_element_sigma(self.h, _dptr(out)))
        return out

    def features(self, out=None):
        """Element features [E, 2(N+1)] (float32 CUDA tensor)."""
        import torch
        if out is None:
            out = torch.empty((self.E, 2 * (self.N + 1)), dtype=torch.float32, device="cuda")
        self._check(self.lib.selbm_features(self.h, C.c_void_p(out.data_ptr())))
        return out

    def element_errors(self, ref, out=None):
        """Per-element error against a higher-order handle on the same mesh (float64 CUDA tensor [E])."""
        import torch
        if out is None:
            out = torch.empty(self.E, dtype=torch.float64, device="cuda")
        self._check(self.lib.selbm_element_errors(self.h, ref.h, C.c_void_p(out.data_ptr())))
        return out


# --------------------------------------------------------------------------- MLP
def _cur_stream():
    import torch
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _chk(rc, what):
    if rc != 0:
        raise SelbmError(rc, what)


def mlp_nparams(nin):
    return int(load_library().selbm_mlp_nparams(int(nin)))


def mlp_grad(params, x, y, order):
    """(loss, grad) over all samples; params, x, y float32 CUDA tensors."""
    import torch
    lib = load_library()
    grad = torch.empty_like(params)
    loss = torch.empty(1, dtype=torch.float32, device=params.device)
    _chk(lib.selbm_mlp_grad(C.c_void_p(params.data_ptr()), x.shape[1], int(order), C.c_void_p(x.data_ptr()),
                            C.c_void_p(y.data_ptr()), x.shape[0], C.c_void_p(grad.data_ptr()),
                            C.c_void_p(loss.data_ptr()), _cur_stream()), "mlp_grad")
    return float(loss.item()), grad


def mlp_forward(params, x, order, bf16=True):
    import torch
    lib = load_library()
    out = torch.empty((x.shape[0], 2), dtype=torch.float32, device=x.device)
    _chk(lib.selbm_mlp_forward(C.c_void_p(params.data_ptr()), x.shape[1], int(order), C.c_void_p(x.data_ptr()),
                               x.shape[0], int(bf16), C.c_void_p(out.data_ptr()), _cur_stream()), "mlp_forward")
    return out


def mlp_train(params, m, v, x, y, order, batch=1024, epochs=10, lr=1e-3, seed=0, adam_t=0):
    """Adam training in place on CUDA tensors; returns (per-epoch mean loss, adam_t)."""
    lib = load_library()
    hist = np.zeros(max(epochs, 1), np.float32)
    t = C.c_int64(int(adam_t))
    _chk(lib.selbm_mlp_train(C.c_void_p(params.data_ptr()), C.c_void_p(m.data_ptr()), C.c_void_p(v.data_ptr()),
                             x.shape[1], int(order), C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr()), x.shape[0],
                             int(batch), int(epochs), float(lr), int(seed), C.byref(t),
                             hist.ctypes.data_as(C.POINTER(C.c_float)), _cur_stream()), "mlp_train")
    return hist[:epochs].tolist(), int(t.value)


def from_case(case, precision=FP64, **kw):
    """Handle for a ``workloads.Case``."""
    return SELBM(case.mesh, case.lattice, case.order, case.nu, cfl=case.cfl, rho0=case.rho0,
                 precision=precision, filt=kw.pop("filt", case.filt), body_accel=kw.pop("body_accel", case.body_accel),
                 **kw)
