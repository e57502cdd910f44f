"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module holds *data only*: element corner coordinates, boundary tags,
periodic lengths, wall velocities and closed-form initial fields, and the node
form of a mesh (node coordinates of the element maps at reference points the
caller supplies, face connectivity found by matching faces).  It contains none
of the method's arithmetic (no GLL points, no metrics, no lattice tables): both
the CUDA library and the CPU oracle map the corners (or interpolate the nodes) to
their own GLL nodes and evaluate the initial fields there.

Mesh conventions (shared interface, documented in include/selbm.h):

* ``verts[e, c, k]``: corner ``c`` of element ``e``, coordinate ``k``.  The
  corner index is ``c = a + 2 b (+ 4 g)`` where ``a, b, g`` in {0, 1} select
  reference coordinate ``r, s (, t) = -1 or +1``.
* ``curved[e, f]``: 1 if face ``f`` of element ``e`` lies on the circle
  (2D) / cylinder (3D, axis = z) of radius ``radius`` centred on the origin,
  else 0.  Face ids: 0: r=-1, 1: r=+1, 2: s=-1, 3: s=+1, 4: t=-1, 5: t=+1.
  Curved 3D elements are extrusions along z (corners c and c+4 share x, y).
* ``bc[e, f]``: 0 for interior or periodic faces, k >= 1 for a wall with
  velocity ``wall_velocity[k-1]``.
* ``period[k]``: periodic length along axis k (0 if not periodic),
  ``origin[k]`` the domain origin along that axis.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


@dataclass
class MeshSpec:
    dim: int
    verts: np.ndarray            # [E, 2**dim, dim] float64
    curved: np.ndarray           # [E, 2*dim] int32
    bc: np.ndarray               # [E, 2*dim] int32
    period: np.ndarray           # [dim] float64
    origin: np.ndarray           # [dim] float64
    wall_velocity: np.ndarray    # [nwalls, dim] float64
    radius: float = 0.0
    name: str = ""

    @property
    def nelem(self) -> int:
        return int(self.verts.shape[0])


@dataclass
class Case:
    """A workload: mesh + lattice + order + physics + closed-form initial field."""
    name: str
    mesh: MeshSpec
    lattice: str                 # "D2Q9" | "D3Q19" | "D3Q27"
    order: int
    nu: float                    # kinematic viscosity; lambda = nu / cs^2
    cfl: float
    rho0: float
    init: object                 # callable(x: [n, dim]) -> (rho [n], u [n, dim])
    body_accel: np.ndarray = field(default_factory=lambda: np.zeros(3))
    filt: dict = field(default_factory=lambda: {"shape": 0, "gamma": 0.0, "kc": 0.0, "p": 8.0})
    steps: int = 0
    U0: float = 1.0


# ----------------------------------------------------------------------------
# box meshes
# ----------------------------------------------------------------------------

def box_mesh(shape, lo, hi, periodic, walls=None, wall_velocity=None, name="box") -> MeshSpec:
    """Structured box of ``shape`` elements between ``lo`` and ``hi``.

    ``periodic[k]`` makes axis k periodic.  ``walls`` maps a face id of the
    box (0: x-, 1: x+, 2: y-, 3: y+, 4: z-, 5: z+) to a wall id >= 1.
    """
    dim = len(shape)
    walls = walls or {}
    nw = max(walls.values()) if walls else 0
    wv = np.zeros((nw, dim)) if wall_velocity is None else np.asarray(wall_velocity, float).reshape(nw, dim)
    edges = [np.linspace(lo[k], hi[k], shape[k] + 1) for k in range(dim)]
    E = int(np.prod(shape))
    verts = np.zeros((E, 2 ** dim, dim))
    bc = np.zeros((E, 2 * dim), np.int32)
    order = []   # element order: x index fastest
    for ijk in np.ndindex(*shape[::-1]):
        order.append(ijk[::-1])
    for e, ijk in enumerate(order):
        for c in range(2 ** dim):
            bits = [(c >> k) & 1 for k in range(dim)]
            verts[e, c] = [edges[k][ijk[k] + bits[k]] for k in range(dim)]
        for k in range(dim):
            if not periodic[k]:
                if ijk[k] == 0 and (2 * k) in walls:
                    bc[e, 2 * k] = walls[2 * k]
                if ijk[k] == shape[k] - 1 and (2 * k + 1) in walls:
                    bc[e, 2 * k + 1] = walls[2 * k + 1]
    period = np.array([(hi[k] - lo[k]) if periodic[k] else 0.0 for k in range(dim)])
    return MeshSpec(dim=dim, verts=verts, curved=np.zeros((E, 2 * dim), np.int32), bc=bc,
                    period=period, origin=np.array(lo, float), wall_velocity=wv, name=name)


# ----------------------------------------------------------------------------
# butterfly O-grid pipe
# ----------------------------------------------------------------------------

def pipe_mesh(n_core=8, n_radial=6, grading=1.3, n_axial=32, length=10.0, radius=1.0,
              core_half=0.5, name="pipe") -> MeshSpec:
    """Butterfly (O-grid) pipe of radius ``radius`` along z, periodic axially.

    Cross-section: an ``n_core x n_core`` square core of half-width
    ``core_half * radius`` and four outer blocks of ``n_core`` azimuthal by
    ``n_radial`` radial elements whose radial sizes shrink by ``grading``
    from one ring to the next toward the wall.  Only the outermost ring's wall
    face is curved (a circular arc); every other edge is straight.  Wall id 1,
    no-slip.
    """
    a = core_half * radius
    quads = []         # (4 corners (x,y) in corner order, curved face id or -1)
    g = np.linspace(-a, a, n_core + 1)
    for j in range(n_core):
        for i in range(n_core):
            quads.append(([(g[i], g[j]), (g[i + 1], g[j]), (g[i], g[j + 1]), (g[i + 1], g[j + 1])], -1))
    sizes = np.array([grading ** (-k) for k in range(n_radial)])
    s = np.concatenate([[0.0], np.cumsum(sizes) / sizes.sum()])
    for blk in range(4):
        rot = blk * math.pi / 2
        c, sn = math.cos(rot), math.sin(rot)

        def R2(p):
            return (c * p[0] - sn * p[1], sn * p[0] + c * p[1])

        for m in range(n_core):
            for k in range(n_radial):
                pts = []
                # corner order: r (radial, outward) fastest, s (azimuth, counter-clockwise)
                for mm in (m, m + 1):
                    ys = -a + 2 * a * mm / n_core
                    th = -math.pi / 4 + (math.pi / 2) * mm / n_core
                    ps = np.array([a, ys])
                    pc = np.array([radius * math.cos(th), radius * math.sin(th)])
                    for kk in (k, k + 1):
                        p = ps + s[kk] * (pc - ps)
                        if kk == n_radial:
                            p = pc
                        pts.append(R2(p))
                # pts order: (m,k),(m,k+1),(m+1,k),(m+1,k+1) -> corners a + 2b with a radial, b azimuth
                corners = [pts[0], pts[1], pts[2], pts[3]]
                quads.append((corners, 1 if k == n_radial - 1 else -1))
    nq = len(quads)
    E = nq * n_axial
    verts = np.zeros((E, 8, 3))
    curved = np.zeros((E, 6), np.int32)
    bc = np.zeros((E, 6), np.int32)
    zs = np.linspace(0.0, length, n_axial + 1)
    e = 0
    for kz in range(n_axial):
        for corners, cf in quads:
            for cc in range(8):
                x, y = corners[cc & 3]
                verts[e, cc] = (x, y, zs[kz + (cc >> 2)])
            if cf >= 0:
                curved[e, cf] = 1
                bc[e, cf] = 1
            e += 1
    return MeshSpec(dim=3, verts=verts, curved=curved, bc=bc,
                    period=np.array([0.0, 0.0, length]), origin=np.array([0.0, 0.0, 0.0]),
                    wall_velocity=np.zeros((1, 3)), radius=radius, name=name)


# ----------------------------------------------------------------------------
# closed-form initial fields (paper's test problems)
# ----------------------------------------------------------------------------

@dataclass
class NodeMeshSpec:
    """Mesh given by the node coordinates of each element's map and its face connectivity
    (the selbm_mesh_nodes form of include/selbm.h).

    * ``xyz[e, k, p]``: coordinate k of the element's node p = i + n j (+ n^2 l), n = order + 1,
      at the reference points the caller chose (the order-``order`` GLL points for the library).
    * ``face_nbr[e, f]``: neighbour element across face f or -1; ``face_nbr_face[e, f]`` its face;
      ``face_orient[e, f]``: bit 0 swaps the face coordinates (a, b), bit 1 flips a, bit 2 flips b
      (face coordinates: the two tangential node indices in increasing axis order).
    * ``bc[e, f]``: 0 interior / periodic / open, k >= 1 wall k with ``wall_velocity[k-1]``.
    """
    dim: int
    order: int
    xyz: np.ndarray              # [E, dim, (order+1)**dim] float64
    face_nbr: np.ndarray         # [E, 2*dim] int32
    face_nbr_face: np.ndarray    # [E, 2*dim] int8
    face_orient: np.ndarray      # [E, 2*dim] int8
    bc: np.ndarray               # [E, 2*dim] int32
    wall_velocity: np.ndarray    # [nwalls, dim] float64
    name: str = "nodes"

    @property
    def nelem(self) -> int:
        return int(self.xyz.shape[0])


def _face_local(n, dim, f):
    """Local node indices of face f in face-coordinate order (a fastest)."""
    axis, fixed = f // 2, (n - 1) * (f % 2)
    out = []
    tang = [k for k in range(dim) if k != axis]
    rng_b = range(n) if dim == 3 else range(1)
    for b in rng_b:
        for a in range(n):
            idx = [0, 0, 0]
            idx[axis] = fixed
            idx[tang[0]] = a
            if dim == 3:
                idx[tang[1]] = b
            out.append(idx[0] + n * idx[1] + n * n * idx[2])
    return np.array(out)


def _orient(code, m, a, b):
    u, v = (b, a) if code & 1 else (a, b)
    return (m - u if code & 2 else u), (m - v if code & 4 else v)


def node_mesh(mesh, ref_points, deform=None, rotate=(), name="nodes"):
    """Node form of a straight-sided corner mesh: the (bi/tri)linear map of each element's
    corners evaluated at the tensor product of ``ref_points`` (reference coordinates in
    [-1, 1], ascending, symmetric), then ``deform`` (x[n, dim] -> x[n, dim]) applied to every
    node, and the local frames of the elements in ``rotate`` turned by 90 degrees about t (in 2D
    about the normal): their new node (i, j, l) is the old node (m - j, i, l), m = len - 1.
    Connectivity comes from matching faces whose nodes coincide up to one translation (zero
    inside the domain, a period of ``mesh`` across periodic faces)."""
    xi = np.asarray(ref_points, float)
    n, dim, E = len(xi), mesh.dim, mesh.nelem
    m = n - 1
    idx = np.indices((n,) * dim).reshape(dim, -1)[::-1]           # row 0 = i (fastest)
    Np = n ** dim
    xyz = np.zeros((E, dim, Np))
    bc = np.array(mesh.bc, np.int32).copy()
    rot = set(int(e) for e in rotate)
    for e in range(E):
        C = mesh.verts[e]
        ii = idx.copy()
        if e in rot:
            ii = np.stack([m - idx[1], idx[0]] + ([idx[2]] if dim == 3 else []))
        lam = [np.stack([(1 - xi[ii[k]]) / 2, (1 + xi[ii[k]]) / 2]) for k in range(dim)]
        x = np.zeros((Np, dim))
        for c in range(2 ** dim):
            bits = [(c >> k) & 1 for k in range(dim)]
            wgt = np.prod([lam[k][bits[k]] for k in range(dim)], axis=0)
            x += wgt[:, None] * C[c][None, :]
        if deform is not None:
            x = deform(x)
        xyz[e] = x.T
        if e in rot:
            perm = [2, 3, 1, 0] + ([4, 5] if dim == 3 else [])
            bc[e] = np.array(mesh.bc[e])[perm]
    nf = 2 * dim
    period = np.asarray(mesh.period, float)
    faces = {}
    for e in range(E):
        for f in range(nf):
            faces[(e, f)] = xyz[e][:, _face_local(n, dim, f)].T         # [nface, dim]
    scale = float(np.ptp(xyz.transpose(0, 2, 1).reshape(-1, dim), axis=0).max())
    tol = 1e-9 * scale

    def wrapped_key(P):
        c = P.mean(0).copy()
        for k in range(dim):
            if period[k] > 0:
                c[k] = np.mod(c[k] - mesh.origin[k] + 0.5 * tol, period[k])
        return tuple(np.round(c / (1e-6 * scale)).astype(np.int64))
    buckets = {}
    for key, P in faces.items():
        buckets.setdefault(wrapped_key(P), []).append(key)
    face_nbr = np.full((E, nf), -1, np.int32)
    face_nbr_face = np.zeros((E, nf), np.int8)
    face_orient = np.zeros((E, nf), np.int8)
    nb = n if dim == 3 else 1
    for keys in buckets.values():
        for (e, f) in keys:
            for (e2, f2) in keys:
                if (e2, f2) == (e, f):
                    continue
                A, B = faces[(e, f)], faces[(e2, f2)]
                for code in (range(8) if dim == 3 else (0, 2)):
                    mp = [_orient(code, m, a, b) for b in range(nb) for a in range(n)]
                    d = np.array([B[a2 + n * b2] for a2, b2 in mp]) - A
                    if np.abs(d - d[0]).max() > tol:
                        continue
                    ok = all(abs(d[0][k]) <= tol or (period[k] > 0 and abs(abs(d[0][k]) - period[k]) <= tol)
                             for k in range(dim))
                    if ok and face_nbr[e, f] < 0:
                        face_nbr[e, f], face_nbr_face[e, f], face_orient[e, f] = e2, f2, code
    return NodeMeshSpec(dim, m, xyz, face_nbr, face_nbr_face, face_orient, bc,
                        np.asarray(mesh.wall_velocity, float).reshape(-1, dim), name)


def couette_init(rho0=1.0):
    def f(x):
        n = x.shape[0]
        return np.full(n, rho0), np.zeros((n, 2))
    return f


def shear_layer_init(U0=0.04, kappa=80.0, delta=0.05, rho0=1.0):
    """Double shear layer (paper Sec. 3.1): tanh layers at y = 0.25, 0.75."""
    def f(x):
        X, Y = x[:, 0], x[:, 1]
        ux = np.where(Y <= 0.5, U0 * np.tanh(kappa * (Y - 0.25)), U0 * np.tanh(kappa * (0.75 - Y)))
        uy = delta * U0 * np.sin(2 * np.pi * (X + 0.25))
        return np.full(x.shape[0], rho0), np.stack([ux, uy], 1)
    return f


def tgv3d_init(U0=0.05, rho0=1.0, cs2=1.0 / 3.0):
    """3D Taylor-Green vortex (paper Sec. 3.4), density from the incompressible
    pressure p - p0 = rho0 U0^2/16 (cos 2x + cos 2y)(cos 2z + 2), rho = rho0 + (p-p0)/cs^2."""
    def f(x):
        X, Y, Z = x[:, 0], x[:, 1], x[:, 2]
        u = np.stack([U0 * np.sin(X) * np.cos(Y) * np.cos(Z),
                      -U0 * np.cos(X) * np.sin(Y) * np.cos(Z),
                      np.zeros_like(X)], 1)
        p = rho0 * U0 ** 2 / 16.0 * (np.cos(2 * X) + np.cos(2 * Y)) * (np.cos(2 * Z) + 2.0)
        return rho0 + p / cs2, u
    return f


def tgv2d_init(U0=0.01, rho0=1.0, cs2=1.0 / 3.0):
    """2D Taylor-Green vortex on [0, 2pi]^2 (low Re decay test)."""
    def f(x):
        X, Y = x[:, 0], x[:, 1]
        u = np.stack([U0 * np.sin(X) * np.cos(Y), -U0 * np.cos(X) * np.sin(Y)], 1)
        p = -rho0 * U0 ** 2 / 4.0 * (np.cos(2 * X) + np.cos(2 * Y))
        return rho0 + p / cs2, u
    return f


def poiseuille_init(G, mu, L=1.0, rho0=1.0, parabola=True):
    """Planar Poiseuille: u_x = G/(2 mu) y (L - y) driven by a body force G along x."""
    def f(x):
        Y = x[:, 1]
        ux = G / (2 * mu) * Y * (L - Y) if parabola else np.zeros_like(Y)
        return np.full(x.shape[0], rho0), np.stack([ux, np.zeros_like(Y)], 1)
    return f


def pipe_init(U_bulk, radius=1.0, length=10.0, noise=0.05, seed=1234, nmodes=24, rho0=1.0):
    """Laminar parabola with bulk velocity U_bulk plus a seeded smooth random
    velocity perturbation of amplitude ``noise * U_bulk`` (sum of random
    Fourier modes, axially periodic, damped to zero at the wall)."""
    rng = np.random.default_rng(seed)
    kz = rng.integers(1, 5, size=(3, nmodes)) * 2 * np.pi / length
    kxy = rng.uniform(-3.0, 3.0, size=(3, nmodes, 2))
    ph = rng.uniform(0, 2 * np.pi, size=(3, nmodes))
    amp = rng.uniform(-1.0, 1.0, size=(3, nmodes))
    amp /= np.abs(amp).sum(axis=1, keepdims=True)

    def f(x):
        X, Y, Z = x[:, 0], x[:, 1], x[:, 2]
        r2 = (X ** 2 + Y ** 2) / radius ** 2
        damp = np.clip(1.0 - r2, 0.0, None)
        u = np.zeros((x.shape[0], 3))
        u[:, 2] = 2.0 * U_bulk * damp
        for c in range(3):
            arg = kxy[c, :, 0][None] * X[:, None] + kxy[c, :, 1][None] * Y[:, None] + kz[c][None] * Z[:, None] + ph[c][None]
            u[:, c] += noise * U_bulk * damp * (amp[c][None] * np.sin(arg)).sum(1)
        return np.full(x.shape[0], rho0), u
    return f


def loglaw_uplus(y_plus, kappa=0.41, c_plus=5.0):
    """Mean velocity of a turbulent wall layer in wall units (Sec. 4, pipe initial profile):
    u+ = y+ in the viscous sublayer, (1/kappa) ln y+ + C+ in the inertial sublayer, switched at the
    upper crossing y_c of the two branches (y_c = 10.80 for kappa = 0.41, C+ = 5), so that the
    profile is continuous and u+ = 0 on the wall."""
    lo, hi = 1.0, 100.0                        # y - ln(y)/kappa - C+ changes sign once in [1, 100]
    for _ in range(80):
        mid = 0.5 * (lo + hi)
        if mid - math.log(mid) / kappa - c_plus < 0:
            lo = mid
        else:
            hi = mid
    y = np.asarray(y_plus, float)
    return np.where(y < hi, y, np.log(np.maximum(y, hi)) / kappa + c_plus)


def pipe_loglaw_init(u_tau, nu, radius=1.0, length=10.0, noise=0.05, seed=1234, nmodes=24, rho0=1.0):
    """Pipe initial field of Sec. 4: axial velocity u_tau u+(y+) with y+ = (R - r) u_tau / nu from
    ``loglaw_uplus``, plus the seeded smooth perturbation of ``pipe_init`` scaled by the centreline
    velocity u_tau u+(R u_tau / nu)."""
    base = pipe_init(1.0, radius=radius, length=length, noise=noise, seed=seed, nmodes=nmodes, rho0=rho0)
    Uc = u_tau * float(loglaw_uplus(radius * u_tau / nu))

    def f(x):
        X, Y = x[:, 0], x[:, 1]
        r = np.sqrt(X ** 2 + Y ** 2)
        rho, up = base(x)                       # 2 (1 - r^2/R^2) + perturbation, per unit bulk velocity
        u = up * Uc
        u[:, 2] = u_tau * loglaw_uplus(np.clip(radius - r, 0.0, None) * u_tau / nu) + \
            (up[:, 2] - 2.0 * np.clip(1.0 - r ** 2 / radius ** 2, 0.0, None)) * Uc
        return rho, u
    return f


def peng_forcing(g, radius=1.0, length=10.0, kz=3, ktheta=4, B0=50.0, kappa=0.5, l0=0.2, l=0.4):
    """Spatial part of the pipe's divergence-free perturbation force (Sec. 4, after Peng et al.),
    as an acceleration field for a pipe along z through the origin: the time factor
    sin(2 pi t / P) is left out (it is applied per step).  In cylindrical components, with
    phi = 2 pi (R - r - l0) / l and only inside l0 <= R - r <= l0 + l (l0, l in units of R):
      F_r     = -g kappa B0 (R / r) (kz l / L) (1 - cos phi) cos(2 pi kz z / L) cos(ktheta theta)
      F_theta =  g (1 - kappa) B0 (kz / ktheta) (2 pi R / L) sin phi cos(2 pi kz z / L) sin(ktheta theta)
      F_z     = -g B0 (R / r) sin phi sin(2 pi kz z / L) cos(ktheta theta)
    turned to Cartesian components.  The paper does not give kz and ktheta."""
    R, L = float(radius), float(length)
    L0, Lb = l0 * R, l * R

    def f(x):
        X, Y, Z = x[:, 0], x[:, 1], x[:, 2]
        r = np.sqrt(X ** 2 + Y ** 2)
        th = np.arctan2(Y, X)
        inside = (R - r >= L0) & (R - r <= L0 + Lb)
        rs = np.where(inside, r, R)                     # keeps R / r finite off the band
        phi = 2.0 * np.pi * (R - rs - L0) / Lb
        cz, sz = np.cos(2.0 * np.pi * kz * Z / L), np.sin(2.0 * np.pi * kz * Z / L)
        ct, st = np.cos(ktheta * th), np.sin(ktheta * th)
        Fr = -g * kappa * B0 * (R / rs) * (kz * Lb / L) * (1.0 - np.cos(phi)) * cz * ct
        Ft = g * (1.0 - kappa) * B0 * (kz / ktheta) * (2.0 * np.pi * R / L) * np.sin(phi) * cz * st
        Fz = -g * B0 * (R / rs) * np.sin(phi) * sz * ct
        out = np.zeros((x.shape[0], 3))
        out[:, 0] = np.where(inside, Fr * np.cos(th) - Ft * np.sin(th), 0.0)
        out[:, 1] = np.where(inside, Fr * np.sin(th) + Ft * np.cos(th), 0.0)
        out[:, 2] = np.where(inside, Fz, 0.0)
        return out
    return f


# ----------------------------------------------------------------------------
# the configurations of the benchmark suite (sizes as stated for each case)
# ----------------------------------------------------------------------------

CS2 = 1.0 / 3.0


def couette_case(order=4, nx=8, ny=4, U0=0.01, nu=0.002) -> Case:
    mesh = box_mesh((nx, ny), (0.0, 0.0), (1.0, 1.0), (True, False), walls={2: 1, 3: 2},
                    wall_velocity=[[0.0, 0.0], [U0, 0.0]], name="couette")
    return Case("couette", mesh, "D2Q9", order, nu, 0.5, 1.0, couette_init(), np.zeros(2),
                {"shape": 0, "gamma": 0.0, "kc": float(order), "p": 8.0}, 2000, U0)


def shear_layer_case(n=32, order=8, U0=0.04, Re=1.0e4, gamma=0.1) -> Case:
    mesh = box_mesh((n, n), (0.0, 0.0), (1.0, 1.0), (True, True), name="shear_layer")
    return Case("shear_layer", mesh, "D2Q9", order, U0 * 1.0 / Re, 0.5, 1.0, shear_layer_init(U0),
                np.zeros(2), {"shape": 1, "gamma": gamma, "kc": float(order - 2), "p": 8.0}, 20000, U0)


def tgv3d_case(n=16, order=7, lattice="D3Q27", U0=0.05, Re=1600.0, gamma=0.1) -> Case:
    L = 2 * np.pi
    mesh = box_mesh((n, n, n), (0.0, 0.0, 0.0), (L, L, L), (True, True, True), name="tgv3d")
    return Case("tgv3d", mesh, lattice, order, U0 * 1.0 / Re, 0.5, 1.0, tgv3d_init(U0), np.zeros(3),
                {"shape": 0, "gamma": gamma, "kc": float(order - 2), "p": 8.0}, 31767, U0)


def pipe_case(order=7, n_axial=32, n_core=8, n_radial=6, Re_tau=180.0, u_tau=0.0025, gamma=0.1) -> Case:
    R = 1.0
    mesh = pipe_mesh(n_core=n_core, n_radial=n_radial, n_axial=n_axial, radius=R)
    nu = u_tau * R / Re_tau
    U_b = 5300.0 * nu / (2 * R)
    g = 2 * u_tau ** 2 / R
    return Case("pipe", mesh, "D3Q19", order, nu, 0.5, 1.0, pipe_init(U_b), np.array([0.0, 0.0, g]),
                {"shape": 0, "gamma": gamma, "kc": float(order - 2), "p": 8.0}, 1000, U_b)
