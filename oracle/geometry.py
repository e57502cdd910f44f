"""Isoparametric element map, geometric factors, lumped mass, global node
numbering and wall-face data (paper Sec. 2.2: lumped mass M = J rho_i rho_j rho_k,
chain rule with dr/dx and J; Sec. 2.2.1: surface integral R on wall faces).

Node ordering inside an element: i_hat = i + (N+1) j + (N+1)^2 k, r index
fastest (Sec. 2.2).  Arrays indexed [E, Np, ...] use that ordering.
"""
import math

import numpy as np
from scipy.spatial import cKDTree


# ----------------------------------------------------------------------------
# tensor-product helpers (plain reshapes; no blocking)
# ----------------------------------------------------------------------------

def apply_axis(A, u, axis, N, dim):
    """Apply the 1D matrix A along reference axis ``axis`` (0 = r, 1 = s, 2 = t)
    of a field u[..., Np] laid out r-fastest.  Returns the same shape."""
    n = N + 1
    lead = u.shape[:-1]
    v = u.reshape(lead + (n,) * dim)          # [..., (t), s, r]
    ax = v.ndim - 1 - axis
    w = np.moveaxis(np.tensordot(v, A, axes=([ax], [1])), -1, ax)
    return w.reshape(lead + (n ** dim,))


def node_index_grid(N, dim):
    """Per local node, its (i, j[, k]) reference indices -> [Np, dim]."""
    n = N + 1
    idx = np.indices((n,) * dim).reshape(dim, -1).T     # C order: last fastest
    return idx[:, ::-1]                                   # column 0 = i (r), fastest


# ----------------------------------------------------------------------------
# isoparametric map (Gordon-Hall blending with circular-arc edges)
# ----------------------------------------------------------------------------

def _edge_point(Pa, Pb, xi, arc, radius):
    """Point at parameter xi in [-1, 1] on the edge from Pa to Pb: a straight
    segment, or (arc) the circular arc of the given radius about the z axis
    with the angle linear in xi (z, if present, linear in xi)."""
    la, lb = (1.0 - xi) / 2.0, (1.0 + xi) / 2.0
    if not arc:
        return la[:, None] * Pa[None, :] + lb[:, None] * Pb[None, :]
    ta, tb = math.atan2(Pa[1], Pa[0]), math.atan2(Pb[1], Pb[0])
    if tb - ta > math.pi:
        tb -= 2 * math.pi
    if ta - tb > math.pi:
        tb += 2 * math.pi
    th = la * ta + lb * tb
    out = la[:, None] * Pa[None, :] + lb[:, None] * Pb[None, :]
    out[:, 0] = radius * np.cos(th)
    out[:, 1] = radius * np.sin(th)
    return out


def _quad_map(C, curved4, r, s, radius):
    """Gordon-Hall transfinite map of a quad with corners C[4] (corner a + 2b
    at (r, s) = (2a-1, 2b-1)) and faces 0: r=-1, 1: r=+1, 2: s=-1, 3: s=+1
    (curved4[f] = 1: that edge is a circular arc).  r, s: [n] -> [n, dim]."""
    E0 = _edge_point(C[0], C[2], s, curved4[0], radius)   # r = -1, parameter s
    E1 = _edge_point(C[1], C[3], s, curved4[1], radius)   # r = +1
    E2 = _edge_point(C[0], C[1], r, curved4[2], radius)   # s = -1, parameter r
    E3 = _edge_point(C[2], C[3], r, curved4[3], radius)   # s = +1
    rm, rp, sm, sp = (1 - r) / 2, (1 + r) / 2, (1 - s) / 2, (1 + s) / 2
    bil = (rm * sm)[:, None] * C[0] + (rp * sm)[:, None] * C[1] + (rm * sp)[:, None] * C[2] + (rp * sp)[:, None] * C[3]
    return rm[:, None] * E0 + rp[:, None] * E1 + sm[:, None] * E2 + sp[:, None] * E3 - bil


def element_nodes(mesh, xi):
    """Physical coordinates of every GLL node: X[E, Np, dim]."""
    N = len(xi) - 1
    dim = mesh.dim
    ijk = node_index_grid(N, dim)
    r, s = xi[ijk[:, 0]], xi[ijk[:, 1]]
    X = np.zeros((mesh.nelem, len(ijk), dim))
    for e in range(mesh.nelem):
        C = mesh.verts[e]
        cv = mesh.curved[e, :4]
        if dim == 2:
            X[e] = _quad_map(C, cv, r, s, mesh.radius)
        else:
            t = xi[ijk[:, 2]]
            bot = _quad_map(C[0:4], cv, r, s, mesh.radius)
            top = _quad_map(C[4:8], cv, r, s, mesh.radius)
            X[e] = ((1 - t) / 2)[:, None] * bot + ((1 + t) / 2)[:, None] * top
    return X


def element_nodes_from_map(mesh, xi):
    """Node form of the mesh (Sec. 2.2, isoparametric elements): the element map is the
    tensor-product Lagrange interpolant through the given coordinates at the GLL points of
    order mesh.order; evaluated at the points xi -> X[E, Np, dim]."""
    from . import gll
    Ng, dim = int(mesh.order), mesh.dim
    xg = gll.gll_nodes(Ng)
    # l_j(x) = prod_{m != j} (x - xg_m) / (xg_j - xg_m)
    Imat = np.ones((len(xi), Ng + 1))
    for j in range(Ng + 1):
        for m in range(Ng + 1):
            if m != j:
                Imat[:, j] *= (xi - xg[m]) / (xg[j] - xg[m])
    n_to, n_from = len(xi), Ng + 1
    E = mesh.nelem
    X = np.zeros((E, n_to ** dim, dim))
    for k in range(dim):
        v = mesh.xyz[:, k, :].reshape((E,) + (n_from,) * dim)      # [E, (l), j, i]
        for axis in range(dim):
            ax = dim - axis                                         # array axis of reference axis
            v = np.moveaxis(np.tensordot(v, Imat, axes=([ax], [1])), -1, ax)
        X[:, :, k] = v.reshape(E, -1)
    return X


def face_local_nodes(N, dim, f):
    """Local indices of the nodes of face f listed by face coordinates (a, b), a fastest: a and b
    are the tangential node indices in increasing axis order."""
    ijk = node_index_grid(N, dim)
    axis, side = f // 2, f % 2
    tang = [k for k in range(dim) if k != axis]
    on = np.nonzero(ijk[:, axis] == (N if side else 0))[0]
    a = ijk[on, tang[0]]
    b = ijk[on, tang[1]] if dim == 3 else np.zeros_like(a)
    order = np.lexsort((a, b))                # b slowest, a fastest
    return on[order]


def global_numbering_connectivity(mesh, N):
    """Global numbering of the node form from its face connectivity alone -> glo[E, Np]: the
    nodes (a, b) of face f of e and (a', b') of the neighbour's face are one node, with
    (u, v) = (b, a) if bit 0 of the orientation code is set else (a, b), a' = N - u if bit 1,
    b' = N - v if bit 2.  Ids in order of first appearance (element-major, node-minor)."""
    dim, E = mesh.dim, mesh.nelem
    n = N + 1
    Np = n ** dim
    parent = np.arange(E * Np)

    def find(x):
        while parent[x] != x:
            parent[x] = parent[parent[x]]
            x = parent[x]
        return x
    nb = n if dim == 3 else 1
    for e in range(E):
        for f in range(2 * dim):
            e2 = int(mesh.face_nbr[e, f])
            if e2 < 0:
                continue
            f2, code = int(mesh.face_nbr_face[e, f]), int(mesh.face_orient[e, f])
            here, there = face_local_nodes(N, dim, f), face_local_nodes(N, dim, f2)
            for b in range(nb):
                for a in range(n):
                    u, v = (b, a) if code & 1 else (a, b)
                    a2 = N - u if code & 2 else u
                    b2 = N - v if code & 4 else v
                    r1 = find(e * Np + here[a + n * b])
                    r2 = find(e2 * Np + there[a2 + n * b2])
                    if r1 != r2:
                        parent[max(r1, r2)] = min(r1, r2)
    roots = np.array([find(q) for q in range(E * Np)])
    _, first, inv = np.unique(roots, return_index=True, return_inverse=True)
    order = np.argsort(first)
    rank = np.empty_like(order)
    rank[order] = np.arange(len(order))
    return rank[inv].reshape(E, Np)


# ----------------------------------------------------------------------------
# geometric factors
# ----------------------------------------------------------------------------

def metrics(X, D, N, dim, w):
    """dxdr[e,i,k,l] = dx_k/dr_l (isoparametric: D applied to the nodal
    coordinates), J = det, drdx[e,i,l,k] = dr_l/dx_k, wJ = rho_i rho_j rho_k J."""
    E, Np, _ = X.shape
    dxdr = np.zeros((E, Np, dim, dim))
    for k in range(dim):
        for l in range(dim):
            dxdr[:, :, k, l] = apply_axis(D, X[:, :, k], l, N, dim)
    J = np.linalg.det(dxdr)
    drdx = np.linalg.inv(dxdr)                     # inv(dx/dr)[l, k] = dr_l/dx_k
    ijk = node_index_grid(N, dim)
    wq = np.prod(w[ijk], axis=1)                   # rho_i rho_j (rho_k)
    return dxdr, J, drdx, wq[None, :] * J


def global_numbering(X, mesh, tol=1e-9):
    """Identify coincident GLL nodes (periodic images included) -> glo[E, Np].

    Global ids are assigned in order of first appearance in the element-major,
    node-minor local ordering.  Coincidence: distance below tol * domain size
    after wrapping periodic coordinates into [0, period).
    """
    E, Np, dim = X.shape
    P = X.reshape(-1, dim).copy()
    scale = float(np.max(np.ptp(P, axis=0)))
    eps = tol * scale
    for k in range(dim):
        L = mesh.period[k]
        if L > 0:
            y = np.mod(P[:, k] - mesh.origin[k], L)
            y[y > L - eps] -= L
            P[:, k] = y
    tree = cKDTree(P)
    pairs = tree.query_pairs(r=eps, output_type="ndarray")
    parent = np.arange(len(P))

    def find(a):
        while parent[a] != a:
            parent[a] = parent[parent[a]]
            a = parent[a]
        return a

    for a, b in pairs:
        ra, rb = find(a), find(b)
        if ra != rb:
            parent[max(ra, rb)] = min(ra, rb)
    roots = np.array([find(a) for a in range(len(P))])
    _, first, inv = np.unique(roots, return_index=True, return_inverse=True)
    # relabel clusters by first appearance
    order = np.argsort(first)
    rank = np.empty_like(order)
    rank[order] = np.arange(len(order))
    return rank[inv].reshape(E, Np)


def face_nodes(N, dim, f):
    """Local node indices on face f (0: r=-1, 1: r=+1, 2: s=-1, 3: s=+1, 4: t=-1, 5: t=+1)."""
    ijk = node_index_grid(N, dim)
    axis, side = f // 2, f % 2
    return np.nonzero(ijk[:, axis] == (N if side else 0))[0]


def wall_faces(mesh, drdx, J, w, N):
    """For every wall face: (element, local nodes, outward unit normal n [nf, dim],
    surface weight w_s J_s [nf], wall id).  Normal n = +-grad r_l / |grad r_l|,
    surface Jacobian J_s = J |grad r_l| (Nanson), w_s = product of the GLL
    weights of the tangential indices."""
    dim = mesh.dim
    ijk = node_index_grid(N, dim)
    out = []
    for e in range(mesh.nelem):
        for f in range(2 * dim):
            wid = int(mesh.bc[e, f])
            if wid <= 0:
                continue
            axis, side = f // 2, f % 2
            nodes = face_nodes(N, dim, f)
            g = drdx[e, nodes, axis, :]                 # grad r_axis [nf, dim]
            gn = np.linalg.norm(g, axis=1)
            n = (1.0 if side else -1.0) * g / gn[:, None]
            tang = [a for a in range(dim) if a != axis]
            ws = np.prod(w[ijk[nodes][:, tang]], axis=1)
            out.append((e, nodes, n, ws * J[e, nodes] * gn, wid))
    return out


def min_node_spacing(X, N, dim):
    """Smallest physical distance between neighbouring GLL nodes along any
    reference axis, over all elements."""
    n = N + 1
    E = X.shape[0]
    v = X.reshape((E,) + (n,) * dim + (dim,))
    best = np.inf
    for axis in range(dim):
        ax = dim - axis            # array axis of reference axis `axis` (after the E axis)
        d = np.diff(v, axis=ax)
        best = min(best, float(np.sqrt((d * d).sum(-1)).min()))
    return best
