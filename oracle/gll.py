"""Gauss-Lobatto-Legendre quadrature, Lagrange derivative matrix and the
explicit modal filter (paper Sec. 2.2 and Sec. 2.4 "Filter & Stabilization").
"""
import numpy as np
from numpy.polynomial import legendre as npleg


def legendre(n, x):
    """L_n(x) by the three-term recurrence (k+1) L_{k+1} = (2k+1) x L_k - k L_{k-1}."""
    x = np.asarray(x, dtype=float)
    p0, p1 = np.ones_like(x), x.copy()
    if n == 0:
        return p0
    for k in range(1, n):
        p0, p1 = p1, ((2 * k + 1) * x * p1 - k * p0) / (k + 1)
    return p1


def gll_nodes(N):
    """GLL nodes: -1, +1 and the N-1 roots of L'_N (Sec. 2.2)."""
    c = np.zeros(N + 1)
    c[N] = 1.0
    interior = np.sort(npleg.legroots(npleg.legder(c)).real)
    return np.concatenate([[-1.0], interior, [1.0]])


def gll_weights(N, xi):
    """rho_i = 2 / (N (N+1) L_N(xi_i)^2) (Sec. 2.2, lumped mass)."""
    return 2.0 / (N * (N + 1) * legendre(N, xi) ** 2)


def derivative_matrix(xi):
    """D_hat[i, j] = l_j'(xi_i) for the Lagrange basis l_j on the nodes xi.

    From the product form l_j(x) = prod_{m != j} (x - x_m)/(x_j - x_m):
    l_j'(x_i) = 1/(x_j - x_i) prod_{m != i, j} (x_i - x_m)/(x_j - x_m)  (i != j),
    l_j'(x_j) = sum_{k != j} 1/(x_j - x_k).
    """
    n = len(xi)
    D = np.zeros((n, n))
    for i in range(n):
        for j in range(n):
            if i == j:
                D[i, j] = sum(1.0 / (xi[j] - xi[k]) for k in range(n) if k != j)
            else:
                p = 1.0 / (xi[j] - xi[i])
                for m in range(n):
                    if m != i and m != j:
                        p *= (xi[i] - xi[m]) / (xi[j] - xi[m])
                D[i, j] = p
    return D


def modal_basis(N, xi):
    """V[i, k] = phi_k(xi_i) with phi_0 = 1, phi_1 = xi, phi_k = L_k - L_{k-2}.

    The hierarchical basis of the Fischer-Mullen filter the paper cites for
    its explicit filter: phi_k (k >= 2) vanish at +-1, so filtering modes
    k >= 2 leaves element-boundary values unchanged.
    """
    V = np.zeros((len(xi), N + 1))
    V[:, 0] = 1.0
    V[:, 1] = xi
    for k in range(2, N + 1):
        V[:, k] = legendre(k, xi) - legendre(k - 2, xi)
    return V


def filter_sigma(N, shape, gamma, kc, p=8.0):
    """Transfer function sigma_k, k = 0..N.

    shape 0 (paper, Sec. 2.4): sigma_k = 1 - gamma ((k - kc)/(N - kc))^2 for k > kc, else 1.
    shape 1 (exponential):     sigma_k = (1 - gamma) ** (((k - kc)/(N - kc)) ** p) for k > kc, else 1.
    Both give sigma_N = 1 - gamma.  kc may be real-valued.
    """
    sig = np.ones(N + 1)
    for k in range(N + 1):
        if k > kc:
            r = (k - kc) / (N - kc)
            sig[k] = 1.0 - gamma * r * r if shape == 0 else (1.0 - gamma) ** (r ** p)
    return sig


def filter_matrix(N, xi, sigma):
    """F = V diag(sigma) V^{-1}: nodal values -> modal coefficients -> damp -> nodal."""
    V = modal_basis(N, xi)
    return V @ np.diag(sigma) @ np.linalg.inv(V)
