"""FP64 oracle of the learned per-element filter control (not in the paper; the
paper's fixed explicit filter of Sec. 2.4 is the fallback and the yardstick).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Definitions used by both the oracle and the CUDA library:

* modal coefficients of a nodal element field q: a = (V^-1 x V^-1 (x V^-1)) q, with V the
  hierarchical basis 1, xi, L_k - L_{k-2} of the filter (Sec. 2.4);
* shell energy E_k = sum of a^2 over modes whose largest index is k (k = 0..N);
* features: x = [log10(E_k(rho - rho0) + 1e-30)]_k ++ [log10(E_k(|u|) + 1e-30)]_k  (2(N+1) values);
* scaled input s = 2 (x - lo)/(hi - lo) - 1 with the training range [lo, hi];
* MLP: h1 = tanh(W1 s + b1), h2 = tanh(W2 h1 + b2), o = W3 h2 + b3 (64, 64, 2 units);
* gamma = 0.5 sigmoid(o0), kc = 2 + (N - 3) sigmoid(o1); the element's filter has the
  paper's quadratic transfer function with that (gamma, kc);
* loss = mean(((gamma - gamma*)/0.5)^2 + ((kc - kc*)/(N - 3))^2);
* labels (gamma*, kc*) = the sweep setting with the smallest element error against the
  same case at order N + 4 interpolated to the order-N nodes;
* parameter vector: W1[64][nin], b1[64], W2[64][64], b2[64], W3[2][64], b3[2].
"""
import numpy as np

from . import geometry as geo
from . import gll

H = 64
EPS_LOG = 1e-30


# ----------------------------------------------------------------------------- features
def modal_coefficients(q, N, dim):
    """q[E, Np] nodal -> modal coefficients [E, Np] (same r-fastest index order)."""
    xi = gll.gll_nodes(N)
    Vi = np.linalg.inv(gll.modal_basis(N, xi))
    a = q
    for l in range(dim):
        a = geo.apply_axis(Vi, a, l, N, dim)
    return a


def shell_energies(q, N, dim):
    """E_k = sum over modes with max index k of a^2 -> [E, N+1]."""
    a = modal_coefficients(q, N, dim)
    idx = geo.node_index_grid(N, dim)
    shell = idx.max(axis=1)
    out = np.zeros((q.shape[0], N + 1))
    for k in range(N + 1):
        out[:, k] = (a[:, shell == k] ** 2).sum(axis=1)
    return out


def features(rho, u, rho0, N, dim):
    """rho [E, Np], u [E, Np, dim] -> x [E, 2(N+1)]."""
    umag = np.sqrt((u * u).sum(-1))
    return np.concatenate([np.log10(shell_energies(rho - rho0, N, dim) + EPS_LOG),
                           np.log10(shell_energies(umag, N, dim) + EPS_LOG)], axis=1)


# ----------------------------------------------------------------------------- MLP
def n_params(nin):
    return H * nin + H + H * H + H + 2 * H + 2


def unpack(p, nin):
    o = 0
    W1 = p[o:o + H * nin].reshape(H, nin); o += H * nin
    b1 = p[o:o + H]; o += H
    W2 = p[o:o + H * H].reshape(H, H); o += H * H
    b2 = p[o:o + H]; o += H
    W3 = p[o:o + 2 * H].reshape(2, H); o += 2 * H
    b3 = p[o:o + 2]
    return W1, b1, W2, b2, W3, b3


def init_params(nin, seed=0):
    """Glorot-uniform weights, zero biases."""
    rng = np.random.default_rng(seed)
    parts = []
    for fan_out, fan_in in ((H, nin), (H, H), (2, H)):
        lim = np.sqrt(6.0 / (fan_in + fan_out))
        parts += [rng.uniform(-lim, lim, fan_out * fan_in), np.zeros(fan_out)]
    return np.concatenate(parts)


def scale_inputs(x, lo, hi):
    return 2.0 * (x - lo) / (hi - lo) - 1.0


def forward(p, s):
    """s [M, nin] scaled inputs -> (o [M, 2], cache)."""
    nin = s.shape[1]
    W1, b1, W2, b2, W3, b3 = unpack(p, nin)
    z1 = s @ W1.T + b1
    h1 = np.tanh(z1)
    z2 = h1 @ W2.T + b2
    h2 = np.tanh(z2)
    o = h2 @ W3.T + b3
    return o, (s, h1, h2)


def sigmoid(z):
    return 1.0 / (1.0 + np.exp(-z))


def outputs_to_filter(o, N):
    """(gamma, kc) per sample from the network outputs."""
    return 0.5 * sigmoid(o[:, 0]), 2.0 + (N - 3) * sigmoid(o[:, 1])


def loss_and_grad(p, s, y, N):
    """Mean loss over the batch and its gradient w.r.t. p (analytic backprop)."""
    M, nin = s.shape
    W1, b1, W2, b2, W3, b3 = unpack(p, nin)
    o, (s_, h1, h2) = forward(p, s)
    sg0, sg1 = sigmoid(o[:, 0]), sigmoid(o[:, 1])
    gam, kc = 0.5 * sg0, 2.0 + (N - 3) * sg1
    r0 = (gam - y[:, 0]) / 0.5
    r1 = (kc - y[:, 1]) / (N - 3)
    loss = float(np.mean(r0 * r0 + r1 * r1))
    # dL/do
    do = np.zeros_like(o)
    do[:, 0] = 2.0 * r0 / 0.5 * 0.5 * sg0 * (1 - sg0) / M
    do[:, 1] = 2.0 * r1 / (N - 3) * (N - 3) * sg1 * (1 - sg1) / M
    gW3 = do.T @ h2
    gb3 = do.sum(0)
    dh2 = do @ W3
    dz2 = dh2 * (1 - h2 * h2)
    gW2 = dz2.T @ h1
    gb2 = dz2.sum(0)
    dh1 = dz2 @ W2
    dz1 = dh1 * (1 - h1 * h1)
    gW1 = dz1.T @ s
    gb1 = dz1.sum(0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])
    return loss, g


def adam_step(p, m, v, g, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (bias-corrected), t = 1-based step count."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


def bf16_round(x):
    """Round float64 values to bfloat16 (round to nearest, ties to even), returned as float64."""
    f = np.asarray(x, dtype=np.float32)
    b = f.view(np.uint32).astype(np.uint64)
    lsb = (b >> 16) & 1
    b = ((b + 0x7FFF + lsb) >> 16) << 16
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def infer_filter(p, x, lo, hi, N, bf16=True):
    """Element features x [E, nin] -> (gamma, kc, in_range) with BF16-rounded weights (FP64 math)."""
    q = bf16_round(p) if bf16 else p
    s = scale_inputs(x, lo, hi)
    o, _ = forward(q, s)
    gam, kc = outputs_to_filter(o, N)
    in_range = np.all((x >= lo) & (x <= hi), axis=1)
    return gam, kc, in_range


# ----------------------------------------------------------------------------- labels
def lagrange_interp_matrix(x_from, x_to):
    """I[i, j] = l_j(x_to[i]) for the Lagrange basis on x_from."""
    I = np.ones((len(x_to), len(x_from)))
    for j, xj in enumerate(x_from):
        for m, xm in enumerate(x_from):
            if m != j:
                I[:, j] *= (x_to - xm) / (xj - xm)
    return I


def interpolate_elements(q, N_from, N_to, dim):
    """Element-wise tensor-product interpolation q[E, (N_from+1)^dim] -> [E, (N_to+1)^dim]."""
    I = lagrange_interp_matrix(gll.gll_nodes(N_from), gll.gll_nodes(N_to))
    n_from, n_to = N_from + 1, N_to + 1
    E = q.shape[0]
    a = q.reshape((E,) + (n_from,) * dim)
    for l in range(dim):
        ax = a.ndim - 1 - l
        a = np.moveaxis(np.tensordot(a, I, axes=([ax], [1])), -1, ax)
    return a.reshape(E, n_to ** dim)


def element_errors(rho, u, rho_ref, u_ref, wJ, N, N_ref, dim):
    """Per-element quadrature error sum wJ ((rho - rho_ref)^2 + |u - u_ref|^2) with the
    reference interpolated element-wise from order N_ref to order N."""
    rr = interpolate_elements(rho_ref, N_ref, N, dim)
    ur = np.stack([interpolate_elements(u_ref[..., k], N_ref, N, dim) for k in range(dim)], -1)
    return (wJ * ((rho - rr) ** 2 + ((u - ur) ** 2).sum(-1))).sum(1)
