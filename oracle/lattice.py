"""Discrete velocity sets D2Q9, D3Q19, D3Q27 (paper Sec. 2.1, equilibrium Eq. geq_s).

The paper uses D2Q9 and D3Q19 and cites their standard weights without
printing them; D3Q27 is the standard 27-velocity set.  Velocities are ordered
by speed class |e|^2 = 0, 1, 2, 3 and, within a class, by the ternary code
(e_x+1) + 3 (e_y+1) + 9 (e_z+1) ascending.  This ordering is the population
index used in every state array of the library and the oracle.
"""
import itertools

import numpy as np

CS2 = 1.0 / 3.0

_CLASS_WEIGHTS = {
    "D2Q9": {0: 4.0 / 9.0, 1: 1.0 / 9.0, 2: 1.0 / 36.0},
    "D3Q19": {0: 1.0 / 3.0, 1: 1.0 / 18.0, 2: 1.0 / 36.0},
    "D3Q27": {0: 8.0 / 27.0, 1: 2.0 / 27.0, 2: 1.0 / 54.0, 3: 1.0 / 216.0},
}


def lattice(name):
    """Return (e [Q, d] int, t [Q] float64, opposite [Q] int)."""
    dim = 2 if name == "D2Q9" else 3
    weights = _CLASS_WEIGHTS[name]
    vel = []
    for comps in itertools.product((-1, 0, 1), repeat=dim):
        ev = np.array(comps[::-1])          # comps iterates last component slowest -> reverse
        speed2 = int((ev * ev).sum())
        if speed2 in weights:
            code = sum((int(ev[k]) + 1) * 3 ** k for k in range(dim))
            vel.append((speed2, code, ev))
    vel.sort(key=lambda v: (v[0], v[1]))
    e = np.array([v[2] for v in vel], dtype=np.int64)
    t = np.array([weights[v[0]] for v in vel])
    opp = np.array([next(b for b in range(len(e)) if np.all(e[b] == -e[a])) for a in range(len(e))])
    return e, t, opp


def equilibrium(e, t, rho, u):
    """f^eq_alpha = t_alpha rho (1 + e.u/cs2 + (e.u)^2/(2 cs2^2) - |u|^2/(2 cs2)).

    Eq. (geq_s).  rho [n], u [n, d] -> [Q, n].
    """
    eu = e.astype(float) @ u.T                  # [Q, n]
    uu = (u * u).sum(axis=1)                    # [n]
    return t[:, None] * rho[None, :] * (1.0 + eu / CS2 + eu ** 2 / (2 * CS2 ** 2) - uu[None, :] / (2 * CS2))


def force_split(e, t, u, F):
    """Leading-order and higher-order forcing terms (Sec. 2.1, Eqs. body and f_c).

    F*_alpha  = t_alpha (e_alpha / cs2) . F
    F**_alpha = t_alpha ((e_alpha . u) e_alpha / cs2^2 - u / cs2) . F
    u [n, d], F [n, d] -> (Fstar [Q, n], Fss [Q, n]).
    """
    ef = e.astype(float)
    eF = ef @ F.T                               # [Q, n]
    eu = ef @ u.T                               # [Q, n]
    uF = (u * F).sum(axis=1)                    # [n]
    Fstar = t[:, None] * eF / CS2
    Fss = t[:, None] * (eu * eF / CS2 ** 2 - uF[None, :] / CS2)
    return Fstar, Fss
