"""Spatial convergence of the unsteady Couette flow (Sec. 3.2): L-infinity error of u_x against
the series solution at T / t0 = 40 (t0 = L / u_top) for polynomial orders N, at Re = 2000 and
Ma = 0.05, with the Shu-Osher scheme and with the printed four-stage scheme (taken literally,
and with its source terms kept for the state arguments only).

Unit square, 6 x 6 quads, D2Q9, periodic in x, wall at rest at y = 0, wall moving at u_top at
y = 1, fluid at rest at t = 0, no filter, CFL 0.5.  The series solution of the impulsively
started flow is u_x = u_top y + sum_n 2 u_top (-1)^n / (n pi) sin(n pi y) exp(-nu (n pi)^2 t).
Every number of the run comes from the library (steps, selbm_moments); this module
evaluates the series and the error.

python -m paper_2509_19171_gb300.couette_convergence --out couette.json
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

from . import FP64, SELBM


def series(y, t, u_top, nu, terms=400):
    n = np.arange(1, terms + 1)[:, None]
    return u_top * y + (2.0 * u_top * (-1.0) ** n / (n * math.pi) * np.sin(n * math.pi * y[None, :])
                        * np.exp(-nu * (n * math.pi) ** 2 * t)).sum(0)


def run(orders=(4, 6, 8, 10, 12, 14), schemes=(0, 1, 2), ne=6, Re=2000.0, Ma=0.05, t_over_t0=40.0, cfl=0.5):
    import workloads as W
    u_top = Ma / math.sqrt(3.0)
    nu = u_top / Re
    mesh = W.box_mesh((ne, ne), (0.0, 0.0), (1.0, 1.0), (True, False), walls={2: 1, 3: 2},
                      wall_velocity=[[0.0, 0.0], [u_top, 0.0]])
    T = t_over_t0 / u_top
    out = []
    for scheme in schemes:
        for N in orders:
            s = SELBM(mesh, "D2Q9", N, nu, cfl=cfl, precision=FP64)
            s.set_time_scheme(scheme)
            s.init_from(lambda x: (np.ones(x.shape[0]), np.zeros((x.shape[0], 2))))
            steps = int(math.ceil(T / s.dt))
            t0 = time.time()
            s.step(steps)
            _, u = s.moments()
            wall_s = time.time() - t0
            y = s.node_coords()[..., 1].reshape(-1)
            ua = series(y, steps * s.dt, u_top, nu)
            err = float(np.abs(u.reshape(-1, 2)[:, 0] - ua).max() / u_top)
            name = ["Shu-Osher SSPRK3", "printed four stages, literal", "printed four stages, sources weighted"][scheme]
            out.append({"scheme": name, "N": N, "dt": s.dt,
                        "steps": steps, "t_over_t0": steps * s.dt * u_top, "linf_err_over_utop": err,
                        "wall_s": round(wall_s, 2)})
            print(json.dumps(out[-1]), flush=True)
            s.close()
    return {"case": f"unsteady Couette, {ne}x{ne} quads, D2Q9, Re={Re}, Ma={Ma}, T/t0={t_over_t0}", "results": out}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default="couette.json")
    ap.add_argument("--orders", default="4,6,8,10,12,14")
    ap.add_argument("--schemes", default="0,1,2")
    args = ap.parse_args()
    res = run(orders=tuple(int(x) for x in args.orders.split(",")),
              schemes=tuple(int(x) for x in args.schemes.split(",")))
    with open(args.out, "w") as fh:
        json.dump(res, fh, indent=1)


if __name__ == "__main__":
    main()
