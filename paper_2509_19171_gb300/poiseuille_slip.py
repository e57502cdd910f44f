"""Numerical slip of the flux bounce-back wall in planar Poiseuille flow (Sec. 3.3): the
dimensionless wall velocity u_slip* = u_x(y = 0) / u_max at steady state for a sweep of the
relaxation time tau = lambda / dt and of the time step dt (through the CFL number), and the wall
normal stress T_xx = -Pi_xx (selbm_stress) against -2 mu lambda (u')^2.

Unit square, 4 x 4 quads, N = 8, D2Q9, periodic in x, walls at y = 0 and 1, driven by the
body force G = 8 nu u_max with u_max = 0.1 / 3 (Ma = 0.1 / sqrt(3)), nu = tau dt cs^2.  Each
case starts on the analytic parabola and runs until u_slip* changes by less than a tolerance
between two checks.  Every number comes from the library (steps, selbm_moments, selbm_stress); this module
schedules the runs and reads the wall nodes.

python -m paper_2509_19171_gb300.poiseuille_slip --out slip.json
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import FP64, SELBM


def run(taus=(0.1, 0.2, 0.3, 0.4), cfls=(0.5, 0.25, 0.125), ne=4, order=8, check=2000, max_steps=200000,
        tol=1e-8, precision=FP64):
    import workloads as W
    mesh = W.box_mesh((ne, ne), (0.0, 0.0), (1.0, 1.0), (True, False), walls={2: 1, 3: 1}, wall_velocity=[[0.0, 0.0]])
    umax = 0.1 / 3.0
    out = []
    for cfl in cfls:
        probe = SELBM(mesh, "D2Q9", order, 1.0, cfl=cfl, precision=precision)
        dt = probe.dt
        probe.close()
        for tau in taus:
            nu = tau * dt / 3.0
            G = 8.0 * nu * umax
            s = SELBM(mesh, "D2Q9", order, nu, dt=dt, precision=precision, body_accel=[G, 0.0])
            s.init_from(W.poiseuille_init(G, nu))
            y = s.node_coords()[..., 1].reshape(-1)
            wall = np.abs(y) < 1e-12
            ua = G / (2.0 * nu) * y * (1.0 - y)
            t0 = time.time()
            steps, prev, slip, err = 0, None, None, None
            while steps < max_steps:
                s.step(check)
                steps += check
                _, u = s.moments()
                ux = u.reshape(-1, 2)[:, 0]
                slip = float(np.abs(ux[wall]).max() / umax)
                err = float(np.abs(ux - ua).max() / umax)
                if prev is not None and abs(slip - prev) < tol:
                    break
                prev = slip
            # wall normal stress T_xx = -Pi_xx against -2 mu lambda (u')^2 with the analytic u'
            rho, _ = s.moments()
            pi = s.stress()
            txx = -pi.reshape(-1, 2, 2)[wall, 0, 0]
            lam = tau * dt
            expect = -2.0 * rho.reshape(-1)[wall] * nu * lam * (G / (2.0 * nu)) ** 2
            out.append({"cfl": cfl, "tau": tau, "dt": dt, "nu": nu, "steps": steps, "u_slip_star": slip,
                        "profile_err_over_umax": err, "converged": prev is not None and abs(slip - prev) < tol,
                        "txx_wall_over_burnett": float(np.mean(txx / expect)),
                        "wall_s": round(time.time() - t0, 2)})
            s.close()
    return {"case": f"planar Poiseuille, {ne}x{ne} quads, N={order}, D2Q9, u_max={umax:.6f}", "results": out}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default="slip.json")
    ap.add_argument("--check", type=int, default=2000)
    ap.add_argument("--max-steps", type=int, default=200000)
    args = ap.parse_args()
    res = run(check=args.check, max_steps=args.max_steps)
    with open(args.out, "w") as fh:
        json.dump(res, fh, indent=1)
    for r in res["results"]:
        print(json.dumps(r))


if __name__ == "__main__":
    main()
