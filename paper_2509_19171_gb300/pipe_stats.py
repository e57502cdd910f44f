"""Turbulent-pipe statistics run (Sec. 4): the butterfly pipe at Re_tau = 180 started from the
log-law profile, driven by the body force g = 2 u_tau^2 / R (with --peng also by the
divergence-free perturbation force of the first three eddy turnover times), sampling the wall shear stress
tau_w / (rho0 u_tau^2) and the space- and time-averaged axial velocity in wall units u+(y+).

Every number comes from the library (steps, selbm_wall_stress, selbm_radial_profile); this
module schedules the samples and averages the profiles over time (mass-weighted).

python -m paper_2509_19171_gb300.pipe_stats --steps 20000 --every 2000 --out pipe_stats.json
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import FP32DEV, FP64, SelbmError, from_case


def run(steps, every, nbins=48, precision=FP32DEV, n_axial=32, init="loglaw", peng=False):
    import workloads as W
    case = W.pipe_case(n_axial=n_axial)
    R, u_tau, L = 1.0, 0.0025, 10.0
    nu = case.nu
    s = from_case(case, precision=precision)
    if peng:
        # perturbation force for the first 3 t0, period 8 t0, amplitude B0 g (g = 2 u_tau^2 / R)
        t0 = R / u_tau
        s.set_force_field(W.peng_forcing(2.0 * u_tau ** 2 / R, radius=R, length=L), 8.0 * t0, 3.0 * t0)
    s.init_from(W.pipe_loglaw_init(u_tau, nu, radius=R, length=L) if init == "loglaw" else case.init)
    hist = []
    acc_mean, acc_mass = np.zeros(nbins), np.zeros(nbins)
    t0 = time.time()
    done = 0
    for k in range(0, steps + 1, every):
        if k > done:
            s.step(k - done)
            done = k
        try:
            d = s.diagnostics()
        except SelbmError as err:
            hist.append({"step": k, "diverged": str(err)})
            break
        tau = s.wall_stress([0, 0, 1])
        mean, mass = s.radial_profile([0, 0, 0], [0, 0, 1], R, nbins)
        acc_mean += mean * mass
        acc_mass += mass
        hist.append({"step": k, "time": float(d[7]), "tau_w_over_rho_utau2": tau / (1.0 * u_tau ** 2),
                     "kinetic_energy": float(d[4])})
    wall_s = time.time() - t0
    ubar = np.divide(acc_mean, acc_mass, out=np.zeros(nbins), where=acc_mass > 0)
    r_mid = (np.arange(nbins) + 0.5) * R / nbins
    y_plus = (R - r_mid) * u_tau / nu
    prof = [{"y_plus": float(y), "u_plus": float(u / u_tau), "u_plus_loglaw": float(W.loglaw_uplus(y))}
            for y, u in zip(y_plus, ubar)]
    out = {"case": "pipe Re_tau=180, 8192 hexes, N=7, D3Q19", "precision": "fp64" if precision == 0 else "fp32dev",
           "dt": s.dt, "t0_over_dt": (R / u_tau) / s.dt, "steps": steps, "wall_s": round(wall_s, 1),
           "history": hist, "profile_time_average": prof}
    s.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--steps", type=int, default=20000)
    ap.add_argument("--every", type=int, default=2000)
    ap.add_argument("--nbins", type=int, default=48)
    ap.add_argument("--out", default="pipe_stats.json")
    ap.add_argument("--fp64", action="store_true")
    ap.add_argument("--init", default="loglaw", choices=["loglaw", "laminar"])
    ap.add_argument("--peng", action="store_true", help="perturbation force for the first 3 t0")
    args = ap.parse_args()
    res = run(args.steps, args.every, args.nbins, precision=FP64 if args.fp64 else FP32DEV, init=args.init,
              peng=args.peng)
    with open(args.out, "w") as fh:
        json.dump(res, fh, indent=1)
    h = res["history"]
    print(json.dumps({"t0_over_dt": res["t0_over_dt"], "wall_s": res["wall_s"], "first": h[0], "last": h[-1]}))


if __name__ == "__main__":
    main()
