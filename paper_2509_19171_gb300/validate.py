"""Accuracy of the FP32-deviation and learned-control forms against the FP64 form.

For each workload the forms start from the same initial field and run the same
steps; at checkpoints the node RMS and max of |u - u_fp64| / U0 and of
|rho - rho_fp64| are recorded, with the kinetic energy and dissipation histories
(selbm_diagnostics).  Taylor-Green 16^3 N=7 D3Q27 to t = 5 L0/U0 with pointwise
comparisons at t = 2 and 5 L0/U0 (before the chaotic decorrelation of the transition),
the learned control also against the fixed filter it replaces and, for its arithmetic
error, against the FP64 form with the same control ("fp64_learned"); the butterfly pipe
(8192 hexes, N=7, D3Q19, curved walls, body force) for 1000 steps, the double
shear layer (32^2, N=8, D2Q9) for 2000 steps.

Sensitivity control ("fp64_perturbed"): the FP64 form started from the same field with
every deviation f - t rho0 multiplied by 1 + 2^-24 xi (xi = +-1, seeded), i.e. a
perturbation of the size of one FP32 storage rounding of the state.  Its distance from the
unperturbed FP64 run is what any FP32-level difference grows to by the flow itself; an
FP32 form at that distance is at the floor the flow sets, not limited by its arithmetic.

python -m paper_2509_19171_gb300.validate --out validation.json
"""
from __future__ import annotations

import argparse
import json
import os
import time

import numpy as np

from . import FP32DEV, FP64, from_case

HERE = os.path.dirname(os.path.abspath(__file__))
WEIGHTS = os.path.join(HERE, "weights", "learned_filter_tgv3d_shear_n7.npz")


def _errors(a, b, U0):
    (ra, ua), (rb, ub) = a, b
    du = np.linalg.norm(ua - ub, axis=-1)
    return {"u_rms_over_U0": float(np.sqrt((du ** 2).mean()) / U0), "u_max_over_U0": float(du.max() / U0),
            "rho_rms": float(np.sqrt(((ra - rb) ** 2).mean())), "rho_max": float(np.abs(ra - rb).max())}


def perturb_fp32_level(h, rho0=1.0, seed=5):
    """Multiply every deviation f - t rho0 of the handle's state by 1 + 2^-24 xi, xi = +-1."""
    f = h.get_state()
    _, t, _ = h.lattice_table()
    rng = np.random.default_rng(seed)
    dev = f - t[:, None, None] * rho0
    xi = rng.integers(0, 2, size=f.shape) * 2.0 - 1.0
    h.set_state(np.ascontiguousarray(t[:, None, None] * rho0 + dev * (1.0 + 2.0 ** -24 * xi)))


def run_case(case, forms, steps, checkpoints, history_every, learned=None):
    handles = {}
    for f in forms:
        h = from_case(case, precision=FP64 if f.startswith("fp64") else FP32DEV)
        h.init_from(case.init)
        if f == "fp64_perturbed":
            perturb_fp32_level(h, case.rho0)
        if f.endswith("_learned"):
            w = np.load(learned)
            h.set_learned_filter(w["params"], w["lo"], w["hi"], mass_bound=1e-6)
        handles[f] = h
    hist = {f: [] for f in forms}
    errs = []
    done = 0
    t0 = time.time()
    marks = sorted(set([c for c in checkpoints if c <= steps] + list(range(history_every, steps + 1, history_every))))
    for m in marks:
        for f, h in handles.items():
            h.step(m - done)
            d = h.diagnostics()
            hist[f].append({"step": m, "time": float(d[7]), "mass": float(d[0]), "ke": float(d[4]),
                            "eps": float(d[5])})
        done = m
        if m in checkpoints:
            fields = {f: h.moments() for f, h in handles.items()}
            row = {"step": m}
            for f in forms:
                if f != "fp64":
                    row[f] = _errors(fields[f], fields["fp64"], case.U0)
            if "fp32dev_learned" in handles:
                row["learned_status"] = handles["fp32dev_learned"].learned_status()
                if "fp32dev" in fields:
                    row["learned_vs_fixed"] = _errors(fields["fp32dev_learned"], fields["fp32dev"], case.U0)
                if "fp64_learned" in fields:
                    # the arithmetic error of the learned form: FP32 against FP64 with the same control
                    row["learned_fp32_vs_learned_fp64"] = _errors(fields["fp32dev_learned"], fields["fp64_learned"],
                                                                  case.U0)
                    row["learned_fp64_status"] = handles["fp64_learned"].learned_status()
            errs.append(row)
    out = {"case": case.name, "elements": case.mesh.nelem, "order": case.order, "lattice": case.lattice,
           "U0": case.U0, "steps": steps, "dt": handles["fp64"].dt, "wall_s": round(time.time() - t0, 1),
           "errors_vs_fp64": errs, "history": hist}
    for h in handles.values():
        h.close()
    # relative KE / dissipation history differences vs FP64
    for f in forms:
        if f == "fp64":
            continue
        ke = np.array([r["ke"] for r in hist[f]])
        ke64 = np.array([r["ke"] for r in hist["fp64"]])
        ep = np.array([r["eps"] for r in hist[f]])
        ep64 = np.array([r["eps"] for r in hist["fp64"]])
        out[f"{f}_ke_rel_max"] = float(np.abs(ke / ke64 - 1).max())
        out[f"{f}_eps_rel_max"] = float(np.abs(ep / ep64 - 1).max())
    m0 = hist["fp64"][0]["mass"]
    out["fp64_mass_rel_drift"] = float(max(abs(r["mass"] / m0 - 1) for r in hist["fp64"]))
    return out


def main():
    import workloads as W
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default="validation.json")
    ap.add_argument("--quick", action="store_true")
    ap.add_argument("--weights", default=WEIGHTS, help="learned-control weights (.npz)")
    ap.add_argument("--cases", default="tgv,pipe,shear")
    args = ap.parse_args()
    res = []
    cases = args.cases.split(",")
    weights = args.weights
    tgv = W.tgv3d_case()
    tgv_steps = 200 if args.quick else 8000     # t = 5 L0/U0 at dt = 0.0126
    lforms = ["fp64_learned", "fp32dev_learned"] if os.path.exists(weights) else []
    forms = ["fp64", "fp64_perturbed", "fp32dev"] + lforms
    if "tgv" in cases:
        res.append(run_case(tgv, forms, tgv_steps, [tgv_steps * 2 // 5, tgv_steps], max(tgv_steps // 40, 1), weights))
    if "pipe" in cases:
        pipe = W.pipe_case()
        pipe_steps = 100 if args.quick else 1000
        pforms = ["fp64", "fp64_perturbed", "fp32dev"] + lforms
        res.append(run_case(pipe, pforms, pipe_steps, [pipe_steps], max(pipe_steps // 10, 1), weights))
    if "shear" in cases:
        shear = W.shear_layer_case()
        sh_steps = 200 if args.quick else 2000
        res.append(run_case(shear, ["fp64", "fp32dev"], sh_steps, [sh_steps], max(sh_steps // 10, 1)))
    with open(args.out, "w") as fh:
        json.dump(res, fh, indent=1)
    for r in res:
        print(r["case"], r["wall_s"], "s", json.dumps(r["errors_vs_fp64"][-1]),
              {k: v for k, v in r.items() if k.endswith("_rel_max") or k.endswith("drift")})


if __name__ == "__main__":
    main()
