"""Learned per-element filter control: dataset generation, training, evaluation.

Every number here is computed by the CUDA library (features, per-element errors
against the order N+4 run, network training and inference); this module only
schedules the runs and moves tensors.

Data: runs of the same case at the fixed filter strengths of a sweep
(default gamma in {0.01, 0.03, 0.1, 0.3} at kc = N-2, optionally kc in
{N-3, N-2, N-1}) and one run at order N+4 with a time step dividing the
order-N step.  At each snapshot every element gets the features of the
default-filter run (the one the control replaces) and the label (gamma*, kc*)
of the sweep setting whose element error against the N+4 run is smallest;
when the default setting's error is within `tie_margin` of the smallest, the
label is the default (in well-resolved regions the settings differ by less
than the noise of the reference and the control should keep the fixed filter).

python -m paper_2509_19171_gb300.learn --case tgv3d --out weights/...npz
"""
from __future__ import annotations

import argparse
import math
import os
import time

import numpy as np

from . import FP32DEV, SELBM

DEFAULT_GAMMAS = (0.01, 0.03, 0.1, 0.3)
WEIGHTS_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights")


def glorot_params(nin, seed):
    rng = np.random.default_rng(seed)
    parts = []
    for fan_out, fan_in in ((64, nin), (64, 64), (2, 64)):
        lim = math.sqrt(6.0 / (fan_in + fan_out))
        parts += [rng.uniform(-lim, lim, fan_out * fan_in), np.zeros(fan_out)]
    return np.concatenate(parts).astype(np.float32)


def _handles(mesh, lattice, N, nu, sweep, default, precision, dt, ref_sub, init):
    runs = [SELBM(mesh, lattice, N, nu, dt=dt, precision=precision, filt=f) for f in sweep]
    base_i = sweep.index(default)
    ref = SELBM(mesh, lattice, N + 4, nu, dt=dt / ref_sub, precision=FP32DEV,
                filt={"shape": 0, "gamma": default["gamma"], "kc": float(N + 2)})
    for h in runs + [ref]:
        h.init_from(init)
    return runs, base_i, ref


def generate(mesh, lattice, N, nu, inits, snapshots, interval, start=0, gammas=DEFAULT_GAMMAS, kcs=None,
             default_gamma=0.1, precision=FP32DEV, cfl=0.5, tie_margin=0.0, verbose=False):
    """Returns X [M, 2(N+1)] raw features (float32) and Y [M, 2] labels (gamma*, kc*)."""
    import torch
    kcs = kcs or (float(N - 2),)
    sweep = [{"shape": 0, "gamma": g, "kc": k} for g in gammas for k in kcs]
    default = {"shape": 0, "gamma": default_gamma, "kc": float(N - 2)}
    if default not in sweep:
        sweep.append(default)
    probe = SELBM(mesh, lattice, N, nu, cfl=cfl, precision=precision)
    dt = probe.dt
    probe_r = SELBM(mesh, lattice, N + 4, nu, cfl=cfl, precision=FP32DEV)
    ref_sub = int(math.ceil(dt / probe_r.dt - 1e-9))
    probe.close()
    probe_r.close()
    X, Y = [], []
    labels = torch.tensor([[f["gamma"], f["kc"]] for f in sweep], dtype=torch.float32, device="cuda")
    for si, init in enumerate(inits):
        t0 = time.time()
        runs, base_i, ref = _handles(mesh, lattice, N, nu, sweep, default, precision, dt, ref_sub, init)
        if start:
            for h in runs:
                h.step(start)
            ref.step(start * ref_sub)
        for k in range(snapshots):
            for h in runs:
                h.step(interval)
            ref.step(interval * ref_sub)
            feat = runs[base_i].features()
            errs = torch.stack([h.element_errors(ref) for h in runs])         # [runs, E]
            best = torch.argmin(errs, dim=0)
            if tie_margin > 0:
                emin = errs.min(dim=0).values
                best = torch.where(errs[base_i] <= (1.0 + tie_margin) * emin, torch.full_like(best, base_i), best)
            X.append(feat.clone())
            Y.append(labels[best])
        for h in runs + [ref]:
            h.close()
        if verbose:
            print(f"seed {si}: {snapshots} snapshots in {time.time() - t0:.1f} s", flush=True)
    return torch.cat(X), torch.cat(Y)


def feature_range(X, pad=0.25):
    lo = X.min(dim=0).values
    hi = X.max(dim=0).values
    span = (hi - lo).clamp_min(1e-3)
    return (lo - pad * span).cpu().numpy(), (hi + pad * span).cpu().numpy()


def train(X, Y, N, epochs=30, batch=1024, lr=2e-3, seed=0, verbose=False):
    """Train on raw features X and labels Y (CUDA tensors); returns (params, lo, hi, history)."""
    import torch
    from . import mlp_train
    lo, hi = feature_range(X)
    lo_t = torch.from_numpy(lo).cuda()
    hi_t = torch.from_numpy(hi).cuda()
    xs = (2.0 * (X - lo_t) / (hi_t - lo_t) - 1.0).contiguous()
    p = torch.from_numpy(glorot_params(X.shape[1], seed)).cuda()
    m = torch.zeros_like(p)
    v = torch.zeros_like(p)
    hist, _ = mlp_train(p, m, v, xs, Y.contiguous(), N, batch=batch, epochs=epochs, lr=lr, seed=seed)
    if verbose:
        print("loss per epoch:", " ".join(f"{l:.4f}" for l in hist), flush=True)
    return p.cpu().numpy(), lo.astype(np.float32), hi.astype(np.float32), hist


def evaluate(mesh, lattice, N, nu, init, steps, params, lo, hi, default_gamma=0.1, precision=FP32DEV, cfl=0.5,
             checkpoints=4):
    """Total error against the N+4 run for the fixed default filter and for the learned control."""
    default = {"shape": 0, "gamma": default_gamma, "kc": float(N - 2)}
    fixed = SELBM(mesh, lattice, N, nu, cfl=cfl, precision=precision, filt=default)
    learned = SELBM(mesh, lattice, N, nu, dt=fixed.dt, precision=precision, filt=default)
    probe_r = SELBM(mesh, lattice, N + 4, nu, cfl=cfl, precision=FP32DEV)
    ref_sub = int(math.ceil(fixed.dt / probe_r.dt - 1e-9))
    probe_r.close()
    ref = SELBM(mesh, lattice, N + 4, nu, dt=fixed.dt / ref_sub, precision=FP32DEV,
                filt={"shape": 0, "gamma": default_gamma, "kc": float(N + 2)})
    for h in (fixed, learned, ref):
        h.init_from(init)
    learned.set_learned_filter(params, lo, hi)
    out = []
    per = max(steps // checkpoints, 1)
    fallback = 0
    for c in range(checkpoints):
        for h in (fixed, learned):
            h.step(per)
        ref.step(per * ref_sub)
        ef = float(fixed.element_errors(ref).sum().item())
        el = float(learned.element_errors(ref).sum().item())
        st = learned.learned_status()
        fallback += st["fixed_element_steps"]
        out.append({"step": (c + 1) * per, "err_fixed": ef, "err_learned": el, "fallback_flag": st["fallback_flag"]})
    for h in (fixed, learned, ref):
        h.close()
    return out, fallback


def tgv_inits(count, seed0=1, U0=0.05):
    """Taylor-Green initial fields with seeded phase shifts (relative to the element grid)."""
    import workloads as W
    rng = np.random.default_rng(seed0)
    out = []
    for _ in range(count):
        ph = rng.uniform(0, 2 * np.pi, 3)
        base = W.tgv3d_init(U0)
        out.append(lambda x, ph=ph, base=base: base(x + ph[None, :]))
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--case", default="tgv3d", choices=["tgv3d"])
    ap.add_argument("--n", type=int, default=8, help="elements per side of the training cube")
    ap.add_argument("--seeds", type=int, default=3)
    ap.add_argument("--snapshots", type=int, default=24)
    ap.add_argument("--interval", type=int, default=100)
    ap.add_argument("--start", type=int, default=400)
    ap.add_argument("--epochs", type=int, default=40)
    ap.add_argument("--all-kc", action="store_true", help="sweep kc in {N-3, N-2, N-1} as well as gamma")
    ap.add_argument("--eval-steps", type=int, default=0, help="held-out evaluation length (0: data horizon)")
    ap.add_argument("--tie-margin", type=float, default=0.0)
    ap.add_argument("--extra-n", type=int, default=0, help="also take data from a cube of this size")
    ap.add_argument("--extra-start", type=int, default=1600)
    ap.add_argument("--extra-interval", type=int, default=200)
    ap.add_argument("--extra-seeds", type=int, default=3)
    ap.add_argument("--out", default=os.path.join(WEIGHTS_DIR, "learned_filter_tgv3d_n7_d3q27.npz"))
    ap.add_argument("--check-n", type=int, default=16, help="cube size at which to report the fallback rate")
    ap.add_argument("--check-steps", type=int, default=400)
    args = ap.parse_args()
    import workloads as W
    case = W.tgv3d_case(n=args.n)
    N = case.order
    t0 = time.time()
    kcs = (float(N - 3), float(N - 2), float(N - 1)) if args.all_kc else None
    X, Y = generate(case.mesh, case.lattice, N, case.nu, tgv_inits(args.seeds), args.snapshots, args.interval,
                    start=args.start, kcs=kcs, tie_margin=args.tie_margin, verbose=True)
    extra_eval = None
    if args.extra_n:
        import torch
        ec = W.tgv3d_case(n=args.extra_n)
        X2, Y2 = generate(ec.mesh, ec.lattice, N, ec.nu, tgv_inits(args.extra_seeds, seed0=7), args.snapshots,
                          args.extra_interval, start=args.extra_start, kcs=kcs, tie_margin=args.tie_margin, verbose=True)
        X, Y = torch.cat([X, X2]), torch.cat([Y, Y2])
        extra_eval = ec
    t1 = time.time()
    params, lo, hi, hist = train(X, Y, N, epochs=args.epochs, verbose=True)
    t2 = time.time()
    res, fb = evaluate(case.mesh, case.lattice, N, case.nu, tgv_inits(1, seed0=99)[0],
                       args.eval_steps or (args.start + args.snapshots * args.interval), params, lo, hi)
    res_extra = None
    if extra_eval is not None:
        res_extra = evaluate(extra_eval.mesh, extra_eval.lattice, N, extra_eval.nu, tgv_inits(1, seed0=99)[0],
                             args.extra_start + args.snapshots * args.extra_interval, params, lo, hi)
    os.makedirs(os.path.dirname(args.out), exist_ok=True)
    np.savez(args.out, params=params, lo=lo, hi=hi, N=N, lattice=case.lattice, samples=int(X.shape[0]),
             loss=np.array(hist, np.float32))
    big = W.tgv3d_case(n=args.check_n)
    h = SELBM(big.mesh, big.lattice, N, big.nu, cfl=big.cfl, precision=FP32DEV, filt=big.filt)
    h.init_from(big.init)
    h.set_learned_filter(params, lo, hi)
    h.step(args.check_steps)
    st = h.learned_status()
    h.close()
    print({"samples": int(X.shape[0]), "data_s": round(t1 - t0, 1), "train_s": round(t2 - t1, 1),
           "label_hist": {f"{g:.2f}/{k:.0f}": int(c) for (g, k), c in
                          zip(*np.unique(Y.cpu().numpy().round(3), axis=0, return_counts=True))},
           "eval": res, "fallback_element_steps": fb, "eval_extra": res_extra,
           "check": {"n": args.check_n, "steps": args.check_steps,
                     "fallback_fraction": st["fixed_element_steps"] / (big.mesh.nelem * (args.check_steps - 1)),
                     "flag": st["fallback_flag"]}})


if __name__ == "__main__":
    main()
