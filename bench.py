"""Throughput of the filtered SELBM hot path on GB300.

Metric: GLL-node x population updates per second (local nodes, i.e. element
copies of shared nodes counted once per element: E * (N+1)^d * Q per step).
Default workload: 3D Taylor-Green vortex, D3Q27, 16^3 hex elements at N=7
(2,097,152 local nodes, 56.6M populations), quadratic filter gamma=0.1,
kc=N-2.  One step = collision, three SSPRK3 stages (element kernel +
assembly kernel each), filter.  Inputs are larger than L2 (one FP64 state
array = 303 MB), so no flush is needed between steps.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun (N > 1) every rank runs an independent replica (weak scaling).
"""
from __future__ import annotations

import os

# The CPU oracle arm is timed single-threaded: pin BLAS threads before numpy loads.
for _v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import argparse
import json
import math
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12     # 152 SMs x 2 DFMA/clk x 2 flop x 2070 MHz


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return d, "measured"
    return PEAKS_FALLBACK, "fallback"


# --------------------------------------------------------------------------- workload
def workload(name, n=16):
    if name == "tgv3d":
        case = W.tgv3d_case(n=n)
    elif name == "pipe":
        case = W.pipe_case()
    elif name == "shear":
        case = W.shear_layer_case()
    else:
        raise SystemExit(f"unknown workload {name}")
    return case


def counts(case, info):
    """Unique / interior / boundary node counts and bytes-per-launch model of the
    unique-node layout ('Algorithmic bytes')."""
    E, N, dim = case.mesh.nelem, case.order, case.mesh.dim
    n = N + 1
    Np = n ** dim
    Gint = E * (N - 1) ** dim
    Nb = Np - (N - 1) ** dim
    return dict(E=E, Np=Np, Nb=Nb, G=info["G"], Gb=info["Gb"], Gint=Gint, ENb=E * Nb)


def bytes_per_step(c, Q, rsz, affine):
    """Algorithmic DRAM bytes of one step: (stage1, stage2+3 per launch, assembly s1, assembly s2/3)."""
    G, Gint, ENb, Gb = c["G"], c["Gint"], c["ENb"], c["Gb"]
    geo = 0 if affine else (c["E"] * c["Np"] * 10 * rsz)     # per-node metrics + wJ read by each stage
    s1 = (G + G + Gint + ENb) * Q * rsz + geo
    s23 = (G + Gint + Gint + ENb) * Q * rsz + geo
    a1 = (ENb + 2 * Gb) * Q * rsz
    a23 = (ENb + 3 * Gb) * Q * rsz
    return s1, s23, a1, a23


def flops_per_step(case, e_nonzero_axes, Q):
    """Algorithmic FP operations of the stage kernels per step."""
    E, N, dim = case.mesh.nelem, case.order, case.mesh.dim
    pops = E * (N + 1) ** dim * Q
    n = N + 1
    deriv = 2 * n * e_nonzero_axes + 2 * e_nonzero_axes       # per pop per stage
    rk = 5
    collide = 20
    filt = dim * 2 * n
    stage1 = pops * (deriv + rk + collide + filt)
    stage23 = pops * (deriv + rk)
    return stage1, stage23


# --------------------------------------------------------------------------- clocks
class ClockSampler:
    def __init__(self):
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self, device_index=0):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9 or not parts[0].isdigit() or int(parts[0]) != device_index:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx = max(mx, float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower() in ("active", "0x1", "1"):
                        reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------------- our arm
def run_form(P, torch, case, precision, steps, warmup, dev_index):
    s = P.from_case(case, precision=precision, stream=torch.cuda.current_stream().cuda_stream)
    s.init_from(case.init)
    s.step(warmup)
    s.sync()
    return s


def time_steps(torch, s, steps, dist):
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    s.timers(True)
    e0.record(st)
    s.step(steps)
    e1.record(st)
    torch.cuda.synchronize()
    t = s.timers_read()
    s.timers(False)
    if dist:
        dist.barrier()
    return e0.elapsed_time(e1), t


def e2e_run(P, torch, case, precision, steps):
    """Public-API end to end: initial fields H2D from pinned host, K steps, moments D2H to pinned host."""
    s = P.from_case(case, precision=precision, stream=torch.cuda.current_stream().cuda_stream)
    x = s.node_coords().reshape(-1, s.dim)
    rho, u = case.init(x)
    rho_h = torch.from_numpy(np.ascontiguousarray(rho, np.float64)).pin_memory()
    u_h = torch.from_numpy(np.ascontiguousarray(u[:, : s.dim], np.float64)).pin_memory()
    rho_o = torch.empty_like(rho_h).pin_memory()
    u_o = torch.empty_like(u_h).pin_memory()
    # warm-up of the same sequence
    s.init(rho_h, u_h)
    s.step(2)
    s.moments(rho_o, u_o)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s.init(rho_h, u_h)
    s.step(steps)
    s.moments(rho_o, u_o)
    torch.cuda.synchronize()
    ms = (time.perf_counter() - t0) * 1e3
    h2d = rho_h.numel() * 8 + u_h.numel() * 8
    d2h = rho_o.numel() * 8 + u_o.numel() * 8
    s.close()
    return ms, h2d, d2h


def cpu_baseline(case, seconds=12.0):
    """The oracle, as it stands, on a bounded sample of the workload: same
    lattice, order and filter on 4^3 elements of the same periodic cube."""
    from oracle.selbm import OracleSELBM
    L = 2 * math.pi
    n = 4
    mesh = W.box_mesh((n, n, n), (0, 0, 0), (L, L, L), (True, True, True))
    o = OracleSELBM(mesh, case.lattice, case.order, case.nu, cfl=case.cfl, filt=case.filt)
    f = o.initial_state_from(case.init)
    f = o.step(f)
    t0 = time.perf_counter()
    k = 0
    while time.perf_counter() - t0 < seconds:
        f = o.step(f)
        k += 1
    dt = time.perf_counter() - t0
    upd = o.E * o.Np * o.Q * k
    return {"value": upd / dt, "unit": "node-pop updates/s", "cores": 1, "kind": "oracle",
            "sample": f"{case.lattice} N={case.order} TGV on {n}^3 elements ({o.E * o.Np * o.Q} updates/step), "
                      f"{k} steps in {dt:.1f} s, numpy float64, 1 thread"}


def workload_config(case, form, world):
    dim = case.mesh.dim
    Q = {"D2Q9": 9, "D3Q19": 19, "D3Q27": 27}[case.lattice]
    nloc = case.mesh.nelem * (case.order + 1) ** dim
    return {"workload": f"{case.name}: {case.lattice}, {case.mesh.nelem} elements, N={case.order}, "
                        f"{nloc} local nodes, {nloc * Q} populations",
            "form": form, "filter": case.filt, "l2": "inputs larger than L2 (no flush)",
            "parallelism": f"replicas x{world}"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="tgv3d", choices=["tgv3d", "pipe", "shear"])
    ap.add_argument("--forms", default="fp64,fp32dev")
    ap.add_argument("--n", type=int, default=16, help="TGV elements per side")
    ap.add_argument("--no-extras", action="store_true", help="skip e2e, cpu baseline and clock sampling")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    case = workload(args.workload, args.n)
    metric = "node-population updates/s"

    if args.impl == "reference":
        if rank != 0:
            return
        cb = None
        vals = []
        for _ in range(args.warmup):
            cpu_baseline(case, seconds=2.0)
        for _ in range(args.steps):
            cb = cpu_baseline(case, seconds=3.0)
            vals.append(cb["value"])
        v = statistics.median(vals)
        cb["value"] = v
        print(json.dumps({"metric": metric, "value": v, "unit": "node-pop updates/s", "n_gpus": args.gpus,
                          "steps": args.steps, "warmup": args.warmup, "impl": "reference",
                          "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                          "data": "synthetic", "config": workload_config(case, "fp64", args.gpus),
                          "cpu_baseline": cb,
                          "e2e": {"value": v, "unit": "node-pop updates/s", "h2d_bytes_per_step": 0,
                                  "d2h_bytes_per_step": 0}}))
        return

    import torch
    dist = None
    if world > 1:
        import torch.distributed as tdist
        local = int(os.environ.get("LOCAL_RANK", "0"))
        torch.cuda.set_device(local)
        tdist.init_process_group("nccl")
        dist = tdist
    dev_index = torch.cuda.current_device()

    import paper_2509_19171_gb300 as P
    from paper_2509_19171_gb300 import build
    if rank == 0:
        build.build()
    if dist:
        dist.barrier()
    info = P.mesh_check(case.mesh, case.lattice, case.order)
    c = counts(case, info)
    pk, pk_kind = peaks()
    hbm = float(pk["hbm_gbs"])

    forms = [f for f in args.forms.split(",") if f]
    results = {}
    clocks = None
    for form in forms:
        prec = P.FP64 if form == "fp64" else P.FP32DEV
        rsz = 8 if form == "fp64" else 4
        s = run_form(P, torch, case, prec, args.steps, args.warmup, dev_index)
        sampler = ClockSampler() if (not args.no_extras and form == forms[0]) else None
        if sampler:
            sampler.start()
        ms, t = time_steps(torch, s, args.steps, dist)
        if sampler:
            clocks = sampler.stop(dev_index)
        if dist:
            tt = torch.tensor([ms], device="cuda")
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
            ms = float(tt.item())
        e, _, _ = s.lattice_table()
        nz_axes = float(np.abs(e).astype(bool).sum(1).mean()) if info["affine"] else float(case.mesh.dim)
        Q = s.Q
        upd_step = case.mesh.nelem * info["Np"] * Q
        value = upd_step * args.steps * world / (ms * 1e-3)
        s1, s23, a1, a23 = bytes_per_step(c, Q, rsz, info["affine"])
        f1, f23 = flops_per_step(case, nz_axes, Q)
        st1_ms = t["stage1"][0] / max(t["stage1"][1], 1)
        st23_ms = t["stage23"][0] / max(t["stage23"][1], 1)
        as_ms = t["assembly"][0] / max(t["assembly"][1], 1)
        stage_ms = (t["stage1"][0] + t["stage23"][0]) / max(t["stage1"][1] + t["stage23"][1], 1)
        stage_bytes = (s1 + 2 * s23) / 3
        stage_flops = (f1 + 2 * f23) / 3
        step_bytes = s1 + 2 * s23 + a1 + 2 * a23
        results[form] = {
            "value": value, "ms_per_step": ms / args.steps, "dtype": "f64" if form == "fp64" else "f32",
            "kernel_ms": {"stage1": st1_ms, "stage2_3": st23_ms, "assembly": as_ms},
            "launches": {k: v[1] for k, v in t.items()},
            "hbm_gbs_alg_step": step_bytes / (ms / args.steps * 1e-3) / 1e9,
            "stage_hbm_frac": stage_bytes / (stage_ms * 1e-3) / 1e9 / hbm,
            "stage_fp64_frac": (stage_flops / (stage_ms * 1e-3) / 1e12 / FP64_PEAK_TFLOPS) if form == "fp64" else None,
            "stage_bytes": stage_bytes, "stage_flops": stage_flops, "stage_ms": stage_ms,
            "bytes_per_update": step_bytes / upd_step,
        }
        s.close()
        del s
        torch.cuda.empty_cache()

    main_form = forms[0]
    r = results[main_form]
    if main_form == "fp64":
        achieved = r["stage_flops"] / (r["stage_ms"] * 1e-3) / 1e12
        roof = {"bound": "alu", "kernel": "stage_kernel (FP64 pipe)", "achieved": achieved,
                "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS,
                "peak_source": "derived: 152 SMs x 2 DFMA/clk x 2 flop x 2070 MHz (DFMA probe: 2.07/clk/SM)",
                "traffic": None, "hbm_frac_alg": r["stage_hbm_frac"]}
    else:
        achieved = r["stage_bytes"] / (r["stage_ms"] * 1e-3) / 1e9
        roof = {"bound": "hbm", "kernel": "stage_kernel", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                "frac": achieved / hbm, "peak_source": f"{pk_kind} hbm_gbs", "traffic": None}

    line = {"metric": metric, "value": r["value"], "unit": "node-pop updates/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": r["dtype"],
            "data": "synthetic",
            "config": workload_config(case, main_form, world),
            "roofline": roof, "forms": results, "gpu_launches": int(sum(results[main_form]["launches"].values()))}
    if clocks:
        line["clocks"] = clocks
    if rank == 0 and not args.no_extras:
        ms_e2e, h2d, d2h = e2e_run(P, torch, case, P.FP64 if main_form == "fp64" else P.FP32DEV, args.steps)
        upd = case.mesh.nelem * info["Np"] * info["Q"] * args.steps
        line["e2e"] = {"value": upd / (ms_e2e * 1e-3), "unit": "node-pop updates/s",
                       "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps,
                       "note": "selbm_init from pinned host (rho, u), K steps, selbm_moments to pinned host"}
        line["cpu_baseline"] = cpu_baseline(case)
    if rank == 0:
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
