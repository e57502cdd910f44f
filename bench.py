"""Throughput of the filtered SELBM hot path on GB300.

Metric: GLL-node x population updates per second (local nodes, i.e. element
copies of shared nodes counted once per element: E * (N+1)^d * Q per step).
Default workload: 3D Taylor-Green vortex, D3Q27, 16^3 hex elements at N=7
(2,097,152 local nodes, 56.6M populations), quadratic filter gamma=0.1,
kc=N-2.  One step = (learned filter control) + collision, three SSPRK3
stages (element kernel + assembly kernel each), filter.  Inputs are larger
than L2 (one FP32 state array = 152 MB, FP64 303 MB), so no flush is needed.

Forms: fp64 (the paper's method in FP64), fp32dev (FP32 deviations), and the
headline fp32dev_learned (FP32 deviations + learned per-element filter
control with the fixed filter as fallback).  Each form is timed with
captured-graph launches; per-kernel times come from a separate short run
with the library's event timers.

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


def fp64_peak(torch, n=4096, reps=3):
    """Measured FP64 arithmetic peak of this GPU: best of `reps` cuBLAS DGEMMs of n^3 (2 n^3
    flops each), CUDA events on the current stream.  On GB300 the FP64 tensor rate equals the
    FP64 FMA rate, so this is the ceiling of the FP64 form's DFMA-bound kernels."""
    a = torch.randn(n, n, dtype=torch.float64, device="cuda")
    b = torch.randn(n, n, dtype=torch.float64, device="cuda")
    torch.mm(a, b)
    best = None
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        torch.mm(a, b)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        best = ms if best is None else min(best, ms)
    del a, b
    return 2.0 * n ** 3 / (best * 1e-3) / 1e12


def measured_traffic(kernel_key, units):
    """DRAM bytes (read + write) per launch of `kernel_key` from the committed ncu summary
    (profiles/traffic.json: bytes per element measured on a smaller mesh, scaled by the
    elements one launch processes); None when the kernel source has changed since."""
    import hashlib
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as fh:
        d = json.load(fh).get(kernel_key)
    if not d:
        return None
    src = os.path.join(ROOT, d["source"])
    if not os.path.exists(src) or hashlib.sha256(open(src, "rb").read()).hexdigest() != d["source_sha256"]:
        return None
    return d["dram_bytes_per_element"] * units


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
    unique-node layout: every unique value a launch needs is read once and every value it
    produces is written once."""
    E, N, dim = case.mesh.nelem, case.order, case.mesh.dim
    n = N + 1
    Np = n ** dim
    Gint = E * (N - 1) ** dim
    Nb = Np - (N - 1) ** dim
    return dict(E=E, Np=Np, Nb=Nb, G=info["G"], Gb=info["Gb"], Gint=Gint, ENb=E * Nb)


def kernel_bytes(c, Q, rsz, affine, split, learned):
    """Algorithmic DRAM bytes per launch of each kernel kind on the unique-node layout:
    every unique value read once and written once per pass, shares of element-boundary
    nodes (E*Nb per population) written and read once, per-node metrics on curved meshes."""
    G, Gint, ENb, Gb, E, Np = c["G"], c["Gint"], c["ENb"], c["Gb"], c["E"], c["Np"]
    geo = 0 if affine else E * Np * 10 * rsz          # per-node metrics + wJ read by each stage
    kb = {"stage23": (G + Gint + Gint + ENb) * Q * rsz + geo,          # f^{s-1}, f^0 (interior), f^s, trace
          "assembly": ((ENb + 2 * Gb) + 2 * (ENb + 3 * Gb)) * Q * rsz / 3}
    if split:
        kb["stage1"] = (G + Gint + ENb) * Q * rsz + geo                # f^0 -> f^1 (interior), trace
        kb["prologue"] = 2 * G * Q * rsz                               # f -> (filter, collision) -> f^0
        # learned: f -> features, network, per-element filter; interior f^0 + boundary shares;
        # then the shares' assembly + collision on shared nodes
        kb["learned"] = (G + Gint + ENb) * Q * rsz + (ENb + Gb) * Q * rsz + (0 if affine else E * Np * rsz)
    else:
        kb["stage1"] = (G + G + Gint + ENb) * Q * rsz + geo            # f, f^0 out, f^1 (interior), trace
        kb["learned"] = (G + Gint + ENb) * Q * rsz + (ENb + Gb) * Q * rsz + (0 if affine else E * Np * rsz)
    return kb


def launches_per_step(split, learned):
    """Kernels one step launches: 3 x (stage + assembly), plus the collision/filter
    prologue of the split form, plus control + drift check + share assembly when learned."""
    if split:
        return 6 + (3 if learned else 1)
    return 6 + (3 if learned else 0)


def flops_per_step(case, e_nonzero_axes, Q):
    """Algorithmic FP operations of the stage kernels per step: per node-population and stage
    2(N+1) per non-zero derivative axis, 2 per axis for the metric combination and 5 for the
    stage combination; stage 1 adds 20 (collision) and 2 d (N+1) (dense filter)."""
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
                                          "-lms", "50"], stdout=self.fh, stderr=subprocess.DEVNULL)
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
WEIGHTS = os.path.join(ROOT, "paper_2509_19171_gb300", "weights", "learned_filter_tgv3d_shear_n7.npz")


def make_form(P, torch, case, form):
    prec = P.FP64 if form == "fp64" else P.FP32DEV
    s = P.from_case(case, precision=prec, stream=torch.cuda.current_stream().cuda_stream)
    s.init_from(case.init)
    if form == "fp32dev_learned":
        w = np.load(WEIGHTS)
        s.set_learned_filter(w["params"], w["lo"], w["hi"], mass_bound=1e-6)
    return s


def max_over_ranks(ms, dist, device):
    """Largest per-rank time (ms) of the timed region, identical on every rank."""
    if not dist:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(updates_per_rank_step, steps, world, ms_max):
    """Whole-job updates/s: all ranks' units over the slowest rank's time (weak scaling)."""
    return updates_per_rank_step * steps * world / (ms_max * 1e-3)


def time_steps(torch, s, steps, dist):
    """CUDA-event time of `steps` steps on the launching stream (captured-graph launches)."""
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0.record(st)
    s.step(steps)
    e1.record(st)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    return e0.elapsed_time(e1)


def kernel_times(torch, s, steps):
    """Per-kernel CUDA-event times of `steps` eager steps (library timers)."""
    torch.cuda.synchronize()
    s.timers(True)
    s.step(steps)
    t = s.timers_read()
    s.timers(False)
    return t


def e2e_run(P, torch, case, form, steps):
    """Public-API end to end: initial fields H2D from pinned host, K steps, moments D2H to pinned host."""
    s = make_form(P, torch, case, form)
    x = s.node_coords().reshape(-1, s.dim)
    rho, u = case.init(x)
    rho_h = torch.from_numpy(np.ascontiguousarray(rho, np.float64)).pin_memory()
    u_h = torch.from_numpy(np.ascontiguousarray(u[:, : s.dim], np.float64)).pin_memory()
    rho_o = torch.empty_like(rho_h).pin_memory()
    u_o = torch.empty_like(u_h).pin_memory()
    s.init(rho_h, u_h)
    s.step(3)
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


def _oracle_sample(case, n=4):
    from oracle.selbm import OracleSELBM
    L = 2 * math.pi
    mesh = W.box_mesh((n, n, n), (0, 0, 0), (L, L, L), (True, True, True))
    return OracleSELBM(mesh, case.lattice, case.order, case.nu, cfl=case.cfl, filt=case.filt)


def _oracle_rate(args):
    """Updates/s of the oracle stepping the sample for about `seconds` (one process, 1 thread)."""
    case_name, n_el, seconds = args
    case = workload(case_name)
    o = _oracle_sample(case, n_el)
    f = o.step(o.initial_state_from(case.init))
    t0 = time.perf_counter()
    k = 0
    while time.perf_counter() - t0 < seconds:
        f = o.step(f)
        k += 1
    dt = time.perf_counter() - t0
    return o.E * o.Np * o.Q * k / dt, k, dt, o.E * o.Np * o.Q


def cpu_model():
    """CPU model of this host (lscpu's model name, else /proc/cpuinfo, else platform)."""
    import platform
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return platform.processor() or platform.machine()


def cpu_baseline(case, seconds=12.0, all_cores=True):
    """The oracle, as it stands, on a bounded sample of the workload: same lattice, order and
    filter on 4^3 elements of the same periodic cube; one thread, and every host core running
    its own copy of the sample (spawned processes, one BLAS thread each)."""
    rate1, k, dt, upd = _oracle_rate((case.name, 4, seconds))
    ncpu = os.cpu_count() or 1
    out = {"value": rate1, "unit": "node-pop updates/s", "cores": 1, "kind": "oracle",
           "cpu_model": cpu_model(), "nproc": ncpu,
           "sample": f"{case.lattice} N={case.order} TGV on 4^3 elements ({upd} updates/step), "
                     f"{k} steps in {dt:.1f} s, numpy float64, 1 thread"}
    if all_cores and ncpu > 1:
        import multiprocessing as mp
        ctx = mp.get_context("spawn")
        with ctx.Pool(ncpu) as pool:
            res = pool.map(_oracle_rate, [(case.name, 4, seconds)] * ncpu)
        total = sum(r[0] for r in res)
        out.update({"value": total, "cores": ncpu, "value_1thread": rate1,
                    "sample": out["sample"] + f"; all cores: {ncpu} processes x the same sample for "
                              f"{seconds:.0f} s each, summed"})
    return out


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
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="tgv3d", choices=["tgv3d", "pipe", "shear"])
    ap.add_argument("--forms", default="fp64,fp32dev,fp32dev_learned")
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
            cpu_baseline(case, seconds=2.0, all_cores=False)
        for _ in range(args.steps):
            cb = cpu_baseline(case, seconds=3.0, all_cores=False)
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
    if "fp32dev_learned" in forms and not os.path.exists(WEIGHTS):
        forms.remove("fp32dev_learned")
    main_form = "fp32dev_learned" if "fp32dev_learned" in forms else forms[-1]
    order = [f for f in forms if f != main_form] + [main_form]
    results, fields, clocks = {}, {}, None
    fp64_tflops = None
    ksteps = min(args.steps, 5)
    for form in order:
        rsz = 8 if form == "fp64" else 4
        s = make_form(P, torch, case, form)
        s.step(args.warmup)
        s.sync()
        sampler = ClockSampler() if (not args.no_extras and form == main_form) else None
        if sampler:
            sampler.start()
        ms = time_steps(torch, s, args.steps, dist)
        if sampler:
            clocks = sampler.stop(dev_index)
        ms = max_over_ranks(ms, dist, "cuda")
        t = kernel_times(torch, s, ksteps)
        e, _, _ = s.lattice_table()
        nz_axes = float(np.abs(e).astype(bool).sum(1).mean()) if info["affine"] else float(case.mesh.dim)
        Q = s.Q
        upd_step = case.mesh.nelem * info["Np"] * Q
        value = job_throughput(upd_step, args.steps, world, ms)
        learned = form == "fp32dev_learned"
        kb = kernel_bytes(c, Q, rsz, info["affine"], s.split, learned)
        f1, f23 = flops_per_step(case, nz_axes, Q)
        per = {k: t[k][0] / t[k][1] for k in t if t[k][1] > 0}          # ms per launch (group)
        kernel_ms = {k: per[k] for k in per}
        kernel_frac = {k: kb[k] / (per[k] * 1e-3) / 1e9 / hbm for k in per if k in kb}
        step_bytes = kb["stage1"] + 2 * kb["stage23"] + 3 * kb["assembly"]
        step_bytes += kb["learned"] if learned else (kb["prologue"] if s.split else 0)
        entry = {
            "value": value, "ms_per_step": ms / args.steps, "dtype": "f64" if form == "fp64" else "f32",
            "step_form": "population-split" if s.split else "whole-element",
            "kernel_ms": kernel_ms, "kernel_hbm_frac_alg": kernel_frac,
            "launches_per_step": launches_per_step(s.split, learned),
            "hbm_gbs_alg_step": step_bytes / (ms / args.steps * 1e-3) / 1e9,
            "bytes_per_update": step_bytes / upd_step,
            "stage23_bytes": kb["stage23"], "stage23_ms": per.get("stage23"),
        }
        if form == "fp64":
            # FP64 pipe roofline of the stage 2/3 kernel (derivative, metric and stage-combination
            # flops; the filter and collision run in the prologue or in stage 1)
            if fp64_tflops is None:
                fp64_tflops = fp64_peak(torch)
            entry["stage23_flops"] = f23
            entry["fp64_peak_tflops"] = fp64_tflops
            entry["stage23_fp64_frac"] = f23 / (per["stage23"] * 1e-3) / 1e12 / fp64_tflops
        if learned:
            st = s.learned_status()
            entry["learned"] = {"fallback_flag": st["fallback_flag"],
                                "fixed_element_steps": st["fixed_element_steps"],
                                "weights": os.path.relpath(WEIGHTS, ROOT)}
        rho, u = s.moments()
        fields[form] = (rho, u)
        results[form] = entry
        s.close()
        del s
        torch.cuda.empty_cache()
    if "fp64" in fields:
        r64, u64 = fields["fp64"]
        for form in results:
            if form == "fp64":
                continue
            r, u = fields[form]
            du = np.linalg.norm(u - u64, axis=-1)
            results[form]["err_vs_fp64"] = {
                "after_steps": args.warmup + args.steps + ksteps,
                "u_max_over_U0": float(du.max() / case.U0), "u_rms_over_U0": float(np.sqrt((du ** 2).mean()) / case.U0),
                "rho_max": float(np.abs(r - r64).max()), "rho_rms": float(np.sqrt(((r - r64) ** 2).mean()))}
        if main_form != "fp64":
            results[main_form]["speedup_vs_fp64"] = results[main_form]["value"] / results["fp64"]["value"]
    r = results[main_form]
    if main_form == "fp64":
        achieved = r["stage23_flops"] / (r["stage23_ms"] * 1e-3) / 1e12
        roof = {"bound": "alu", "kernel": "stage kernel, stages 2 and 3 (FP64 pipe)", "achieved": achieved,
                "peak": fp64_tflops, "unit": "TFLOP/s", "frac": achieved / fp64_tflops,
                "peak_source": "measured on this GPU: best cuBLAS DGEMM 4096^3", "traffic": None}
    else:
        # dominant kernel: the stage 2/3 kernel (two launches per step)
        geom = "affine" if info["affine"] else "curved"
        kern = "stage_split_kernel" if r["step_form"] == "population-split" else "stage_fast_kernel"
        name = f"{kern}<float, {case.lattice}, N={case.order}, {geom}> (stages 2, 3)"
        # ncu traffic only for the kernel instantiation it was captured on
        tkey = f"{kern}_float_{case.lattice.lower()}_n{case.order + 1}_{geom}_stage23"
        achieved = r["stage23_bytes"] / (r["stage23_ms"] * 1e-3) / 1e9
        roof = {"bound": "hbm", "kernel": name, "achieved": achieved, "peak": hbm,
                "unit": "GB/s", "frac": achieved / hbm, "peak_source": f"{pk_kind} hbm_gbs (of {pk_kind})",
                "bytes_per_launch": r["stage23_bytes"],
                "traffic": measured_traffic(tkey, case.mesh.nelem)}

    line = {"metric": metric, "value": r["value"], "unit": "node-pop updates/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": r["dtype"],
            "data": "synthetic",
            "config": workload_config(case, main_form, world),
            "roofline": roof, "forms": results,
            "gpu_launches": int(results[main_form]["launches_per_step"] * args.steps)}
    if clocks:
        line["clocks"] = clocks
    if rank == 0 and not args.no_extras:
        ms_e2e, h2d, d2h = e2e_run(P, torch, case, main_form, args.steps)
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
