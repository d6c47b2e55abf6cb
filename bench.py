#!/usr/bin/env python
"""Benchmark of the spaQR hot path: seconds to ||A^T (A x - b)|| / ||A^T b|| < 1e-10
(factorization + W-preconditioned CGLS) on the 2D 1024x1024 grid least-squares
problem with high-contrast weights w = 10^U[-3,3] (N = 1,048,576 unknowns,
M = 3,143,680 rows), nested dissection depth 16.

One step = spaqr_factor (host CSR in, every floating-point step on the GPU)
followed by spaqr_solve with b and x in device memory.  The end-to-end figure
(e2e) repeats the step through the C ABI with host b and x (copies inside).
With --gpus N > 1 every rank solves an independent replica (seed = rank); the
path has no exchange between ranks, so no collective touches the data path.

--impl reference times the CPU oracle (oracle/) on a bounded sample of the
same workload (a smaller grid of the same family) and scales it to the full
size by M log2 N (the paper's Section 3 factorization cost).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "factor+solve seconds to ||A^T r||/||A^T b|| < 1e-10"
UNIT = "s"
WORKLOAD = "grid2d_1024"
PEAKS = {"fp64_alu_tflops": 1.25, "fp32_alu_tflops": 80.5}  # recipe FP64 figure; FP32 = 152 SM x 128 x 2 x 2.07 GHz


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--eps", type=float, default=1e-6)
    ap.add_argument("--precision", default="mixed", choices=["fp64", "mixed"])
    ap.add_argument("--compare", default="fp64", choices=["fp64", "mixed", "none"],
                    help="also time this precision on the same workload (reported under config.compare)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--clocks-dir", default=None, help="where the nvidia-smi clock samples of the timed region go "
                                                        "(default: the system temporary directory)")
    ap.add_argument("--sample", default=None,
                    help="oracle sample for the CPU baseline (default: a 128^2 grid of the workload's family)")
    args = ap.parse_args()
    if args.sample is None:
        args.sample = "invpoisson2d_128" if args.workload.startswith("invpoisson") else "grid2d_128_c3"
    return args


# --------------------------------------------------------------------- oracle
def _oracle_sample_spec(name):
    # same family (2D grid, w = 10^U[-3,3], or the Inverse-Poisson J^T), smaller
    # size; depth from the paper's default ceil(log2(N/64)) so that leaves keep
    # the full-size leaf size
    sizes = {"grid2d_64_c3": 64, "grid2d_96_c3": 96, "grid2d_128_c3": 128, "grid2d_160_c3": 160,
             "invpoisson2d_64": 64, "invpoisson2d_128": 128}
    nx = sizes[name]
    depth = max(2, math.ceil(math.log2(nx * nx / 64)))
    return nx, depth


def oracle_sample_seconds(name: str, eps: float) -> dict:
    """Time the oracle (factor + solve) on the sample in a fresh single-threaded process."""
    nx, depth = _oracle_sample_spec(name)
    make = ("from inputs.inverse_poisson import inverse_poisson\np = inverse_poisson(%d, 2, seed=0)\n" % nx
            if name.startswith("invpoisson") else
            "from inputs.grid_ls import grid_problem\np = grid_problem(%d, %d, 1, 'c3', 0)\n" % (nx, nx))
    code = (
        "import sys,time,json; sys.path.insert(0, %r)\n"
        "%s"
        "from oracle.spaqr import OracleSpaQR\n"
        "t = time.perf_counter(); o = OracleSpaQR(p, %d, %r).factor(); x, info = o.solve(p.b); t = time.perf_counter() - t\n"
        "print(json.dumps(dict(seconds=t, iters=info['iters'], m=p.m, n=p.n)))\n"
    ) % (ROOT, make, depth, eps)
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, check=True)
    r = json.loads(out.stdout.strip().splitlines()[-1])
    r.update(nx=nx, depth=depth)
    return r


def scale_to_full(sample: dict, m_full: int, n_full: int) -> float:
    return sample["seconds"] * (m_full * math.log2(n_full)) / (sample["m"] * math.log2(sample["n"]))


# ------------------------------------------------------------------- clocks
class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int, directory: str | None = None):
        import tempfile

        self.index = index
        self.proc = None
        self.path = os.path.join(directory or tempfile.gettempdir(), f"spaqr_clocks_rank{index}.csv")

    def start(self):
        os.makedirs(os.path.dirname(self.path), exist_ok=True)
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm), "reasons": sorted(reasons)}


# -------------------------------------------------------------------- main
def reduce_max(value, device=None):
    """Largest value over all ranks (the timing of the slowest replica)."""
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_seconds(max_secs, world):
    """Whole-job seconds per problem: `world` independent replicas finish in the
    slowest rank's time."""
    return max_secs / world


def run_gpu(args, rank, world):
    import numpy as np
    import torch

    import paper_2102_09878_gb300 as sq
    from inputs.grid_ls import workload

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    prob, depth = workload(args.workload, seed=rank)
    an = sq.Analysis(prob.dims, depth)
    stream = torch.cuda.Stream()
    b_dev = torch.from_numpy(prob.b).to(dev)
    torch.cuda.synchronize()

    def step(host_io=False):
        g = sq.SpaQR(prob, an, eps=args.eps, precision=args.precision, stream=stream)
        with torch.cuda.stream(stream):
            x = g.solve(prob.b) if host_io else g.solve(b_dev)
        return g, x

    for _ in range(args.warmup):
        g, x = step()
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.barrier()
    torch.cuda.synchronize()
    clk = ClockSampler(dev.index, args.clocks_dir)
    clk.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    kt = {k: 0.0 for k in ["copy", "front_qr", "qrcp", "other", "apply", "spmv"]}
    kn = {k: 0 for k in kt}
    flops_front = 0.0
    flops_qrcp = 0.0
    bytes_qrcp = 0.0
    launches = 0
    iters = []
    t_factor, t_solve = [], []
    ev0.record(stream)
    for _ in range(args.steps):
        g, x = step()
        st = g.stats()
        for k in kt:
            kt[k] += st["t_kernel"][k]
            kn[k] += st["n_kernel"][k]
        flops_front += st["flops_front"]
        flops_qrcp += st["flops_qrcp"]
        bytes_qrcp += st["bytes_qrcp"]
        launches += st["launches"] + st["n_kernel"]["apply"] + 9 * st["iters"]
        iters.append(st["iters"])
        t_factor.append(st["t_factor"])
        t_solve.append(st["t_solve"])
    ev1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = clk.stop()
    secs = ev0.elapsed_time(ev1) / 1e3 / args.steps
    A = prob.to_scipy()
    xh = x.cpu().numpy()
    rel = float(np.linalg.norm(A.T @ (A @ xh - prob.b)) / np.linalg.norm(A.T @ prob.b))
    stats = g.stats()

    e2e = None
    if not args.no_e2e:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ne = max(1, min(args.steps, 2))
        for _ in range(ne):
            g2, xh2 = step(host_io=True)
        torch.cuda.synchronize()
        te = (time.perf_counter() - t0) / ne
        e2e = {"value": te, "unit": UNIT, "h2d_bytes_per_step": int(prob.rowptr.nbytes + prob.colidx.nbytes
                                                                     + prob.vals.nbytes + prob.b.nbytes),
               "d2h_bytes_per_step": int(xh2.nbytes)}
    if dist:
        secs = reduce_max(secs, dev)
    compare = None
    if args.compare != "none" and args.compare != args.precision:
        # the other precision on the same workload, same timing (device events over K steps)
        for _ in range(max(1, args.warmup)):
            sq.SpaQR(prob, an, eps=args.eps, precision=args.compare, stream=stream).solve(b_dev)
        torch.cuda.synchronize()
        c0 = torch.cuda.Event(enable_timing=True)
        c1 = torch.cuda.Event(enable_timing=True)
        its = []
        c0.record(stream)
        for _ in range(args.steps):
            gc = sq.SpaQR(prob, an, eps=args.eps, precision=args.compare, stream=stream)
            with torch.cuda.stream(stream):
                gc.solve(b_dev)
            its.append(gc.stats()["iters"])
        c1.record(stream)
        torch.cuda.synchronize()
        sc = gc.stats()
        compare = {"precision": args.compare, "seconds": c0.elapsed_time(c1) / 1e3 / args.steps, "iters": its,
                   "t_factor": sc["t_factor"], "t_solve": sc["t_solve"],
                   "kernel_seconds": {k: v for k, v in sc["t_kernel"].items()}}
    return dict(secs=secs, prob=prob, depth=depth, stats=stats, kt=kt, kn=kn, flops_front=flops_front, workload=args.workload,
                flops_qrcp=flops_qrcp, bytes_qrcp=bytes_qrcp, compare=compare,
                launches=launches, iters=iters, rel=rel, e2e=e2e, clocks=clocks, t_factor=t_factor,
                t_solve=t_solve, t_analyze=stats["t_analyze"])


HBM_PEAK = 6660.3  # GB/s, MEASURED_PEAKS.json hbm_gbs
# DRAM bytes of all QRCP launches of one factorization, from one ncu capture of
# the current kernels (profiles/qrcp_dram_grid2d_1024_mixed.md); empty while the
# kernels have changed since the last capture
QRCP_DRAM_BYTES = {("grid2d_1024", "mixed"): 1.851e9}


def family_rooflines(res, precision):
    """Live roofline of every device kernel family over the timed steps (CUDA
    events recorded by the library on its stream around each launch)."""
    kt = res["kt"]
    st = res["stats"]
    alu = PEAKS["fp64_alu_tflops"] if precision == "fp64" else PEAKS["fp32_alu_tflops"]
    alu_src = ("FP64 rate of the recipe table, 1.25 TFLOP/s (of nominal)" if precision == "fp64" else
               "FP32 lanes: 152 SMs x 128 x 2 flops x 2.07 GHz = 80.5 TFLOP/s (derived, of nominal)")
    out = {}
    if kt["qrcp"] > 0:
        steps = max(1, len(res["iters"]))
        ach = res["flops_qrcp"] / kt["qrcp"] / 1e12
        dram = QRCP_DRAM_BYTES.get((res["workload"], precision))
        out["qrcp"] = {"kernel": "column-pivoted QR (sparsification steps 1 and 2)", "bound": "alu", "achieved": ach,
                       "peak": alu, "unit": "TFLOP/s", "frac": ach / alu,
                       "traffic": dram, "traffic_basis": "DRAM bytes of all QRCP launches of one factorization (ncu, "
                                                         "profiles/qrcp_dram_grid2d_1024_mixed.md)" if dram else None,
                       "peak_source": alu_src,
                       "memory_view": {"algorithmic_bytes_per_step": res["bytes_qrcp"] / steps,
                                       "algorithmic_gbs": res["bytes_qrcp"] / kt["qrcp"] / 1e9,
                                       "dram_gbs": (dram * steps / kt["qrcp"] / 1e9) if dram else None,
                                       "note": "per-step passes over the trailing block stay on chip (shared "
                                               "memory or L2); the kernels are bound by the sequential pivot "
                                               "chain"}}
    if kt["front_qr"] > 0:
        ach = res["flops_front"] / kt["front_qr"] / 1e12
        out["front_qr"] = {"kernel": "front QR (eliminate + scale)", "bound": "alu", "achieved": ach, "peak": alu,
                           "unit": "TFLOP/s", "frac": ach / alu, "traffic": None, "peak_source": alu_src}
    if kt["apply"] > 0:
        ach = st["bytes_apply"] * sum(res["iters"]) / kt["apply"] / 1e9
        out["apply"] = {"kernel": "W^-1/W^-T apply", "bound": "hbm", "achieved": ach, "peak": HBM_PEAK,
                        "unit": "GB/s", "frac": ach / HBM_PEAK, "traffic": None,
                        "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)"}
    return out


def roofline(res, precision):
    """Roofline of the device kernel family with the largest share of the timed steps."""
    kt = res["kt"]
    dom = max(kt, key=lambda k: kt[k])
    fam = family_rooflines(res, precision)
    key = dom if dom in fam else max(fam, key=lambda k: kt[k])
    out = dict(fam[key])
    out["share"] = kt[key] / max(sum(kt.values()), 1e-12)
    return out


def main():
    args = parse()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    if args.impl == "reference":
        if rank != 0:
            return 0
        from inputs.grid_ls import WORKLOADS

        nx, ny, nz = WORKLOADS[args.workload]["dims"]
        n_full = nx * ny * nz
        m_full = (nx - 1) * ny * nz + nx * (ny - 1) * nz + (nx * ny * (nz - 1) if nz > 1 else 0) + n_full
        sample = "invpoisson2d_64" if args.workload.startswith("invpoisson") else "grid2d_64_c3"
        vals = []
        for i in range(args.warmup + args.steps):
            r = oracle_sample_seconds(sample, args.eps)
            if i >= args.warmup:
                vals.append(scale_to_full(r, m_full, n_full))
        v = statistics.median(vals)
        desc = f"oracle factor+solve on the {r['nx']}x{r['nx']} grid of the same family (depth {r['depth']}, " \
               f"eps {args.eps}, {r['iters']} CGLS iterations), scaled by M log2 N to the full workload"
        line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": v * 1e3, "higher_is_better": False,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": args.workload, "eps": args.eps},
                "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": desc},
                "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return 0

    if world > 1:
        import torch
        import torch.distributed as dist

        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        dist.init_process_group("nccl")
    res = run_gpu(args, rank, world)
    if rank != 0:
        return 0
    prob, st = res["prob"], res["stats"]
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        try:
            r = oracle_sample_seconds(args.sample, args.eps)
            v = scale_to_full(r, prob.m, prob.n)
            cpu = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                   "sample": f"oracle factor+solve on the {r['nx']}x{r['nx']} grid of the same family "
                             f"(depth {r['depth']}, eps {args.eps}) took {r['seconds']:.2f} s, scaled by M log2 N"}
        except Exception as e:  # pragma: no cover
            cpu = {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": f"failed: {e}"}
    value = job_seconds(res["secs"], world)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": res["secs"] * 1e3, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f32-factor/f64-cgls",
        "data": "synthetic",
        "config": {"workload": args.workload, "grid": list(prob.dims), "n": prob.n, "m": prob.m, "depth": res["depth"],
                   "eps": args.eps, "precision": args.precision, "weights": {"u12": "U[1,2)", "c3": "10^U[-3,3]", "c2": "10^U[-2,2]",
                                                         "ip": "Inverse-Poisson J^T, u ~ U[-1,1), z ~ U[1,2)"}[prob.law], "tol": 1e-10,
                   "l2": "inputs larger than L2 (no flush needed)", "parallelism": f"replicas{world}"},
        "e2e": res["e2e"], "gpu_launches": int(res["launches"]), "clocks": res["clocks"],
        "roofline": roofline(res, args.precision), "cpu_baseline": cpu,
        "compare": res["compare"],
        "detail": {"iters": res["iters"], "rel_resid": res["rel"], "t_factor": res["t_factor"],
                   "t_solve": res["t_solve"], "t_analyze": res["t_analyze"], "nnz_W": st["nnz_W"],
                   "kernel_seconds": res["kt"], "kernel_launches": res["kn"], "flops_front": res["flops_front"],
                   "flops_qrcp": res["flops_qrcp"], "bytes_qrcp": res["bytes_qrcp"],
                   "rooflines": family_rooflines(res, args.precision),
                   "phase_seconds": st["t_phase"], "syncs": st["syncs"], "top_front": [st["top_rows"], st["top_cols"]],
                   "max_front": [st["max_front_rows"], st["max_front_cols"]]},
    }
    print(json.dumps(line))
    return 0


if __name__ == "__main__":
    sys.exit(main())
