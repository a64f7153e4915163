"""Benchmark: one pass of the w-BFBT Stokes hot path per step, on GB300.

A step is the whole path over one synthetic multi-sinker problem (Sec. 2.1):
viscosity/forcing setup on the GPU, the viscosity-dependent setup (sqrt(mu)
weights, three multigrid hierarchies, Chebyshev bounds, FP64 coarsest
inverses; no allocation), and the FGMRES(50) solve to a 1e-6 relative
residual with the w-BFBT block preconditioner.  Default workload: 32^3 Q2 x
P1disc, 24 seeded sinkers, omega = 0.05, delta = 200, DR = 1e6, FP64.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the CPU oracle (oracle/, FP64 SciPy) as the reference
arm.  One JSON line is printed by rank 0.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Stokes solve s to 1e-6 rel. residual & A-apply DOF/s, mixed+learned vs FP64"
WORKLOAD = "32^3-Q2-S24-DR1e6"
RTOL = 1e-6
ORACLE_SAMPLE_N = 16          # the CPU oracle runs the same problem family on a 16^3 mesh
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12   # 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz


def a_apply_flops_per_elem(k: int) -> float:
    """Algorithmic flops of one sum-factorised A element apply: 36 n^4 + 30 n^3, n = k + 1."""
    n = k + 1
    return 36.0 * n ** 4 + 30.0 * n ** 3


def a_apply_bytes_per_node(dtype_bytes: int) -> float:
    """Algorithmic HBM bytes per node of one A apply: u (3) + y (3) + mu (1) words."""
    return 7.0 * dtype_bytes


# --------------------------------------------------------------------------- CPU oracle arm

def oracle_sample(cfg: dict, n_sample: int, its_target: int | None) -> dict:
    """Run the oracle (setup + solve) on an n_sample^3 mesh in a fresh single-threaded process.

    Returns seconds for the sample and the estimate scaled to the workload size:
    (setup + solve * its_target / its_sample) * dof_workload / dof_sample.
    """
    code = f"""
import json, time, sys
sys.path.insert(0, {ROOT!r})
from oracle import mesh as M, wbfbt as W
from paper_1607_03936_gb300 import inputs
n, k = {n_sample}, {cfg['k']}
m = M.Mesh(n, n, n, k)
c = inputs.sinker_centres({cfg['seed']}, {cfg['n_sinkers']})
t0 = time.perf_counter()
mu, f = W.sinker_problem(m, c, {cfg['omega']}, {cfg['delta']}, {cfg['dr']})
prob = W.StokesProblem(m, mu)
pc = W.BlockPreconditioner(prob, 'vcycle', -1.0)
import numpy as np
from oracle import operators as op, krylov
F = np.concatenate([op.load_vector(m, f), np.zeros(m.n_p)])
t1 = time.perf_counter()
x, its, rel = krylov.fgmres(prob.apply_K, pc.apply, F, rtol={RTOL}, restart=50)
t2 = time.perf_counter()
print(json.dumps(dict(setup=t1 - t0, solve=t2 - t1, its=its, rel=rel, dof=m.n_u + m.n_p)))
"""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=900)
    if out.returncode != 0:
        raise RuntimeError("oracle sample failed: " + out.stderr[-2000:])
    r = json.loads(out.stdout.strip().splitlines()[-1])
    n, k = cfg["n"], cfg["k"]
    dof_w = 3 * (k * n + 1) ** 3 + n ** 3 * k * (k + 1) * (k + 2) // 6
    its = its_target if its_target else r["its"]
    r["estimate_s"] = (r["setup"] + r["solve"] * its / r["its"]) * dof_w / r["dof"]
    r["dof_workload"] = dof_w
    return r


def run_reference(args, cfg, rank, world):
    if rank != 0:
        return
    for _ in range(args.warmup):
        oracle_sample(cfg, ORACLE_SAMPLE_N, None)
    runs = [oracle_sample(cfg, ORACLE_SAMPLE_N, None) for _ in range(args.steps)]
    est = [r["estimate_s"] for r in runs]
    v = statistics.mean(est)
    sample = (f"oracle setup+solve on a {ORACLE_SAMPLE_N}^3 mesh of the same problem family "
              f"({runs[0]['its']} its, {runs[0]['setup'] + runs[0]['solve']:.1f} s), scaled by DOF "
              f"({runs[0]['dof']} -> {runs[0]['dof_workload']})")
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "s", "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * v, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded multi-sinker, Sec. 2.1)",
        "config": config_dict(cfg, "fp64"),
        "cpu_baseline": {"value": v, "unit": "s", "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def config_dict(cfg, precision):
    n, k = cfg["n"], cfg["k"]
    return {"workload": WORKLOAD, "mesh": f"{n}x{n}x{n} Q{k} x P{k - 1}disc",
            "u_dof": 3 * (k * n + 1) ** 3, "p_dof": n ** 3 * k * (k + 1) * (k + 2) // 6,
            "sinkers": cfg["n_sinkers"], "omega": cfg["omega"], "delta": cfg["delta"], "dr": cfg["dr"],
            "rtol": RTOL, "krylov": "FGMRES(50)", "precision": precision, "parallelism": "replicas",
            "l2": "flushed between steps (256 MiB write)"}


# --------------------------------------------------------------------------- clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.proc = None
        self.index = index
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (FileNotFoundError, OSError):
            self.proc = None

    def stop(self) -> dict | None:
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=10)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# --------------------------------------------------------------------------- multi-rank helpers

def replica_seed(base_seed: int, rank: int) -> int:
    """Replicas: rank r solves the seeded problem base_seed + r (no data-path collective)."""
    return base_seed + rank


def max_over_ranks(value: float, world: int, device=None) -> float:
    """Max of a per-rank timing over all ranks (the job's step time); identity for one rank."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# --------------------------------------------------------------------------- GPU arm

def traffic_for(kernel: str):
    """DRAM bytes per launch from the committed ncu summary, if the kernel source is unchanged."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(path):
        return None
    data = json.load(open(path))
    ent = data.get(kernel)
    if not ent:
        return None
    srcs = ent["source"] if isinstance(ent["source"], list) else [ent["source"]]
    shas = ent["source_sha256"] if isinstance(ent["source_sha256"], list) else [ent["source_sha256"]]
    for src, want in zip(srcs, shas):
        if hashlib.sha256(open(os.path.join(ROOT, src), "rb").read()).hexdigest() != want:
            return None
    return ent["dram_bytes_per_launch"]


def run_ours(args, cfg, rank, world):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_1607_03936_gb300 import build
    build.build()
    from paper_1607_03936_gb300 import inputs
    from paper_1607_03936_gb300 import wbfbt as wb

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    n, k = cfg["n"], cfg["k"]
    seed = replica_seed(cfg["seed"], rank)
    centres = inputs.sinker_centres(seed, cfg["n_sinkers"])
    mu, f = wb.sinker_setup(n, k, centres, cfg["omega"], cfg["delta"], cfg["dr"])
    precision = wb.MIXED if args.precision == "mixed" else wb.F64
    solver = wb.Solver(n, k, mu, precision=precision)
    u = torch.empty(solver.n_u, dtype=torch.float64, device=dev)
    p = torch.empty(solver.n_p, dtype=torch.float64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    st = torch.cuda.current_stream()

    def step():
        m2, f2 = wb.sinker_setup(n, k, centres, cfg["omega"], cfg["delta"], cfg["dr"])
        e_a = torch.cuda.Event(enable_timing=True)
        e_a.record(st)
        solver.setup(m2)
        e_b = torch.cuda.Event(enable_timing=True)
        e_b.record(st)
        _, _, res = solver.solve(f2, rtol=RTOL, u=u, p=p)
        e_c = torch.cuda.Event(enable_timing=True)
        e_c.record(st)
        return res, (e_a, e_b, e_c)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = ClockSampler(dev.index) if rank == 0 else None
    launches0 = wb.launch_count()
    times, setups, solves, iters, rels = [], [], [], [], []
    wall0 = time.perf_counter()
    for _ in range(args.steps):
        flush.fill_(float(len(times)))        # evict L2 between steps (outside the step's events)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(st)
        res, (ea, eb, ec) = step()
        e1.record(st)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1) / 1e3)
        setups.append(ea.elapsed_time(eb) / 1e3)
        solves.append(eb.elapsed_time(ec) / 1e3)
        iters.append(res.iters)
        rels.append(res.rel_res)
        if res.status != 0:
            raise RuntimeError(f"solve failed: {res}")
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    if world > 1:
        dist.barrier()
    launches = wb.launch_count() - launches0
    clk = clocks.stop() if clocks else None
    t_step = max_over_ranks(statistics.mean(times), world, dev)

    # dominant kernel: the fine-level A apply, timed on the launching stream with CUDA events
    xk = torch.randn(solver.n_u, dtype=torch.float64, device=dev)
    xk32 = xk.float()

    def time_apply(x, reps=20):
        for _ in range(3):
            solver.apply_A(x)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(reps):
            solver.apply_A(x)
        e1.record(st)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3 / reps

    t_a64 = time_apply(xk)
    t_a32 = time_apply(xk32)
    n_elem, n_nodes = solver.n_elem, solver.n_nodes
    flops = a_apply_flops_per_elem(k) * n_elem
    achieved = flops / t_a64 / 1e12
    hbm_peak = None
    peaks_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(peaks_path):
        hbm_peak = json.load(open(peaks_path)).get("hbm_gbs")
    hbm_note = "of measured" if hbm_peak else "of fallback"
    hbm_peak = hbm_peak or 6800.0
    bytes32 = a_apply_bytes_per_node(4) * n_nodes
    roofline = {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved / FP64_PEAK_TFLOPS, "traffic": traffic_for("apply_A_f64"),
                "kernel": "k_q2_elem64<OP_A,iso> + k_q2_gather<double,3,STORE> (one A apply)",
                "per_launch": ("one fine-level A apply (element pass + node pass), 36n^4+30n^3 flops per element "
                               "(the kernel executes about 1300 FP64 operations per element: constant GLL "
                               "derivative sums)"),
                "peak_note": "FP64 ALU peak derived from 152 SMs x 2 DFMA/clk x 2.07 GHz"}
    roofline_fp32 = {"bound": "hbm", "achieved": bytes32 / t_a32 / 1e9, "peak": hbm_peak, "unit": "GB/s",
                     "frac": bytes32 / t_a32 / 1e9 / hbm_peak, "traffic": traffic_for("apply_A_f32"),
                     "kernel": "k_q2_elem<OP_A> + k_q2_gather<3,STORE> (one A apply)", "peak_note": hbm_note}

    # end-to-end through the C ABI with host buffers (copies inside the timed region)
    mu_h = torch.empty(solver.n_nodes, dtype=torch.float64).pin_memory()
    f_h = torch.empty(solver.n_u, dtype=torch.float64).pin_memory()
    mu_h.copy_(mu)
    f_h.copy_(f)
    u_h = torch.empty(solver.n_u, dtype=torch.float64).pin_memory()
    p_h = torch.empty(solver.n_p, dtype=torch.float64).pin_memory()
    torch.cuda.synchronize()
    e2e = []
    for i in range(max(1, min(args.steps, 3))):
        flush.fill_(float(i))
        torch.cuda.synchronize()
        w0 = time.perf_counter()
        solver.setup(mu_h)
        solver.solve(f_h, rtol=RTOL, u=u_h, p=p_h)
        e2e.append(time.perf_counter() - w0)
    h2d = 8 * solver.n_nodes + 8 * solver.n_u
    d2h = 8 * solver.n_u + 8 * solver.n_p

    # the metric's other side: the mixed-precision solve of the same problem, timed the same way
    # (outside the FP64 timed region), and its distance from the FP64 solution
    mixed = None
    if precision == wb.F64:
        u64, p64 = u.clone(), p.clone()
        sm = wb.Solver(n, k, mu, precision=wb.MIXED)
        um = torch.empty_like(u)
        pm = torch.empty_like(p)

        def step_mixed():
            m2, f2 = wb.sinker_setup(n, k, centres, cfg["omega"], cfg["delta"], cfg["dr"])
            sm.setup(m2)
            return sm.solve(f2, rtol=RTOL, u=um, p=pm)[2]

        for _ in range(args.warmup):
            step_mixed()
        tm = []
        for i in range(args.steps):
            flush.fill_(float(i))
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(st)
            rm = step_mixed()
            e1.record(st)
            torch.cuda.synchronize()
            tm.append(e0.elapsed_time(e1) / 1e3)
        t_mixed = max_over_ranks(statistics.mean(tm), world, dev)
        mixed = {"s_per_step": t_mixed, "speedup_vs_fp64": t_step / t_mixed, "iters": rm.iters,
                 "final_rel_res": rm.rel_res,
                 "rel_err_u_vs_fp64": float(torch.linalg.norm(um - u64) / torch.linalg.norm(u64)),
                 "rel_err_p_vs_fp64": float(torch.linalg.norm(pm - p64) / torch.linalg.norm(p64)),
                 "learned": "not attached (no measured gain; every learned step was rejected on held-out problems)"}
        sm.close()

    if rank != 0:
        return
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        r = oracle_sample(cfg, ORACLE_SAMPLE_N, iters[-1])
        cpu = {"value": r["estimate_s"], "unit": "s", "cores": 1, "kind": "oracle",
               "sample": (f"oracle setup+solve on a {ORACLE_SAMPLE_N}^3 mesh of the same problem family "
                          f"({r['its']} its, {r['setup'] + r['solve']:.1f} s single-threaded), scaled by DOF "
                          f"and by the GPU iteration count ({iters[-1]})")}
    line = {
        "metric": METRIC, "value": t_step, "unit": "s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t_step, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if precision == wb.F64 else "f32+f64",
        "data": "synthetic (seeded multi-sinker, Sec. 2.1)", "config": config_dict(cfg, args.precision),
        "iters": iters[-1], "final_rel_res": rels[-1], "setup_s": statistics.mean(setups),
        "solve_s": statistics.mean(solves), "wall_s": wall,
        "a_apply_dof_per_s": {"fp64": solver.n_u / t_a64, "fp32": solver.n_u / t_a32},
        "roofline": roofline, "roofline_fp32": roofline_fp32, "cpu_baseline": cpu,
        "e2e": {"value": statistics.mean(e2e), "unit": "s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": launches, "clocks": clk, "mixed": mixed,
    }
    print(json.dumps(line), flush=True)
    solver.close()


def run_profile(args, cfg):
    import torch

    from paper_1607_03936_gb300 import build
    build.build()
    from paper_1607_03936_gb300 import inputs
    from paper_1607_03936_gb300 import wbfbt as wb

    n, k = cfg["n"], cfg["k"]
    centres = inputs.sinker_centres(cfg["seed"], cfg["n_sinkers"])
    mu, f = wb.sinker_setup(n, k, centres, cfg["omega"], cfg["delta"], cfg["dr"])
    solver = wb.Solver(n, k, mu, precision=wb.MIXED if args.precision == "mixed" else wb.F64)
    n0 = wb.launch_count()
    _, _, res = solver.solve(f, rtol=RTOL)
    torch.cuda.synchronize()
    print(json.dumps({"profile": WORKLOAD, "create_launches": n0, "solve_launches": wb.launch_count() - n0,
                      "iters": res.iters, "rel_res": res.rel_res}), flush=True)
    solver.close()


def run_profile_apply(args, cfg):
    """One fine-level A apply in FP64 and one in FP32 inside an NVTX range "prof" (after three
    warm-up applies each), for ncu --nvtx --nvtx-include prof/ captures of the operator kernels."""
    import torch

    from paper_1607_03936_gb300 import build
    build.build()
    from paper_1607_03936_gb300 import inputs
    from paper_1607_03936_gb300 import wbfbt as wb

    n, k = cfg["n"], cfg["k"]
    centres = inputs.sinker_centres(cfg["seed"], cfg["n_sinkers"])
    mu, _ = wb.sinker_setup(n, k, centres, cfg["omega"], cfg["delta"], cfg["dr"])
    s64 = wb.Solver(n, k, mu, precision=wb.F64, restart=5)
    s32 = wb.Solver(n, k, mu, precision=wb.MIXED, restart=5)
    u64 = torch.randn(s64.n_u, dtype=torch.float64, device="cuda", generator=torch.Generator("cuda").manual_seed(0))
    u32 = u64.float()
    for _ in range(3):
        s64.apply_A(u64)
        s32.apply_A(u32)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("prof")
    s64.apply_A(u64)
    s32.apply_A(u32)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    print(json.dumps({"profile_apply": WORKLOAD, "n_u": s64.n_u}), flush=True)
    s64.close()
    s32.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["fp64", "mixed"], default="fp64")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--profile", action="store_true",
                    help="one setup + solve of the workload and nothing else (for an ncu launch list)")
    ap.add_argument("--profile-apply", action="store_true",
                    help="one FP64 and one FP32 A apply in an NVTX range 'prof' (for ncu --set full)")
    args = ap.parse_args()
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    from paper_1607_03936_gb300 import inputs
    cfg = dict(inputs.WORKLOADS[WORKLOAD])
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        run_reference(args, cfg, rank, world)
        return
    if args.profile_apply:
        run_profile_apply(args, cfg)
        return
    if args.profile:
        run_profile(args, cfg)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        dist.init_process_group("nccl")
    run_ours(args, cfg, rank, world)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
