"""Benchmark: one pass of the w-BFBT Stokes hot path per step, on GB300.

A step is the whole path over one synthetic multi-sinker problem (Sec. 2.1):
viscosity and forcing at the nodes on the GPU, the viscosity-dependent setup
(sqrt(mu) weights, three multigrid hierarchies, Chebyshev bounds, FP64
coarsest inverses; no allocation), and the FGMRES(50) solve to a 1e-6
relative residual with the w-BFBT block preconditioner.

Default workload: 64^3 Q2 x P1disc, 64 seeded sinkers, omega = 0.04,
delta = 400, DR = 1e10 (the largest single-GPU configuration).  `value` is
the mixed-precision step (FP32 preconditioner, FP64 Krylov, true residual and
coarsest solve); the plain FP64 step of the same problem is timed beside it
(`fp64`), and both solutions are compared.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload NAME] [--precision mixed|fp64]

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
DEFAULT_WORKLOAD = "64^3-Q2-S64-DR1e10"
ORACLE_WORKLOAD = "32^3-Q2-S24-DR1e6"     # the largest configuration the oracle solves in bounded time
RTOL = 1e-6
ORACLE_SAMPLE_ITERS = 2                   # FGMRES iterations per reference-arm step
# FP64 FGMRES iteration counts of the GPU path per workload (the GPU FP64 solve takes the oracle's
# count +-1 where the oracle runs: 40 at 32^3); the reference arm scales its per-iteration time by them.
FP64_ITERS = {"8^3-Q2-S4-DR1e4": 50, "32^3-Q2-S24-DR1e6": 40, "24^3-Q3-S32-DR1e8": 43, "64^3-Q2-S64-DR1e10": 104}
L2_FLUSH_BYTES = 256 * 1024 * 1024


def a_apply_flops_per_elem(k: int) -> float:
    """Algorithmic flops of one sum-factorised A element apply: 36 n^4 + 30 n^3, n = k + 1."""
    n = k + 1
    return 36.0 * n ** 4 + 30.0 * n ** 3


def a_apply_bytes_per_node(dtype_bytes: int) -> float:
    """Algorithmic HBM bytes per node of one A apply: u (3) + y (3) + mu (1) words."""
    return 7.0 * dtype_bytes


def dof_counts(cfg: dict) -> tuple[int, int]:
    n, k = cfg["n"], cfg["k"]
    return 3 * (k * n + 1) ** 3, n ** 3 * k * (k + 1) * (k + 2) // 6


def config_dict(name: str, cfg: dict, precision: str) -> dict:
    n, k = cfg["n"], cfg["k"]
    u_dof, p_dof = dof_counts(cfg)
    return {"workload": name, "mesh": f"{n}x{n}x{n} Q{k} x P{k - 1}disc", "u_dof": u_dof, "p_dof": p_dof,
            "sinkers": cfg["n_sinkers"], "omega": cfg["omega"], "delta": cfg["delta"], "dr": cfg["dr"],
            "rtol": RTOL, "krylov": "FGMRES(50)", "precision": precision, "parallelism": "replicas",
            "l2": "flushed between steps (256 MiB write)"}


# --------------------------------------------------------------------------- CPU oracle legs

_ORACLE_CODE = """
import json, sys, time
sys.path.insert(0, {root!r})
import numpy as np
from oracle import krylov, mesh as M, operators as op, wbfbt as W
from paper_1607_03936_gb300 import inputs
cfg = {cfg!r}
m = M.Mesh(cfg['n'], cfg['n'], cfg['n'], cfg['k'])
c = inputs.sinker_centres(cfg['seed'], cfg['n_sinkers'])
t0 = time.perf_counter()
mu, f = W.sinker_problem(m, c, cfg['omega'], cfg['delta'], cfg['dr'])
prob = W.StokesProblem(m, mu)
pc = W.BlockPreconditioner(prob, 'vcycle', -1.0)
F = np.concatenate([op.load_vector(m, f), np.zeros(m.n_p)])
t1 = time.perf_counter()
x, its, rel = krylov.fgmres(prob.apply_K, pc.apply, F, rtol={rtol}, restart=50)
t2 = time.perf_counter()
if {save!r}:
    np.savez({save!r}, u=x[:m.n_u], p=op.project_pressure(m, x[m.n_u:]))
print(json.dumps(dict(setup=t1 - t0, solve=t2 - t1, its=its, rel=rel, dof=m.n_u + m.n_p)))
"""


def _oracle_env() -> dict:
    return dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
                CUDA_VISIBLE_DEVICES="")


def start_oracle_solve(cfg: dict, save: str = "") -> subprocess.Popen:
    """The oracle's full setup + solve of `cfg`, single-threaded, in a separate process (started
    before this process touches the GPU); the solution goes to the .npz file `save` if given."""
    code = _ORACLE_CODE.format(root=ROOT, cfg=cfg, rtol=RTOL, save=save)
    return subprocess.Popen([sys.executable, "-c", code], env=_oracle_env(), stdout=subprocess.PIPE,
                            stderr=subprocess.PIPE, text=True)


def finish_oracle_solve(proc: subprocess.Popen, timeout: float = 1200.0) -> dict:
    out, err = proc.communicate(timeout=timeout)
    if proc.returncode != 0:
        raise RuntimeError("oracle solve failed: " + err[-2000:])
    return json.loads(out.strip().splitlines()[-1])


def run_reference(args, name, cfg, rank, world):
    """The reference arm: the CPU oracle, single-threaded, on the host cores.

    The oracle cannot run the 64^3 workload in bounded time (CSR A alone holds ~2.4e9
    nonzeros, ~29 GB, and a solve would take hours), so each step is a bounded sample of the
    same problem family at 32^3 (Q2, S24, DR 1e6, the configuration the oracle solves in ~1.5
    min): ORACLE_SAMPLE_ITERS FGMRES iterations from x0 = 0 with the V-cycle preconditioner.  The
    oracle's setup (assembly, hierarchies) is timed once in the warm-up.  `value` scales setup
    and per-iteration time by DOF to the workload and by its FP64 iteration count.
    """
    if rank != 0:
        return
    import numpy as np

    from oracle import krylov
    from oracle import mesh as M
    from oracle import operators as op
    from oracle import wbfbt as W
    from paper_1607_03936_gb300 import inputs

    ocfg = dict(inputs.WORKLOADS[ORACLE_WORKLOAD])
    m = M.Mesh(ocfg["n"], ocfg["n"], ocfg["n"], ocfg["k"])
    c = inputs.sinker_centres(ocfg["seed"], ocfg["n_sinkers"])
    t0 = time.perf_counter()
    mu, f = W.sinker_problem(m, c, ocfg["omega"], ocfg["delta"], ocfg["dr"])
    prob = W.StokesProblem(m, mu)
    pc = W.BlockPreconditioner(prob, "vcycle", -1.0)
    F = np.concatenate([op.load_vector(m, f), np.zeros(m.n_p)])
    setup_s = time.perf_counter() - t0

    def sample():
        krylov.fgmres(prob.apply_K, pc.apply, F, rtol=RTOL, restart=50, maxit=ORACLE_SAMPLE_ITERS)

    for _ in range(args.warmup):
        sample()
    times = []
    for _ in range(args.steps):
        s0 = time.perf_counter()
        sample()
        times.append(time.perf_counter() - s0)
    t_step = statistics.mean(times)
    dof_o = m.n_u + m.n_p
    dof_w = sum(dof_counts(cfg))
    its = FP64_ITERS.get(name, FP64_ITERS[ORACLE_WORKLOAD])
    value = (setup_s + t_step / ORACLE_SAMPLE_ITERS * its) * dof_w / dof_o
    sample_txt = (f"per step: {ORACLE_SAMPLE_ITERS} FGMRES(50) iterations (V-cycle w-BFBT) of the oracle on "
                  f"{ORACLE_WORKLOAD} ({dof_o} DOF), {t_step:.2f} s; setup once {setup_s:.1f} s; value = "
                  f"(setup + per-iteration x {its} FP64 iterations) x DOF ratio {dof_w}/{dof_o}")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_step, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded multi-sinker, Sec. 2.1)",
        "config": config_dict(name, cfg, "fp64"),
        "cpu_baseline": {"value": value, "unit": "s", "cores": 1, "kind": "oracle", "sample": sample_txt,
                         "host_cpus": os.cpu_count(), "threads": 1, "oracle_setup_s": setup_s,
                         "oracle_s_per_iteration": t_step / ORACLE_SAMPLE_ITERS},
        "e2e": {"value": value, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


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

def traffic_for(kernel: str, workload: str):
    """DRAM bytes per launch of `kernel` on `workload` from the committed ncu summary, if the
    kernel sources are unchanged since the capture (else None)."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(path):
        return None
    data = json.load(open(path))
    ent = data.get(f"{kernel}@{workload}")
    if not ent:
        return None
    srcs = ent["source"] if isinstance(ent["source"], list) else [ent["source"]]
    shas = ent["source_sha256"] if isinstance(ent["source_sha256"], list) else [ent["source_sha256"]]
    for src, want in zip(srcs, shas):
        if hashlib.sha256(open(os.path.join(ROOT, src), "rb").read()).hexdigest() != want:
            return None
    return ent["dram_bytes_per_launch"]


def fp64_alu_peak_tflops(sm_mhz: float | None) -> float:
    """FP64 ALU peak from the unit counts: 152 SMs x 2 DFMA per clock x 2 flop, at the SM clock
    sampled during the run (the maximum clock, 2070 MHz, when no sample is available)."""
    return 152 * 2 * 2 * (sm_mhz or 2070.0) * 1e6 / 1e12


def fp32_alu_peak_tflops(sm_mhz: float | None) -> float:
    """FP32 ALU peak from the unit counts: 152 SMs x 128 FP32 lanes x 2 flop (one FMA per lane and
    clock), at the given SM clock (2070 MHz by default)."""
    return 152 * 128 * 2 * (sm_mhz or 2070.0) * 1e6 / 1e12


def hbm_peak_gbs() -> tuple[float, str]:
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        v = json.load(open(path)).get("hbm_gbs")
        if v:
            return float(v), "of measured"
    return 6800.0, "of fallback"


def _events(n):
    import torch
    return [torch.cuda.Event(enable_timing=True) for _ in range(n)]


def run_ours(args, name, cfg, rank, world):
    import tempfile

    import numpy as np

    # the CPU baseline runs concurrently on one host core: started before any CUDA call
    oracle_proc, oracle_npz = None, None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        oracle_npz = os.path.join(tempfile.mkdtemp(prefix="wbfbt_bench_"), "oracle.npz")
        oracle_proc = start_oracle_solve(inputs_workload(ORACLE_WORKLOAD), oracle_npz)

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
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    st = torch.cuda.current_stream()

    def step(s, uu, pp):
        ea, eb, ec = _events(3)
        m2, f2 = wb.sinker_setup(n, k, centres, cfg["omega"], cfg["delta"], cfg["dr"])
        ea.record(st)
        s.setup(m2)
        eb.record(st)
        _, _, res = s.solve(f2, rtol=RTOL, u=uu, p=pp)
        ec.record(st)
        return res, (ea, eb, ec)

    def timed(s, uu, pp, steps):
        times, setups, solves, res_all = [], [], [], []
        for i in range(steps):
            flush.fill_(float(i))                 # evict L2 between steps (outside the step's events)
            e0, e1 = _events(2)
            e0.record(st)
            res, (ea, eb, ec) = step(s, uu, pp)
            e1.record(st)
            torch.cuda.synchronize()
            if res.status != 0:
                raise RuntimeError(f"solve failed: {res}")
            times.append(e0.elapsed_time(e1) / 1e3)
            setups.append(ea.elapsed_time(eb) / 1e3)
            solves.append(eb.elapsed_time(ec) / 1e3)
            res_all.append(res)
        return times, setups, solves, res_all

    for _ in range(args.warmup):
        step(solver, u, p)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = ClockSampler(dev.index) if rank == 0 else None
    launches0 = wb.launch_count()
    wall0 = time.perf_counter()
    times, setups, solves, results = timed(solver, u, p, args.steps)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    if world > 1:
        dist.barrier()
    launches = wb.launch_count() - launches0
    clk = clocks.stop() if clocks else None
    t_step = max_over_ranks(statistics.mean(times), world, dev)
    iters = results[-1].iters

    # the other side of the metric: the plain FP64 solve of the same problem (fewer steps: it is
    # the comparison, not the headline), and the distance between the two solutions
    other = None
    if precision == wb.MIXED:
        s64 = wb.Solver(n, k, mu, precision=wb.F64)
        u64 = torch.empty_like(u)
        p64 = torch.empty_like(p)
        step(s64, u64, p64)
        t64, su64, so64, r64 = timed(s64, u64, p64, max(1, min(args.steps, 3)))
        t64m = max_over_ranks(statistics.mean(t64), world, dev)
        other = {"precision": "fp64", "s_per_step": t64m, "setup_s": statistics.mean(su64),
                 "solve_s": statistics.mean(so64), "iters": r64[-1].iters, "final_rel_res": r64[-1].rel_res,
                 "steps": len(t64), "mixed_speedup": t64m / t_step,
                 "rel_err_u_mixed_vs_fp64": float(torch.linalg.norm(u - u64) / torch.linalg.norm(u64)),
                 "rel_err_p_mixed_vs_fp64": float(torch.linalg.norm(p - p64) / torch.linalg.norm(p64))}
        s64.close()
        del u64, p64
    torch.cuda.synchronize()
    return dict(solver=solver, wb=wb, torch=torch, np=np, dev=dev, st=st, flush=flush, centres=centres, mu=mu,
                f=f, u=u, p=p, t_step=t_step, times=times, setups=setups, solves=solves, iters=iters,
                rel=results[-1].rel_res, wall=wall, launches=launches, clk=clk, other=other,
                oracle_proc=oracle_proc, oracle_npz=oracle_npz, precision=precision)


def finish_ours(args, name, cfg, rank, world, R):
    torch, wb, np = R["torch"], R["wb"], R["np"]
    solver, st, flush, dev = R["solver"], R["st"], R["flush"], R["dev"]
    n, k = cfg["n"], cfg["k"]

    def time_op(fn, reps=20):
        for _ in range(3):
            fn()
        e0, e1 = _events(2)
        e0.record(st)
        for _ in range(reps):
            fn()
        e1.record(st)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3 / reps

    # operator applies on the fine level, timed on the launching stream with CUDA events.  The
    # mixed context applies A in FP32 (the preconditioner's) and FP64 (the Krylov side's).
    x64 = torch.randn(solver.n_u, dtype=torch.float64, device=dev)
    t_a32 = None
    xk = torch.randn(solver.n_u + solver.n_p, dtype=torch.float64, device=dev)
    t_k64 = time_op(lambda: solver.apply_K(xk))
    t_a64 = time_op(lambda: solver.apply_A(x64))
    if R["precision"] == wb.MIXED:
        x32 = x64.float()
        t_a32 = time_op(lambda: solver.apply_A(x32))
    n_elem, n_nodes = solver.n_elem, solver.n_nodes
    clk = R["clk"]
    peak64 = fp64_alu_peak_tflops(clk["sm_mhz"] if clk else None)
    hbm, hbm_note = hbm_peak_gbs()
    flops_a = a_apply_flops_per_elem(k) * n_elem
    # fused Stokes K apply: A (36n^4+30n^3) plus what B and B^T add at each of the n^3 points
    # (their derivative sums are A's): B: the divergence (2 adds), its weight (1) and Np
    # basis FMAs (2 Np); B^T: the pressure at the point (2 Np), its weight (1) and the
    # three diagonal stress updates (3)
    np_e = k * (k + 1) * (k + 2) // 6
    flops_k = flops_a + (k + 1) ** 3 * (4 * np_e + 7) * n_elem
    roof64 = {"bound": "alu", "achieved": flops_k / t_k64 / 1e12, "peak": peak64, "unit": "TFLOP/s",
              "frac": flops_k / t_k64 / 1e12 / peak64, "traffic": traffic_for("apply_K_f64", name),
              "kernel": "k_q2_elem64<OP_A|OP_BT|OP_B,iso> + k_q2_gather<double,3,STORE> (the FP64 Arnoldi K apply)",
              "per_launch": ("one fine-level K = [A B^T; B 0] apply: (36n^4 + 30n^3 + n^3 (4 Np + 7)) flops per "
                             f"element x {n_elem} elements"),
              "peak_note": "FP64 ALU peak from 152 SMs x 2 DFMA/clk x 2 flop at the sampled SM clock"}
    bytes32 = a_apply_bytes_per_node(4) * n_nodes
    roof32 = None
    if t_a32:
        roof32 = {"bound": "hbm", "achieved": bytes32 / t_a32 / 1e9, "peak": hbm, "unit": "GB/s",
                  "frac": bytes32 / t_a32 / 1e9 / hbm, "traffic": traffic_for("apply_A_f32", name),
                  "kernel": ("k_q2_fused<OP_A,STORE> + k_q2_fused_fix<3,STORE> (one FP32 A apply, single-kernel "
                             "form)" if solver.n_elem >= (1 << 17) else
                             "k_q2_elem<OP_A> + k_q2_gather<3,STORE> (one FP32 A apply)"), "peak_note": hbm_note,
                  "per_launch": f"7 words x 4 B per node x {n_nodes} nodes (u, y, mu)"}
    roofA64 = {"bound": "alu", "achieved": flops_a / t_a64 / 1e12, "peak": peak64, "unit": "TFLOP/s",
               "frac": flops_a / t_a64 / 1e12 / peak64, "traffic": traffic_for("apply_A_f64", name),
               "kernel": "k_q2_elem64<OP_A,iso> + k_q2_gather<double,3,STORE> (one FP64 A apply)"}

    # end to end through the C ABI, the call a user with host data makes: every step copies the
    # viscosity and the forcing from pinned host memory (in place of the on-GPU sinker setup),
    # runs setup and solve, and reads the solution back into pinned host memory.
    mu_h = torch.empty(solver.n_nodes, dtype=torch.float64).pin_memory()
    f_h = torch.empty(solver.n_u, dtype=torch.float64).pin_memory()
    mu_h.copy_(R["mu"])
    f_h.copy_(R["f"])
    u_h = torch.empty(solver.n_u, dtype=torch.float64).pin_memory()
    p_h = torch.empty(solver.n_p, dtype=torch.float64).pin_memory()
    torch.cuda.synchronize()
    e2e = []
    for i in range(args.steps):
        flush.fill_(float(i))
        torch.cuda.synchronize()
        w0 = time.perf_counter()
        solver.setup(mu_h)
        _, _, res = solver.solve(f_h, rtol=RTOL, u=u_h, p=p_h)
        e2e.append(time.perf_counter() - w0)
        if res.status != 0:
            raise RuntimeError(f"e2e solve failed: {res}")
    h2d = 8 * solver.n_nodes + 8 * solver.n_u
    d2h = 8 * solver.n_u + 8 * solver.n_p
    e2e_v = max_over_ranks(statistics.mean(e2e), world, dev)

    # the oracle's 32^3 solve (running since the start) and the GPU's solve of the same problem in
    # this run's precision: the error against the oracle, and the CPU baseline
    cpu, vs_oracle = None, None
    if R["oracle_proc"] is not None:
        o = finish_oracle_solve(R["oracle_proc"])
        ocfg = inputs_workload(ORACLE_WORKLOAD)
        from paper_1607_03936_gb300 import inputs
        oc = inputs.sinker_centres(ocfg["seed"], ocfg["n_sinkers"])
        mo, fo = wb.sinker_setup(ocfg["n"], ocfg["k"], oc, ocfg["omega"], ocfg["delta"], ocfg["dr"])
        so = wb.Solver(ocfg["n"], ocfg["k"], mo, precision=R["precision"])
        ug, pg, ro = so.solve(fo, rtol=RTOL)
        ref = np.load(R["oracle_npz"])
        ug, pg = ug.cpu().numpy(), pg.cpu().numpy()
        vs_oracle = {"workload": ORACLE_WORKLOAD, "precision": args.precision, "iters_gpu": ro.iters,
                     "iters_oracle": o["its"],
                     "rel_err_u": float(np.linalg.norm(ug - ref["u"]) / np.linalg.norm(ref["u"])),
                     "rel_err_p": float(np.linalg.norm(pg - ref["p"]) / np.linalg.norm(ref["p"]))}
        so.close()
        dof_o = o["dof"]
        dof_w = sum(dof_counts(cfg))
        its_w = R["other"]["iters"] if R["other"] else R["iters"]
        est = (o["setup"] + o["solve"] * its_w / o["its"]) * dof_w / dof_o
        cpu = {"value": est, "unit": "s", "cores": 1, "kind": "oracle",
               "sample": (f"full oracle setup + FP64 solve of {ORACLE_WORKLOAD} ({dof_o} DOF, {o['its']} its, "
                          f"{o['setup']:.1f} s + {o['solve']:.1f} s on one host core, run concurrently with the GPU "
                          f"measurement); the {name} workload is beyond the oracle (CSR A ~2.4e9 nonzeros); "
                          f"value = (setup + solve x {its_w}/{o['its']} FP64 iterations) x DOF ratio "
                          f"{dof_w}/{dof_o}"),
               "measured_s": o["setup"] + o["solve"], "measured_workload": ORACLE_WORKLOAD,
               "host_cpus": os.cpu_count(), "threads": 1}
    if rank != 0:
        return
    prec_name = "mixed" if R["precision"] == wb.MIXED else "fp64"
    line = {
        "metric": METRIC, "value": R["t_step"], "unit": "s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * R["t_step"], "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64" if R["precision"] == wb.MIXED else "f64",
        "data": "synthetic (seeded multi-sinker, Sec. 2.1)", "config": config_dict(name, cfg, prec_name),
        "iters": R["iters"], "final_rel_res": R["rel"], "setup_s": statistics.mean(R["setups"]),
        "solve_s": statistics.mean(R["solves"]), "wall_s": R["wall"],
        "learned": "not attached (no measured gain: every learned step was rejected on held-out problems)",
        "fp64": R["other"],
        "a_apply_dof_per_s": {"fp64": solver.n_u / t_a64, "fp32": solver.n_u / t_a32 if t_a32 else None},
        "roofline": roof64, "roofline_fp32_A": roof32, "roofline_fp64_A": roofA64,
        "cpu_baseline": cpu, "vs_oracle": vs_oracle,
        "e2e": {"value": e2e_v, "unit": "s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": R["launches"], "clocks": clk,
    }
    print(json.dumps(line), flush=True)
    solver.close()


def inputs_workload(name: str) -> dict:
    from paper_1607_03936_gb300 import inputs
    return dict(inputs.WORKLOADS[name])


def run_profile(args, name, cfg):
    """One solve of the workload inside an NVTX range "prof" (after the context's creation and
    setup), for an ncu launch list of the solve."""
    import torch

    from paper_1607_03936_gb300 import build
    build.build()
    from paper_1607_03936_gb300 import inputs
    from paper_1607_03936_gb300 import wbfbt as wb

    n, k = cfg["n"], cfg["k"]
    centres = inputs.sinker_centres(cfg["seed"], cfg["n_sinkers"])
    mu, f = wb.sinker_setup(n, k, centres, cfg["omega"], cfg["delta"], cfg["dr"])
    solver = wb.Solver(n, k, mu, precision=wb.MIXED if args.precision == "mixed" else wb.F64)
    torch.cuda.synchronize()
    n0 = wb.launch_count()
    torch.cuda.nvtx.range_push("prof")
    _, _, res = solver.solve(f, rtol=RTOL)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    print(json.dumps({"profile": name, "precision": args.precision, "create_launches": n0,
                      "solve_launches": wb.launch_count() - n0, "iters": res.iters, "rel_res": res.rel_res}),
          flush=True)
    solver.close()


def run_profile_setup(args, name, cfg):
    """One viscosity-dependent setup (wbfbt_setup) inside an NVTX range "prof", after the
    context's creation, for an ncu launch list of the setup."""
    import torch

    from paper_1607_03936_gb300 import build
    build.build()
    from paper_1607_03936_gb300 import inputs
    from paper_1607_03936_gb300 import wbfbt as wb

    n, k = cfg["n"], cfg["k"]
    centres = inputs.sinker_centres(cfg["seed"], cfg["n_sinkers"])
    mu, _ = wb.sinker_setup(n, k, centres, cfg["omega"], cfg["delta"], cfg["dr"])
    solver = wb.Solver(n, k, mu, precision=wb.MIXED if args.precision == "mixed" else wb.F64)
    torch.cuda.synchronize()
    n0 = wb.launch_count()
    torch.cuda.nvtx.range_push("prof")
    solver.setup(mu)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    print(json.dumps({"profile_setup": name, "precision": args.precision, "setup_launches": wb.launch_count() - n0}),
          flush=True)
    solver.close()


def run_profile_apply(args, name, cfg):
    """One fine-level A apply in FP64, one in FP32, one fused FP64 K apply and one FP32 B^T apply
    inside an NVTX range "prof" (after three warm-up applies each), for ncu --nvtx --nvtx-include
    prof/ captures of the operator kernels (launch order: FP64 A element + node pass, FP32 A element
    + node pass, FP64 K element + node pass, FP32 B^T element + node pass)."""
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
    x64 = torch.randn(s64.n_u + s64.n_p, dtype=torch.float64, device="cuda",
                      generator=torch.Generator("cuda").manual_seed(1))
    p32 = x64[s64.n_u:].float()
    for _ in range(3):
        s64.apply_A(u64)
        s32.apply_A(u32)
        s64.apply_K(x64)
        s32.apply_BT(p32)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("prof")
    s64.apply_A(u64)
    s32.apply_A(u32)
    s64.apply_K(x64)
    s32.apply_BT(p32)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    print(json.dumps({"profile_apply": name, "n_u": s64.n_u}), flush=True)
    s64.close()
    s32.close()


def run_profile_mapped(args, name, cfg):
    """One fused FP64 K apply on a mapped mesh of the workload's size (vertex offsets of amp 0.1,
    seed 7) inside an NVTX range "prof" (after three warm-up applies), for ncu captures of the mapped
    element pass (launch order: mapped K element pass, node pass)."""
    import numpy as np
    import torch

    from paper_1607_03936_gb300 import build
    build.build()
    from paper_1607_03936_gb300 import inputs
    from paper_1607_03936_gb300 import wbfbt as wb

    n, k = cfg["n"], cfg["k"]
    centres = inputs.sinker_centres(cfg["seed"], cfg["n_sinkers"])
    X0 = wb.node_coords(n, k).view(3, -1).T.cpu().numpy()
    X = torch.tensor(np.ascontiguousarray(inputs.deform_vertices(X0, (n, n, n), (1.0, 1.0, 1.0), 0.1, 7).T).ravel(),
                     device="cuda")
    mu, _ = wb.sinker_setup_at(X, n, k, centres, cfg["omega"], cfg["delta"], cfg["dr"])
    s = wb.Solver(n, k, mu, precision=wb.F64, restart=5)
    s.set_geometry(X)
    x64 = torch.randn(s.n_u + s.n_p, dtype=torch.float64, device="cuda",
                      generator=torch.Generator("cuda").manual_seed(1))
    for _ in range(3):
        s.apply_K(x64)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("prof")
    s.apply_K(x64)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    print(json.dumps({"profile_mapped": name, "n_u": s.n_u}), flush=True)
    s.close()


SWEEP_SINKERS = (1, 4, 8, 12, 16, 20, 24, 28)
SWEEP_DR = (1e4, 1e6, 1e8, 1e10)


def run_sweep(args):
    """Iteration-count sweeps in the style of the paper's tables, one JSON line per solve.

    robustness (Sec. 4, Table 1): w-BFBT (sqrt(mu) and viscosity-gradient weights) against
      diag(A)-BFBT and the inverse-viscosity pressure mass (lumped, Eq. lumping, and its diagonal)
      over sinker counts x dynamic ratios, n^3 Q2, omega 0.1, delta 200, seeded centres;
    amplification (Sec. 5, Table 2): w-BFBT with a_l = 1 and a_r in {1, 2, 4, 8, 16, 32};
    order (Sec. 7, Table 3b): w-BFBT for k = 2, 3, 4 on the same mesh, a_r by the Table 3 rule;
    alone (Sec. 7, Table 3): the viscous block and K_{w_r} solved on their own with their V-cycles
      beside the Stokes solve, over mesh size and order;
    kcycles: Stokes iterations with 1-8 V-cycles per K~_w^-1, and the cost of one K_w V-cycle
      against one U-Net forward pass (what a learned K~_w^-1 could at best save);
    cheb: Stokes iterations and solve time against the Chebyshev smoothing degree;
    acycles: the same against the number of V-cycles per A~^-1 application;
    restart: the same against the FGMRES restart length;
    mapped: mapped-hexahedron applies beside the brick's, and iterations against the distortion;
    applies: every fine-level operator apply of --workload against its HBM and ALU rooflines.
    """
    import numpy as np
    import torch

    from paper_1607_03936_gb300 import build
    build.build()
    from paper_1607_03936_gb300 import inputs
    from paper_1607_03936_gb300 import wbfbt as wb

    prec = wb.MIXED if args.precision == "mixed" else wb.F64
    n = args.sweep_n

    def solve(k, ns, dr, schur=wb.SCHUR_WBFBT, a_r=0.0, seed=0, weights=wb.WEIGHTS_SQRT_MU):
        c = inputs.sinker_centres(seed, ns)
        mu, f = wb.sinker_setup(n, k, c, 0.1, 200.0, dr)
        s = wb.Solver(n, k, mu, precision=prec, schur=schur, a_r=a_r, weights=weights)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, _, res = s.solve(f, rtol=RTOL, maxit=args.sweep_maxit)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        s.close()
        return {"iters": res.iters, "converged": res.status == 0, "rel_res": res.rel_res, "solve_s": dt}

    names = {wb.SCHUR_WBFBT: "w-BFBT", wb.SCHUR_MASS: "M_p(1/mu) lumped", wb.SCHUR_MASS_DIAG: "M_p(1/mu) diagonal"}
    base = {"mesh": f"{n}^3", "precision": args.precision, "omega": 0.1, "delta": 200.0, "rtol": RTOL,
            "maxit": args.sweep_maxit}
    if args.sweep == "robustness":
        for ns in SWEEP_SINKERS:
            for dr in SWEEP_DR:
                for schur in (wb.SCHUR_WBFBT, wb.SCHUR_MASS_DIAG, wb.SCHUR_MASS):
                    r = solve(2, ns, dr, schur)
                    print(json.dumps({"sweep": "robustness", **base, "k": 2, "sinkers": ns, "dr": dr,
                                      "schur": names[schur], **r}), flush=True)
                r = solve(2, ns, dr, weights=wb.WEIGHTS_GRAD)
                print(json.dumps({"sweep": "robustness", **base, "k": 2, "sinkers": ns, "dr": dr,
                                  "schur": "w-BFBT, gradient weights", **r}), flush=True)
                r = solve(2, ns, dr, weights=wb.WEIGHTS_DIAG_A)
                print(json.dumps({"sweep": "robustness", **base, "k": 2, "sinkers": ns, "dr": dr,
                                  "schur": "diag(A)-BFBT", **r}), flush=True)
    elif args.sweep == "amplification":
        for k in (2, 3, 4):
            for a_r in (1.0, 2.0, 4.0, 8.0, 16.0, 32.0):
                r = solve(k, 16, 1e6, a_r=a_r)
                print(json.dumps({"sweep": "amplification", **base, "k": k, "sinkers": 16, "dr": 1e6, "a_l": 1.0,
                                  "a_r": a_r, **r}), flush=True)
    elif args.sweep == "alone":
        # Table 3: the viscous block and the weighted pressure Poisson operator K_{w_r} solved on
        # their own (FGMRES + their V-cycles, rhs: the load vector / a seeded mean-free vector)
        # beside the full Stokes solve, S16 DR 1e6, over mesh size (k = 2) and order (n = 32)
        for nn_, k in ((16, 2), (32, 2), (64, 2), (32, 3), (32, 4)):
            c = inputs.sinker_centres(0, 16)
            mu, f = wb.sinker_setup(nn_, k, c, 0.1, 200.0, 1e6)
            s = wb.Solver(nn_, k, mu, precision=prec)
            _, ra = s.solve_block(wb.BLOCK_A, f.clone(), rtol=RTOL, maxit=args.sweep_maxit)
            gen = torch.Generator(device="cuda").manual_seed(9)
            b = torch.randn(s.n_p, dtype=torch.float64, device="cuda", generator=gen)
            _, rk = s.solve_block(wb.BLOCK_KR, b, rtol=RTOL, maxit=args.sweep_maxit)
            _, _, rs = s.solve(f, rtol=RTOL, maxit=args.sweep_maxit)
            print(json.dumps({"sweep": "alone", **base, "mesh": f"{nn_}^3", "k": k, "sinkers": 16, "dr": 1e6,
                              "u_dof": s.n_u, "p_dof": s.n_p, "its_A_alone": ra.iters, "its_Kwr_alone": rk.iters,
                              "its_stokes": rs.iters}), flush=True)
            s.close()
    elif args.sweep == "kcycles":
        # how much a better K~_w^-1 could gain (the learned correction stands in for it): Stokes
        # iterations and solve time with 1, 2, 4 and 8 V-cycles per K~_w^-1 application on the
        # 32^3 and 64^3 workloads, beside the measured cost of one K_w V-cycle and of one U-Net
        # forward pass on the same element grid
        for wname in ("32^3-Q2-S24-DR1e6", "64^3-Q2-S64-DR1e10"):
            cfg = inputs.WORKLOADS[wname]
            c = inputs.sinker_centres(cfg["seed"], cfg["n_sinkers"])
            mu, f = wb.sinker_setup(cfg["n"], cfg["k"], c, cfg["omega"], cfg["delta"], cfg["dr"])
            for cyc in (1, 2, 4, 8):
                s = wb.Solver(cfg["n"], cfg["k"], mu, precision=prec, kinv_cycles=cyc)
                s.solve(f)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                _, _, res = s.solve(f, rtol=RTOL, maxit=args.sweep_maxit)
                torch.cuda.synchronize()
                row = {"sweep": "kcycles", "workload": wname, "precision": args.precision, "kinv_cycles": cyc,
                       "iters": res.iters, "converged": res.status == 0, "solve_s": time.perf_counter() - t0}
                if cyc == 1:
                    r = torch.randn(s.n_p, device="cuda", dtype=s.pdtype)
                    ev = _events(2)
                    for _ in range(3):
                        s.apply_Kinv(1, r)
                    ev[0].record()
                    for _ in range(20):
                        s.apply_Kinv(1, r)
                    ev[1].record()
                    torch.cuda.synchronize()
                    row["kw_vcycle_s"] = ev[0].elapsed_time(ev[1]) / 20 / 1e3
                    net = wb.Net(1 + s.np, s.np, cfg["n"])
                    net.set_params(torch.tensor(inputs.unet_init_params(3, 1 + s.np, s.np), device="cuda"))
                    x = torch.randn(1, cfg["n"] ** 3, 1 + s.np, device="cuda")
                    for _ in range(3):
                        net.forward(x)
                    ev[0].record()
                    for _ in range(20):
                        net.forward(x)
                    ev[1].record()
                    torch.cuda.synchronize()
                    row["unet_forward_s"] = ev[0].elapsed_time(ev[1]) / 20 / 1e3
                    net.close()
                print(json.dumps(row), flush=True)
                s.close()
    elif args.sweep == "acycles":
        # V-cycles per A~^-1 application (Sec. 6 approximates A^-1 by V-cycles without fixing their
        # number): Stokes iterations and solve time on the bench workloads
        for wname in ("32^3-Q2-S24-DR1e6", "64^3-Q2-S64-DR1e10"):
            cfg = inputs.WORKLOADS[wname]
            c = inputs.sinker_centres(cfg["seed"], cfg["n_sinkers"])
            mu, f = wb.sinker_setup(cfg["n"], cfg["k"], c, cfg["omega"], cfg["delta"], cfg["dr"])
            for cyc in (1, 2, 3, 4):
                s = wb.Solver(cfg["n"], cfg["k"], mu, precision=prec, ainv_cycles=cyc)
                s.solve(f)
                ts = []
                for _ in range(2):
                    torch.cuda.synchronize()
                    t0 = time.perf_counter()
                    _, _, res = s.solve(f, rtol=RTOL, maxit=args.sweep_maxit)
                    torch.cuda.synchronize()
                    ts.append(time.perf_counter() - t0)
                print(json.dumps({"sweep": "acycles", "workload": wname, "precision": args.precision,
                                  "ainv_cycles": cyc, "iters": res.iters, "converged": res.status == 0,
                                  "solve_s": min(ts)}), flush=True)
                s.close()
    elif args.sweep == "cheb":
        # Chebyshev smoothing degree of every V-cycle (Sec. 6 fixes the smoother family, not its
        # degree): Stokes iterations and solve time on the bench workloads
        for wname in ("32^3-Q2-S24-DR1e6", "64^3-Q2-S64-DR1e10"):
            cfg = inputs.WORKLOADS[wname]
            c = inputs.sinker_centres(cfg["seed"], cfg["n_sinkers"])
            mu, f = wb.sinker_setup(cfg["n"], cfg["k"], c, cfg["omega"], cfg["delta"], cfg["dr"])
            for deg in (2, 3, 4, 5, 6, 8):
                s = wb.Solver(cfg["n"], cfg["k"], mu, precision=prec, cheb_degree=deg)
                s.solve(f)
                ts = []
                for _ in range(2):
                    torch.cuda.synchronize()
                    t0 = time.perf_counter()
                    _, _, res = s.solve(f, rtol=RTOL, maxit=args.sweep_maxit)
                    torch.cuda.synchronize()
                    ts.append(time.perf_counter() - t0)
                print(json.dumps({"sweep": "cheb", "workload": wname, "precision": args.precision,
                                  "cheb_degree": deg, "iters": res.iters, "converged": res.status == 0,
                                  "solve_s": min(ts)}), flush=True)
                s.close()
    elif args.sweep == "restart":
        # FGMRES restart length: iterations against the per-iteration cost of the Arnoldi basis
        # (CGS2 is 4 (j + 1) n FP64 multiply-adds at step j)
        for wname in ("32^3-Q2-S24-DR1e6", "64^3-Q2-S64-DR1e10"):
            cfg = inputs.WORKLOADS[wname]
            c = inputs.sinker_centres(cfg["seed"], cfg["n_sinkers"])
            mu, f = wb.sinker_setup(cfg["n"], cfg["k"], c, cfg["omega"], cfg["delta"], cfg["dr"])
            for m in (10, 20, 30, 50, 100):
                s = wb.Solver(cfg["n"], cfg["k"], mu, precision=prec, restart=m)
                s.solve(f)
                ts = []
                for _ in range(2):
                    torch.cuda.synchronize()
                    t0 = time.perf_counter()
                    _, _, res = s.solve(f, rtol=RTOL, maxit=args.sweep_maxit)
                    torch.cuda.synchronize()
                    ts.append(time.perf_counter() - t0)
                print(json.dumps({"sweep": "restart", "workload": wname, "precision": args.precision, "restart": m,
                                  "iters": res.iters, "converged": res.status == 0, "solve_s": min(ts)}), flush=True)
                s.close()
    elif args.sweep == "applies":
        # every fine-level operator apply of the workload against its own roofline: algorithmic
        # bytes (each vector word moved once) and flops per apply, the time each would take at the
        # HBM and the ALU peak, and the fraction of the larger of the two that the apply reaches
        # (CUDA events around each apply, warm, a 256 MiB write before each so L2 starts cold; median
        # of 20)
        cfg = inputs.WORKLOADS[args.workload]
        nn_, k = cfg["n"], cfg["k"]
        if k != 2:
            raise SystemExit("--sweep applies counts Q2 operators")
        c = inputs.sinker_centres(cfg["seed"], cfg["n_sinkers"])
        mu, f = wb.sinker_setup(nn_, k, c, cfg["omega"], cfg["delta"], cfg["dr"])
        hbm, hbm_note = hbm_peak_gbs()
        E, NN, NP = nn_ ** 3, (2 * nn_ + 1) ** 3, 4
        nq = 3                                            # points per axis
        fl_A = 36 * nq ** 4 + 30 * nq ** 3                # per element (sum factorisation)
        fl_B = 6 * nq ** 4 + 2 * nq ** 3 * NP
        rows = []
        for prec_name, sprec, es in (("fp32", wb.MIXED, 4), ("fp64", wb.F64, 8)):
            s = wb.Solver(nn_, k, mu, precision=sprec)
            dt = torch.float32 if es == 4 else torch.float64
            gen = torch.Generator(device="cuda").manual_seed(3)
            u = torch.randn(s.n_u, device="cuda", generator=gen).to(dt)
            p = torch.randn(s.n_p, device="cuda", generator=gen).to(dt)
            x = torch.cat([u, p])
            peak_alu = fp32_alu_peak_tflops(None) if es == 4 else fp64_alu_peak_tflops(None)
            cases = [("A", lambda: s.apply_A(u), 7 * NN, fl_A * E),
                     ("B", lambda: s.apply_B(u), 3 * NN + NP * E, fl_B * E),
                     ("BT", lambda: s.apply_BT(p), NP * E + 3 * NN, fl_B * E),
                     ("K", lambda: s.apply_K(x), 7 * NN + 2 * NP * E, (fl_A + 2 * fl_B) * E),
                     ("Kw", lambda: s.apply_Kw(1, p), 2 * NP * E + NN, 2 * fl_B * E + 3 * NN)]
            flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
            for name, fn, words, flops in cases:
                for _ in range(3):
                    fn()
                ts = []
                for _ in range(20):
                    flush.zero_()                        # L2 (129 MB) holds none of the apply's data
                    ev = _events(2)
                    ev[0].record()
                    fn()
                    ev[1].record()
                    ts.append(ev)
                torch.cuda.synchronize()
                t = statistics.median(e0.elapsed_time(e1) for e0, e1 in ts) / 1e3
                t_mem = words * es / (hbm * 1e9)
                t_alu = flops / (peak_alu * 1e12)
                bound = "hbm" if t_mem >= t_alu else "alu"
                rows.append({"sweep": "applies", "workload": args.workload, "precision": prec_name, "apply": name,
                             "t_us": t * 1e6, "alg_bytes": words * es, "alg_flops": flops,
                             "flop_per_byte": flops / (words * es), "bound": bound,
                             "hbm_frac": words * es / t / (hbm * 1e9), "alu_frac": flops / t / (peak_alu * 1e12),
                             "bound_frac": max(t_mem, t_alu) / t, "hbm_peak_gbs": hbm, "hbm_note": hbm_note,
                             "alu_peak_tflops": peak_alu})
                print(json.dumps(rows[-1]), flush=True)
            s.close()
    elif args.sweep == "mapped":
        # mapped hexahedra (isoparametric Q2 from moved nodes, the fields of Sec. 2.1 at the moved
        # nodes): the mapped operator applies beside the brick's on the same mesh (CUDA events),
        # and Stokes iterations and solve time against the distortion, the preconditioner staying
        # the brick's
        k = 2
        c = inputs.sinker_centres(0, 16)
        X0 = wb.node_coords(n, k).view(3, -1).T.cpu().numpy()
        geoms = (("brick", 0.0), ("trilinear", 0.05), ("trilinear", 0.1), ("trilinear", 0.15), ("smooth", 0.05),
                 ("smooth", 0.1), ("smooth", 0.15))

        def apply_s(fn, x, reps=20):
            for _ in range(3):
                fn(x)
            ev = _events(2)
            ev[0].record()
            for _ in range(reps):
                fn(x)
            ev[1].record()
            torch.cuda.synchronize()
            return ev[0].elapsed_time(ev[1]) / reps / 1e3

        for kind, amp in geoms:
            if kind == "brick":
                X = X0
            elif kind == "trilinear":
                X = inputs.deform_vertices(X0, (n, n, n), (1.0, 1.0, 1.0), amp, 7)
            else:
                X = inputs.deform_smooth(X0, (1.0, 1.0, 1.0), amp)
            Xt = torch.tensor(np.ascontiguousarray(X.T).ravel(), device="cuda")
            mu, f = wb.sinker_setup_at(Xt, n, k, c, 0.1, 200.0, 1e6)
            s = wb.Solver(n, k, mu, precision=prec)
            s.set_geometry(Xt)
            gen = torch.Generator(device="cuda").manual_seed(5)
            x64 = torch.randn(s.n_u + s.n_p, dtype=torch.float64, device="cuda", generator=gen)
            u32 = x64[: s.n_u].float()
            row = {"sweep": "mapped", **base, "k": k, "sinkers": 16, "dr": 1e6, "geometry": kind, "amp": amp,
                   "A64_mapped_s": apply_s(s.apply_A, x64[: s.n_u]), "K64_mapped_s": apply_s(s.apply_K, x64),
                   "A32_mapped_s": apply_s(s.apply_A, u32)}
            s.set_geometry(None)
            row.update({"A64_brick_s": apply_s(s.apply_A, x64[: s.n_u]), "K64_brick_s": apply_s(s.apply_K, x64),
                        "A32_brick_s": apply_s(s.apply_A, u32)})
            if kind == "brick":
                _, _, rb = s.solve(f, rtol=RTOL, maxit=args.sweep_maxit)
                row["iters_brick_path"] = rb.iters
            s.set_geometry(Xt)
            s.solve(f, rtol=RTOL, maxit=args.sweep_maxit)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, _, res = s.solve(f, rtol=RTOL, maxit=args.sweep_maxit)
            torch.cuda.synchronize()
            row.update({"iters": res.iters, "converged": res.status == 0, "rel_res": res.rel_res,
                        "solve_s": time.perf_counter() - t0})
            print(json.dumps(row), flush=True)
            s.close()
    elif args.sweep == "order":
        for k in (2, 3, 4):
            r = solve(k, 16, 1e6)
            print(json.dumps({"sweep": "order", **base, "k": k, "sinkers": 16, "dr": 1e6,
                              "a_r": max(1.0, n / 16.0 * 2.0 ** (k - 2)), **r}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--precision", choices=["fp64", "mixed"], default="mixed")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--profile", action="store_true",
                    help="one setup + solve of the workload and nothing else (for an ncu launch list)")
    ap.add_argument("--profile-setup", action="store_true",
                    help="one viscosity-dependent setup in an NVTX range 'prof' (for an ncu launch list)")
    ap.add_argument("--profile-mapped", action="store_true",
                    help="one FP64 K apply on a mapped mesh in an NVTX range 'prof' (for ncu)")
    ap.add_argument("--profile-apply", action="store_true",
                    help="one FP64 A, one FP32 A and one FP64 K apply in an NVTX range 'prof' (for ncu)")
    ap.add_argument("--sweep", choices=["robustness", "amplification", "order", "alone", "kcycles", "cheb", "restart",
                                        "mapped", "applies", "acycles"],
                    help="iteration-count sweeps in the style of Tables 1, 2 and 3b (many JSON lines)")
    ap.add_argument("--sweep-n", type=int, default=32)
    ap.add_argument("--sweep-maxit", type=int, default=2000)
    args = ap.parse_args()
    if args.sweep:
        run_sweep(args)
        return
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    cfg = inputs_workload(args.workload)
    name = args.workload
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        run_reference(args, name, cfg, rank, world)
        return
    if args.profile_mapped:
        run_profile_mapped(args, name, cfg)
        return
    if args.profile_apply:
        run_profile_apply(args, name, cfg)
        return
    if args.profile:
        run_profile(args, name, cfg)
        return
    if args.profile_setup:
        run_profile_setup(args, name, cfg)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        dist.init_process_group("nccl")
    R = run_ours(args, name, cfg, rank, world)
    finish_ours(args, name, cfg, rank, world, R)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    if "reference" in sys.argv:
        # the oracle's timing is single-threaded: pin the BLAS pools before numpy loads
        for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            os.environ[_v] = "1"
    main()
