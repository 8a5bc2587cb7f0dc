#!/usr/bin/env python
"""GenEO-PCG time-to-solution benchmark on GB300.

Workload (default): the 64x32x24-element laminated block (160,875 dofs,
12 plies drawn from {0, +-45, 90} with 11 one-element resin interlayers),
clamped at x = 0 under 1 MPa top pressure, 4x4x2 subdomains with overlap 1,
GenEO threshold rule capped at 20 modes per subdomain, PCG to ||r||/||b|| <= 1e-8.

One step = the whole method on one synthetic problem: assembly of A u = b,
the GenEO set-up (eigenproblems, coarse space, subdomain factors) and the
(F)PCG solve, all on the GPU through the library's C ABI.  `value` times
steps whose inputs already sit in device memory; `e2e` times the same step
from host arrays with the host<->device copies inside the timed region.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--config c2] [--precision fp64|mixed]

Multi-GPU: the path does not shard (one GPU per problem, no collectives), so
N ranks run N independent replicas (weak scaling); value = max-over-ranks time
divided by the solves all ranks completed.
`--impl reference` times the FP64 CPU oracle on a bounded sample of the same
workload and extrapolates to one full solve.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GenEO-PCG time-to-1e-8 relative residual"
UNIT = "ms"
TOL = 1e-8


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="c2")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-darcy", action="store_true")
    ap.add_argument("--no-c3", action="store_true",
                    help="skip the 128x64x48 mixed-precision leg")
    ap.add_argument("--batch-blocks", type=int, default=32,
                    help="blocks of the uneven batched-solve workload to run (0 skips it)")
    ap.add_argument("--serve-requests", type=int, default=10,
                    help="requests of the serving sample (uneven laminate blocks)")
    return ap.parse_args()


def workload_config(p, prec):
    s = dict(workload=f"{p['name']}: {p['nx']}x{p['ny']}x{p['nz']} Q1 hex laminate, "
                      f"{3 * (p['nx'] + 1) * (p['ny'] + 1) * (p['nz'] + 1)} dofs",
             partition="x".join(str(v) for v in p["partition"][:3]) + f", overlap {p['partition'][3]}",
             modes=("fixed %d" % p["modes"]["fixed_modes"] if p["modes"]["fixed_modes"]
                    else "threshold rule, cap %d" % p["modes"]["max_modes"]),
             precision=prec, tol=TOL,
             l2="working set (BSR + band factors) > 129 MB L2; no flush needed")
    return s


# ---------------------------------------------------------------------------
# clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                rows.append((float(f[1]), float(f[2]), f[5], f[6], f[7], f[8]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({n for r in rows for n, v in zip(names, r[2:]) if v.lower() == "active"})
        return dict(sm_mhz=statistics.median(r[0] for r in rows), sm_max_mhz=max(r[1] for r in rows),
                    samples=len(rows), reasons=reasons)


FP64_PEAK_TFLOPS = 1.25


def profiled_traffic(kernel, args):
    """DRAM bytes per launch of `kernel` from the committed ncu summary of this
    workload (profiles/dram_<config>_<precision>.md), or None when the summary
    is missing or was taken on a different version of the kernel's source."""
    import hashlib
    path = os.path.join(ROOT, "profiles", f"dram_{args.config}_{args.precision}.md")
    if not os.path.exists(path):
        return None
    srcs = {"k_schwarz_cluster": "schwarz.cu", "k_band_solve_dense": "band.cu"}
    src = os.path.join(ROOT, "paper_1901_05188_gb300", "csrc", srcs.get(kernel, ""))
    h = hashlib.sha1(open(src, "rb").read()).hexdigest()[:12] if os.path.isfile(src) else None
    for line in open(path):
        f = line.strip().strip("|").split("|")
        f = [x.strip() for x in f]
        if len(f) >= 3 and f[0] == kernel and f[1] == h:
            try:
                return float(f[2])
            except ValueError:
                return None
    return None


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ---------------------------------------------------------------------------
# CPU oracle sample (the baseline arm)

def oracle_sample(p, gpu_iterations):
    """Time a bounded sample of the oracle on this workload and extrapolate to
    one full solve: 1/8 of the element assembly (x8), one of the GenEO
    eigensolves (x subdomains), four subdomain factorisations (x subdomains/4),
    and per iteration an SpMV on the sampled rows (x8) plus the four subdomain
    solves (x subdomains/4), times the iteration count.
    Returns (ms, sample description, threads used)."""
    import contextlib
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    from oracle import decomp, fem, geneo
    try:
        from threadpoolctl import threadpool_limits
        ctx, threads = threadpool_limits(limits=1), 1
    except ImportError:           # BLAS keeps its default; the sparse kernels are serial
        ctx, threads = contextlib.nullcontext(), os.cpu_count() or 1
    with ctx:
        nel = p["nx"] * p["ny"] * p["nz"]
        t0 = time.perf_counter()
        A8 = fem.assemble_stiffness(p, np.arange(0, nel, 8))
        t_asm = (time.perf_counter() - t0) * 8
        subs = decomp.partition(p)
        ns = len(subs)
        j = min(ns - 1, ns // 2 + 1)
        m = p["modes"]
        nev = (m["fixed_modes"] if m["fixed_modes"] > 0 else m["max_modes"]) + 1
        t0 = time.perf_counter()
        Aj, Aoj = geneo.local_matrices(p, subs[j])
        Xd = sp.diags(subs[j].X)
        geneo.eigenpairs(Aj, (Xd @ Aoj @ Xd).tocsr(), nev, m["shift"])
        t_eig = (time.perf_counter() - t0) * ns
        idx = sorted({min(ns - 1, k * ns // 4) for k in range(4)})
        t0 = time.perf_counter()
        lus = []
        for k in idx:
            Ak, _ = geneo.local_matrices(p, subs[k])
            lus.append((spla.splu(Ak.tocsc()), Ak.shape[0]))
        t_fac = (time.perf_counter() - t0) * ns / len(idx)
        x = np.ones(A8.shape[0])
        t0 = time.perf_counter()
        for _ in range(3):
            A8 @ x
        t_spmv = (time.perf_counter() - t0) / 3 * 8
        t0 = time.perf_counter()
        for _ in range(3):
            for lu, n in lus:
                lu.solve(np.ones(n))
        t_sub = (time.perf_counter() - t0) / 3 * ns / len(idx)
        total = t_asm + t_eig + t_fac + gpu_iterations * (t_spmv + t_sub)
    sample = (f"FP64 oracle sample: assembly of 1/8 of the elements (x8), 1 of {ns} GenEO "
              f"eigensolves (x{ns}), {len(idx)} of {ns} subdomain factorisations, per-iteration "
              f"SpMV on 1/8 of the elements (x8) + {len(idx)} subdomain solves, "
              f"x {gpu_iterations} iterations")
    return total * 1000.0, sample, threads


def run_reference(args):
    import workloads
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    p = workloads.config(args.config)
    iters = 103 if args.config == "c2" else 60
    gold = os.path.join(ROOT, "tests", "golden", f"{args.config}_oracle.json")
    if os.path.exists(gold):
        iters = json.load(open(gold))["iterations"]
    for _ in range(args.warmup):
        oracle_sample(p, iters)
    times = []
    sample, threads = "", 1
    for _ in range(args.steps):
        ms, sample, threads = oracle_sample(p, iters)
        times.append(ms)
    v = statistics.mean(times)
    line = dict(metric=METRIC, value=v, unit=UNIT, n_gpus=args.gpus, steps=args.steps,
                warmup=args.warmup, ms_per_step=v, higher_is_better=False, scaling="weak",
                vs_baseline=None, dtype="f64", data="synthetic", impl="reference",
                config=workload_config(p, "fp64"),
                cpu_baseline=dict(value=v, unit=UNIT, cores=threads, kind="oracle", sample=sample),
                e2e=dict(value=v, unit=UNIT, h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(line))


# ---------------------------------------------------------------------------
# GPU arm

def device_problem(p, torch, dev):
    q = dict(p)
    for k in ("x", "y", "z", "elem_theta", "elem_phi", "dirichlet_values"):
        q[k] = torch.as_tensor(np.ascontiguousarray(p[k], dtype=np.float64), device=dev)
    for k in ("elem_mat", "dirichlet_dofs"):
        q[k] = torch.as_tensor(np.ascontiguousarray(p[k], dtype=np.int32), device=dev)
    return q


def host_bytes(p):
    n = 0
    for k in ("x", "y", "z", "elem_theta", "elem_phi", "dirichlet_values", "elem_mat",
              "dirichlet_dofs", "materials"):
        n += np.asarray(p[k]).nbytes
    return n


def job_ms_per_solve(ms_local, steps, world, device="cpu"):
    """(ms per step of the slowest rank, whole-job ms per solve) for `world`
    replicas that each timed `steps` solves in `ms_local` ms: the max over
    ranks, divided by every solve of the job."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms_local)], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_step = float(t.item()) / steps
    return ms_step, ms_step / world


def one_solve(pkg, s, p, prec, out):
    s.assemble(p)
    s.setup(p, prec)
    u, st = s.solve(tol=TOL, max_it=5000, out=out)
    return st


def run_ours(args):
    import torch
    import torch.distributed as dist
    import workloads
    import paper_1901_05188_gb300 as pkg

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    pkg.load(build_if_missing=True)
    prec = pkg.GENEO_FP64 if args.precision == "fp64" else pkg.GENEO_MIXED_FP32
    p = workloads.config(args.config)
    pd = device_problem(p, torch, dev)
    s = pkg.GeneoSolver()
    ndof = 3 * (p["nx"] + 1) * (p["ny"] + 1) * (p["nz"] + 1)
    u_dev = torch.empty(ndof, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    for _ in range(args.warmup):
        st = one_solve(pkg, s, pd, prec, u_dev)
    barrier()
    clocks = ClockSampler(local)
    clocks.start()
    l0 = pkg.geneo_launch_count()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    stats = []
    for _ in range(args.steps):
        stats.append(one_solve(pkg, s, pd, prec, u_dev))
    e1.record(stream)
    barrier()
    launches = pkg.geneo_launch_count() - l0
    clk = clocks.stop()
    ms_total = e0.elapsed_time(e1)
    ms_step, value = job_ms_per_solve(ms_total, args.steps, world, dev)
    st = stats[-1]

    # end-to-end through the C ABI from host arrays (copies inside the region)
    e2e = None
    if not args.no_e2e:
        u_host = torch.empty(ndof, dtype=torch.float64, pin_memory=True).numpy()
        one_solve(pkg, s, p, prec, u_host)
        barrier()
        e0.record(stream)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            one_solve(pkg, s, p, prec, u_host)
        e1.record(stream)
        barrier()
        wall = (time.perf_counter() - t0) * 1000.0
        _, e2e_ms = job_ms_per_solve(max(e0.elapsed_time(e1), wall), args.steps, world, dev)
        e2e = dict(value=e2e_ms, unit=UNIT,
                   h2d_bytes_per_step=host_bytes(p), d2h_bytes_per_step=8 * ndof)

    # roofline of the dominant kernel: the larger of the Schwarz local solves
    # (per iteration) and the eigensolver's FP64 band solves (per Lanczos step)
    peak, peak_kind = measured_peaks()
    ms_k, by_k, fl_k = pkg.geneo_profile(s.ctx, 0, 20)
    n_schwarz = st["iterations"] + 1
    cand = []
    hbm = dict(bound="hbm", kernel="k_schwarz_cluster (one-level local band solves, "
                                   f"{'FP64' if args.precision == 'fp64' else 'FP32'})",
               achieved=by_k / (ms_k * 1e-3) / 1e9, peak=peak, unit="GB/s",
               peak_source=f"{peak_kind} hbm_gbs", ms_per_launch=ms_k,
               algorithmic_bytes=by_k, launches_per_solve=n_schwarz)
    hbm["frac"] = hbm["achieved"] / peak
    hbm["traffic"] = profiled_traffic("k_schwarz_cluster", args)
    cand.append((ms_k * n_schwarz, hbm))
    if st["n_coarse"] > 0:
        ms_l, by_l, fl_l = pkg.geneo_profile(s.ctx, 3, 5)
        n_lanczos = 2 * st["lanczos_steps"] + 1   # two sweeps per block step + the Ritz vectors
        alu = dict(bound="alu", kernel="k_band_solve_dense (GenEO shift-invert band solves, FP64, "
                                       "8 right-hand sides)",
                   achieved=fl_l / (ms_l * 1e-3) / 1e12, peak=FP64_PEAK_TFLOPS, unit="TFLOP/s",
                   peak_source="nominal FP64 1.25 TFLOP/s (152 SMs x 2 FMA/clk x 2.07 GHz); "
                               "torch DGEMM measured 1.10",
                   ms_per_launch=ms_l, algorithmic_flops=fl_l, launches_per_solve=n_lanczos)
        alu["frac"] = alu["achieved"] / FP64_PEAK_TFLOPS
        alu["traffic"] = profiled_traffic("k_band_solve_dense", args)
        cand.append((ms_l * n_lanczos, alu))
    cand.sort(key=lambda t: -t[0])
    roof = cand[0][1]
    ms_sp, by_sp, _ = pkg.geneo_profile(s.ctx, 1, 50)
    ms_pc, by_pc, _ = pkg.geneo_profile(s.ctx, 2, 20)
    kernels = dict(spmv=dict(ms=ms_sp, gbs=by_sp / (ms_sp * 1e-3) / 1e9),
                   precond_apply=dict(ms=ms_pc, gbs=by_pc / (ms_pc * 1e-3) / 1e9),
                   other_roofline=[c[1] for c in cand[1:]])

    # accuracy against the oracle's stored summary (sampled displacements)
    acc = None
    gold = os.path.join(ROOT, "tests", "golden", f"{args.config}_oracle.json")
    if os.path.exists(gold):
        g = json.load(open(gold))
        u = u_dev.cpu().numpy()
        us = u[::g["sample_stride"]][:len(g["u_samples"])]
        ref = np.asarray(g["u_samples"])
        acc = dict(rel_err_samples=float(np.linalg.norm(us - ref) / np.linalg.norm(ref)),
                   oracle_iterations=g["iterations"])

    mixed = None
    if not args.no_mixed and args.precision == "fp64":
        for _ in range(2):
            stm = one_solve(pkg, s, pd, pkg.GENEO_MIXED_FP32, u_dev)
        torch.cuda.synchronize(dev)
        e0.record(stream)
        for _ in range(args.steps):
            stm = one_solve(pkg, s, pd, pkg.GENEO_MIXED_FP32, u_dev)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        mixed = dict(ms_per_solve=e0.elapsed_time(e1) / args.steps, iterations=stm["iterations"],
                     rel_res_true=stm["rel_res_true"],
                     phases_ms=dict(setup_eig_coarse=stm["ms_setup_eig"],
                                    setup_factor=stm["ms_setup_factor"], solve=stm["ms_solve"]),
                     schwarz_launch=dict(cluster=stm["schwarz_cluster"], rows=stm["schwarz_rows"],
                                         staged=stm["schwarz_staged"]))
        if acc is not None:
            u = u_dev.cpu().numpy()
            us = u[::g["sample_stride"]][:len(g["u_samples"])]
            mixed["rel_err_samples"] = float(np.linalg.norm(us - ref) / np.linalg.norm(ref))

    # serving: a seeded stream of uneven solve requests through the
    # continuous-batching server (burst, then Poisson at half its throughput)
    serving = None
    if rank == 0 and world == 1 and not args.no_serve and args.serve_requests > 0:
        from paper_1901_05188_gb300.serve import serve_benchmark
        sv = serve_benchmark(n=args.serve_requests, seed=6, prec=pkg.GENEO_MIXED_FP32, slots=4,
                             rate_factors=(None, 0.5), darcy_frac=0.3)
        serving = dict(workload=f"{sv['requests']} requests: {sv['requests'] - sv['darcy']} laminate "
                                f"blocks and {sv['darcy']} Darcy blocks (layered permeability), "
                                f"{min(sv['dofs'])}-{max(sv['dofs'])} unknowns (log-uniform 2e4-2e6, "
                                f"seed 6), {sv['repeats']} repeated structures with new loads",
                       precision=sv["precision"], slots=sv["slots"],
                       runs=[{k: r[k] for k in ("arrivals", "n", "p50_ms", "p99_ms", "mean_ms",
                                                "solves_per_s", "reused", "peak_inflight",
                                                "peak_mem_gb", "failed") if k in r}
                             for r in sv["runs"]])

    # batched uneven solves: the first blocks of the seeded batch (8e3-1e5
    # elements, 4-24 plies, 2-64 subdomains), all submitted at once to the
    # concurrent-slot server (mixed precision), throughput and latency
    batch = None
    if rank == 0 and world == 1 and args.batch_blocks > 0:
        from paper_1901_05188_gb300.serve import GeneoServer, latency_summary
        from workloads.batch import batch_blocks
        blocks = batch_blocks(args.batch_blocks, seed=3)
        srv = GeneoServer(slots=4)
        try:
            t0 = time.perf_counter()
            reqs = [srv.submit(pb, prec=pkg.GENEO_MIXED_FP32, tol=TOL, key=pb["name"], arrival=t0)
                    for pb in blocks]
            for rq in reqs:
                rq.wait()
            wall = time.perf_counter() - t0
        finally:
            srv.close()
        summ = latency_summary(reqs)
        dofs = [3 * (pb["nx"] + 1) * (pb["ny"] + 1) * (pb["nz"] + 1) for pb in blocks]
        parts = [pb["partition"][0] * pb["partition"][1] * pb["partition"][2] for pb in blocks]
        batch = dict(workload=f"first {len(blocks)} blocks of the seeded batch (seed 3): "
                              f"{min(dofs)}-{max(dofs)} dofs, {min(parts)}-{max(parts)} subdomains, "
                              "4-24 plies, burst of independent solves",
                     precision="mixed", slots=4, wall_s=wall,
                     solves_per_s=len(blocks) / wall, dofs_per_s=sum(dofs) / wall,
                     p50_ms=summ.get("p50_ms"), p99_ms=summ.get("p99_ms"),
                     failed=summ.get("failed", len(blocks)))

    # the paper's second application at its full grid: Darcy on SPE10's 60x220x85
    # cells with a synthetic layered permeability (contrast 1.4e10), FP64
    darcy = None
    if rank == 0 and world == 1 and not args.no_darcy:
        from workloads.darcy import darcy_config
        pdz = darcy_config("d-spe10")
        sd = pkg.GeneoSolver()
        for _ in range(2):                       # warm-up, then one timed solve
            e0.record(stream)
            sd.assemble(pdz)
            sd.setup(pdz, pkg.GENEO_FP64)
            _, std = sd.solve(tol=TOL, max_it=5000)
            e1.record(stream)
            torch.cuda.synchronize(dev)
        darcy = dict(workload="Darcy, 60x220x85 cells (1,159,366 unknowns), 6x18 subdomains, "
                              "synthetic layered log-normal permeability, f = 1",
                     ms_per_solve=e0.elapsed_time(e1), iterations=std["iterations"],
                     n_coarse=std["n_coarse"], rel_res_true=std["rel_res_true"],
                     phases_ms=dict(assemble=std["ms_assemble"], setup_eig_coarse=std["ms_setup_eig"],
                                    setup_factor=std["ms_setup_factor"], solve=std["ms_solve"]))
        sd.close()

    # the 1.2M-dof wrinkled laminate (128x64x48, 8x4x4 subdomains): time to
    # 1e-8 with the FP32-factor preconditioner against the all-FP64 one, and the
    # HBM fraction of its Schwarz local solves
    c3 = None
    if rank == 0 and world == 1 and not args.no_c3 and args.config != "c3":
        p3 = workloads.config("c3")
        pd3 = device_problem(p3, torch, dev)
        s3 = pkg.GeneoSolver()
        n3 = 3 * (p3["nx"] + 1) * (p3["ny"] + 1) * (p3["nz"] + 1)
        u3 = torch.empty(n3, dtype=torch.float64, device=dev)
        c3 = dict(workload=f"c3: 128x64x48 Q1 hex laminate with a fibre wrinkle, {n3} dofs, "
                           "8x4x4 subdomains")
        for key, pr in (("mixed", pkg.GENEO_MIXED_FP32), ("fp64", pkg.GENEO_FP64)):
            for _ in range(2):                   # warm-up (and tuning), then one timed solve
                e0.record(stream)
                st3 = one_solve(pkg, s3, pd3, pr, u3)
                e1.record(stream)
                torch.cuda.synchronize(dev)
            leg = dict(ms_per_solve=e0.elapsed_time(e1), iterations=st3["iterations"],
                       rel_res_true=st3["rel_res_true"], n_coarse=st3["n_coarse"],
                       phases_ms=dict(assemble=st3["ms_assemble"],
                                      setup_eig_coarse=st3["ms_setup_eig"],
                                      setup_factor=st3["ms_setup_factor"], solve=st3["ms_solve"]),
                       schwarz_launch=dict(cluster=st3["schwarz_cluster"], rows=st3["schwarz_rows"],
                                           staged=st3["schwarz_staged"]))
            ms3, by3, _ = pkg.geneo_profile(s3.ctx, 0, 10)
            leg["schwarz_apply"] = dict(ms=ms3, gbs=by3 / (ms3 * 1e-3) / 1e9,
                                        frac_of_measured_hbm=by3 / (ms3 * 1e-3) / 1e9 / peak)
            c3[key] = leg
        s3.close()
        del pd3, u3

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        ms_cpu, sample, threads = oracle_sample(p, st["iterations"])
        cpu = dict(value=ms_cpu, unit=UNIT, cores=threads, kind="oracle", sample=sample)

    if rank == 0:
        line = dict(metric=METRIC, value=value, unit=UNIT, n_gpus=world, steps=args.steps,
                    warmup=args.warmup, ms_per_step=ms_step, higher_is_better=False,
                    scaling="weak", vs_baseline=None,
                    dtype="f64" if args.precision == "fp64" else "f64+f32",
                    data="synthetic", config=workload_config(p, args.precision),
                    roofline=roof, cpu_baseline=cpu, e2e=e2e, gpu_launches=int(launches),
                    clocks=clk, iterations=st["iterations"], rel_res_true=st["rel_res_true"],
                    n_coarse=st["n_coarse"], kappa_est=st["kappa_est"],
                    phases_ms=dict(assemble=st["ms_assemble"], setup_eig_coarse=st["ms_setup_eig"],
                                   setup_factor=st["ms_setup_factor"], solve=st["ms_solve"]),
                    bytes_per_iter=st["bytes_per_iter"], kernels=kernels,
                    schwarz_launch=dict(cluster=st["schwarz_cluster"], rows=st["schwarz_rows"],
                                        staged=st["schwarz_staged"],
                                        chosen_by="set-up autotuner"),
                    accuracy_vs_oracle=acc, mixed_precision=mixed, serving=serving,
                    darcy_spe10=darcy, c3_mixed_vs_fp64=c3, batched_uneven=batch)
        print(json.dumps(line))
    s.close()
    if world > 1:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
