#!/usr/bin/env python
"""GenEO-PCG time-to-solution benchmark on GB300.

Workload (default): the 128x64x48-element laminated block with a fibre
wrinkle (1,232,595 dofs, 24 plies of a seeded random stacking, out-of-plane
Gaussian wrinkle of 8 degrees and width 10 elements), clamped at x = 0 under
1 MPa top pressure, 8x4x4 subdomains with overlap 1, GenEO threshold rule
capped at 20 modes per subdomain, (F)PCG to ||r||/||b|| <= 1e-8.  `value` is
the mixed-precision path (FP32 subdomain factors with 3xTF32 tensor-core
updates inside FP64 flexible CG); the all-FP64 path is timed beside it
(`fp64`), and both carry their error against the FP64 oracle's stored
solution (tests/golden/c3_oracle.json).

One step = the whole method on one synthetic problem: assembly of A u = b,
the GenEO set-up (eigenproblems, coarse space, subdomain factors) and the
(F)PCG solve, all on the GPU through the library's C ABI.  `value` times
steps whose inputs already sit in device memory; `e2e` times the same step
from host arrays with the host<->device copies inside the timed region.
Secondary legs: the 64x32x24 laminate (160,875 dofs) with GenEO in FP64 and
mixed precision, one-level additive Schwarz and unpreconditioned CG; Darcy
flow on SPE10's 60x220x85 grid; a batch of uneven blocks; a serving stream.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--config c3] [--precision mixed|fp64]

Multi-GPU: the path does not shard (one GPU per problem, no collectives), so
N ranks run N independent replicas (weak scaling); value = max-over-ranks time
divided by the solves all ranks completed.
`--impl reference` times the FP64 CPU oracle on a bounded sample of the same
workload per step (one subdomain's share of every stage) and reports the
extrapolation to one full solve, labelled as such.
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
    ap.add_argument("--config", default="c3")
    ap.add_argument("--precision", default="mixed", choices=["fp64", "mixed"])
    ap.add_argument("--other-steps", type=int, default=5,
                    help="timed solves of the other precision (at most --steps)")
    ap.add_argument("--no-other", action="store_true", help="skip the other precision's leg")
    ap.add_argument("--no-c2", action="store_true",
                    help="skip the 64x32x24 legs (GenEO FP64/mixed, one-level AS, plain CG)")
    ap.add_argument("--no-profile", action="store_true", help="skip the per-kernel rooflines")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-darcy", action="store_true")
    ap.add_argument("--batch-blocks", type=int, default=256,
                    help="blocks of the uneven batched-solve workload to run (0 skips it)")
    ap.add_argument("--batch-concurrency", type=int, default=8,
                    help="contexts that assemble and set up the batch's blocks concurrently")
    ap.add_argument("--serve-requests", type=int, default=10,
                    help="requests of the serving sample (uneven laminate blocks)")
    ap.add_argument("--serve-rates", default="0.5,0.8",
                    help="Poisson arrival rates of the serving runs after the burst, as "
                         "fractions of the burst's solves/s (comma-separated)")
    ap.add_argument("--serve-darcy-grid", default=None, choices=[None, "spe10"],
                    help="spe10: the stream's Darcy requests are the 60x220x85 SPE10 grid")
    ap.add_argument("--serve-only", action="store_true",
                    help="run only the serving stream and print its summary")
    ap.add_argument("--profile-case", default=None, choices=["schwarz", "chol", "spmv"],
                    help="the small cases the ncu captures under profiles/ use: a 32x32x24 "
                         "laminate in 2x2x2 subdomains of the 128x64x48 workload's size, set up "
                         "in mixed precision, then the local solves (schwarz) or the band "
                         "Cholesky of the shifted Neumann matrices (chol) through geneo_profile; "
                         "spmv: five SpMVs of a 96x48x36 laminate (361 MB of BSR, above L2)")
    return ap.parse_args()


def workload_config(p, prec):
    wr = " with a fibre wrinkle" if np.any(np.asarray(p.get("elem_phi", 0.0)) != 0) else ""
    s = dict(workload=f"{p['name']}: {p['nx']}x{p['ny']}x{p['nz']} Q1 hex laminate{wr}, "
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
FP64_PEAK_SOURCE = ("nominal FP64 1.25 TFLOP/s (152 SMs x 2 FMA/clk x 2.07 GHz); "
                    "torch DGEMM measured 1.10")


def profiled_traffic(kernel, args):
    """DRAM bytes per launch of `kernel` from the committed ncu summary of this
    workload (profiles/dram_<config>_<precision>.md), or None when the summary
    is missing or was taken on a different version of the kernel's source."""
    import hashlib
    path = os.path.join(ROOT, "profiles", f"dram_{args.config}_{args.precision}.md")
    if not os.path.exists(path):
        return None
    srcs = {"k_schwarz_cluster": "schwarz.cu", "k_band_solve_dense": "band.cu",
            "band_cholesky_neumann": "band.cu"}
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

def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def blas_threads():
    try:
        from threadpoolctl import threadpool_info
        n = [d.get("num_threads") for d in threadpool_info() if d.get("user_api") == "blas"]
        if n:
            return int(max(n)), "threadpoolctl"
    except ImportError:
        pass
    for k in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
        if os.environ.get(k):
            return int(os.environ[k]), k
    return os.cpu_count() or 1, "library default (all cores)"


def oracle_sample(p, A, subs, gpu_iterations, step=0):
    """Time one subdomain's share of the oracle's whole solve on this workload:
    1/nsub of the element assembly, the GenEO eigensolve and the subdomain
    factorisation (sparse LU of A_j = R_j A R_j^T, as the oracle's one-level
    term builds it) of one subdomain (rotating with `step`), and per iteration
    an SpMV over 1/nsub of the elements plus that subdomain's solve.  A is the
    oracle's assembled global matrix (built once, outside the samples).
    Returns (measured ms of the sample, ms extrapolated to one full solve
    (x nsub), sample description).  The coarse space and the vector updates
    are not sampled."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    from oracle import fem, geneo
    t_start = time.perf_counter()
    ns = len(subs)
    nel = p["nx"] * p["ny"] * p["nz"]
    t0 = time.perf_counter()
    Ae = fem.assemble_stiffness(p, np.arange(step % ns, nel, ns)).tocsr()
    t_asm = time.perf_counter() - t0
    j = (ns // 2 + 1 + step) % ns
    m = p["modes"]
    nev = (m["fixed_modes"] if m["fixed_modes"] > 0 else m["max_modes"]) + 1
    t0 = time.perf_counter()
    Aj, Aoj = geneo.local_matrices(p, subs[j])
    Xd = sp.diags(subs[j].X)
    geneo.eigenpairs(Aj, (Xd @ Aoj @ Xd).tocsr(), nev, m["shift"])
    t_eig = time.perf_counter() - t0
    t0 = time.perf_counter()
    d = subs[j].int_dofs
    lu = spla.splu(A[d][:, d].tocsc())
    t_fac = time.perf_counter() - t0
    x = np.ones(Ae.shape[0])
    rj = np.ones(d.size)
    t0 = time.perf_counter()
    for _ in range(gpu_iterations):
        Ae @ x
        lu.solve(rj)
    t_it = time.perf_counter() - t0
    measured = time.perf_counter() - t_start
    full = (t_asm + t_eig + t_fac + t_it) * ns
    sample = (f"one subdomain's share of the FP64 oracle: 1/{ns} of the element assembly, "
              f"subdomain {j}'s GenEO eigensolve (ARPACK shift-invert) and sparse LU, "
              f"{gpu_iterations} iterations of an SpMV over 1/{ns} of the elements plus its local "
              f"solve; extrapolated x{ns}; coarse space and vector updates not sampled")
    return measured * 1000.0, full * 1000.0, sample


def golden(config):
    path = os.path.join(ROOT, "tests", "golden", f"{config}_oracle.json")
    return json.load(open(path)) if os.path.exists(path) else None


def run_reference(args):
    import workloads
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import decomp, fem
    p = workloads.config(args.config)
    g = golden(args.config)
    iters = g["iterations"] if g else 100
    A, _ = fem.assemble_system(p)
    A = A.tocsr()
    subs = decomp.partition(p)
    for w in range(args.warmup):
        oracle_sample(p, A, subs, iters, step=w)
    meas, full = [], []
    sample = ""
    for k in range(args.steps):
        ms, est, sample = oracle_sample(p, A, subs, iters, step=args.warmup + k)
        meas.append(ms)
        full.append(est)
    v = statistics.mean(full)
    threads, how = blas_threads()
    cpu = dict(value=v, unit=UNIT, cores=os.cpu_count() or 1, kind="oracle", sample=sample,
               estimate="extrapolated from the sample, not a timed full solve",
               cpu_model=cpu_model(), blas_threads=threads, blas_threads_set_by=how,
               sparse_lu_threads=1)
    if g and "oracle_seconds" in g:
        cpu["full_solve_recorded_s"] = g["oracle_seconds"].get("total")
        cpu["full_solve_recorded_on"] = "the machine that wrote tests/golden (x86, 8 cores)"
    line = dict(metric=METRIC, value=v, unit=UNIT, n_gpus=args.gpus, steps=args.steps,
                warmup=args.warmup, ms_per_step=statistics.mean(meas), higher_is_better=False,
                scaling="weak", vs_baseline=None, dtype="f64", data="synthetic", impl="reference",
                config=workload_config(p, "fp64"), cpu_baseline=cpu,
                extrapolation=dict(ms_per_step_measured=statistics.mean(meas),
                                   factor=int(p["partition"][0] * p["partition"][1] *
                                              p["partition"][2]),
                                   note="value = one full solve extrapolated from each step's "
                                        "sample; ms_per_step = the sample actually timed"),
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


def one_solve(pkg, s, p, prec, out, schwarz=0, coarse=0, max_it=5000):
    s.assemble(p)
    s.setup(p, prec, schwarz, coarse)
    u, st = s.solve(tol=TOL, max_it=max_it, out=out, raise_on_nonconvergence=False)
    return st


def oracle_error(u, g):
    """Error of the displacement u against the FP64 oracle's stored solution:
    relative L2 over the stored samples, the norm of u, and the largest
    deviation of the per-chunk norms (every dof is in one chunk) relative to
    the largest chunk norm."""
    if g is None:
        return None
    us = u[::g["sample_stride"]][:len(g["u_samples"])]
    ref = np.asarray(g["u_samples"])
    out = dict(rel_l2_err_samples=float(np.linalg.norm(us - ref) / np.linalg.norm(ref)),
               n_samples=int(ref.size),
               rel_err_u_norm=float(abs(np.linalg.norm(u) - g["u_norm"]) / g["u_norm"]),
               oracle_iterations=g["iterations"])
    if "u_chunk_norms" in g:
        ch = int(g["chunk"])
        cn = np.sqrt(np.add.reduceat(u * u, np.arange(0, u.size, ch)))
        rc = np.asarray(g["u_chunk_norms"])
        out["max_dev_chunk_norms"] = float(np.max(np.abs(cn - rc)) / np.max(rc))
    return out


def leg_summary(st):
    return dict(iterations=st["iterations"], rel_res_true=st["rel_res_true"],
                n_coarse=st["n_coarse"], kappa_est=st["kappa_est"],
                phases_ms=dict(assemble=st["ms_assemble"], setup_eig_coarse=st["ms_setup_eig"],
                               setup_factor=st["ms_setup_factor"], solve=st["ms_solve"]),
                schwarz_launch=dict(cluster=st["schwarz_cluster"], rows=st["schwarz_rows"],
                                    staged=st["schwarz_staged"]))


def tf32_peak():
    """Dense TF32 tensor peak: the measured bf16 burst peak times the nominal
    TF32 / bf16 ratio (1.1 / 2.25 PFLOP/s)."""
    try:
        d = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        return float(d["bf16_tflops"]) * 1.1 / 2.25, "measured bf16 x nominal TF32/bf16"
    except Exception:
        return 1900.0 * 1.1 / 2.25, "fallback bf16 x nominal TF32/bf16"


def rooflines(pkg, s, st, args, peak, peak_kind):
    """Per-kernel rooflines of one solve of the resident set-up, each with its
    time share: (ms per solve, record) for the Schwarz local solves, the SpMV,
    the eigensolver's band solves, the Cholesky of the shifted Neumann
    matrices and the subdomain factorisation."""
    mixed = args.precision == "mixed"
    cand = []
    n_it = st["iterations"] + 1
    ms, by, fl = pkg.geneo_profile(s.ctx, 0, 10)
    cand.append((ms * n_it, dict(
        bound="hbm", kernel="k_schwarz_cluster* (one-level local band solves, "
                            f"{'FP32' if mixed else 'FP64'})",
        achieved=by / (ms * 1e-3) / 1e9, peak=peak, unit="GB/s", peak_source=f"{peak_kind} hbm_gbs",
        ms_per_launch=ms, algorithmic_bytes=by, launches_per_solve=n_it)))
    ms, by, fl = pkg.geneo_profile(s.ctx, 1, 50)
    cand.append((ms * n_it, dict(
        bound="hbm", kernel="k_cg_spmv_pq / k_spmv (3x3 BSR SpMV, FP64)",
        achieved=by / (ms * 1e-3) / 1e9, peak=peak, unit="GB/s", peak_source=f"{peak_kind} hbm_gbs",
        ms_per_launch=ms, algorithmic_bytes=by, launches_per_solve=n_it)))
    if st["n_coarse"] > 0 and st["lanczos_steps"] > 0:
        n_l = 2 * st["lanczos_steps"] + 1     # two sweeps per block step + the Ritz vectors
        ms, by, fl = pkg.geneo_profile(s.ctx, 3, 5)
        cand.append((ms * n_l, dict(
            bound="alu", kernel="k_band_solve_dense (GenEO shift-invert band solves, FP64, "
                                "8 right-hand sides)",
            achieved=fl / (ms * 1e-3) / 1e12, peak=FP64_PEAK_TFLOPS, unit="TFLOP/s",
            peak_source=FP64_PEAK_SOURCE, ms_per_launch=ms, algorithmic_flops=fl,
            algorithmic_bytes=by, launches_per_solve=n_l)))
        ms, by, fl = pkg.geneo_profile(s.ctx, 4, 2)
        cand.append((ms, dict(
            bound="alu", kernel="band Cholesky of S_j = A_j - sigma B_j (k_chol_diag/trsm/"
                                "update<double>, FP64)",
            achieved=fl / (ms * 1e-3) / 1e12, peak=FP64_PEAK_TFLOPS, unit="TFLOP/s",
            peak_source=FP64_PEAK_SOURCE, ms_per_launch=ms, algorithmic_flops=fl,
            algorithmic_bytes=by, launches_per_solve=1)))
    ms, by, fl = pkg.geneo_profile(s.ctx, 5, 2)
    if mixed:
        tp, tsrc = tf32_peak()
        rec = dict(bound="tensor", kernel="band Cholesky of A_j, FP32 with 3xTF32 tcgen05 trailing "
                                          "updates (k_chol_update_tc)",
                   achieved=3 * fl / (ms * 1e-3) / 1e12, peak=tp, unit="TFLOP/s",
                   peak_source=tsrc, ms_per_launch=ms, algorithmic_flops=fl,
                   tensor_flops=3 * fl, launches_per_solve=1,
                   note="runs beside the GenEO eigensolve on its own streams")
    else:
        rec = dict(bound="alu", kernel="band Cholesky of A_j (k_chol_*<double>, FP64)",
                   achieved=fl / (ms * 1e-3) / 1e12, peak=FP64_PEAK_TFLOPS, unit="TFLOP/s",
                   peak_source=FP64_PEAK_SOURCE, ms_per_launch=ms, algorithmic_flops=fl,
                   launches_per_solve=1, note="runs beside the GenEO eigensolve on its own streams")
    cand.append((ms, rec))
    for t, r in cand:
        r["frac"] = r["achieved"] / r["peak"]
        r["ms_per_solve"] = t
    cand.sort(key=lambda t: -t[0])
    return cand


def serving_leg(pkg, args):
    """The continuous-batching server on a seeded stream of uneven requests:
    a burst (saturated throughput), then Poisson arrivals at the given
    fractions of the burst's solves/s; errors against the oracle's stored
    solutions of the stream's small requests where they exist."""
    from paper_1901_05188_gb300.serve import serve_benchmark
    gpath = os.path.join(ROOT, "tests", "golden", "serving_oracle.json")
    golden = None
    if os.path.exists(gpath):
        g = json.load(open(gpath))
        if (g["n"], g["seed"], g["darcy_grid"]) == (args.serve_requests, 6, args.serve_darcy_grid):
            golden = g["requests"]
    rates = tuple(float(x) for x in args.serve_rates.split(",") if x.strip())
    sv = serve_benchmark(n=args.serve_requests, seed=6, prec=pkg.GENEO_MIXED_FP32, slots=4,
                         rate_factors=(None,) + rates, darcy_frac=0.3,
                         darcy_grid=args.serve_darcy_grid, golden=golden,
                         progress=lambda r: print(json.dumps({k: v for k, v in r.items()
                                                              if k != "iterations"}),
                                                  file=sys.stderr, flush=True))
    dgrid = "the 60x220x85 SPE10 grid" if args.serve_darcy_grid == "spe10" else "SPE10 proportions"
    return dict(workload=f"{sv['requests']} requests: {sv['requests'] - sv['darcy']} laminate "
                         f"blocks and {sv['darcy']} Darcy problems (layered permeability, {dgrid}), "
                         f"{min(sv['dofs'])}-{max(sv['dofs'])} unknowns (laminates log-uniform "
                         f"2e4-2e6, seed 6), {sv['repeats']} repeated structures with new loads",
                precision=sv["precision"], slots=sv["slots"],
                runs=[{k: r[k] for k in ("arrivals", "n", "p50_ms", "p99_ms", "mean_ms",
                                         "solves_per_s", "reused", "peak_inflight",
                                         "peak_mem_gb", "failed", "oracle_checked",
                                         "max_rel_err_vs_oracle") if k in r}
                      for r in sv["runs"]])


def batched_uneven(pkg, torch, dev, nblocks, nconc=8):
    import concurrent.futures as cf
    from paper_1901_05188_gb300.serve import request_memory
    from workloads.batch import batch_blocks
    prec = pkg.GENEO_MIXED_FP32
    blocks = batch_blocks(nblocks, seed=3)
    est = [request_memory(pb, prec) for pb in blocks]
    torch.cuda.synchronize(dev)
    torch.cuda.empty_cache()                  # the earlier legs' cached blocks
    budget = 0.6 * torch.cuda.mem_get_info(dev)[0]
    waves, cur, used = [], [], 0
    for k, e in enumerate(est):
        if cur and used + e > budget:
            waves.append(cur)
            cur, used = [], 0
        cur.append(k)
        used += e
    waves.append(cur)
    streams = [torch.cuda.Stream(dev) for _ in range(nconc)]

    def build(k, st):
        with torch.cuda.stream(st):
            sv = pkg.GeneoSolver(stream=st.cuda_stream, device=dev.index)
            sv.assemble(blocks[k])
            sv.setup(blocks[k], prec)
        return sv

    iters, failed, t_setup, t_solve, shapes = [], 0, 0.0, 0.0, set()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(nconc) as ex:
        for wv in waves:
            ta = time.perf_counter()
            futs = [ex.submit(build, k, streams[i % nconc]) for i, k in enumerate(wv)]
            solvers = [f.result() for f in futs]
            for st in streams:
                st.synchronize()
            tb = time.perf_counter()
            bt = pkg.GeneoBatch(solvers)
            outs = [torch.empty(sv.ndof, dtype=torch.float64, device=dev) for sv in solvers]
            _, stats = bt.solve(tol=TOL, max_it=5000, outs=outs, raise_on_nonconvergence=False)
            torch.cuda.synchronize(dev)
            tc = time.perf_counter()
            bt.close()
            for sv in solvers:
                sv.close()
            t_setup += tb - ta
            t_solve += tc - tb
            iters += [st["iterations"] for st in stats]
            failed += sum(1 for st in stats if not st["rel_res_recursive"] <= TOL)
            shapes.add((stats[0]["schwarz_rows"], stats[0]["schwarz_staged"]))
    wall = time.perf_counter() - t0
    dofs = [3 * (pb["nx"] + 1) * (pb["ny"] + 1) * (pb["nz"] + 1) for pb in blocks]
    parts = [pb["partition"][0] * pb["partition"][1] * pb["partition"][2] for pb in blocks]
    return dict(workload=f"{len(blocks)} blocks of the seeded batch (seed 3): {min(dofs)}-{max(dofs)} "
                         f"dofs ({sum(dofs)} in all), {min(parts)}-{max(parts)} subdomains "
                         f"({sum(parts)} in all), 4-24 plies",
                precision="mixed", waves=len(waves), wave_sizes=[len(w) for w in waves],
                memory_budget_gb=budget / 1e9, wall_s=wall, setup_s=t_setup, batched_solve_s=t_solve,
                solves_per_s=len(blocks) / wall, dofs_per_s=sum(dofs) / wall,
                iterations=dict(min=min(iters), max=max(iters),
                                mean=float(np.mean(iters))),
                local_solve_shapes=sorted([dict(rows=r, staged=st) for r, st in shapes],
                                          key=lambda d: (d["rows"], d["staged"])),
                setup=f"{nconc} concurrent contexts", failed=failed)


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
    mixed = args.precision == "mixed"
    prec = pkg.GENEO_MIXED_FP32 if mixed else pkg.GENEO_FP64
    other = pkg.GENEO_FP64 if mixed else pkg.GENEO_MIXED_FP32
    p = workloads.config(args.config)
    g = golden(args.config)
    pd = device_problem(p, torch, dev)
    s = pkg.GeneoSolver()
    ndof = 3 * (p["nx"] + 1) * (p["ny"] + 1) * (p["nz"] + 1)
    u_dev = torch.empty(ndof, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    def timed(prob, pr, out, steps, warm, **kw):
        for _ in range(warm):
            st = one_solve(pkg, s, prob, pr, out, **kw)
        torch.cuda.synchronize(dev)
        e0.record(stream)
        for _ in range(steps):
            st = one_solve(pkg, s, prob, pr, out, **kw)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1) / steps, st

    for _ in range(args.warmup):
        st = one_solve(pkg, s, pd, prec, u_dev)
    barrier()
    clocks = ClockSampler(local)
    clocks.start()
    l0 = pkg.geneo_launch_count()
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
    acc = oracle_error(u_dev.cpu().numpy(), g)

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
        e2e = dict(value=e2e_ms, unit=UNIT, steps=args.steps,
                   h2d_bytes_per_step=host_bytes(p), d2h_bytes_per_step=8 * ndof)

    # rooflines of the resident set-up's kernels; the headline object is the
    # kernel with the largest share of one solve
    peak, peak_kind = measured_peaks()
    roof, kernels = None, None
    if not args.no_profile:
        cand = rooflines(pkg, s, st, args, peak, peak_kind)
        roof = dict(cand[0][1])
        for k in ("k_band_solve_dense", "k_schwarz_cluster"):
            if roof["kernel"].startswith(k):
                roof["traffic"] = profiled_traffic(k, args)
        if roof["kernel"].startswith("band Cholesky of S_j"):
            roof["traffic"] = profiled_traffic("band_cholesky_neumann", args)
        roof.setdefault("traffic", None)
        ms_pc, by_pc, _ = pkg.geneo_profile(s.ctx, 2, 10)
        kernels = dict(precond_apply=dict(ms=ms_pc, gbs=by_pc / (ms_pc * 1e-3) / 1e9),
                       other_rooflines=[c[1] for c in cand[1:]])

    # the other precision on the same workload, at equal accuracy
    other_leg = None
    if rank == 0 and world == 1 and not args.no_other:
        k = max(1, min(args.steps, args.other_steps))
        ms_o, st_o = timed(pd, other, u_dev, k, 1)
        other_leg = dict(precision="fp64" if mixed else "mixed", ms_per_solve=ms_o, steps=k,
                         **leg_summary(st_o), oracle_error=oracle_error(u_dev.cpu().numpy(), g))
        other_leg["speedup_of_mixed"] = (ms_o / value) if mixed else (value / ms_o)

    # the 64x32x24 laminate: GenEO in both precisions against one-level
    # additive Schwarz and unpreconditioned CG
    c2 = None
    if rank == 0 and world == 1 and not args.no_c2 and args.config != "c2":
        p2 = workloads.config("c2")
        g2 = golden("c2")
        pd2 = device_problem(p2, torch, dev)
        n2 = 3 * (p2["nx"] + 1) * (p2["ny"] + 1) * (p2["nz"] + 1)
        u2 = torch.empty(n2, dtype=torch.float64, device=dev)
        c2 = dict(workload=workload_config(p2, "fp64")["workload"],
                  partition=workload_config(p2, "fp64")["partition"])
        k2 = max(1, min(args.steps, 3))
        for key, pr, sw, co, mi in (("geneo_fp64", pkg.GENEO_FP64, pkg.GENEO_AS, 0, 5000),
                                    ("geneo_mixed", pkg.GENEO_MIXED_FP32, pkg.GENEO_AS, 0, 5000),
                                    ("one_level_as_fp64", pkg.GENEO_FP64, pkg.GENEO_AS,
                                     pkg.GENEO_COARSE_NONE, 20000),
                                    ("plain_cg", pkg.GENEO_FP64, pkg.GENEO_NO_PRECOND, 0, 20000)):
            kk = k2 if key.startswith("geneo") else 1
            ms2, st2 = timed(pd2, pr, u2, kk, 1, schwarz=sw, coarse=co, max_it=mi)
            c2[key] = dict(ms_per_solve=ms2, steps=kk, converged=st2["rel_res_recursive"] <= TOL,
                           **leg_summary(st2), oracle_error=oracle_error(u2.cpu().numpy(), g2))
        # threshold scaling (Sec. 3.2: the eigenvalue threshold trades coarse
        # dimension and set-up time against iterations).  The default rule's
        # threshold (diam / width, about 250 here) lies far above the 32nd
        # eigenvalue (below 0.2), so the cap decides there; the sweep takes
        # absolute thresholds across the computed spectrum, cap 32 modes
        keep = []
        taus = pkg.geneo_default_thresholds(pkg.GeneoSolver.mesh_of(p2, keep),
                                            pkg.GeneoSolver.partition_of(p2))
        sweep = []
        for tau in (0.003, 0.01, 0.03, 0.06, 0.12):
            q = dict(p2, modes=dict(fixed_modes=0, threshold=tau, max_modes=32, shift=-0.01))
            ms_t, st_t = timed(device_problem(q, torch, dev), pkg.GENEO_FP64, u2, 1, 1)
            sweep.append(dict(threshold=tau, ms_per_solve=ms_t,
                              n_coarse=st_t["n_coarse"], iterations=st_t["iterations"],
                              kappa_est=st_t["kappa_est"],
                              setup_ms=st_t["ms_setup_eig"], solve_ms=st_t["ms_solve"]))
        c2["threshold_sweep"] = dict(default_threshold_median=float(np.median(taus)), cap=32,
                                     precision="fp64", runs=sweep)
        del pd2, u2

    # serving: a seeded stream of uneven solve requests through the
    # continuous-batching server (burst, then Poisson at half its throughput)
    serving = None
    if rank == 0 and world == 1 and not args.no_serve and args.serve_requests > 0:
        serving = serving_leg(pkg, args)

    # batched uneven solves: the seeded batch of laminated blocks (8e3-1e5
    # elements, 4-24 plies, 2-64 subdomains), in waves that fit the device
    # memory: each wave's instances are assembled and set up by eight
    # concurrent contexts, then solved together by one batched FCG (one
    # launch per step over the wave, local solves in one persistent
    # work-queue launch, iterations in a CUDA graph)
    batch = None
    if rank == 0 and world == 1 and args.batch_blocks > 0:
        batch = batched_uneven(pkg, torch, dev, args.batch_blocks, args.batch_concurrency)

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

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        from oracle import decomp, fem
        A, _ = fem.assemble_system(p)
        ms_s, ms_cpu, sample = oracle_sample(p, A.tocsr(), decomp.partition(p), st["iterations"])
        threads, how = blas_threads()
        cpu = dict(value=ms_cpu, unit=UNIT, cores=os.cpu_count() or 1, kind="oracle",
                   sample=sample, sample_ms=ms_s,
                   estimate="extrapolated from the sample, not a timed full solve",
                   cpu_model=cpu_model(), blas_threads=threads, blas_threads_set_by=how,
                   sparse_lu_threads=1)
        if g and "oracle_seconds" in g:
            cpu["full_solve_recorded_s"] = g["oracle_seconds"].get("total")
            cpu["full_solve_recorded_on"] = "the machine that wrote tests/golden (x86, 8 cores)"

    if rank == 0:
        line = dict(metric=METRIC, value=value, unit=UNIT, n_gpus=world, steps=args.steps,
                    warmup=args.warmup, ms_per_step=ms_step, higher_is_better=False,
                    scaling="weak", vs_baseline=None,
                    dtype="f64" if args.precision == "fp64" else "f64+f32",
                    data="synthetic", config=workload_config(p, args.precision),
                    roofline=roof, cpu_baseline=cpu, e2e=e2e, gpu_launches=int(launches),
                    clocks=clk, **leg_summary(st), bytes_per_iter=st["bytes_per_iter"],
                    oracle_error=acc, kernels=kernels,
                    **{("fp64" if mixed else "mixed"): other_leg},
                    c2=c2, serving=serving, darcy_spe10=darcy, batched_uneven=batch)
        line["schwarz_launch"]["chosen_by"] = "set-up autotuner"
        print(json.dumps(line))
    s.close()
    if world > 1:
        dist.destroy_process_group()


def profile_case(args):
    import paper_1901_05188_gb300 as pkg
    from workloads.laminate import make_block
    pkg.load(build_if_missing=True)
    if args.profile_case == "spmv":
        import torch
        p = make_block(96, 48, 36, [0.0, 45.0, -45.0, 90.0] * 3, partition=(1, 1, 1, 1),
                       name="spmv-96x48x36")
        s = pkg.GeneoSolver()
        s.assemble(p)
        x = torch.ones(s.ndof, dtype=torch.float64, device="cuda")
        y = torch.empty_like(x)
        for _ in range(5):
            pkg.geneo_spmv(s.ctx, x, y)
        torch.cuda.synchronize()
        print(json.dumps(dict(spmv_nnzb=s.nnzb, ndof=s.ndof,
                              bsr_bytes=s.nnzb * 76 + 4 * (s.nnode + 1))))
        s.close()
        return
    thr = dict(fixed_modes=0, threshold=0.0, max_modes=20, shift=-0.01)
    p = make_block(32, 32, 24, [0.0, 45.0, -45.0, 90.0] * 3, partition=(2, 2, 2, 1), modes=thr,
                   name="c3-subdomains-8")
    s = pkg.GeneoSolver()
    s.assemble(p)
    s.setup(p, pkg.GENEO_MIXED_FP32)
    out = {}
    if args.profile_case == "schwarz":
        ms, by, _ = pkg.geneo_profile(s.ctx, 0, 3)
        out["schwarz"] = dict(ms=ms, bytes=by)
    else:
        ms, by, fl = pkg.geneo_profile(s.ctx, 4, 1)
        out["chol_neumann"] = dict(ms=ms, bytes=by, flops=fl)
    s.close()
    print(json.dumps(out))


def main():
    args = parse()
    if args.profile_case:
        profile_case(args)
        return
    if args.serve_only:
        import torch
        import paper_1901_05188_gb300 as pkg
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        pkg.load(build_if_missing=True)
        print(json.dumps(dict(serving=serving_leg(pkg, args))))
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
