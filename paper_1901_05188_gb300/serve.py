"""Serving loop for GenEO-PCG solve requests with continuous batching.

Requests arrive at any time and wait in a FIFO queue.  A dispatcher admits the
request at the head of the queue as soon as a slot is free and the request's
device memory (the library's host-only workspace estimate) fits in the
remaining budget; a request arriving while others run on the GPU is admitted
the moment a slot and memory free up, and its kernels overlap with theirs
(every slot owns a CUDA stream and a solver context; the library releases the
GIL during its calls).  A slot keeps its last problem's assembly and
preconditioner resident: a later request with the same `key` (same structure,
any load) skips assembly and set-up, replaces the load and only solves.

The scheduling logic is plain host code; the execution step is pluggable
(`executor`), so the admission rules are tested on the CPU with a fake
executor, while the default executor runs the library on the GPU.
"""
from __future__ import annotations

import collections
import threading
import time
from dataclasses import dataclass, field
from typing import Any, Callable, Optional

import numpy as np


@dataclass
class Request:
    rid: int
    problem: dict
    prec: int = 0
    tol: float = 1e-8
    # same key = same structure (mesh, materials, Dirichlet data, partition,
    # modes); the load may differ, so resident factors can be reused
    key: Optional[str] = None
    mem: int = 0                        # admitted device bytes (estimate)
    t_arrival: float = 0.0
    t_start: float = 0.0
    t_done: float = 0.0
    slot: int = -1
    u: Any = None
    stats: dict = field(default_factory=dict)
    error: Optional[str] = None
    reused: bool = False
    _done: threading.Event = field(default_factory=threading.Event, repr=False)

    def wait(self, timeout=None):
        if not self._done.wait(timeout):
            raise TimeoutError(f"request {self.rid} not finished")
        return self

    @property
    def latency(self):
        return self.t_done - self.t_arrival


def request_memory(problem, prec):
    """Device bytes a request needs (host-only estimate from the library)."""
    from . import GeneoSolver, geneo_estimate_workspace_bytes
    keep = []
    mesh = GeneoSolver.mesh_of(problem, keep)
    a, s = geneo_estimate_workspace_bytes(mesh, GeneoSolver.partition_of(problem),
                                          GeneoSolver.modes_of(problem), prec,
                                          GeneoSolver.unknowns_per_node(problem))
    return int(a + s)


class GpuSlotExecutor:
    """Runs a request on the GPU in slot `slot` (one stream + solver per slot).

    With `reuse` the slot's resident matrix and preconditioner (from its last
    request, same key) are kept: the request's load replaces the right-hand
    side and only the PCG solve runs.
    """

    def __init__(self, device=0):
        import torch
        self.torch = torch
        self.device = torch.device("cuda", device)
        self.streams = {}
        self.solvers = {}

    def _slot(self, slot):
        torch = self.torch
        if slot not in self.solvers:
            from . import GeneoSolver
            torch.cuda.set_device(self.device)
            st = torch.cuda.Stream(self.device)
            self.streams[slot] = st
            self.solvers[slot] = GeneoSolver(stream=st.cuda_stream, device=self.device.index)
        return self.solvers[slot]

    def __call__(self, slot, req, reuse):
        torch = self.torch
        torch.cuda.set_device(self.device)
        s = self._slot(slot)
        with torch.cuda.stream(self.streams[slot]):
            if reuse:
                scalar = req.problem["source" if req.problem.get("kind") == "darcy" else "top_pressure"]
                s.set_load(req.problem.get("nodal_load"), scalar)
            else:
                s.assemble(req.problem)
                s.setup(req.problem, req.prec)
            u, st = s.solve(tol=req.tol, max_it=5000)
        req.u, req.stats = u, st

    def release(self, slot):
        """Release the slot's resident problem and workspaces (the slot is idle)."""
        s = self.solvers.pop(slot, None)
        if s is not None:
            self.streams[slot].synchronize()
            s.close()
            self.torch.cuda.empty_cache()

    def close(self):
        for slot, s in self.solvers.items():
            self.streams[slot].synchronize()
            s.close()
        self.solvers.clear()
        self.torch.cuda.empty_cache()       # the next server sees the memory as free


class GeneoServer:
    """Continuous-batching server: up to `slots` concurrent solves within `mem_budget` bytes.

    Memory model: a slot keeps the device workspace of its largest request
    (the library's workspaces only grow), so the budget is charged with the
    sum over slots of their resident bytes.  Admission is FIFO (a request
    whose key is resident in a busy slot waits for that slot and lets later
    requests pass): a request is placed on an idle slot that holds its key (no
    assembly or set-up), else on an idle slot holding no resident problem,
    else on the idle slot whose growth to the request's size keeps the total
    lowest; in every case only if the new total fits the budget.
    """

    def __init__(self, slots=4, mem_budget=None, executor: Optional[Callable] = None,
                 memory_of: Optional[Callable] = None, device=0):
        if executor is None:
            executor = GpuSlotExecutor(device)
            if mem_budget is None:
                import torch
                free, _ = torch.cuda.mem_get_info(device)
                mem_budget = int(0.8 * free)
        self.executor = executor
        self.memory_of = memory_of or (lambda r: request_memory(r.problem, r.prec))
        self.mem_budget = int(mem_budget if mem_budget is not None else 1 << 62)
        self.nslots = slots
        self.idle = [True] * slots
        self.slot_mem = [0] * slots          # resident device bytes per slot
        self.slot_key = [None] * slots       # (key, precision) of the slot's resident problem
        self.queue = collections.deque()
        self.lock = threading.Condition()
        self.closed = False
        self.next_id = 0
        self.done = []
        self.peak_mem = 0
        self.peak_inflight = 0
        self.inflight = 0
        self.evictions = 0
        self.dispatcher = threading.Thread(target=self._dispatch, daemon=True)
        self.dispatcher.start()

    @property
    def mem_in_use(self):
        return sum(self.slot_mem)

    def submit(self, problem, prec=0, tol=1e-8, key=None, arrival=None):
        req = Request(rid=self.next_id, problem=problem, prec=prec, tol=tol, key=key)
        self.next_id += 1
        req.t_arrival = time.perf_counter() if arrival is None else arrival
        req.mem = int(self.memory_of(req))
        if req.mem > self.mem_budget:
            req.error = f"request needs {req.mem} bytes, budget is {self.mem_budget}"
            req.t_done = time.perf_counter()
            req._done.set()
            return req
        with self.lock:
            self.queue.append(req)
            self.lock.notify_all()
        return req

    def cancel(self, req):
        """Remove a request that is still queued; returns True if it was removed."""
        with self.lock:
            try:
                self.queue.remove(req)
            except ValueError:
                return False
        req.error = "cancelled"
        req.t_done = time.perf_counter()
        req._done.set()
        return True

    def _place(self, req):
        """(slot, reuse, evict) for the queue head, or None if it must wait.  Lock held.

        evict lists idle slots whose resident workspaces must be released
        first.  Without eviction a slot only grows to the request's size; when
        that fits nowhere, the idle slots are released one at a time, the
        largest first (the slot the request runs on is released first when
        its own memory is not enough), until the request fits; when even
        releasing every idle slot is not enough it waits for a busy slot."""
        idle = [s for s in range(self.nslots) if self.idle[s]]
        if not idle:
            return None
        if req.key is not None:
            for s in idle:
                if self.slot_key[s] == (req.key, req.prec) and self.slot_mem[s] >= req.mem:
                    return s, True, []
        total = self.mem_in_use
        best = None
        for s in idle:
            t = total - self.slot_mem[s] + max(self.slot_mem[s], req.mem)
            # keep resident problems while an empty slot fits; then the lowest total
            rank = (self.slot_key[s] is not None, t, s)
            if t <= self.mem_budget and (best is None or rank < best[0]):
                best = (rank, s)
        if best is not None:
            return best[1], False, []
        # release idle slots, largest first, until the request fits on one of them
        order = sorted(idle, key=lambda s: (-self.slot_mem[s], s))
        target = order[0]
        evict = [target]
        t = total - self.slot_mem[target] + req.mem
        for s in order[1:]:
            if t <= self.mem_budget:
                break
            evict.append(s)
            t -= self.slot_mem[s]
        if t > self.mem_budget:
            return None
        return target, False, evict

    def _next(self):
        """(request, slot, reuse) to start now, or None.  Lock held.

        FIFO, except that a request whose structure is resident in a busy slot
        waits for that slot (it will only solve there) and lets the requests
        behind it go first; the first request that may start anywhere but does
        not fit the memory budget stops the scan (no bypass by size).
        """
        busy_keys = {self.slot_key[s] for s in range(self.nslots)
                     if not self.idle[s] and self.slot_key[s] is not None}
        for req in self.queue:
            if req.key is not None and (req.key, req.prec) in busy_keys:
                continue
            placed = self._place(req)
            if placed is None:
                return None
            return (req,) + placed
        return None

    def _dispatch(self):
        while True:
            with self.lock:
                nxt = None
                while not self.closed or self.queue:
                    if self.queue:
                        nxt = self._next()
                        if nxt is not None:
                            break
                    self.lock.wait(0.05)
                if nxt is None:
                    return
                req, slot, reuse, evict = nxt
                self.queue.remove(req)
                for e in evict:                      # idle slots: nothing runs on them
                    if hasattr(self.executor, "release"):
                        self.executor.release(e)
                    self.slot_mem[e] = 0
                    self.slot_key[e] = None
                    self.evictions += 1
                self.idle[slot] = False
                self.slot_mem[slot] = max(self.slot_mem[slot], req.mem)
                self.slot_key[slot] = None if req.key is None else (req.key, req.prec)
                self.inflight += 1
                self.peak_mem = max(self.peak_mem, self.mem_in_use)
                self.peak_inflight = max(self.peak_inflight, self.inflight)
            req.slot, req.reused = slot, reuse
            threading.Thread(target=self._run, args=(slot, req, reuse), daemon=True).start()

    def _run(self, slot, req, reuse):
        req.t_start = time.perf_counter()
        try:
            self.executor(slot, req, reuse)
        except Exception as e:  # reported on the request, the server keeps going
            req.error = f"{type(e).__name__}: {e}"
        req.t_done = time.perf_counter()
        with self.lock:
            if req.error is not None:
                self.slot_key[slot] = None       # the resident state is not trusted
            self.inflight -= 1
            self.idle[slot] = True
            self.done.append(req)
            self.lock.notify_all()
        req._done.set()

    def drain(self, timeout=None):
        t0 = time.perf_counter()
        while True:
            with self.lock:
                if not self.queue and self.inflight == 0:
                    return
            if timeout is not None and time.perf_counter() - t0 > timeout:
                raise TimeoutError("server did not drain")
            time.sleep(0.005)

    def close(self):
        self.drain()
        with self.lock:
            self.closed = True
            self.lock.notify_all()
        self.dispatcher.join(timeout=5)
        if hasattr(self.executor, "close"):
            self.executor.close()


def latency_summary(reqs):
    ok = [r for r in reqs if r.error is None]
    if not ok:
        return dict(n=0)
    lat = np.array([r.latency for r in ok]) * 1000.0
    t0 = min(r.t_arrival for r in ok)
    t1 = max(r.t_done for r in ok)
    return dict(n=len(ok), p50_ms=float(np.percentile(lat, 50)), p99_ms=float(np.percentile(lat, 99)),
                mean_ms=float(lat.mean()), max_ms=float(lat.max()),
                solves_per_s=len(ok) / max(t1 - t0, 1e-9),
                failed=len(reqs) - len(ok))


def run_poisson(server, problems, rate_hz, seed=0, prec=0, tol=1e-8, keys=None):
    """Submit `problems` with exponential inter-arrival times (rate_hz) and wait."""
    rng = np.random.default_rng(seed)
    reqs = []
    t_next = time.perf_counter()
    for i, p in enumerate(problems):
        now = time.perf_counter()
        if t_next > now:
            time.sleep(t_next - now)
        reqs.append(server.submit(p, prec=prec, tol=tol, key=None if keys is None else keys[i],
                                  arrival=t_next))
        t_next += rng.exponential(1.0 / rate_hz)
    for r in reqs:
        r.wait()
    return reqs


def serve_benchmark(n=10, seed=4, prec=1, slots=4, rate_factors=(None, 0.5), tol=1e-8,
                    dof_lo=2e4, dof_hi=2e6, warmup=True, darcy_frac=0.0, darcy_grid=None,
                    golden=None, progress=None):
    """Serve a seeded request stream; one summary per arrival pattern.

    rate_factors: None = every request arrives at t = 0 (a burst, which gives
    the saturated throughput); a number f = Poisson arrivals at f times the
    burst's solves/s; progress(summary) is called after every run.  golden:
    stored reference solutions of some requests of
    this stream ({request index: summary with sample_stride, u_samples,
    u_norm}); every run reports the largest relative error of those requests.
    Returns a dict with the stream description and the summaries.
    """
    from workloads.serving import dofs_of, request_stream
    base = request_stream(n, seed=seed, dof_lo=dof_lo, dof_hi=dof_hi, darcy_frac=darcy_frac,
                          darcy_grid=darcy_grid)
    if warmup:   # load the library and build every kernel variant once
        from workloads import config
        w = GeneoServer(slots=1)
        w.submit(config("c1"), prec=prec).wait()
        w.close()
    out = dict(requests=n, seed=seed, slots=slots, precision="mixed" if prec else "fp64",
               dofs=[dofs_of(p) for _, p, _ in base],
               darcy=sum(1 for _, p, _ in base if p.get("kind") == "darcy"),
               repeats=sum(1 for i, (k, _, _) in enumerate(base)
                           if any(k == kk for kk, _, _ in base[:i])),
               runs=[])
    burst_rate = None
    for f in rate_factors:
        srv = GeneoServer(slots=slots)
        try:
            t0 = time.perf_counter()
            if f is None:
                reqs = [srv.submit(p, prec=prec, tol=tol, key=k, arrival=t0) for k, p, _ in base]
                for r in reqs:
                    r.wait()
            else:
                rate = f * (burst_rate or 1.0)
                rng = np.random.default_rng(seed + 1)
                gaps = rng.exponential(1.0 / rate, size=n)
                reqs = []
                t_next = t0
                for (k, p, _), g in zip(base, gaps):
                    now = time.perf_counter()
                    if t_next > now:
                        time.sleep(t_next - now)
                    reqs.append(srv.submit(p, prec=prec, tol=tol, key=k, arrival=t_next))
                    t_next += g
                for r in reqs:
                    r.wait()
        finally:
            srv.close()
        s = latency_summary(reqs)
        s["arrivals"] = "burst" if f is None else f"poisson {rate:.3g}/s"
        s["reused"] = sum(1 for r in reqs if r.reused)
        s["evictions"] = srv.evictions
        s["peak_inflight"] = srv.peak_inflight
        s["peak_mem_gb"] = srv.peak_mem / 1e9
        s["iterations"] = [int(r.stats.get("iterations", -1)) for r in reqs]
        if golden:
            errs = []
            for i, r in enumerate(reqs):
                g = golden.get(str(i))
                if g is None or r.u is None:
                    continue
                ref = np.asarray(g["u_samples"])
                us = np.asarray(r.u)[::g["sample_stride"]][:ref.size]
                errs.append(float(np.linalg.norm(us - ref) / np.linalg.norm(ref)))
            s["oracle_checked"] = len(errs)
            s["max_rel_err_vs_oracle"] = max(errs) if errs else None
        for r in reqs:
            r.u = None                                   # results are not kept
        errs = [r.error for r in reqs if r.error]
        if errs:
            s["errors"] = errs[:3]
        if f is None:
            burst_rate = s.get("solves_per_s")
        out["runs"].append(s)
        if progress:
            progress(s)
    return out


def main(argv=None):
    import argparse
    import json
    ap = argparse.ArgumentParser(description="serve a seeded stream of GenEO-PCG solves")
    ap.add_argument("--requests", type=int, default=10)
    ap.add_argument("--seed", type=int, default=4)
    ap.add_argument("--slots", type=int, default=4)
    ap.add_argument("--precision", choices=["fp64", "mixed"], default="mixed")
    ap.add_argument("--rates", default="burst,0.5",
                    help="comma list: 'burst' or a fraction of the burst throughput")
    ap.add_argument("--dof-lo", type=float, default=2e4)
    ap.add_argument("--dof-hi", type=float, default=2e6)
    a = ap.parse_args(argv)
    rates = tuple(None if r == "burst" else float(r) for r in a.rates.split(","))
    res = serve_benchmark(a.requests, a.seed, 1 if a.precision == "mixed" else 0, a.slots,
                          rates, dof_lo=a.dof_lo, dof_hi=a.dof_hi)
    print(json.dumps(res))


if __name__ == "__main__":
    main()
