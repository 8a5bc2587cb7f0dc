"""Whole GenEO-PCG pipeline on one problem (Sec. 2 + Sec. 3), FP64.

solve(p) assembles A u = b (eqn:fe_matrix_system), builds the overlapping box
decomposition (Sec. 3.1), the GenEO coarse space (Sec. 3.2-3.3) and runs
(flexible) PCG (Sec. 3.1) to ||r|| <= tol ||b||.
"""
from __future__ import annotations

import time

import numpy as np

from . import decomp, fem, geneo, krylov


def setup(p, precond="geneo", weight="none", eig_method="auto", A=None, b=None,
          coarse="direct", coarse_tol=1e-2):
    t0 = time.perf_counter()
    if A is None:
        A, b = fem.assemble_system(p)
    t1 = time.perf_counter()
    subs = decomp.partition(p)
    info = None
    if precond in ("geneo", "zem"):
        if precond == "geneo":
            Z, info = geneo.coarse_space(p, subs, A, eig_method)
        else:
            Z, info = geneo.zem_space(p, subs, A)
        M = krylov.TwoLevelAS(A, subs, Z, weight, coarse=coarse, coarse_tol=coarse_tol,
                              block_sizes=[d["m"] for d in info])
    elif precond == "as":
        M = krylov.OneLevelAS(A, subs, weight)
    elif precond == "none":
        M = None
    else:
        raise ValueError(precond)
    t2 = time.perf_counter()
    return dict(A=A, b=b, subs=subs, M=M, info=info,
                t_assemble=t1 - t0, t_setup=t2 - t1)


def solve(p, precond="geneo", tol=1e-8, maxit=2000, flexible=None,
          weight="none", eig_method="auto", coarse="direct", coarse_tol=1e-2):
    """Returns dict(u, iterations, rel_res, true_rel_res, kappa, n_coarse, ...).

    coarse="cg" solves the coarse problem by block-Jacobi PCG to coarse_tol
    (an inexact coarse solve: flexible CG outside, Sec. 3.3.3)."""
    st = setup(p, precond, weight, eig_method, coarse=coarse, coarse_tol=coarse_tol)
    if flexible is None:
        flexible = weight != "none" or coarse != "direct"
    t0 = time.perf_counter()
    u, it = krylov.pcg(st["A"], st["b"], st["M"], tol=tol, maxit=maxit,
                       flexible=flexible)
    t1 = time.perf_counter()
    kappa = krylov.lanczos_condition(it["alphas"], it["betas"]) if not flexible else None
    out = dict(u=u, iterations=it["iterations"], rel_res=it["rel_res"],
               true_rel_res=it["true_rel_res"], kappa=kappa,
               history=it["history"], t_assemble=st["t_assemble"],
               t_setup=st["t_setup"], t_solve=t1 - t0, A=st["A"], b=st["b"],
               subs=st["subs"], M=st["M"])
    if st["info"] is not None:
        out["modes"] = [d["m"] for d in st["info"]]
        out["lambdas"] = [d["lam"] for d in st["info"]]
        out["taus"] = [d.get("tau") for d in st["info"]]
        out["n_coarse"] = int(sum(out["modes"]))
        out["eig_info"] = st["info"]
    else:
        out["n_coarse"] = 0
    return out
