"""The library's condition estimate (stats.kappa_est, host-only) against the
oracle's, on the CPU.

Both take the extreme eigenvalues of the CG Lanczos tridiagonal; the library
by Sturm bisection, the oracle with LAPACK's tridiagonal eigensolver.  On the
coefficients of the oracle's own PCG runs (GenEO and one-level AS on c1, the
Darcy block) and on seeded random coefficient sequences they agree to 1e-9;
the estimate is 0 without coefficients.
"""
import numpy as np
import pytest

import paper_1901_05188_gb300 as pkg
import workloads
from oracle import krylov, solver


def _oracle_run(p, pre):
    st = solver.setup(p, pre)
    _, it = krylov.pcg(st["A"], st["b"], st["M"], tol=1e-8, maxit=2000)
    return np.array(it["alphas"]), np.array(it["betas"])


@pytest.mark.parametrize("case", [("c1", "geneo"), ("c1", "as"), ("d-small", "geneo")])
def test_kappa_of_oracle_runs(case):
    name, pre = case
    if name.startswith("d-"):
        from workloads.darcy import darcy_config
        p = darcy_config(name)
    else:
        p = workloads.config(name)
    al, be = _oracle_run(p, pre)
    k = krylov.lanczos_condition(al, be)
    assert pkg.geneo_kappa_from_cg(al, be[: len(al) - 1]) == pytest.approx(k, rel=1e-9)


def test_kappa_of_random_sequences():
    rng = np.random.default_rng(17)
    for k in (1, 2, 5, 40, 200):
        al = rng.uniform(0.05, 2.0, size=k)
        be = rng.uniform(0.0, 0.9, size=max(k - 1, 0))
        want = krylov.lanczos_condition(al, be)
        assert pkg.geneo_kappa_from_cg(al, be) == pytest.approx(want, rel=1e-9), k


def test_kappa_without_coefficients():
    assert pkg.geneo_kappa_from_cg([], []) == 0.0


def test_too_few_betas_is_refused():
    with pytest.raises(ValueError):
        pkg.geneo_kappa_from_cg([1.0, 2.0, 3.0], [0.5])
