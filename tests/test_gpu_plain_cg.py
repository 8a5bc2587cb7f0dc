"""Plain CG (GENEO_NO_PRECOND, M = I) against the oracle's unpreconditioned CG.

The comparison leg of the 64x32x24 workload (Sec. 3.1 with no
preconditioner).  On the small blocks the GPU solution matches the oracle's
(1e-6 relative L2 at tol 1e-8) and the iteration count agrees within 2 % + 2
(without a preconditioner CG runs hundreds of steps on these layered blocks,
and the step at which the recursive residual crosses the tolerance moves with
the summation order).  The preconditioner is the identity: z = r exactly.
"""
import numpy as np
import pytest

import workloads
from oracle import solver

from gpu_common import rel, require_gpu

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name", ["tiny", "small", "c1"])
def test_plain_cg_matches_oracle(name):
    pkg = require_gpu()
    p = workloads.config(name)
    ref = solver.solve(p, precond="none", tol=1e-8, maxit=20000)
    s = pkg.GeneoSolver()
    s.assemble(p)
    s.setup(p, pkg.GENEO_FP64, pkg.GENEO_NO_PRECOND)
    r = np.random.default_rng(3).normal(size=s.ndof)
    assert np.array_equal(s.apply_preconditioner(r), r)
    u, st = s.solve(tol=1e-8, max_it=20000)
    s.close()
    assert rel(u, ref["u"]) <= 1e-6
    assert abs(st["iterations"] - ref["iterations"]) <= 0.02 * ref["iterations"] + 2
    assert st["n_coarse"] == 0 and st["flexible"] == 0
    assert st["rel_res_true"] <= 2e-8
