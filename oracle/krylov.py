"""Additive Schwarz preconditioners and Krylov iterations (Sec. 3.1).

One-level AS (eqn:onelevelAS):  M1^-1 = sum_j R_j^T D_j A_j^-1 R_j with
A_j = R_j A R_j^T on V_{h,0}(Omega_j) and D_j = I (the paper's operator) or
D_j = X_j (PoU-weighted variant; not symmetric, so only with flexible CG).
Two-level AS (Sec. 3.1):  M2^-1 = R_H^T A_H^-1 R_H + M1^-1.  The coarse
problem is solved directly (Cholesky of A_H) or, as the paper does when the
coarse space is too large for a direct solve (Sec. 3.3.3), by preconditioned
CG to a relative tolerance; that solve is inexact, so the preconditioner
varies from one application to the next and the outer iteration must be
flexible.  The paper preconditions the coarse CG with BoomerAMG; here a
block-Jacobi preconditioner over the subdomain blocks Z_j^T A Z_j of A_H
(factored exactly) stands in for it.

CG (Sec. 3.1, Hestenes-Stiefel) from x0 = 0, stopped when the recursive
residual satisfies ||r_k|| <= tol ||b||.  The flexible variant (needed when
the preconditioner is not a fixed symmetric operator, Sec. 3.3.3 end) is
Notay's FCG(1): the new direction is A-orthogonalised against the previous
one only.  Condition estimates come from the Lanczos tridiagonal matrix
built from the CG coefficients (Tables 1-2 report such estimates).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse.linalg as spla


class OneLevelAS:
    def __init__(self, A, subs, weight="none"):
        self.subs = subs
        self.solvers = []
        self.weights = []
        for s in subs:
            Aj = A[s.int_dofs][:, s.int_dofs].tocsc()
            self.solvers.append(spla.splu(Aj))
            if weight == "none":
                self.weights.append(None)
            else:
                pos = np.searchsorted(s.neu_dofs, s.int_dofs)
                self.weights.append(s.X[pos])

    def __call__(self, r):
        z = np.zeros_like(r)
        for s, lu, w in zip(self.subs, self.solvers, self.weights):
            y = lu.solve(r[s.int_dofs])
            if w is not None:
                y = w * y
            z[s.int_dofs] += y
        return z


class TwoLevelAS:
    """Two-level AS.  coarse = "direct" (Cholesky of A_H) or "cg" (block-Jacobi
    preconditioned CG on A_H from y = 0, stopped at ||w - A_H y|| <= coarse_tol ||w||
    or after coarse_maxit iterations; blocks = the coarse columns of each
    subdomain, `block_sizes` in order)."""

    def __init__(self, A, subs, Z, one_level_weight="none", coarse="direct", coarse_tol=1e-2,
                 coarse_maxit=200, block_sizes=None):
        self.one = OneLevelAS(A, subs, one_level_weight)
        self.Z = Z
        self.nH = Z.shape[1]
        self.mode = coarse
        self.coarse_tol = coarse_tol
        self.coarse_maxit = coarse_maxit
        self.inner_iterations = []
        if self.nH:
            AH = (Z.T @ (A @ Z)).toarray()
            self.AH = AH
            if coarse == "direct":
                self.cho = sla.cho_factor(AH, lower=True)
            elif coarse == "cg":
                sizes = list(block_sizes) if block_sizes is not None else [self.nH]
                if sum(sizes) != self.nH:
                    raise ValueError("block sizes do not cover the coarse space")
                self.blocks = []
                o = 0
                for m in sizes:
                    if m:
                        self.blocks.append((o, m, sla.cho_factor(AH[o:o + m, o:o + m], lower=True)))
                    o += m
            else:
                raise ValueError(coarse)

    def _block_jacobi(self, v):
        z = np.empty_like(v)
        for o, m, c in self.blocks:
            z[o:o + m] = sla.cho_solve(c, v[o:o + m])
        return z

    def coarse_solve(self, w):
        """y ~ A_H^-1 w (exact for "direct", inner PCG for "cg")."""
        if self.mode == "direct":
            return sla.cho_solve(self.cho, w)
        y = np.zeros_like(w)
        r = w.copy()
        wn = np.linalg.norm(w)
        it = 0
        if wn > 0.0:
            z = self._block_jacobi(r)
            p = z.copy()
            rz = r @ z
            while it < self.coarse_maxit and np.linalg.norm(r) > self.coarse_tol * wn:
                q = self.AH @ p
                alpha = rz / (p @ q)
                y += alpha * p
                r -= alpha * q
                it += 1
                z = self._block_jacobi(r)
                rz_new = r @ z
                p = z + (rz_new / rz) * p
                rz = rz_new
        self.inner_iterations.append(it)
        return y

    def coarse(self, r):
        if not self.nH:
            return np.zeros_like(r)
        w = self.Z.T @ r
        return self.Z @ self.coarse_solve(w)

    def __call__(self, r):
        return self.one(r) + self.coarse(r)


def pcg(A, b, M=None, tol=1e-8, maxit=1000, flexible=False):
    """(Flexible) preconditioned CG from x0 = 0 (Sec. 3.1).

    Returns x, dict(iterations, rel_res, true_rel_res, alphas, betas, history).
    iterations = number of products A p_k performed.
    """
    if M is None:
        M = lambda v: v.copy()
    x = np.zeros_like(b)
    r = b.copy()
    bn = np.linalg.norm(b)
    hist = [1.0]
    if bn == 0.0:
        return x, dict(iterations=0, rel_res=0.0, true_rel_res=0.0,
                       alphas=[], betas=[], history=hist)
    z = M(r)
    p = z.copy()
    rz = r @ z
    alphas, betas = [], []
    it = 0
    rel = 1.0
    while it < maxit:
        q = A @ p
        pq = p @ q
        if not pq > 0.0:
            raise FloatingPointError("CG breakdown: p^T A p <= 0")
        alpha = rz / pq
        x += alpha * p
        r -= alpha * q
        it += 1
        alphas.append(alpha)
        rel = np.linalg.norm(r) / bn
        hist.append(rel)
        if rel <= tol:
            break
        z = M(r)
        rz_new = r @ z
        if flexible:
            beta = -(z @ q) / pq
        else:
            beta = rz_new / rz
        betas.append(beta)
        p = z + beta * p
        rz = rz_new
    true_rel = np.linalg.norm(b - A @ x) / bn
    return x, dict(iterations=it, rel_res=rel, true_rel_res=true_rel,
                   alphas=alphas, betas=betas, history=hist)


def lanczos_condition(alphas, betas):
    """Extreme eigenvalues of the CG Lanczos matrix -> kappa estimate.

    T_kk = 1/alpha_k + beta_{k-1}/alpha_{k-1};  T_{k,k+1} = sqrt(beta_k)/alpha_k.
    """
    k = len(alphas)
    if k == 0:
        return 1.0
    d = np.zeros(k)
    e = np.zeros(max(k - 1, 0))
    for i in range(k):
        d[i] = 1.0 / alphas[i]
        if i > 0:
            d[i] += betas[i - 1] / alphas[i - 1]
        if i < k - 1:
            e[i] = np.sqrt(max(betas[i], 0.0)) / alphas[i]
    ev = sla.eigh_tridiagonal(d, e, eigvals_only=True)
    return float(ev[-1] / ev[0])
