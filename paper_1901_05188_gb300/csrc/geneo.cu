// GenEO coarse space on the device (Sec. 3.2, Sec. 3.3.1-3.3.3).
//
// Per subdomain j the generalised eigenproblem (eqm:matrixForm)
//   A_{Omega_j} p = lambda X_j A_{Omega_j^o} X_j p
// is solved with the shift-and-invert transformation the paper uses
// (Sec. 3.3.2): S = A - sigma B = L L^T for a small sigma < 0, and the
// symmetric operator C = L^-1 B L^-T has eigenvalues mu = 1 / (lambda - sigma),
// so the wanted smallest lambda are the largest mu.  Instead of ARPACK's
// implicitly restarted Lanczos, a block Lanczos process (block size 8, full
// re-orthogonalisation, Cholesky-QR) runs batched over all subdomains and the
// projected matrix is diagonalised by a cyclic Jacobi method; p = L^-T y.
#include "geneo.cuh"
#include "fem.cuh"

namespace geneo {

namespace {

__device__ __forceinline__ double *tile_at(double *pool, const BandLayout &L, int I, int d) {
  return pool + L.off + (((long long)I * (L.w + 1) + d) << 10);
}

__device__ __forceinline__ int cand_count(const int *c) {
  int n = 0;
  while (n < kMaxCand && c[n] >= 0) ++n;
  return n;
}

// Partition-of-unity weight X_j at node (gi, gj, gk) of subdomain j's
// interior: 1 / multiplicity (Sec. 3.3.1), or Sarkis's d_j / sum_k d_k with
// d the distance to each interior subdomain's artificial boundary in element
// layers (Sec. 3.2).  The caller zeroes it on global Dirichlet dofs.
__device__ double pou_weight(const SubDesc *subs, int j, int gi, int gj, int gk, const int *cand,
                             int co0, int co1, int co2, int px, int py, int nx, int ny, int nz,
                             int kind) {
  const int *ci = cand + (co0 + gi) * kMaxCand;
  const int *cj = cand + (co1 + gj) * kMaxCand;
  const int *ck = cand + (co2 + gk) * kMaxCand;
  const int nci = cand_count(ci), ncj = cand_count(cj), nck = cand_count(ck);
  if (kind == 0) return 1.0 / double(nci * ncj * nck);
  int sum = 0;
  for (int c = 0; c < nck; ++c)
    for (int b = 0; b < ncj; ++b)
      for (int a = 0; a < nci; ++a)
        sum += artificial_distance(subs[ci[a] + px * (cj[b] + py * ck[c])], gi, gj, gk, nx, ny, nz);
  return double(artificial_distance(subs[j], gi, gj, gk, nx, ny, nz)) / double(sum);
}

__global__ void k_pou_neumann(const SubDesc *subs, const int *cand, int co0, int co1, int co2,
                              const uint8_t *mask, int nnx, int nny, int nnz, int px, int py,
                              int kind, double *Xneu) {
  const int j = blockIdx.y;
  const SubDesc &S = subs[j];
  const int nc = S.nc;
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nc * S.nbox.count()) return;
  int l = t / nc, comp = t - nc * l;
  int gi, gj, gk;
  S.nbox.global(l, gi, gj, gk);
  double x = 0.0;
  if (S.ibox.local(gi, gj, gk) >= 0) {
    x = pou_weight(subs, j, gi, gj, gk, cand, co0, co1, co2, px, py, nnx - 1, nny - 1, nnz - 1,
                   kind);
    if (mask[nc * (gi + nnx * (gj + nny * gk)) + comp]) x = 0.0;
  }
  Xneu[S.x_neu + t] = x;
}

// The same weights on the interior dofs, laid out like the local solutions
// (offset v_int): the one-level weight D_j = X_j of the gather.
__global__ void k_pou_interior(const SubDesc *subs, const int *cand, int co0, int co1, int co2,
                               const uint8_t *mask, int nnx, int nny, int nnz, int px, int py,
                               int kind, double *wloc) {
  const int j = blockIdx.y;
  const SubDesc &S = subs[j];
  const int nc = S.nc;
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nc * S.ibox.count()) return;
  int l = t / nc, comp = t - nc * l;
  int gi, gj, gk;
  S.ibox.global(l, gi, gj, gk);
  double x = pou_weight(subs, j, gi, gj, gk, cand, co0, co1, co2, px, py, nnx - 1, nny - 1,
                        nnz - 1, kind);
  if (mask[nc * (gi + nnx * (gj + nny * gk)) + comp]) x = 0.0;
  wloc[S.v_int + t] = x;
}

__global__ void __launch_bounds__(128)
    k_neumann_assemble(const SubDesc *subs, const BandLayout *lay, int nx, int ny, int nz,
                       const double *__restrict__ X, const double *__restrict__ Y,
                       const double *__restrict__ Z, const double *__restrict__ Cel,
                       const double *__restrict__ perm,
                       const int *__restrict__ ecnt, int eo0, int eo1, int eo2,
                       const uint8_t *__restrict__ mask, const double *__restrict__ Xneu,
                       double sigma, double *poolS, double *Bloc) {
  const int j = blockIdx.y;
  const SubDesc &S = subs[j];
  const int nn = S.nbox.count();
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)nn * 27) return;
  const int l = (int)(t / 27), s = (int)(t % 27);
  int gi, gj, gk;
  S.nbox.global(l, gi, gj, gk);
  const int i2 = gi + s % 3 - 1, j2 = gj + (s / 3) % 3 - 1, k2 = gk + s / 9 - 1;
  const int l2 = S.nbox.local(i2, j2, k2);
  const int nc = S.nc, nc2 = nc * nc;
  double *bl = Bloc + (S.b_neu + (long long)l * 27 + s) * nc2;
  if (l2 < 0) {
    for (int q = 0; q < nc2; ++q) bl[q] = 0.0;
    return;
  }
  double KA[9], KO[9];
  for (int q = 0; q < 9; ++q) KA[q] = KO[q] = 0.0;
  for (int ez = max(max(gk, k2) - 1, S.elo[2]); ez <= min(min(gk, k2), S.ehi[2] - 1); ++ez)
    for (int ey = max(max(gj, j2) - 1, S.elo[1]); ey <= min(min(gj, j2), S.ehi[1] - 1); ++ey)
      for (int ex = max(max(gi, i2) - 1, S.elo[0]); ex <= min(min(gi, i2), S.ehi[0] - 1); ++ex) {
        int e = ex + nx * (ey + ny * ez);
        int a = (gi - ex) + 2 * (gj - ey) + 4 * (gk - ez);
        int b = (i2 - ex) + 2 * (j2 - ey) + 4 * (k2 - ez);
        double Kb[9];
        if (nc == 3)
          element_block(Cel + 36 * (size_t)e, X[ex + 1] - X[ex], Y[ey + 1] - Y[ey],
                        Z[ez + 1] - Z[ez], a, b, Kb);
        else
          Kb[0] = darcy_entry(perm + 3 * (size_t)e, X[ex + 1] - X[ex], Y[ey + 1] - Y[ey],
                              Z[ez + 1] - Z[ez], a, b);
        bool ov = ecnt[eo0 + ex] * ecnt[eo1 + ey] * ecnt[eo2 + ez] >= 2;
        for (int q = 0; q < nc2; ++q) {
          KA[q] += Kb[q];
          if (ov) KO[q] += Kb[q];
        }
      }
  const int nnx = nx + 1, nny = ny + 1;
  const int g = gi + nnx * (gj + nny * gk), g2 = i2 + nnx * (j2 + nny * k2);
  const BandLayout L = lay[j];
  for (int r = 0; r < nc; ++r)
    for (int c = 0; c < nc; ++c) {
      int rd = nc * g + r, cd = nc * g2 + c;
      double a = KA[nc * r + c], o = KO[nc * r + c];
      if (mask[rd] || mask[cd]) {
        a = (rd == cd) ? 1.0 : 0.0;
        o = 0.0;
      }
      double bv = Xneu[S.x_neu + nc * l + r] * o * Xneu[S.x_neu + nc * l2 + c];
      bl[nc * r + c] = bv;
      int R = nc * l + r, C = nc * l2 + c;
      if (R >= C) tile_at(poolS, L, R >> 5, (R >> 5) - (C >> 5))[(C & 31) * 32 + (R & 31)] = a - sigma * bv;
    }
}

__global__ void k_bloc_mv(const SubDesc *subs, const double *__restrict__ Bloc,
                          const double *__restrict__ T, double *__restrict__ W,
                          long long stride, int p) {
  const int j = blockIdx.y;
  const SubDesc &S = subs[j];
  const int nc = S.nc;
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nc * S.nbox.count()) return;
  int l = t / nc, r = t - nc * l;
  int gi, gj, gk;
  S.nbox.global(l, gi, gj, gk);
  double acc[kLanczosBlock];
#pragma unroll
  for (int q = 0; q < kLanczosBlock; ++q) acc[q] = 0.0;
  const double *Tj = T + j * stride;
  for (int s = 0; s < 27; ++s) {
    int l2 = S.nbox.local(gi + s % 3 - 1, gj + (s / 3) % 3 - 1, gk + s / 9 - 1);
    if (l2 < 0) continue;
    const double *bl = Bloc + (S.b_neu + (long long)l * 27 + s) * (nc * nc) + nc * r;
    for (int c = 0; c < nc; ++c) {
      double bv = bl[c];
      if (bv == 0.0) continue;
      const double *tr = Tj + (long long)(nc * l2 + c) * p;
#pragma unroll
      for (int q = 0; q < kLanczosBlock; ++q)
        if (q < p) acc[q] += bv * tr[q];
    }
  }
  double *wr = W + j * stride + (long long)t * p;
#pragma unroll
  for (int q = 0; q < kLanczosBlock; ++q)
    if (q < p) wr[q] = acc[q];
}

__device__ __forceinline__ unsigned long long splitmix64(unsigned long long x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

__global__ void k_random_block(const SubDesc *subs, int npad, double *V, int ld, long long stride,
                               int p, unsigned long long seed) {
  const int j = blockIdx.y;
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= npad * p) return;
  int row = t / p, c = t - row * p;
  double v = 0.0;
  if (row < subs[j].n_neu) {
    unsigned long long h = splitmix64(seed ^ splitmix64(((unsigned long long)j << 40) ^
                                                        ((unsigned long long)row << 8) ^ c));
    v = double(h >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0;
  }
  V[j * stride + (long long)row * ld + c] = v;
}

// partial dot products over a chunk of rows, staged 16 rows at a time
__global__ void __launch_bounds__(256)
    k_tsdots(const SubDesc *subs, const double *__restrict__ A, int lda, long long sa, int na,
             const double *__restrict__ B, int ldb, long long sb, int nb, double *Hpart,
             int chunks, const int *gate) {
  const int j = blockIdx.y, ch = blockIdx.x;
  if (gate && !gate[j]) return;                       // the reduction writes zeros
  const int n = subs[j].n_neu;
  const int per = (n + chunks - 1) / chunks;
  const int r0 = ch * per, r1 = min(n, r0 + per);
  const int nout = na * nb;
  extern __shared__ __align__(16) unsigned char smraw[];
  double *sA = reinterpret_cast<double *>(smraw);     // [16][na]
  double *sB = sA + 16 * na;                          // [16][nb]
  double acc[5] = {0, 0, 0, 0, 0};
  const double *Aj = A + j * sa;
  const double *Bj = B + j * sb;
  for (int rb = r0; rb < r1; rb += 16) {
    int nr = min(16, r1 - rb);
    for (int e = threadIdx.x; e < 16 * na; e += 256) {
      int rr = e / na, c = e - rr * na;
      sA[e] = rr < nr ? Aj[(long long)(rb + rr) * lda + c] : 0.0;
    }
    for (int e = threadIdx.x; e < 16 * nb; e += 256) {
      int rr = e / nb, c = e - rr * nb;
      sB[e] = rr < nr ? Bj[(long long)(rb + rr) * ldb + c] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      int o = threadIdx.x + 256 * q;
      if (o < nout) {
        int a = o / nb, b = o - a * nb;
        double s = 0.0;
        for (int rr = 0; rr < 16; ++rr) s += sA[rr * na + a] * sB[rr * nb + b];
        acc[q] += s;
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    int o = threadIdx.x + 256 * q;
    if (o < nout) Hpart[((long long)j * chunks + ch) * nout + o] = acc[q];
  }
}

__global__ void k_tsdots_reduce(const double *Hpart, int chunks, int nout, double *H, long long hs,
                                const int *gate) {
  const int j = blockIdx.x;
  const bool skip = gate && !gate[j];
  for (int o = threadIdx.x; o < nout; o += blockDim.x) {
    double s = 0.0;
    if (!skip)
      for (int ch = 0; ch < chunks; ++ch) s += Hpart[((long long)j * chunks + ch) * nout + o];
    H[j * hs + o] = s;
  }
}

// Second re-orthogonalisation pass needed?  After one projection W -= V H,
// column b of W has squared norm G_bb and lost sum_a H_ab^2; the pass is
// repeated where more than half of the column's squared norm was removed,
// G_bb < sum_a H_ab^2 (the criterion of Daniel, Gragg, Kaufman and Stewart with
// eta = 1/sqrt(2): "twice is enough").
__global__ void k_reorth_gate(const double *G, int p, const double *H, int na, long long hs,
                              int *gate) {
  const int j = blockIdx.x;
  __shared__ int need;
  if (threadIdx.x == 0) need = 0;
  __syncthreads();
  if (threadIdx.x < p) {
    const int b = threadIdx.x;
    double lost = 0.0;
    for (int a = 0; a < na; ++a) {
      const double h = H[j * hs + (long long)a * p + b];
      lost += h * h;
    }
    if (!(G[(long long)j * p * p + b * p + b] >= lost)) atomicOr(&need, 1);
  }
  __syncthreads();
  if (threadIdx.x == 0) gate[j] = need;
}

__global__ void __launch_bounds__(256)
    k_tsgemm(const SubDesc *subs, int npad, const double *__restrict__ A, int lda, long long sa,
             int na, const double *__restrict__ H, int ldh, long long hs, double *C, int ldc,
             long long sc, int nb, double alpha, double beta, const int *gate) {
  const int j = blockIdx.y;
  if (gate && !gate[j]) return;
  extern __shared__ __align__(16) unsigned char smraw[];
  double *sH = reinterpret_cast<double *>(smraw);   // [na][nb]
  for (int e = threadIdx.x; e < na * nb; e += blockDim.x) {
    int a = e / nb, b = e - a * nb;
    sH[e] = H[j * hs + (long long)a * ldh + b];
  }
  __syncthreads();
  const int n = subs[j].n_neu;
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)npad * nb) return;
  int row = (int)(t / nb), b = (int)(t - (long long)row * nb);
  double *cp = C + j * sc + (long long)row * ldc + b;
  if (row >= n) {
    if (beta == 0.0) *cp = 0.0;
    return;
  }
  const double *ar = A + j * sa + (long long)row * lda;
  double s = 0.0;
  for (int a = 0; a < na; ++a) s += ar[a] * sH[a * nb + b];
  *cp = (beta == 0.0 ? 0.0 : beta * *cp) + alpha * s;
}

// Cholesky of the p x p Gram matrix, inverse, and Racc update (one block per subdomain)
__global__ void k_cholqr_small(const double *G, int p, double *Rinv, double *Racc, int first,
                               double abs_tiny) {
  const int j = blockIdx.x;
  __shared__ double R[kLanczosBlock][kLanczosBlock];
  __shared__ double Ri[kLanczosBlock][kLanczosBlock];
  __shared__ double Ra[kLanczosBlock][kLanczosBlock];
  if (threadIdx.x == 0) {
    const double *g = G + (long long)j * p * p;
    for (int a = 0; a < p; ++a)
      for (int b = 0; b < p; ++b) R[a][b] = 0.0;
    // upper factor R with G = R^T R; dead columns get R[k][k] = 0
    for (int k = 0; k < p; ++k) {
      double d = g[k * p + k];
      for (int i = 0; i < k; ++i) d -= R[i][k] * R[i][k];
      // numerically dependent (angle to the block's span below 1e-7) or
      // negligible against the operator scale: deflate the column
      bool dead = !(d > 1e-14 * g[k * p + k]) || !(d > abs_tiny);
      double rk = dead ? 0.0 : sqrt(d);
      R[k][k] = rk;
      for (int c = k + 1; c < p; ++c) {
        double v = g[k * p + c];
        for (int i = 0; i < k; ++i) v -= R[i][k] * R[i][c];
        R[k][c] = dead ? 0.0 : v / rk;
      }
    }
    // Rinv (upper); a dead column maps to zero
    for (int c = 0; c < p; ++c) {
      for (int a = p - 1; a >= 0; --a) {
        if (a > c) {
          Ri[a][c] = 0.0;
          continue;
        }
        if (R[a][a] == 0.0) {
          Ri[a][c] = 0.0;
          continue;
        }
        double s = (a == c) ? 1.0 : 0.0;
        for (int k = a + 1; k <= c; ++k) s -= R[a][k] * Ri[k][c];
        Ri[a][c] = s / R[a][a];
      }
    }
    double *racc = Racc + (long long)j * p * p;
    for (int a = 0; a < p; ++a)
      for (int b = 0; b < p; ++b) {
        double s;
        if (first) {
          s = R[a][b];
        } else {
          s = 0.0;
          for (int k = 0; k < p; ++k) s += R[a][k] * racc[k * p + b];
        }
        Ra[a][b] = s;
      }
    for (int a = 0; a < p; ++a)
      for (int b = 0; b < p; ++b) {
        racc[a * p + b] = Ra[a][b];
        Rinv[(long long)j * p * p + a * p + b] = Ri[a][b];
      }
  }
}

__global__ void k_rowmul(const SubDesc *subs, int npad, double *W, int p, const double *Rinv) {
  const int j = blockIdx.y;
  int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= npad) return;
  double *w = W + ((long long)j * npad + row) * p;
  const double *ri = Rinv + (long long)j * p * p;
  double in[kLanczosBlock];
  for (int q = 0; q < p; ++q) in[q] = w[q];
  for (int b = 0; b < p; ++b) {
    double s = 0.0;
    for (int a = 0; a <= b; ++a) s += in[a] * ri[a * p + b];
    w[b] = row < subs[j].n_neu ? s : 0.0;
  }
}

__global__ void k_hm_accum(double *Hm, int kdim, const double *Hs, int rows, int k, int p) {
  const int j = blockIdx.x;
  for (int e = threadIdx.x; e < rows * p; e += blockDim.x) {
    int r = e / p, b = e - r * p;
    Hm[(long long)j * kdim * kdim + (long long)r * kdim + k * p + b] +=
        Hs[(long long)j * rows * p + e];
  }
}

__global__ void k_hm_subdiag(double *Hm, int kdim, const double *Racc, int k, int p,
                             double *Rblk) {
  const int j = blockIdx.x;
  for (int e = threadIdx.x; e < p * p; e += blockDim.x) {
    int a = e / p, b = e - a * p;
    double v = Racc[(long long)j * p * p + e];
    if ((k + 1) * p < kdim)
      Hm[(long long)j * kdim * kdim + (long long)((k + 1) * p + a) * kdim + k * p + b] = v;
    else
      Rblk[(long long)j * p * p + e] = v;
  }
}

__global__ void k_restart_hm(double *Hm, int kdim, const double *Eval, const double *Evec,
                             const double *Rblk, int kk, int p) {
  const int j = blockIdx.x;
  double *H = Hm + (long long)j * kdim * kdim;
  const double *S = Evec + (long long)j * kdim * kdim;
  const double *R = Rblk + (long long)j * p * p;
  for (int e = threadIdx.x; e < kdim * kdim; e += blockDim.x) {
    int r = e / kdim, c = e - r * kdim;
    double v = 0.0;
    if (r < kk && c < kk) {
      v = (r == c) ? Eval[(long long)j * kdim + r] : 0.0;
    } else if (r >= kk && r < kk + p && c < kk) {
      int a = r - kk;
      for (int b = 0; b < p; ++b) v += R[a * p + b] * S[(long long)(kdim - p + b) * kdim + c];
    }
    H[e] = v;
  }
}

__global__ void k_copy_block(const SubDesc *subs, int npad, const double *W, int ldw,
                             long long sw, double *V, int ldv, long long sv, int p) {
  const int j = blockIdx.y;
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= npad * p) return;
  int row = t / p, b = t - row * p;
  V[j * sv + (long long)row * ldv + b] = W[j * sw + (long long)row * ldw + b];
}

// Ritz pairs of the symmetrised projected matrix H (n x n, n <= kMaxKdim):
// Householder reduction to tridiagonal form (H = Q T Q^T), the nw largest
// eigenvalues of T by Sturm-sequence bisection, their eigenvectors by inverse
// iteration (re-orthogonalised inside clusters of close eigenvalues), and the
// back-transformation y = Q x.  One block per subdomain; eigenvalues are
// returned in descending order, columns nw..n-1 of Evec are zero.
constexpr int kMaxKdim = 128;

__device__ __forceinline__ int sturm_count(const double *d, const double *e2, int n, double x,
                                           double pivmin) {
  // number of eigenvalues of T smaller than x
  int cnt = 0;
  double q = d[0] - x;
  if (fabs(q) < pivmin) q = -pivmin;
  if (q < 0) ++cnt;
  for (int i = 1; i < n; ++i) {
    q = d[i] - x - e2[i - 1] / q;
    if (fabs(q) < pivmin) q = -pivmin;
    if (q < 0) ++cnt;
  }
  return cnt;
}

__global__ void __launch_bounds__(256)
    k_ritz_eig(const double *Hm, int n, int nw, int p, const double *Rblk, double *Eval,
               double *Evec, double *Eres) {
  const int j = blockIdx.x;
  const int ld = n + 1;
  extern __shared__ __align__(16) unsigned char smraw[];
  double *A = reinterpret_cast<double *>(smraw);   // n x ld, Householder vectors below diagonal
  double *d = A + n * ld;                          // diagonal of T
  double *e = d + n;                               // off-diagonal of T
  double *e2 = e + n;                              // squares
  double *lam = e2 + n;                            // wanted eigenvalues (descending)
  double *vs = lam + n;                            // current Householder vector / work
  double *ps = vs + n;                             // A v / q
  __shared__ double red[8];
  __shared__ double bounds[2];
  const double *H = Hm + (long long)j * n * n;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int t = tid; t < n * n; t += blockDim.x) {
    int r = t / n, c = t - r * n;
    A[r * ld + c] = 0.5 * (H[t] + H[c * n + r]);
  }
  __syncthreads();
  // ---- Householder tridiagonalisation (lower)
  for (int k = 0; k + 2 < n; ++k) {
    const int m = n - k - 1;
    double s2 = 0.0;
    for (int i = tid; i < m; i += blockDim.x) {
      double x = A[(k + 1 + i) * ld + k];
      s2 += x * x;
    }
    s2 = warp_sum(s2);
    if (lane == 0) red[warp] = s2;
    __syncthreads();
    if (tid == 0) {
      double t = 0.0;
      for (int w = 0; w < 8; ++w) t += red[w];
      double x0 = A[(k + 1) * ld + k];
      double nrm = sqrt(t);
      double alpha = (x0 >= 0.0) ? -nrm : nrm;
      double vnorm2 = t - x0 * x0 + (x0 - alpha) * (x0 - alpha);
      d[k] = A[k * ld + k];
      if (nrm == 0.0 || vnorm2 <= 0.0) {
        e[k] = 0.0;
        red[0] = 0.0;           // no reflection
      } else {
        e[k] = alpha;
        red[0] = 1.0 / sqrt(vnorm2);
        red[1] = alpha;
      }
    }
    __syncthreads();
    const double inv = red[0];
    if (inv == 0.0) {
      for (int i = tid; i < m; i += blockDim.x) A[(k + 1 + i) * ld + k] = 0.0;
      __syncthreads();
      continue;
    }
    const double alpha = red[1];
    for (int i = tid; i < m; i += blockDim.x) {
      double v = A[(k + 1 + i) * ld + k] - (i == 0 ? alpha : 0.0);
      v *= inv;
      vs[i] = v;
      A[(k + 1 + i) * ld + k] = v;       // keep v for the back-transformation
    }
    __syncthreads();
    // p = A_sub v
    for (int i = tid; i < m; i += blockDim.x) {
      const double *row = A + (k + 1 + i) * ld + (k + 1);
      double s = 0.0;
      for (int c = 0; c < m; ++c) s += row[c] * vs[c];
      ps[i] = s;
    }
    __syncthreads();
    double b = 0.0;
    for (int i = tid; i < m; i += blockDim.x) b += vs[i] * ps[i];
    b = warp_sum(b);
    if (lane == 0) red[warp] = b;
    __syncthreads();
    double beta = 0.0;
    for (int w = 0; w < 8; ++w) beta += red[w];
    __syncthreads();
    for (int i = tid; i < m; i += blockDim.x) ps[i] = 2.0 * ps[i] - 2.0 * beta * vs[i];
    __syncthreads();
    // A_sub -= v q^T + q v^T
    for (int t = tid; t < m * m; t += blockDim.x) {
      int r = t / m, c = t - r * m;
      A[(k + 1 + r) * ld + (k + 1 + c)] -= vs[r] * ps[c] + ps[r] * vs[c];
    }
    __syncthreads();
  }
  if (tid == 0) {
    if (n >= 2) {
      d[n - 2] = A[(n - 2) * ld + (n - 2)];
      e[n - 2] = A[(n - 1) * ld + (n - 2)];
    }
    d[n - 1] = A[(n - 1) * ld + (n - 1)];
    e[n - 1] = 0.0;
    double lo = 1e300, hi = -1e300, mx = 0.0;
    for (int i = 0; i < n; ++i) {
      double r = (i > 0 ? fabs(e[i - 1]) : 0.0) + fabs(e[i]);
      lo = fmin(lo, d[i] - r);
      hi = fmax(hi, d[i] + r);
      mx = fmax(mx, fabs(d[i]) + r);
    }
    bounds[0] = lo - 1e-12 * mx - 1e-300;
    bounds[1] = hi + 1e-12 * mx + 1e-300;
    red[0] = mx;
  }
  __syncthreads();
  for (int i = tid; i < n; i += blockDim.x) e2[i] = e[i] * e[i];
  __syncthreads();
  const double tnorm = red[0];
  const double pivmin = fmax(1e-290, 1e-30 * tnorm * tnorm) / fmax(tnorm, 1e-300);
  // ---- bisection: thread q finds the q-th largest eigenvalue
  for (int q = tid; q < nw; q += blockDim.x) {
    const int target = n - 1 - q;          // index from the bottom
    double a = bounds[0], bnd = bounds[1];
    for (int it = 0; it < 200; ++it) {
      double mid = 0.5 * (a + bnd);
      if (sturm_count(d, e2, n, mid, pivmin) > target) bnd = mid;
      else a = mid;
      if (bnd - a <= 2.2e-16 * (fabs(a) + fabs(bnd)) + 1e-300) break;
    }
    lam[q] = 0.5 * (a + bnd);
  }
  __syncthreads();
  // ---- inverse iteration on T - lam I (partial pivoting), vectors to Evec columns
  double *Ev = Evec + (long long)j * n * n;
  for (int q = tid; q < nw; q += blockDim.x) {
    double u0[kMaxKdim], u1[kMaxKdim], u2[kMaxKdim], lm[kMaxKdim], x[kMaxKdim];
    unsigned char piv[kMaxKdim];
    const double lq = lam[q];
    const double tiny = 1e-15 * fmax(tnorm, 1e-300);
    for (int i = 0; i < n; ++i) {
      u0[i] = d[i] - lq;
      u1[i] = (i + 1 < n) ? e[i] : 0.0;
      u2[i] = 0.0;
    }
    for (int i = 0; i + 1 < n; ++i) {
      double sub = e[i];
      if (fabs(u0[i]) >= fabs(sub)) {
        piv[i] = 0;
        if (fabs(u0[i]) < tiny) u0[i] = (u0[i] >= 0 ? tiny : -tiny);
        lm[i] = sub / u0[i];
        u0[i + 1] -= lm[i] * u1[i];
      } else {
        piv[i] = 1;
        lm[i] = u0[i] / sub;
        double t0 = u0[i + 1], t1 = (i + 2 < n) ? u1[i + 1] : 0.0;
        u0[i] = sub;
        double n11 = u1[i] - lm[i] * t0;
        double n12 = -lm[i] * t1;
        u1[i] = t0;
        u2[i] = t1;
        u0[i + 1] = n11;
        if (i + 2 < n) u1[i + 1] = n12;
      }
    }
    if (fabs(u0[n - 1]) < tiny) u0[n - 1] = (u0[n - 1] >= 0 ? tiny : -tiny);
    // deterministic start vector
    unsigned long long h = 0x9E3779B97F4A7C15ull * (unsigned long long)(q + 1) ^ (unsigned long long)j;
    for (int i = 0; i < n; ++i) {
      h = splitmix64(h + i);
      x[i] = double(h >> 11) * (1.0 / 9007199254740992.0) - 0.5;
    }
    for (int it = 0; it < 3; ++it) {
      for (int i = 0; i + 1 < n; ++i) {
        if (piv[i]) {
          double t = x[i];
          x[i] = x[i + 1];
          x[i + 1] = t;
        }
        x[i + 1] -= lm[i] * x[i];
      }
      x[n - 1] /= u0[n - 1];
      if (n >= 2) x[n - 2] = (x[n - 2] - u1[n - 2] * x[n - 1]) / u0[n - 2];
      for (int i = n - 3; i >= 0; --i) x[i] = (x[i] - u1[i] * x[i + 1] - u2[i] * x[i + 2]) / u0[i];
      double s = 0.0;
      for (int i = 0; i < n; ++i) s += x[i] * x[i];
      s = 1.0 / sqrt(s);
      for (int i = 0; i < n; ++i) x[i] *= s;
    }
    for (int i = 0; i < n; ++i) Ev[(long long)i * n + q] = x[i];
  }
  for (int t = tid; t < n * n; t += blockDim.x) {
    int c = t - (t / n) * n;
    if (c >= nw) Ev[t] = 0.0;
  }
  __syncthreads();
  // ---- re-orthogonalise inside clusters of close eigenvalues (warp 0, in order)
  if (warp == 0) {
    const double ctol = 1e-7 * fmax(fabs(lam[0]), 1e-300);
    int c0 = 0;
    for (int q = 1; q < nw; ++q) {
      if (fabs(lam[q] - lam[q - 1]) > ctol) {
        c0 = q;
        continue;
      }
      for (int pass = 0; pass < 2; ++pass) {
        for (int r = c0; r < q; ++r) {
          double s = 0.0;
          for (int i = lane; i < n; i += 32) s += Ev[(long long)i * n + r] * Ev[(long long)i * n + q];
          s = warp_sum(s);
          for (int i = lane; i < n; i += 32) Ev[(long long)i * n + q] -= s * Ev[(long long)i * n + r];
          __syncwarp();
        }
        double s = 0.0;
        for (int i = lane; i < n; i += 32) s += Ev[(long long)i * n + q] * Ev[(long long)i * n + q];
        s = warp_sum(s);
        s = s > 0.0 ? 1.0 / sqrt(s) : 0.0;
        for (int i = lane; i < n; i += 32) Ev[(long long)i * n + q] *= s;
        __syncwarp();
      }
    }
  }
  __syncthreads();
  // ---- back-transformation y = H_0 H_1 ... H_{n-3} x (thread q owns column q)
  for (int q = tid; q < nw; q += blockDim.x) {
    double x[kMaxKdim];
    for (int i = 0; i < n; ++i) x[i] = Ev[(long long)i * n + q];
    for (int k = n - 3; k >= 0; --k) {
      double s = 0.0;
      for (int i = k + 1; i < n; ++i) s += A[i * ld + k] * x[i];
      s *= 2.0;
      for (int i = k + 1; i < n; ++i) x[i] -= s * A[i * ld + k];
    }
    for (int i = 0; i < n; ++i) Ev[(long long)i * n + q] = x[i];
    Eval[(long long)j * n + q] = lam[q];
    // residual estimate || R_s y[n-p .. n-1] ||
    const double *Rb = Rblk + (long long)j * p * p;
    double r2 = 0.0;
    for (int a = 0; a < p; ++a) {
      double v = 0.0;
      for (int b = 0; b < p; ++b) v += Rb[a * p + b] * x[n - p + b];
      r2 += v * v;
    }
    Eres[(long long)j * n + q] = sqrt(r2);
  }
  for (int q = nw + tid; q < n; q += blockDim.x) {
    Eval[(long long)j * n + q] = 0.0;
    Eres[(long long)j * n + q] = 0.0;
  }
}

__global__ void k_build_Z(const SubDesc *subs, const double *P, int ldp, long long sp,
                          const double *Xneu, double *Zp) {
  const int j = blockIdx.y;
  const SubDesc &S = subs[j];
  if (S.m == 0) return;
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)S.n_int * S.m) return;
  int row = (int)(t / S.m), k = (int)(t - (long long)row * S.m);
  const int nc = S.nc;
  int node = row / nc, comp = row - nc * node;
  int gi, gj, gk;
  S.ibox.global(node, gi, gj, gk);
  int ln = S.nbox.local(gi, gj, gk);
  int nd = nc * ln + comp;
  Zp[S.z_off + t] = Xneu[S.x_neu + nd] * P[j * sp + (long long)nd * ldp + k];
}

__global__ void k_AZ(const SubDesc *subs, int nnx, int nny, int nnz, const int32_t *__restrict__ rp,
                     const int32_t *__restrict__ col, const double *__restrict__ val,
                     const double *__restrict__ Zp, const long long *yoff, double *Yp) {
  const int j = blockIdx.y;
  const SubDesc &S = subs[j];
  const int m = S.m;
  if (m == 0) return;
  const int nc = S.nc;
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nc * S.nbox.count()) return;
  int l = t / nc, r = t - nc * l;
  int gi, gj, gk;
  S.nbox.global(l, gi, gj, gk);
  int g = gi + nnx * (gj + nny * gk);
  double acc[kMaxModes];
#pragma unroll
  for (int q = 0; q < kMaxModes; ++q) acc[q] = 0.0;
  for (int pidx = rp[g]; pidx < rp[g + 1]; ++pidx) {
    int g2 = col[pidx];
    int i2 = g2 % nnx, rr = g2 / nnx, j2 = rr % nny, k2 = rr / nny;
    int l2 = S.ibox.local(i2, j2, k2);
    if (l2 < 0) continue;
    for (int c = 0; c < nc; ++c) {
      double a = val[(size_t)nc * nc * pidx + nc * r + c];
      const double *zr = Zp + S.z_off + (long long)(nc * l2 + c) * m;
#pragma unroll
      for (int q = 0; q < kMaxModes; ++q)
        if (q < m) acc[q] += a * zr[q];
    }
  }
  double *yr = Yp + yoff[j] + (long long)t * m;
#pragma unroll
  for (int q = 0; q < kMaxModes; ++q)
    if (q < m) yr[q] = acc[q];
}

__global__ void __launch_bounds__(256)
    k_coarse_blocks(const SubDesc *subs, const int2 *pairs, const double *__restrict__ Zp,
                    const double *__restrict__ Yp, const long long *yoff, double *AH, int nH) {
  const int2 pr = pairs[blockIdx.x];
  const SubDesc &Sj = subs[pr.x];
  const SubDesc &Sk = subs[pr.y];
  const int mj = Sj.m, mk = Sk.m;
  int lo[3], hi[3];
  for (int d = 0; d < 3; ++d) {
    lo[d] = max(Sj.ibox.lo[d], Sk.nbox.lo[d]);
    hi[d] = min(Sj.ibox.lo[d] + Sj.ibox.n[d], Sk.nbox.lo[d] + Sk.nbox.n[d]);
  }
  const int ex = hi[0] - lo[0], ey = hi[1] - lo[1], ez = hi[2] - lo[2];
  const int nout = mj * mk;
  for (int o = threadIdx.x; o < nout; o += blockDim.x) {
    int a = o / mk, b = o - a * mk;
    double s = 0.0;
    if (ex > 0 && ey > 0 && ez > 0) {
      for (int q = 0; q < ex * ey * ez; ++q) {
        int ii = lo[0] + q % ex, rr = q / ex, jj = lo[1] + rr % ey, kk = lo[2] + rr / ey;
        int lj = Sj.ibox.local(ii, jj, kk), lk = Sk.nbox.local(ii, jj, kk);
        for (int c = 0; c < Sj.nc; ++c)
          s += Zp[Sj.z_off + (long long)(Sj.nc * lj + c) * mj + a] *
               Yp[yoff[pr.y] + (long long)(Sj.nc * lk + c) * mk + b];
      }
    }
    AH[(long long)(Sj.coff + a) * nH + Sk.coff + b] = s;
    if (pr.x != pr.y) AH[(long long)(Sk.coff + b) * nH + Sj.coff + a] = s;
  }
}

__global__ void k_dense_to_tiles(const double *AH, int n, const BandLayout *lay, double *pool) {
  const BandLayout L = lay[0];
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)n * n) return;
  int R = (int)(t / n), C = (int)(t - (long long)R * n);
  if (R < C) return;
  tile_at(pool, L, R >> 5, (R >> 5) - (C >> 5))[(C & 31) * 32 + (R & 31)] = AH[t];
}

__global__ void k_symmetrize(double *M, int n) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)n * n) return;
  int r = (int)(t / n), c = (int)(t - (long long)r * n);
  if (r >= c) return;
  double a = M[(long long)r * n + c], b = M[(long long)c * n + r];
  double v = 0.5 * (a + b);
  M[(long long)r * n + c] = v;
  M[(long long)c * n + r] = v;
}

__global__ void k_identity(double *M, int n) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)n * n) return;
  int r = (int)(t / n), c = (int)(t - (long long)r * n);
  M[t] = r == c ? 1.0 : 0.0;
}

__global__ void k_normalize_cols(const SubDesc *subs, int npad, double *P, int ld, long long sp,
                                 int ncol, const double *G) {
  const int j = blockIdx.y;
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)npad * ncol) return;
  int row = (int)(t / ncol), c = (int)(t - (long long)row * ncol);
  double g = G[(long long)j * ncol * ncol + c * ncol + c];
  double *pv = P + j * sp + (long long)row * ld + c;
  if (row >= subs[j].n_neu) {
    *pv = 0.0;
    return;
  }
  if (g > 0.0) *pv /= sqrt(g);
}

// Rigid displacements of the Neumann nodes of every subdomain (Sec. 5, zero
// energy modes): P[j][row][k] for k < 6 -- translations along x, y, z and
// rotations omega x (X - c) about the axes through the centre c of the
// subdomain's node box; columns 6.. and the padding rows are zero.
__global__ void k_rigid_modes(const SubDesc *subs, int npad, const double *__restrict__ X,
                              const double *__restrict__ Y, const double *__restrict__ Z,
                              double *P, int ld, long long sp) {
  const int j = blockIdx.y;
  const SubDesc &S = subs[j];
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)npad * ld) return;
  const int row = (int)(t / ld), k = (int)(t - (long long)row * ld);
  double v = 0.0;
  if (S.nc == 1) {                // scalar problem: the constants
    v = (row < S.n_neu && k == 0) ? 1.0 : 0.0;
  } else if (row < S.n_neu && k < 6) {
    const int node = row / 3, comp = row - 3 * node;
    int gi, gj, gk;
    S.nbox.global(node, gi, gj, gk);
    const NodeBox &B = S.nbox;
    const double dx = X[gi] - 0.5 * (X[B.lo[0]] + X[B.lo[0] + B.n[0] - 1]);
    const double dy = Y[gj] - 0.5 * (Y[B.lo[1]] + Y[B.lo[1] + B.n[1] - 1]);
    const double dz = Z[gk] - 0.5 * (Z[B.lo[2]] + Z[B.lo[2] + B.n[2] - 1]);
    if (k < 3) {
      v = comp == k ? 1.0 : 0.0;
    } else if (k == 3) {          // about x: (0, -dz, dy)
      v = comp == 1 ? -dz : (comp == 2 ? dy : 0.0);
    } else if (k == 4) {          // about y: (dz, 0, -dx)
      v = comp == 0 ? dz : (comp == 2 ? -dx : 0.0);
    } else {                      // about z: (-dy, dx, 0)
      v = comp == 0 ? -dy : (comp == 1 ? dx : 0.0);
    }
  }
  P[j * sp + t] = v;
}

}  // namespace

void launch_rigid_modes(const SubDesc *d_subs, int nsub, int npad, const double *X,
                        const double *Y, const double *Z, double *P, int ld, long long sp,
                        cudaStream_t s) {
  long long tot = (long long)npad * ld;
  dim3 g((unsigned)((tot + 255) / 256), nsub);
  k_rigid_modes<<<g, 256, 0, s>>>(d_subs, npad, X, Y, Z, P, ld, sp); GENEO_COUNT_LAUNCH();
}

void launch_pou_neumann(const SubDesc *d_subs, int nsub, int max_nodes, const int *cand,
                        const int cand_off[3], const uint8_t *mask, int nnx, int nny, int nnz,
                        int px, int py, int kind, double *Xneu, cudaStream_t s) {
  dim3 g((3 * max_nodes + 255) / 256, nsub);
  k_pou_neumann<<<g, 256, 0, s>>>(d_subs, cand, cand_off[0], cand_off[1], cand_off[2], mask, nnx,
                                  nny, nnz, px, py, kind, Xneu); GENEO_COUNT_LAUNCH();
}

void launch_pou_interior(const SubDesc *d_subs, int nsub, int max_nodes, const int *cand,
                         const int cand_off[3], const uint8_t *mask, int nnx, int nny, int nnz,
                         int px, int py, int kind, double *wloc, cudaStream_t s) {
  dim3 g((3 * max_nodes + 255) / 256, nsub);
  k_pou_interior<<<g, 256, 0, s>>>(d_subs, cand, cand_off[0], cand_off[1], cand_off[2], mask,
                                   nnx, nny, nnz, px, py, kind, wloc); GENEO_COUNT_LAUNCH();
}

void launch_neumann_assemble(const SubDesc *d_subs, const BandLayout *d_lay, int nsub,
                             int max_nodes, int nx, int ny, int nz, const double *X,
                             const double *Y, const double *Z, const double *Cel,
                             const double *perm,
                             const int *ecnt, const int ecnt_off[3], const uint8_t *mask,
                             const double *Xneu, double sigma, double *poolS, double *Bloc,
                             cudaStream_t s) {
  long long tot = (long long)max_nodes * 27;
  dim3 g((unsigned)((tot + 127) / 128), nsub);
  k_neumann_assemble<<<g, 128, 0, s>>>(d_subs, d_lay, nx, ny, nz, X, Y, Z, Cel, perm, ecnt,
                                       ecnt_off[0], ecnt_off[1], ecnt_off[2], mask, Xneu, sigma,
                                       poolS, Bloc); GENEO_COUNT_LAUNCH();
}

void launch_bloc_mv(const SubDesc *d_subs, int nsub, int max_nodes, const double *Bloc,
                    const double *T, double *W, long long sys_stride, int p, cudaStream_t s) {
  dim3 g((3 * max_nodes + 127) / 128, nsub);
  k_bloc_mv<<<g, 128, 0, s>>>(d_subs, Bloc, T, W, sys_stride, p); GENEO_COUNT_LAUNCH();
}

void launch_random_block(const SubDesc *d_subs, int nsub, int npad, double *V, int ld,
                         long long sys_stride, int p, unsigned long long seed, cudaStream_t s) {
  dim3 g((npad * p + 255) / 256, nsub);
  k_random_block<<<g, 256, 0, s>>>(d_subs, npad, V, ld, sys_stride, p, seed); GENEO_COUNT_LAUNCH();
}

void launch_tsdots(const SubDesc *d_subs, int nsub, int npad, const double *A, int lda,
                   long long sa, int na, const double *B, int ldb, long long sb, int nb,
                   double *Hpart, int chunks, double *H, long long hs, cudaStream_t s,
                   const int *gate) {
  (void)npad;
  int sm = 16 * (na + nb) * (int)sizeof(double);
  (void)ensure_smem(k_tsdots, sm);   // a failure surfaces as a launch error
  k_tsdots<<<dim3(chunks, nsub), 256, sm, s>>>(d_subs, A, lda, sa, na, B, ldb, sb, nb, Hpart,
                                               chunks, gate); GENEO_COUNT_LAUNCH();
  k_tsdots_reduce<<<nsub, 256, 0, s>>>(Hpart, chunks, na * nb, H, hs, gate); GENEO_COUNT_LAUNCH();
}

void launch_reorth_gate(int nsub, const double *G, int p, const double *H, int na, long long hs,
                        int *gate, cudaStream_t s) {
  k_reorth_gate<<<nsub, 32, 0, s>>>(G, p, H, na, hs, gate); GENEO_COUNT_LAUNCH();
}

void launch_tsgemm(const SubDesc *d_subs, int nsub, int npad, const double *A, int lda,
                   long long sa, int na, const double *H, int ldh, long long hs, double *C,
                   int ldc, long long sc, int nb, double alpha, double beta, cudaStream_t s,
                   const int *gate) {
  int sm = na * nb * (int)sizeof(double);
  (void)ensure_smem(k_tsgemm, sm);
  long long tot = (long long)npad * nb;
  dim3 g((unsigned)((tot + 255) / 256), nsub);
  k_tsgemm<<<g, 256, sm, s>>>(d_subs, npad, A, lda, sa, na, H, ldh, hs, C, ldc, sc, nb, alpha,
                              beta, gate); GENEO_COUNT_LAUNCH();
}

void launch_cholqr(const SubDesc *d_subs, int nsub, int npad, const double *G, double *W,
                   int p, double *Racc, double *Rinv, int first, double abs_tiny, cudaStream_t s) {
  k_cholqr_small<<<nsub, 32, 0, s>>>(G, p, Rinv, Racc, first, abs_tiny); GENEO_COUNT_LAUNCH();
  dim3 g((npad + 255) / 256, nsub);
  k_rowmul<<<g, 256, 0, s>>>(d_subs, npad, W, p, Rinv); GENEO_COUNT_LAUNCH();
}

void launch_hm_accum(int nsub, double *Hm, int kdim, const double *Hs, int rows, int k, int p,
                     cudaStream_t s) {
  k_hm_accum<<<nsub, 256, 0, s>>>(Hm, kdim, Hs, rows, k, p); GENEO_COUNT_LAUNCH();
}

void launch_hm_subdiag(int nsub, double *Hm, int kdim, const double *Racc, int k, int p,
                       double *Rblk, cudaStream_t s) {
  k_hm_subdiag<<<nsub, 64, 0, s>>>(Hm, kdim, Racc, k, p, Rblk); GENEO_COUNT_LAUNCH();
}

void launch_restart_hm(int nsub, double *Hm, int kdim, const double *Eval, const double *Evec,
                       const double *Rblk, int kk, int p, cudaStream_t s) {
  k_restart_hm<<<nsub, 256, 0, s>>>(Hm, kdim, Eval, Evec, Rblk, kk, p); GENEO_COUNT_LAUNCH();
}

void launch_copy_block(const SubDesc *d_subs, int nsub, int npad, const double *W, int ldw,
                       long long sw, double *V, int ldv, long long sv, int p, cudaStream_t s) {
  dim3 g((npad * p + 255) / 256, nsub);
  k_copy_block<<<g, 256, 0, s>>>(d_subs, npad, W, ldw, sw, V, ldv, sv, p); GENEO_COUNT_LAUNCH();
}

int launch_ritz_eig(int nsub, const double *Hm, int kdim, int nw, int p, const double *Rblk,
                    double *Eval, double *Evec, double *Eres, cudaStream_t s) {
  if (kdim > kMaxKdim || nw > kdim) return GENEO_ERR_INVALID_ARG;
  int sm = (kdim * (kdim + 1) + 6 * kdim) * (int)sizeof(double);
  if (int st = ensure_smem(k_ritz_eig, sm)) return st;
  k_ritz_eig<<<nsub, 256, sm, s>>>(Hm, kdim, nw, p, Rblk, Eval, Evec, Eres); GENEO_COUNT_LAUNCH();
  GENEO_CUDA_TRY(cudaGetLastError());
  return GENEO_OK;
}

void launch_build_Z(const SubDesc *d_subs, int nsub, int max_nint, const double *P, int ldp,
                    long long sp, const double *Xneu, double *Zp, cudaStream_t s) {
  long long tot = (long long)max_nint * kMaxModes;
  dim3 g((unsigned)((tot + 255) / 256), nsub);
  k_build_Z<<<g, 256, 0, s>>>(d_subs, P, ldp, sp, Xneu, Zp); GENEO_COUNT_LAUNCH();
}

void launch_AZ(const SubDesc *d_subs, int nsub, int max_nodes, int nnx, int nny, int nnz,
               const int32_t *rp, const int32_t *col, const double *val, const double *Zp,
               const long long *yoff, double *Yp, cudaStream_t s) {
  dim3 g((3 * max_nodes + 127) / 128, nsub);
  k_AZ<<<g, 128, 0, s>>>(d_subs, nnx, nny, nnz, rp, col, val, Zp, yoff, Yp); GENEO_COUNT_LAUNCH();
}

void launch_coarse_blocks(const SubDesc *d_subs, const int2 *pairs, int npairs, const double *Zp,
                          const double *Yp, const long long *yoff, double *AH, int nH,
                          cudaStream_t s) {
  if (npairs > 0) {
    k_coarse_blocks<<<npairs, 256, 0, s>>>(d_subs, pairs, Zp, Yp, yoff, AH, nH);
    GENEO_COUNT_LAUNCH();
  }
}

void launch_dense_to_tiles(const double *AH, int nH, const BandLayout *d_lay, double *pool,
                           cudaStream_t s) {
  long long tot = (long long)nH * nH;
  k_dense_to_tiles<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(AH, nH, d_lay, pool); GENEO_COUNT_LAUNCH();
}

void launch_symmetrize(double *M, int n, cudaStream_t s) {
  long long tot = (long long)n * n;
  k_symmetrize<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(M, n); GENEO_COUNT_LAUNCH();
}

void launch_identity(double *M, int n, cudaStream_t s) {
  long long tot = (long long)n * n;
  k_identity<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(M, n); GENEO_COUNT_LAUNCH();
}

void launch_normalize_cols(const SubDesc *d_subs, int nsub, int npad, double *P, int ld,
                           long long sp, int ncol, const double *G, cudaStream_t s) {
  long long tot = (long long)npad * ncol;
  dim3 g((unsigned)((tot + 255) / 256), nsub);
  k_normalize_cols<<<g, 256, 0, s>>>(d_subs, npad, P, ld, sp, ncol, G); GENEO_COUNT_LAUNCH();
}

}  // namespace geneo
