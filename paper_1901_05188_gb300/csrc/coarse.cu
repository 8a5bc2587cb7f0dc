// Coarse correction and gather of the two-level Schwarz preconditioner
// (Sec. 3.3: M^-1 r = sum_j R_j^T D_j A_j^-1 R_j r + Z A_H^-1 Z^T r): the
// restriction w = Z^T r, y = A_H^-1 w, the prolongation Z_j y_j, and the
// deterministic gather of the local solutions over the subdomains containing
// each node.
#include <algorithm>

#include "band.cuh"
#include "batch.cuh"

namespace geneo {

namespace {

// ---- gather / coarse --------------------------------------------------------

// Subdomains of node n (global node coordinates i, jj, k): the per-axis
// candidate lists give the overlapping subdomains containing the node (their
// count is the partition-of-unity denominator); `visit(S, l)` is called, in a
// fixed order, for those whose interior holds it (l = local node index).
template <typename F>
__device__ __forceinline__ int for_node_subdomains(int i, int jj, int k, int px, int py,
                                                   const int *__restrict__ cand, int co0, int co1,
                                                   int co2, const SubDesc *subs, F visit) {
  const int *ci = cand + (co0 + i) * kMaxCand;
  const int *cj = cand + (co1 + jj) * kMaxCand;
  const int *ck = cand + (co2 + k) * kMaxCand;
  int nci = 0, ncj = 0, nck = 0;
  while (nci < kMaxCand && ci[nci] >= 0) ++nci;
  while (ncj < kMaxCand && cj[ncj] >= 0) ++ncj;
  while (nck < kMaxCand && ck[nck] >= 0) ++nck;
  // not unrolled: the candidate counts are small and the nest only serves the
  // set-up's gather map and the rare nodes in more than eight interiors (fully
  // unrolled, its 64 copies of `visit` made this file slow to compile)
#pragma unroll 1
  for (int c = 0; c < nck; ++c)
#pragma unroll 1
    for (int b = 0; b < ncj; ++b)
#pragma unroll 1
      for (int a = 0; a < nci; ++a) {
        const SubDesc &S = subs[ci[a] + px * (cj[b] + py * ck[c])];
        const int l = S.ibox.local(i, jj, k);
        if (l >= 0) visit(S, l);
      }
  return nci * ncj * nck;
}

// Gather map: per node the xloc offsets (v_int + nc l) of the subdomains whose
// interior holds it, in the order above (-1 after the last), and the number of
// overlapping subdomains containing it; kMapFull marks a node with more than
// kMapSlots interior subdomains, which the gather then visits directly.
constexpr int kMapSlots = 8;
constexpr uint8_t kMapFull = 0xFF;

__global__ void k_gather_map(int nnx, int nny, int nnz, int px, int py,
                             const int *__restrict__ cand, int co0, int co1, int co2,
                             const SubDesc *subs, int *__restrict__ gmap,
                             uint8_t *__restrict__ gcnt) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= nnx * nny * nnz) return;
  const int i = n % nnx, r = n / nnx, jj = r % nny, k = r / nny;
  int e = 0;
  bool full = false;
  const int cnt = for_node_subdomains(i, jj, k, px, py, cand, co0, co1, co2, subs,
                                      [&](const SubDesc &S, int l) {
                                        if (e < kMapSlots) gmap[n * kMapSlots + e++] = S.v_int + S.nc * l;
                                        else full = true;
                                      });
  for (; e < kMapSlots; ++e) gmap[n * kMapSlots + e] = -1;
  gcnt[n] = full ? kMapFull : (uint8_t)cnt;
}

// z = sum_j R_j^T (D_j x_j + (Z y)_j), one thread per node, deterministic order.
template <typename T>
__device__ __forceinline__ void gather_node(int n, int nnx, int nny, int px, int py,
                                            const int *__restrict__ cand, int co0, int co1,
                                            int co2, const SubDesc *subs,
                                            const int *__restrict__ gmap,
                                            const uint8_t *__restrict__ gcnt,
                                            const T *__restrict__ xloc,
                                            const double *__restrict__ zy, int pou,
                                            const double *__restrict__ wloc,
                                            const uint8_t *__restrict__ mask,
                                            double *__restrict__ z) {
  const int nc = subs[0].nc;
  double o[3] = {0.0, 0.0, 0.0};
  const int cnt = gcnt[n];
  auto add = [&](int off, double wgt) {
    for (int comp = 0; comp < nc; ++comp) {
      double v = double(xloc[off + comp]);
      if (pou) v *= wloc ? wloc[off + comp] : (mask[nc * n + comp] ? 0.0 : wgt);
      if (zy) v += zy[off + comp];
      o[comp] += v;
    }
  };
  if (cnt != kMapFull) {
    const int4 a = reinterpret_cast<const int4 *>(gmap)[2 * n];
    const int4 b = reinterpret_cast<const int4 *>(gmap)[2 * n + 1];
    const int off[kMapSlots] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
    const double wgt = pou ? 1.0 / double(cnt) : 1.0;
#pragma unroll
    for (int e = 0; e < kMapSlots; ++e) {
      if (off[e] < 0) break;
      add(off[e], wgt);
    }
  } else {
    const int i = n % nnx, r = n / nnx, jj = r % nny, k = r / nny;
    const int count = for_node_subdomains(i, jj, k, px, py, cand, co0, co1, co2, subs,
                                          [](const SubDesc &, int) {});
    const double wgt = pou ? 1.0 / double(count) : 1.0;
    for_node_subdomains(i, jj, k, px, py, cand, co0, co1, co2, subs,
                        [&](const SubDesc &S, int l) { add(S.v_int + nc * l, wgt); });
  }
  for (int comp = 0; comp < nc; ++comp) z[nc * n + comp] = o[comp];
}

template <typename T>
__global__ void __launch_bounds__(256)
    k_schwarz_gather(int nnx, int nny, int nnz, int px, int py, const int *__restrict__ cand,
                     int co0, int co1, int co2, const SubDesc *subs,
                     const int *__restrict__ gmap, const uint8_t *__restrict__ gcnt,
                     const T *__restrict__ xloc, const double *__restrict__ zy, int pou,
                     const double *__restrict__ wloc, const uint8_t *__restrict__ mask,
                     double *__restrict__ z, const CGScalars *cg) {
  if (cg && cg->done) return;
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= nnx * nny * nnz) return;
  gather_node<T>(n, nnx, nny, px, py, cand, co0, co1, co2, subs, gmap, gcnt, xloc, zy, pou,
                 wloc, mask, z);
}

// Coarse restriction and prolongation stream Z_j (row-major n_int x m_j) in
// blocks of kZRows rows: the block's m_j * kZRows contiguous values are loaded
// with coalesced loads, all in flight at once, into shared memory.
__device__ __forceinline__ double restrict_r(const SubDesc &S, const double *__restrict__ r,
                                             int nnx, int nny, int l) {
  const int nc = S.nc, node = l / nc, c = l - nc * node;
  int gi, gj, gk;
  S.ibox.global(node, gi, gj, gk);
  return __ldg(r + nc * (gi + nnx * (gj + nny * gk)) + c);
}

// partial w_{j,k} over rows [kZRows b, kZRows (b + 1)): warp g takes rows g, g + 8, ..., lane k
__device__ __forceinline__ void coarse_restrict_block(const SubDesc *subs, int j, int b, int nnx,
                                                      int nny, const double *__restrict__ Zp,
                                                      const double *__restrict__ r,
                                                      double *__restrict__ wpart, int nchunk,
                                                      int mcap) {
  const SubDesc &S = subs[j];
  const int m = S.m, l0 = b * kZRows;
  if (m == 0 || l0 >= S.n_int) return;
  const int rows = min(kZRows, S.n_int - l0), cnt = rows * m;
  __shared__ double zs[kZRows * kMaxModes];
  __shared__ double rs[kZRows];
  __shared__ double acc[8][32];
  const double *Z = Zp + S.z_off + (long long)l0 * m;
#pragma unroll 4
  for (int e = threadIdx.x; e < cnt; e += 256) zs[e] = __ldg(Z + e);
  if (threadIdx.x < rows) rs[threadIdx.x] = restrict_r(S, r, nnx, nny, l0 + threadIdx.x);
  __syncthreads();
  const int k = threadIdx.x & 31, g = threadIdx.x >> 5;
  double s = 0.0;
  if (k < m)
    for (int t = g; t < rows; t += 8) s = fma(zs[t * m + k], rs[t], s);
  acc[g][k] = s;
  __syncthreads();
  if (threadIdx.x < m) {
    double t = 0.0;
#pragma unroll
    for (int q = 0; q < 8; ++q) t += acc[q][k];
    wpart[((long long)j * nchunk + b) * mcap + k] = t;
  }
}

__global__ void __launch_bounds__(256) k_coarse_restrict(const SubDesc *subs, int nnx, int nny,
                                                         const double *__restrict__ Zp,
                                                         const double *__restrict__ r,
                                                         double *__restrict__ wpart, int nchunk,
                                                         int mcap, const CGScalars *cg) {
  if (cg && cg->done) return;
  coarse_restrict_block(subs, blockIdx.y, blockIdx.x, nnx, nny, Zp, r, wpart, nchunk, mcap);
}

// zy_j = Z_j y_j on rows [kZRows b, kZRows (b + 1)) of subdomain j (rows padded
// to m + 1 values in shared memory against bank conflicts)
__device__ __forceinline__ void coarse_prolong_block(const SubDesc *subs, int j, int b,
                                                     const double *__restrict__ Zp,
                                                     const double *__restrict__ yH,
                                                     double *__restrict__ zy) {
  const SubDesc &S = subs[j];
  const int m = S.m, l0 = b * kZRows;
  if (l0 >= S.n_int) return;
  const int rows = min(kZRows, S.n_int - l0);
  if (m == 0) {
    if (threadIdx.x < rows) zy[S.v_int + l0 + threadIdx.x] = 0.0;
    return;
  }
  __shared__ double zs[kZRows * (kMaxModes + 1)];
  __shared__ double yj[kMaxModes];
  if (threadIdx.x < m) yj[threadIdx.x] = yH[S.coff + threadIdx.x];
  const double *Z = Zp + S.z_off + (long long)l0 * m;
  const int cnt = rows * m;
#pragma unroll 4
  for (int e = threadIdx.x; e < cnt; e += 256) {
    const int t = e / m;
    zs[e + t] = __ldg(Z + e);                   // row t at t * (m + 1)
  }
  __syncthreads();
  if (threadIdx.x < rows) {
    const double *zr = zs + threadIdx.x * (m + 1);
    double v0 = 0.0, v1 = 0.0;
    int q = 0;
    for (; q + 1 < m; q += 2) {
      v0 = fma(zr[q], yj[q], v0);
      v1 = fma(zr[q + 1], yj[q + 1], v1);
    }
    if (q < m) v0 = fma(zr[q], yj[q], v0);
    zy[S.v_int + l0 + threadIdx.x] = v0 + v1;
  }
}

__global__ void __launch_bounds__(256) k_coarse_prolong(const SubDesc *subs,
                                                        const double *__restrict__ Zp,
                                                        const double *__restrict__ yH,
                                                        double *__restrict__ zy,
                                                        const CGScalars *cg) {
  if (cg && cg->done) return;
  coarse_prolong_block(subs, blockIdx.y, blockIdx.x, Zp, yH, zy);
}

// w_{j,k} = sum of the row-block partials: warp g adds blocks g, g + 8, ...
__device__ __forceinline__ void coarse_reduce_block(const SubDesc *subs, int j,
                                                    const double *__restrict__ wpart,
                                                    double *__restrict__ wH, int nchunk,
                                                    int mcap) {
  const SubDesc &S = subs[j];
  const int k = threadIdx.x & 31, g = threadIdx.x >> 5, m = S.m;
  __shared__ double acc[8][32];
  if (m == 0) return;
  const int nb = (S.n_int + kZRows - 1) / kZRows;
  double t = 0.0;
  if (k < m)
    for (int ch = g; ch < nb; ch += 8) t += wpart[((long long)j * nchunk + ch) * mcap + k];
  acc[g][k] = t;
  __syncthreads();
  if (threadIdx.x < m) {
    double u = 0.0;
#pragma unroll
    for (int q = 0; q < 8; ++q) u += acc[q][k];
    wH[S.coff + k] = u;
  }
}

__global__ void __launch_bounds__(256) k_coarse_reduce(const SubDesc *subs,
                                                       const double *__restrict__ wpart,
                                                       double *__restrict__ wH, int nchunk,
                                                       int mcap, const CGScalars *cg) {
  if (cg && cg->done) return;
  coarse_reduce_block(subs, blockIdx.x, wpart, wH, nchunk, mcap);
}

// ---- the same steps over the instances of a batch ------------------------------
__global__ void __launch_bounds__(256) k_batch_restrict(const BatchInst *inst, const int4 *items,
                                                        const CGScalars *cg,
                                                        const double *__restrict__ r) {
  const int4 it = items[blockIdx.x];
  if (cg[it.x].done) return;
  const BatchInst &B = inst[it.x];
  coarse_restrict_block(B.subs, it.y, it.z, B.nnx, B.nny, B.Zp, r + B.vbase, B.wpart, B.nchunk,
                        B.mcap);
}

__global__ void __launch_bounds__(256) k_batch_reduce_w(const BatchInst *inst, const int2 *items,
                                                        const CGScalars *cg) {
  const int2 it = items[blockIdx.x];
  const BatchInst &B = inst[it.x];
  if (cg[it.x].done || B.nH == 0) return;
  coarse_reduce_block(B.subs, it.y, B.wpart, B.wH, B.nchunk, B.mcap);
}

// y = A_H^-1 w per instance, one warp per coarse row
__global__ void __launch_bounds__(256) k_batch_gemv(const BatchInst *inst, const int2 *items,
                                                    int nitems, const CGScalars *cg) {
  const int lane = threadIdx.x & 31;
  const int wi = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (wi >= nitems) return;
  const int2 it = items[wi];
  if (cg[it.x].done) return;
  const BatchInst &B = inst[it.x];
  const double *a = B.AHinv + (long long)it.y * B.nH;
  double s = 0.0;
  for (int c = lane; c < B.nH; c += 32) s += a[c] * B.wH[c];
  s = warp_sum(s);
  if (lane == 0) B.yH[it.y] = s;
}

__global__ void __launch_bounds__(256) k_batch_prolong(const BatchInst *inst, const int4 *items,
                                                       const CGScalars *cg) {
  const int4 it = items[blockIdx.x];
  if (cg[it.x].done) return;
  const BatchInst &B = inst[it.x];
  coarse_prolong_block(B.subs, it.y, it.z, B.Zp, B.yH, B.zy);
}

template <typename T>
__global__ void __launch_bounds__(256) k_batch_gather(const BatchInst *inst, const long long *off,
                                                      int n, const CGScalars *cg,
                                                      double *__restrict__ z) {
  // block b covers nodes [256 (b - off[i]), ...) of the instance i it belongs to
  const long long b = blockIdx.x;
  int lo = 0, hi = n;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (off[mid] <= b) lo = mid;
    else hi = mid;
  }
  const int i = lo;
  if (cg[i].done) return;
  const BatchInst &B = inst[i];
  const int node = (int)(b - off[i]) * 256 + threadIdx.x;
  if (node >= B.nnode) return;
  gather_node<T>(node, B.nnx, B.nny, B.px, B.py, B.cand, B.co0, B.co1, B.co2, B.subs, B.gmap,
                 B.gcnt, (const T *)B.xloc, B.nH > 0 ? B.zy : nullptr, B.pou, B.wloc, B.mask,
                 z + B.vbase);
}

// y = AHinv w, one warp per row (AHinv symmetric, row-major)
__global__ void k_coarse_gemv(int nH, const double *__restrict__ Ainv,
                              const double *__restrict__ w, double *__restrict__ y,
                              const CGScalars *cg) {
  if (cg && cg->done) return;
  int lane = threadIdx.x & 31;
  int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (row >= nH) return;
  const double *a = Ainv + (long long)row * nH;
  double s = 0.0;
  for (int c = lane; c < nH; c += 32) s += a[c] * w[c];
  s = warp_sum(s);
  if (lane == 0) y[row] = s;
}

// ---- inexact coarse solve (Sec. 3.3.3) -------------------------------------
// For large coarse spaces the paper solves A_H y = w by preconditioned CG and
// makes the outer Krylov method flexible.  Here: CG preconditioned by the
// inverses of A_H's diagonal blocks (one block per subdomain's modes), run to
// ||w - A_H y|| <= tol ||w|| or max_it steps, inside one cooperative launch
// whose blocks meet at a grid barrier with bounded waits.

// Inverse of subdomain j's diagonal block of A_H (m_j x m_j, SPD) by
// Gauss-Jordan elimination on [B | I] in shared memory; one CTA per subdomain.
__global__ void __launch_bounds__(1024) k_coarse_bj_inverse(const SubDesc *subs, int nH,
                                                            const double *__restrict__ AH,
                                                            double *__restrict__ BJ, int mcap) {
  const int j = blockIdx.x;
  const SubDesc &S = subs[j];
  const int m = S.m, o = S.coff;
  if (m == 0) return;
  __shared__ double G[32][65];
  const int r = threadIdx.x >> 5, c = threadIdx.x & 31;
  G[r][c] = (r < m && c < m) ? AH[(long long)(o + r) * nH + o + c] : (r == c ? 1.0 : 0.0);
  G[r][32 + c] = r == c ? 1.0 : 0.0;
  __syncthreads();
  for (int k = 0; k < m; ++k) {
    const double piv = G[k][k];
    const double f0 = G[r][k];
    __syncthreads();
    if (r == k) {
      G[k][c] /= piv;
      G[k][32 + c] /= piv;
    }
    __syncthreads();
    if (r != k) {
      G[r][c] -= f0 * G[k][c];
      G[r][32 + c] -= f0 * G[k][32 + c];
    }
    __syncthreads();
  }
  if (r < m && c < m) BJ[(long long)j * mcap * mcap + r * mcap + c] = G[r][32 + c];
}

__device__ __forceinline__ uint64_t coarse_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid barrier over the co-resident blocks of a cooperative launch: arrival
// counter and generation word in global memory; a block that waits more than
// about a second records GENEO_ERR_TIMEOUT and returns false.
__device__ bool coarse_grid_barrier(unsigned int *bar, DevStatus *st) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    volatile unsigned int *gen = bar + 1;
    const unsigned int g = *gen;
    __threadfence();
    const unsigned int arrived = atomicAdd(bar, 1u);
    if (arrived == gridDim.x - 1) {
      bar[0] = 0;
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      const uint64_t t0 = coarse_ns();
      while (*gen == g) {
        if (coarse_ns() - t0 > 1000000000ull) {
          atomicCAS(&st->code, 0, (int)GENEO_ERR_TIMEOUT);
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

// Sum of the per-block partials part[b * 4 + k], the same order in every block.
__device__ __forceinline__ double coarse_sum_partials(const double *part, int k) {
  double s = 0.0;
  for (int b = 0; b < (int)gridDim.x; ++b) s += ((volatile const double *)part)[b * 4 + k];
  return s;
}

__device__ __forceinline__ void coarse_block_partials(double *part, double a, double b,
                                                      double c) {
  __shared__ double red[8][3];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  a = warp_sum(a);
  b = warp_sum(b);
  c = warp_sum(c);
  if (lane == 0) {
    red[warp][0] = a;
    red[warp][1] = b;
    red[warp][2] = c;
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += red[w][threadIdx.x];
    part[blockIdx.x * 4 + threadIdx.x] = t;
  }
  __syncthreads();
}

// Block-Jacobi PCG on A_H y = w from y = 0.  work: r, z, p, q [nH each] then
// the per-block partials [gridDim.x][4]; bar: the barrier words.  One warp per
// subdomain block for the vector updates and the block-Jacobi product, one
// warp per row for A_H p.
__global__ void __launch_bounds__(256)
    k_coarse_pcg(const SubDesc *subs, int nsub, int nH, int mcap, const double *__restrict__ AH,
                 const double *__restrict__ BJ, const double *__restrict__ w,
                 double *__restrict__ y, double *work, unsigned int *bar, double tol2, int maxit,
                 const CGScalars *cg, DevStatus *st, int *inner_its) {
  if (cg && cg->done) return;
  double *r = work, *z = r + nH, *p = z + nH, *q = p + nH, *part = q + nH;
  const int lane = threadIdx.x & 31;
  const int gwarp = blockIdx.x * 8 + (threadIdx.x >> 5), nwarps = gridDim.x * 8;
  // r = w, y = 0, z = BJ r, p = z; partials r.z and r.r
  double a0 = 0.0, a1 = 0.0;
  for (int j = gwarp; j < nsub; j += nwarps) {
    const int m = subs[j].m, o = subs[j].coff;
    if (m == 0) continue;
    const double rv = lane < m ? w[o + lane] : 0.0;
    double zv = 0.0;
    for (int k = 0; k < m; ++k)
      zv += (lane < m ? BJ[(long long)j * mcap * mcap + lane * mcap + k] : 0.0) *
            __shfl_sync(0xffffffffu, rv, k);
    if (lane < m) {
      r[o + lane] = rv;
      y[o + lane] = 0.0;
      z[o + lane] = zv;
      p[o + lane] = zv;
      a0 += rv * zv;
      a1 += rv * rv;
    }
  }
  coarse_block_partials(part, a0, a1, 0.0);
  if (!coarse_grid_barrier(bar, st)) return;
  double rz = coarse_sum_partials(part, 0), rr = coarse_sum_partials(part, 1);
  const double ww = rr;
  int it = 0;
  for (; it < maxit && rr > tol2 * ww; ++it) {
    if (!coarse_grid_barrier(bar, st)) return;     // every block has read the partials
    // q = A_H p and p.q
    double pq = 0.0;
    for (int row = gwarp; row < nH; row += nwarps) {
      const double *a = AH + (long long)row * nH;
      double sum = 0.0;
      for (int c = lane; c < nH; c += 32) sum += a[c] * p[c];
      sum = warp_sum(sum);
      if (lane == 0) {
        q[row] = sum;
        pq += p[row] * sum;
      }
    }
    coarse_block_partials(part, pq, 0.0, 0.0);
    if (!coarse_grid_barrier(bar, st)) return;
    const double alpha = rz / coarse_sum_partials(part, 0);
    if (!coarse_grid_barrier(bar, st)) return;     // partials read before they are rewritten
    // y += alpha p, r -= alpha q, z = BJ r; partials r.z, r.r
    a0 = a1 = 0.0;
    for (int j = gwarp; j < nsub; j += nwarps) {
      const int m = subs[j].m, o = subs[j].coff;
      if (m == 0) continue;
      double rv = 0.0;
      if (lane < m) {
        y[o + lane] += alpha * p[o + lane];
        rv = r[o + lane] - alpha * q[o + lane];
        r[o + lane] = rv;
      }
      double zv = 0.0;
      for (int k = 0; k < m; ++k)
        zv += (lane < m ? BJ[(long long)j * mcap * mcap + lane * mcap + k] : 0.0) *
              __shfl_sync(0xffffffffu, rv, k);
      if (lane < m) {
        z[o + lane] = zv;
        a0 += rv * zv;
        a1 += rv * rv;
      }
    }
    coarse_block_partials(part, a0, a1, 0.0);
    if (!coarse_grid_barrier(bar, st)) return;
    const double rz_new = coarse_sum_partials(part, 0);
    rr = coarse_sum_partials(part, 1);
    const double beta = rz_new / rz;
    rz = rz_new;
    for (int j = gwarp; j < nsub; j += nwarps) {
      const int m = subs[j].m, o = subs[j].coff;
      if (lane < m) p[o + lane] = z[o + lane] + beta * p[o + lane];
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0 && inner_its) atomicAdd(inner_its, it);
}

}  // namespace

void launch_coarse_bj_inverse(const SubDesc *d_subs, int nsub, int nH, const double *AH,
                              double *BJ, int mcap, cudaStream_t s) {
  k_coarse_bj_inverse<<<nsub, 1024, 0, s>>>(d_subs, nH, AH, BJ, mcap); GENEO_COUNT_LAUNCH();
}

int coarse_pcg_blocks() {
  static int blocks = 0;
  if (blocks == 0) {
    int dev = 0, sms = 0, per = 0;
    GENEO_CUDA_TRY(cudaGetDevice(&dev));
    GENEO_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    GENEO_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_coarse_pcg, 256, 0));
    blocks = sms * std::max(1, std::min(per, 2));
  }
  return blocks;
}

int launch_coarse_apply_iterative(const SubDesc *d_subs, int nsub, int max_nint, int nnx,
                                  int nny, const double *Zp, const double *r, double *wpart,
                                  double *wH, double *yH, double *zy, const double *AH,
                                  const double *BJ, int nH, int mcap, double *work,
                                  unsigned int *bar, double tol, int maxit, const CGScalars *cg,
                                  DevStatus *st, int *inner_its, cudaStream_t s) {
  const int nchunk = restrict_chunks(max_nint);
  k_coarse_restrict<<<dim3(nchunk, nsub), 256, 0, s>>>(d_subs, nnx, nny, Zp, r, wpart, nchunk,
                                                      mcap, cg); GENEO_COUNT_LAUNCH();
  k_coarse_reduce<<<nsub, 256, 0, s>>>(d_subs, wpart, wH, nchunk, mcap, cg); GENEO_COUNT_LAUNCH();
  const int blocks = coarse_pcg_blocks();
  if (blocks <= 0) return GENEO_ERR_CUDA;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(blocks);
  cfg.blockDim = dim3(256);
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;     // every block resident: the barrier can complete
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  const double tol2 = tol * tol;
  GENEO_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_coarse_pcg, d_subs, nsub, nH, mcap, AH, BJ,
                                    (const double *)wH, yH, work, bar, tol2, maxit, cg, st,
                                    inner_its));
  GENEO_COUNT_LAUNCH();
  k_coarse_prolong<<<dim3(nchunk, nsub), 256, 0, s>>>(d_subs, Zp, yH, zy, cg); GENEO_COUNT_LAUNCH();
  return GENEO_OK;
}

void launch_batch_coarse(const BatchInst *inst, const BatchTables &T, const CGScalars *cg,
                         const double *r, cudaStream_t s) {
  if (T.nchunk_items == 0) return;
  k_batch_restrict<<<T.nchunk_items, 256, 0, s>>>(inst, T.chunk_items, cg, r); GENEO_COUNT_LAUNCH();
  k_batch_reduce_w<<<T.nsub_items, 256, 0, s>>>(inst, T.sub_items, cg); GENEO_COUNT_LAUNCH();
  k_batch_gemv<<<(T.nrow_items * 32 + 255) / 256, 256, 0, s>>>(inst, T.row_items, T.nrow_items,
                                                               cg); GENEO_COUNT_LAUNCH();
  k_batch_prolong<<<T.nchunk_items, 256, 0, s>>>(inst, T.chunk_items, cg); GENEO_COUNT_LAUNCH();
}

void launch_batch_gather(const BatchInst *inst, const BatchTables &T, const CGScalars *cg,
                         bool f32, double *z, cudaStream_t s) {
  if (f32) {
    k_batch_gather<float><<<(unsigned)T.nnodeblk, 256, 0, s>>>(inst, T.node_off, T.n, cg, z); GENEO_COUNT_LAUNCH();
  } else {
    k_batch_gather<double><<<(unsigned)T.nnodeblk, 256, 0, s>>>(inst, T.node_off, T.n, cg, z); GENEO_COUNT_LAUNCH();
  }
}

void launch_gather_map(int nx, int ny, int nz, int px, int py, const int *cand,
                       const int cand_off[3], const SubDesc *d_subs, int *gmap, uint8_t *gcnt,
                       cudaStream_t s) {
  int nn = (nx + 1) * (ny + 1) * (nz + 1);
  k_gather_map<<<(nn + 255) / 256, 256, 0, s>>>(nx + 1, ny + 1, nz + 1, px, py, cand,
                                                cand_off[0], cand_off[1], cand_off[2], d_subs,
                                                gmap, gcnt); GENEO_COUNT_LAUNCH();
}

template <typename T>
void launch_schwarz_gather(int nx, int ny, int nz, int px, int py, const int *cand,
                           const int cand_off[3], const SubDesc *d_subs, const int *gmap,
                           const uint8_t *gcnt, const T *xloc, const double *zy, int pou,
                           const double *wloc, const uint8_t *mask, double *z,
                           const CGScalars *cg, cudaStream_t s) {
  int nn = (nx + 1) * (ny + 1) * (nz + 1);
  k_schwarz_gather<T><<<(nn + 255) / 256, 256, 0, s>>>(nx + 1, ny + 1, nz + 1, px, py, cand,
                                                      cand_off[0], cand_off[1], cand_off[2],
                                                      d_subs, gmap, gcnt, xloc, zy, pou, wloc,
                                                      mask, z, cg); GENEO_COUNT_LAUNCH();
}

void launch_coarse_apply(const SubDesc *d_subs, int nsub, int max_nint, int nnx, int nny,
                         const double *Zp, const double *r, double *wpart, double *wH,
                         double *yH, double *zy, const double *AHinv, int nH, int mcap,
                         const CGScalars *cg, cudaStream_t s) {
  const int nchunk = restrict_chunks(max_nint);
  k_coarse_restrict<<<dim3(nchunk, nsub), 256, 0, s>>>(d_subs, nnx, nny, Zp, r, wpart, nchunk,
                                                      mcap, cg); GENEO_COUNT_LAUNCH();
  k_coarse_reduce<<<nsub, 256, 0, s>>>(d_subs, wpart, wH, nchunk, mcap, cg); GENEO_COUNT_LAUNCH();
  k_coarse_gemv<<<(nH * 32 + 255) / 256, 256, 0, s>>>(nH, AHinv, wH, yH, cg); GENEO_COUNT_LAUNCH();
  k_coarse_prolong<<<dim3(nchunk, nsub), 256, 0, s>>>(d_subs, Zp, yH, zy, cg); GENEO_COUNT_LAUNCH();
}

template void launch_schwarz_gather<double>(int, int, int, int, int, const int *, const int[3],
                                            const SubDesc *, const int *, const uint8_t *,
                                            const double *, const double *, int, const double *,
                                            const uint8_t *, double *, const CGScalars *,
                                            cudaStream_t);
template void launch_schwarz_gather<float>(int, int, int, int, int, const int *, const int[3],
                                           const SubDesc *, const int *, const uint8_t *,
                                           const float *, const double *, int, const double *,
                                           const uint8_t *, double *, const CGScalars *,
                                           cudaStream_t);

}  // namespace geneo
