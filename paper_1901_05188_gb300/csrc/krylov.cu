// BSR SpMV and the fused vector kernels of (flexible) PCG (Sec. 3.1).
//
// All reductions are two-stage and deterministic: every block writes one
// partial sum, and the last block to finish (ticket counter) adds the
// partials in a fixed order and updates the CG scalars on the device, so the
// iteration runs without host round trips and can be captured in a graph.
#include <algorithm>
#include <cstdlib>

#include "batch.cuh"
#include "kernels.cuh"

namespace geneo {

namespace {

constexpr int NT = kRedThreads;
constexpr int NB = kRedBlocks;

// Ticket: true in every thread of the block that finishes last.
__device__ __forceinline__ bool last_block(unsigned int *counter) {
  __shared__ bool is_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned t = atomicAdd(counter, 1u);
    is_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (is_last) __threadfence();
  return is_last;
}

// Sum part[0..n) in a fixed order inside the last block; valid in thread 0.
__device__ __forceinline__ double sum_partials(const double *part, int n, double *sh) {
  double v = 0.0;
  for (int i = threadIdx.x; i < n; i += NT) v += ((volatile const double *)part)[i];
  return block_sum<NT>(v, sh);
}

// One lane per matrix row (the loop over a row's blocks not unrolled and the
// kernels limited to 32 registers, so that 64 warps per SM keep the loads in
// flight; measured on the 128x64x48 workload: 0.187 ms against 0.211 ms
// unrolled three times and 0.308 ms unrolled nine times at 40 registers).
// Lane i of warp group g holds scalar row 32g + i
// (block row (32g + i) / NC, component (32g + i) % NC), so no lane idles; every
// stored value takes exactly one FMA and no sum crosses lanes -- FP64 issue,
// not bandwidth, is the scarce resource on this GPU, and a shuffle reduction
// costs FP64 adds.  The lanes of a block row read the rows of the same blocks
// and the same x entries, so their loads share L1 lines; results go to
// consecutive entries of y.

template <int NC, int U = 1>
__device__ __forceinline__ double spmv_lane_row(const int32_t *__restrict__ rp,
                                                const int32_t *__restrict__ col,
                                                const double *__restrict__ val,
                                                const double *__restrict__ x, int node, int r) {
  const int base = rp[node];
  const int nb = rp[node + 1] - base;
  const double *v = val + (size_t)NC * NC * base + NC * r;
  double a[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) a[c] = 0.0;
#pragma unroll U
  for (int b = 0; b < nb; ++b) {
    const double *xb = x + NC * __ldg(col + base + b);
#pragma unroll
    for (int c = 0; c < NC; ++c) a[c] = fma(__ldg(v + NC * NC * b + c), __ldg(xb + c), a[c]);
  }
  double s = a[0];
#pragma unroll
  for (int c = 1; c < NC; ++c) s += a[c];
  return s;
}

template <int NC>
__global__ void __launch_bounds__(256, 8) k_spmv(int nnode, const int32_t *__restrict__ rp,
                                              const int32_t *__restrict__ col,
                                              const double *__restrict__ val,
                                              const double *__restrict__ x,
                                              double *__restrict__ y) {
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  const int nrow = NC * nnode;
  for (int g = warp; g * 32 < nrow; g += nw) {
    const int row = g * 32 + lane;
    if (row < nrow) {
      const int node = row / NC;
      y[row] = spmv_lane_row<NC>(rp, col, val, x, node, row - NC * node);
    }
  }
}

template <int NC>
__global__ void __launch_bounds__(NT, 8) k_cg_spmv_pq(int nnode, const int32_t *__restrict__ rp,
                                                   const int32_t *__restrict__ col,
                                                   const double *__restrict__ val,
                                                   const double *__restrict__ p,
                                                   double *__restrict__ q, CGScalars *cg,
                                                   double *part) {
  if (cg->done) return;
  __shared__ double sh[32];
  int lane = threadIdx.x & 31;
  int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int nw = (gridDim.x * blockDim.x) >> 5;
  double acc = 0.0;
  const int nrow = NC * nnode;
  for (int g = warp; g * 32 < nrow; g += nw) {
    const int row = g * 32 + lane;
    if (row < nrow) {
      const int node = row / NC;
      const double yv = spmv_lane_row<NC>(rp, col, val, p, node, row - NC * node);
      q[row] = yv;
      acc = fma(p[row], yv, acc);
    }
  }
  double s = block_sum<NT>(acc, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
  if (last_block(&cg->counter)) {
    double pq = sum_partials(part, gridDim.x, sh);
    if (threadIdx.x == 0) {
      cg->counter = 0;
      cg->pq = pq;
      if (!(pq > 0.0)) {
        cg->done = 2;
      } else {
        cg->alpha = cg->rz / pq;
      }
    }
  }
}

__global__ void __launch_bounds__(NT) k_cg_update_xr(int n, const double *__restrict__ p,
                                                     const double *__restrict__ q,
                                                     double *__restrict__ x,
                                                     double *__restrict__ r, CGScalars *cg,
                                                     double *part, double *alphas) {
  if (cg->done) return;
  __shared__ double sh[32];
  double alpha = cg->alpha;
  double acc = 0.0;
  for (int i = blockIdx.x * NT + threadIdx.x; i < n; i += gridDim.x * NT) {
    x[i] += alpha * p[i];
    double ri = r[i] - alpha * q[i];
    r[i] = ri;
    acc += ri * ri;
  }
  double s = block_sum<NT>(acc, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
  if (last_block(&cg->counter)) {
    double rr = sum_partials(part, gridDim.x, sh);
    if (threadIdx.x == 0) {
      cg->counter = 0;
      cg->rr = rr;
      int it = cg->it;
      if (alphas) alphas[it] = alpha;
      cg->it = it + 1;
      if (!(rr == rr)) cg->done = 2;
      else if (rr <= cg->tol2 * cg->bb) cg->done = 1;
      else if (it + 1 >= cg->maxit) cg->done = 3;
    }
  }
}

__global__ void __launch_bounds__(NT) k_cg_dots(int n, const double *__restrict__ r,
                                                const double *__restrict__ z,
                                                const double *__restrict__ q, CGScalars *cg,
                                                double *part, double *betas) {
  if (cg->done) return;
  __shared__ double sh[32];
  double a = 0.0, b = 0.0;
  for (int i = blockIdx.x * NT + threadIdx.x; i < n; i += gridDim.x * NT) {
    double zi = z[i];
    a += r[i] * zi;
    b += zi * q[i];
  }
  double sa = block_sum<NT>(a, sh);
  double sb = block_sum<NT>(b, sh);
  if (threadIdx.x == 0) {
    part[blockIdx.x] = sa;
    part[NB + blockIdx.x] = sb;
  }
  if (last_block(&cg->counter)) {
    double rz = sum_partials(part, gridDim.x, sh);
    double zq = sum_partials(part + NB, gridDim.x, sh);
    if (threadIdx.x == 0) {
      cg->counter = 0;
      double beta = cg->flexible ? -zq / cg->pq : rz / cg->rz;
      if (!(beta == beta) || !(rz == rz)) cg->done = 2;
      cg->beta = beta;
      cg->zq = zq;
      if (betas) betas[cg->it - 1] = beta;
      cg->rz = rz;
    }
  }
}

__global__ void __launch_bounds__(NT) k_cg_update_p(int n, const double *__restrict__ z,
                                                    double *__restrict__ p,
                                                    const CGScalars *cg) {
  if (cg->done) return;
  double beta = cg->beta;
  for (int i = blockIdx.x * NT + threadIdx.x; i < n; i += gridDim.x * NT)
    p[i] = z[i] + beta * p[i];
}

__global__ void __launch_bounds__(NT) k_cg_init(int n, const double *__restrict__ b,
                                                double *__restrict__ x,
                                                double *__restrict__ r, CGScalars *cg,
                                                double *part) {
  __shared__ double sh[32];
  double acc = 0.0;
  for (int i = blockIdx.x * NT + threadIdx.x; i < n; i += gridDim.x * NT) {
    double bi = b[i];
    x[i] = 0.0;
    r[i] = bi;
    acc += bi * bi;
  }
  double s = block_sum<NT>(acc, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
  if (last_block(&cg->counter)) {
    double bb = sum_partials(part, gridDim.x, sh);
    if (threadIdx.x == 0) {
      cg->counter = 0;
      cg->bb = bb;
      cg->rr = bb;
      cg->it = 0;
      cg->done = (bb == 0.0) ? 1 : 0;
    }
  }
}

__global__ void __launch_bounds__(NT) k_cg_init2(int n, const double *__restrict__ r,
                                                 const double *__restrict__ z,
                                                 double *__restrict__ p, CGScalars *cg,
                                                 double *part) {
  if (cg->done) return;
  __shared__ double sh[32];
  double acc = 0.0;
  for (int i = blockIdx.x * NT + threadIdx.x; i < n; i += gridDim.x * NT) {
    double zi = z[i];
    p[i] = zi;
    acc += r[i] * zi;
  }
  double s = block_sum<NT>(acc, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
  if (last_block(&cg->counter)) {
    double rz = sum_partials(part, gridDim.x, sh);
    if (threadIdx.x == 0) {
      cg->counter = 0;
      cg->rz = rz;
      if (!(rz == rz)) cg->done = 2;
    }
  }
}

__global__ void k_copy_if_running(int n, const double *__restrict__ src, double *__restrict__ dst,
                                  const CGScalars *cg) {
  if (cg && cg->done) return;
  for (int i = blockIdx.x * NT + threadIdx.x; i < n; i += gridDim.x * NT) dst[i] = src[i];
}

__global__ void __launch_bounds__(NT) k_norm2(int n, const double *__restrict__ v, double *out,
                                              double *part, unsigned *counter) {
  __shared__ double sh[32];
  double acc = 0.0;
  for (int i = blockIdx.x * NT + threadIdx.x; i < n; i += gridDim.x * NT) acc += v[i] * v[i];
  double s = block_sum<NT>(acc, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
  if (last_block(counter)) {
    double t = sum_partials(part, gridDim.x, sh);
    if (threadIdx.x == 0) {
      *counter = 0;
      *out = t;
    }
  }
}

__global__ void k_sub(int n, const double *__restrict__ a, const double *__restrict__ b,
                      double *__restrict__ out) {
  for (int i = blockIdx.x * NT + threadIdx.x; i < n; i += gridDim.x * NT) out[i] = a[i] - b[i];
}

// ---- batched steps over many instances ---------------------------------------
// A warp task is 32 consecutive scalar rows of one instance; task t belongs to
// the instance i with task_off[i] <= t < task_off[i + 1].  Every lane of a
// warp shares the task, so the instance and its `done` flag are warp-uniform.
// The per-task partial sums are added per instance by k_batch_reduce in a
// fixed order.

__device__ __forceinline__ int find_inst(const long long *off, int n, long long t) {
  int lo = 0, hi = n;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (off[mid] <= t) lo = mid;
    else hi = mid;
  }
  return lo;
}

// Calls f(B, i, row, global index) for this warp's rows; writes the two warp
// sums of the values f returns (a, b) as the task's partials.
template <bool SkipDone, typename F>
__device__ __forceinline__ void batch_rows(const BatchInst *inst, const long long *off, int n,
                                           long long ntask, const CGScalars *cg, double *tpart,
                                           F f) {
  const int lane = threadIdx.x & 31;
  const long long w0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long t = w0; t < ntask; t += nw) {
    const int i = find_inst(off, n, t);
    if (SkipDone && cg[i].done) continue;
    const BatchInst &B = inst[i];
    const int row = (int)(t - off[i]) * 32 + lane;
    double a = 0.0, b = 0.0;
    if (row < B.ndof) f(B, i, row, B.vbase + row, a, b);
    a = warp_sum(a);
    b = warp_sum(b);
    if (tpart && lane == 0) {
      tpart[2 * t] = a;
      tpart[2 * t + 1] = b;
    }
  }
}

__global__ void __launch_bounds__(256) k_batch_init(const BatchInst *inst, const long long *off,
                                                    int n, long long ntask,
                                                    const double *__restrict__ b,
                                                    double *__restrict__ x,
                                                    double *__restrict__ r, double *tpart) {
  batch_rows<false>(inst, off, n, ntask, nullptr, tpart,
                    [&](const BatchInst &, int, int, long long g, double &a, double &) {
                      const double bi = b[g];
                      x[g] = 0.0;
                      r[g] = bi;
                      a = bi * bi;
                    });
}

__global__ void __launch_bounds__(256) k_batch_init2(const BatchInst *inst, const long long *off,
                                                     int n, long long ntask, const CGScalars *cg,
                                                     const double *__restrict__ r,
                                                     const double *__restrict__ z,
                                                     double *__restrict__ p, double *tpart) {
  batch_rows<true>(inst, off, n, ntask, cg, tpart,
                   [&](const BatchInst &, int, int, long long g, double &a, double &) {
                     const double zi = z[g];
                     p[g] = zi;
                     a = r[g] * zi;
                   });
}

__global__ void __launch_bounds__(256, 8) k_batch_spmv_pq(const BatchInst *inst, const long long *off,
                                                       int n, long long ntask,
                                                       const CGScalars *cg,
                                                       const double *__restrict__ p,
                                                       double *__restrict__ q, double *tpart) {
  batch_rows<true>(inst, off, n, ntask, cg, tpart,
                   [&](const BatchInst &B, int, int row, long long g, double &a, double &) {
                     const double *pb = p + B.vbase;
                     double y;
                     if (B.nc == 3) {
                       const int node = row / 3;
                       y = spmv_lane_row<3>(B.row_ptr, B.col, B.val, pb, node, row - 3 * node);
                     } else {
                       y = spmv_lane_row<1>(B.row_ptr, B.col, B.val, pb, row, 0);
                     }
                     q[g] = y;
                     a = pb[row] * y;
                   });
}

__global__ void __launch_bounds__(256, 8) k_batch_residual(const BatchInst *inst,
                                                        const long long *off, int n,
                                                        long long ntask,
                                                        const double *__restrict__ x,
                                                        const double *__restrict__ bv,
                                                        double *tpart) {
  batch_rows<false>(inst, off, n, ntask, nullptr, tpart,
                    [&](const BatchInst &B, int, int row, long long g, double &a, double &) {
                      const double *xb = x + B.vbase;
                      double y;
                      if (B.nc == 3) {
                        const int node = row / 3;
                        y = spmv_lane_row<3>(B.row_ptr, B.col, B.val, xb, node, row - 3 * node);
                      } else {
                        y = spmv_lane_row<1>(B.row_ptr, B.col, B.val, xb, row, 0);
                      }
                      const double d = bv[g] - y;
                      a = d * d;
                    });
}

__global__ void __launch_bounds__(256) k_batch_update_xr(const BatchInst *inst,
                                                         const long long *off, int n,
                                                         long long ntask, const CGScalars *cg,
                                                         const double *__restrict__ p,
                                                         const double *__restrict__ q,
                                                         double *__restrict__ x,
                                                         double *__restrict__ r, double *tpart) {
  batch_rows<true>(inst, off, n, ntask, cg, tpart,
                   [&](const BatchInst &, int i, int, long long g, double &a, double &) {
                     const double alpha = cg[i].alpha;
                     x[g] += alpha * p[g];
                     const double ri = r[g] - alpha * q[g];
                     r[g] = ri;
                     a = ri * ri;
                   });
}

__global__ void __launch_bounds__(256) k_batch_dots(const BatchInst *inst, const long long *off,
                                                    int n, long long ntask, const CGScalars *cg,
                                                    const double *__restrict__ r,
                                                    const double *__restrict__ z,
                                                    const double *__restrict__ q,
                                                    double *tpart) {
  batch_rows<true>(inst, off, n, ntask, cg, tpart,
                   [&](const BatchInst &, int, int, long long g, double &a, double &b) {
                     const double zi = z[g];
                     a = r[g] * zi;
                     b = zi * q[g];
                   });
}

__global__ void __launch_bounds__(256) k_batch_update_p(const BatchInst *inst,
                                                        const long long *off, int n,
                                                        long long ntask, const CGScalars *cg,
                                                        const double *__restrict__ z,
                                                        double *__restrict__ p) {
  batch_rows<true>(inst, off, n, ntask, cg, nullptr,
                   [&](const BatchInst &, int i, int, long long g, double &, double &) {
                     p[g] = z[g] + cg[i].beta * p[g];
                   });
}

// One block per instance: the instance's task partials in a fixed order,
// then the scalar update of the step (the same rules as the single-system
// kernels above).
__global__ void __launch_bounds__(NT) k_batch_reduce(const long long *off, CGScalars *cgs,
                                                     const double *tpart, int kind,
                                                     double *alphas, double *betas, int hist,
                                                     double *out) {
  __shared__ double sh[32];
  const int i = blockIdx.x;
  CGScalars *cg = cgs + i;
  if (kind >= 1 && kind <= 4 && cg->done) return;
  double a = 0.0, b = 0.0;
  for (long long t = off[i] + threadIdx.x; t < off[i + 1]; t += NT) {
    a += tpart[2 * t];
    b += tpart[2 * t + 1];
  }
  a = block_sum<NT>(a, sh);
  b = block_sum<NT>(b, sh);
  if (threadIdx.x != 0) return;
  if (kind == 0) {
    cg->bb = a;
    cg->rr = a;
    cg->it = 0;
    cg->done = (a == 0.0) ? 1 : 0;
  } else if (kind == 1) {
    cg->rz = a;
    if (!(a == a)) cg->done = 2;
  } else if (kind == 2) {
    cg->pq = a;
    if (!(a > 0.0)) cg->done = 2;
    else cg->alpha = cg->rz / a;
  } else if (kind == 3) {
    cg->rr = a;
    const int it = cg->it;
    if (alphas && it < hist) alphas[(long long)i * hist + it] = cg->alpha;
    cg->it = it + 1;
    if (!(a == a)) cg->done = 2;
    else if (a <= cg->tol2 * cg->bb) cg->done = 1;
    else if (it + 1 >= cg->maxit) cg->done = 3;
  } else if (kind == 4) {
    const double beta = cg->flexible ? -b / cg->pq : a / cg->rz;
    if (!(beta == beta) || !(a == a)) cg->done = 2;
    cg->beta = beta;
    cg->zq = b;
    if (betas && cg->it - 1 < hist) betas[(long long)i * hist + cg->it - 1] = beta;
    cg->rz = a;
  } else if (out) {
    out[i] = a;
  }
}

}  // namespace

static unsigned batch_grid(long long ntask) {
  const long long blocks = (ntask + 7) / 8;          // 8 warps per block, one task each
  return (unsigned)std::max(1LL, std::min(blocks, (long long)NB * 8));
}

void launch_batch_init(const BatchInst *inst, const BatchTables &T, const double *b, double *x,
                       double *r, double *tpart, cudaStream_t s) {
  k_batch_init<<<batch_grid(T.ntask), 256, 0, s>>>(inst, T.task_off, T.n, T.ntask, b, x, r, tpart); GENEO_COUNT_LAUNCH();
}
void launch_batch_init2(const BatchInst *inst, const BatchTables &T, const CGScalars *cg,
                        const double *r, const double *z, double *p, double *tpart,
                        cudaStream_t s) {
  k_batch_init2<<<batch_grid(T.ntask), 256, 0, s>>>(inst, T.task_off, T.n, T.ntask, cg, r, z, p, tpart); GENEO_COUNT_LAUNCH();
}
void launch_batch_spmv_pq(const BatchInst *inst, const BatchTables &T, const CGScalars *cg,
                          const double *p, double *q, double *tpart, cudaStream_t s) {
  k_batch_spmv_pq<<<batch_grid(T.ntask), 256, 0, s>>>(inst, T.task_off, T.n, T.ntask, cg, p, q, tpart); GENEO_COUNT_LAUNCH();
}
void launch_batch_update_xr(const BatchInst *inst, const BatchTables &T, const CGScalars *cg,
                            const double *p, const double *q, double *x, double *r,
                            double *tpart, cudaStream_t s) {
  k_batch_update_xr<<<batch_grid(T.ntask), 256, 0, s>>>(inst, T.task_off, T.n, T.ntask, cg, p, q, x, r, tpart); GENEO_COUNT_LAUNCH();
}
void launch_batch_dots(const BatchInst *inst, const BatchTables &T, const CGScalars *cg,
                       const double *r, const double *z, const double *q, double *tpart,
                       cudaStream_t s) {
  k_batch_dots<<<batch_grid(T.ntask), 256, 0, s>>>(inst, T.task_off, T.n, T.ntask, cg, r, z, q, tpart); GENEO_COUNT_LAUNCH();
}
void launch_batch_update_p(const BatchInst *inst, const BatchTables &T, const CGScalars *cg,
                           const double *z, double *p, cudaStream_t s) {
  k_batch_update_p<<<batch_grid(T.ntask), 256, 0, s>>>(inst, T.task_off, T.n, T.ntask, cg, z, p); GENEO_COUNT_LAUNCH();
}
void launch_batch_residual(const BatchInst *inst, const BatchTables &T, const double *x,
                           const double *a, double *tpart, cudaStream_t s) {
  k_batch_residual<<<batch_grid(T.ntask), 256, 0, s>>>(inst, T.task_off, T.n, T.ntask, x, a, tpart); GENEO_COUNT_LAUNCH();
}
void launch_batch_reduce(const BatchInst *inst, const BatchTables &T, CGScalars *cg,
                         const double *tpart, int kind, double *alphas, double *betas,
                         int hist, double *out, cudaStream_t s) {
  (void)inst;
  k_batch_reduce<<<T.n, NT, 0, s>>>(T.task_off, cg, tpart, kind, alphas, betas, hist, out); GENEO_COUNT_LAUNCH();
}

void launch_spmv(const BSR &A, const double *x, double *y, cudaStream_t s) {
  if (A.nc == 1) {
    k_spmv<1><<<NB * 4, 256, 0, s>>>(A.nnode, A.row_ptr, A.col, A.val, x, y); GENEO_COUNT_LAUNCH();
  } else {
    k_spmv<3><<<NB * 4, 256, 0, s>>>(A.nnode, A.row_ptr, A.col, A.val, x, y); GENEO_COUNT_LAUNCH();
  }
}
void launch_cg_init(int n, const double *b, double *x, double *r, CGScalars *cg, double *part,
                    cudaStream_t s) {
  k_cg_init<<<NB, NT, 0, s>>>(n, b, x, r, cg, part); GENEO_COUNT_LAUNCH();
}
void launch_cg_init2(int n, const double *r, const double *z, double *p, CGScalars *cg,
                     double *part, cudaStream_t s) {
  k_cg_init2<<<NB, NT, 0, s>>>(n, r, z, p, cg, part); GENEO_COUNT_LAUNCH();
}
void launch_cg_spmv_pq(const BSR &A, const double *p, double *q, CGScalars *cg, double *part,
                       cudaStream_t s) {
  if (A.nc == 1) {
    k_cg_spmv_pq<1><<<NB * 4, NT, 0, s>>>(A.nnode, A.row_ptr, A.col, A.val, p, q, cg, part); GENEO_COUNT_LAUNCH();
  } else {
    k_cg_spmv_pq<3><<<NB * 4, NT, 0, s>>>(A.nnode, A.row_ptr, A.col, A.val, p, q, cg, part); GENEO_COUNT_LAUNCH();
  }
}
void launch_cg_update_xr(int n, const double *p, const double *q, double *x, double *r,
                         CGScalars *cg, double *part, double *alphas, cudaStream_t s) {
  k_cg_update_xr<<<NB, NT, 0, s>>>(n, p, q, x, r, cg, part, alphas); GENEO_COUNT_LAUNCH();
}
void launch_cg_dots(int n, const double *r, const double *z, const double *q, CGScalars *cg,
                    double *part, double *betas, cudaStream_t s) {
  k_cg_dots<<<NB, NT, 0, s>>>(n, r, z, q, cg, part, betas); GENEO_COUNT_LAUNCH();
}
void launch_cg_update_p(int n, const double *z, double *p, CGScalars *cg, cudaStream_t s) {
  k_cg_update_p<<<NB, NT, 0, s>>>(n, z, p, cg); GENEO_COUNT_LAUNCH();
}
void launch_copy_if_running(int n, const double *src, double *dst, const CGScalars *cg,
                            cudaStream_t s) {
  k_copy_if_running<<<NB, NT, 0, s>>>(n, src, dst, cg); GENEO_COUNT_LAUNCH();
}
void launch_norm2(int n, const double *v, double *out, double *part, unsigned *counter,
                  cudaStream_t s) {
  k_norm2<<<NB, NT, 0, s>>>(n, v, out, part, counter); GENEO_COUNT_LAUNCH();
}
void launch_sub(int n, const double *a, const double *b, double *out, cudaStream_t s) {
  k_sub<<<NB, NT, 0, s>>>(n, a, b, out); GENEO_COUNT_LAUNCH();
}

}  // namespace geneo
