// BSR SpMV and the fused vector kernels of (flexible) PCG (Sec. 3.1).
//
// All reductions are two-stage and deterministic: every block writes one
// partial sum, and the last block to finish (ticket counter) adds the
// partials in a fixed order and updates the CG scalars on the device, so the
// iteration runs without host round trips and can be captured in a graph.
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

// One lane per matrix row: lane i of warp group g holds scalar row 32g + i
// (block row (32g + i) / NC, component (32g + i) % NC), so no lane idles; every
// stored value takes exactly one FMA and no sum crosses lanes -- FP64 issue,
// not bandwidth, is the scarce resource on this GPU, and a shuffle reduction
// costs FP64 adds.  The lanes of a block row read the rows of the same blocks
// and the same x entries, so their loads share L1 lines; results go to
// consecutive entries of y.

template <int NC>
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
#pragma unroll 9
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
__global__ void __launch_bounds__(256) k_spmv(int nnode, const int32_t *__restrict__ rp,
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
__global__ void __launch_bounds__(NT) k_cg_spmv_pq(int nnode, const int32_t *__restrict__ rp,
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

}  // namespace

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
