// Band-tiled Cholesky factors of the one-level additive Schwarz term
// sum_j R_j^T D_j A_j^-1 R_j  (Sec. 3.1, eqn:onelevelAS) and of the GenEO
// shift-invert operators (whose multi-right-hand-side solves run the local
// solves' look-ahead sweep), and the extraction of A_j from the global
// matrix.  The coarse correction and the
// gather are in coarse.cu, the cluster sweeps of the local solves in
// schwarz.cu.
//
// The paper factors A_j with a sparse direct solver (UMFPack).  Here each
// A_j is a band matrix in a box numbering whose longest axis runs slowest, held
// as dense 32 x 32 tiles; the factorisation is a right-looking tile Cholesky
// (one launch per tile column for the diagonal block, one for the panel, one
// for the trailing update, batched over all subdomains), and the diagonal
// blocks are stored inverted so both triangular sweeps become streams of
// small matrix-vector products.
#include "band.cuh"

namespace geneo {

namespace {

template <typename T>
__device__ __forceinline__ T *tile_ptr(T *base, const BandLayout &L, int I, int d) {
  return base + L.off + (((long long)I * (L.w + 1) + d) << 10);
}
template <typename T>
__device__ __forceinline__ const T *tile_ptr(const T *base, const BandLayout &L, int I, int d) {
  return base + L.off + (((long long)I * (L.w + 1) + d) << 10);
}

template <typename T>
__global__ void k_band_pad(const BandLayout *lay, int nsys, T *pool) {
  int j = blockIdx.x;
  if (j >= nsys) return;
  BandLayout L = lay[j];
  int last = L.nt - 1;
  for (int idx = L.n + threadIdx.x; idx < L.nt * 32; idx += blockDim.x) {
    int r = idx - last * 32;
    tile_ptr(pool, L, last, 0)[r * 32 + r] = T(1);
  }
}

// ---- tile Cholesky ---------------------------------------------------------

// 1/sqrt(d) for d > 0: single-precision estimate refined by Newton's iteration
// for f(y) = 1/y^2 - d, y <- y (3 - d y^2) / 2, which doubles the number of
// correct bits per step (24 -> 48 -> full double).  The pivot is on the serial
// path of the diagonal-block factorisation, where a few dependent FP64
// operations are much cheaper than a correctly rounded square root and
// division; the factor only needs the pivot to working precision.
__device__ __forceinline__ double inv_sqrt_pos(double d) {
  double y = (double)rsqrtf((float)d);
  if (!(d >= 1e-30 && d <= 1e30)) return 1.0 / sqrt(d);   // outside float range: exact path
  y = y * (1.5 - 0.5 * d * y * y);
  y = y * (1.5 - 0.5 * d * y * y);
  return y;
}
__device__ __forceinline__ float inv_sqrt_pos(float d) {
  float y = rsqrtf(d);
  return y * (1.5f - 0.5f * d * y * y);
}

template <typename T>
__global__ void __launch_bounds__(1024) k_chol_diag(const BandLayout *lay, int nsys, int J,
                                                    T *poolL, T *poolU, DevStatus *st) {
  int j = blockIdx.x;
  BandLayout L = lay[j];
  if (J >= L.nt) return;
  __shared__ T A[32][33];
  __shared__ T X[32][33];
  __shared__ T Y[32][33];
  __shared__ T piv[2];
  __shared__ int bad;
  const int tid = threadIdx.x, r = tid & 31, cc = tid >> 5;   // thread (r, cc) owns entry (r, cc)
  T *t = tile_ptr(poolL, L, J, 0);
  A[r][cc] = t[cc * 32 + r];
  if (tid == 0) bad = -1;
  __syncthreads();
  // right-looking Cholesky, one entry per thread: three barriers per column
  for (int k = 0; k < 32; ++k) {
    if (tid == 0) {
      T d = A[k][k];
      if (!(d > T(0))) {
        if (bad < 0) bad = J * 32 + k;
        d = T(1);
      }
      const T y = inv_sqrt_pos(d);
      piv[0] = d * y;          // sqrt(d)
      piv[1] = y;              // 1 / sqrt(d)
    }
    __syncthreads();
    if (cc == k && r >= k) A[r][k] = (r == k) ? piv[0] : A[r][k] * piv[1];
    __syncthreads();
    if (cc > k && r >= cc) A[r][cc] -= A[r][k] * A[cc][k];
    __syncthreads();
  }
  // inverse of the lower-triangular factor by recursive doubling:
  // inv([[P, 0], [Q, R]]) = [[iP, 0], [-iR Q iP, iR]]
  X[r][cc] = (r == cc) ? T(1) / A[r][r] : T(0);
  __syncthreads();
  for (int b = 1; b < 32; b <<= 1) {
    // pairs of b x b diagonal blocks at s and s + b, s = multiple of 2b
    const int s = (r / (2 * b)) * (2 * b);
    const bool lower = (r >= s + b) && (cc >= s) && (cc < s + b);   // block (R-row, P-col)
    T v = T(0);
    if (lower) {   // Y = Q iP  (Q = A[s+b.., s..s+b), iP = X[s.., s..])
      for (int k = cc; k < s + b; ++k) v += A[r][k] * X[k][cc];
    }
    Y[r][cc] = v;
    __syncthreads();
    if (lower) {   // X_lower = -iR Y
      T w = T(0);
      for (int k = s + b; k <= r; ++k) w += X[r][k] * Y[k][cc];
      X[r][cc] = -w;
    }
    __syncthreads();
  }
  T *u = tile_ptr(poolU, L, J, 0);
  t[cc * 32 + r] = X[r][cc];    // inv(L_JJ), column-major
  u[cc * 32 + r] = X[cc][r];    // inv(L_JJ)^T
  if (tid == 0 && bad >= 0) {
    if (atomicCAS(&st->code, 0, GENEO_ERR_NOT_SPD) == 0) {
      st->where = j;
      st->detail = bad;
    }
  }
}

// L(J+d, J) = A(J+d, J) inv(L_JJ)^T for d = 1..w (blockIdx.y = d - 1).
template <typename T>
__global__ void __launch_bounds__(256) k_chol_trsm(const BandLayout *lay, int nsys, int J,
                                                   T *poolL, T *poolU) {
  int j = blockIdx.x, d = blockIdx.y + 1;
  BandLayout L = lay[j];
  if (J >= L.nt || d > L.w || J + d >= L.nt) return;
  __shared__ T Aa[32][33];
  __shared__ T D[32][33];
  T *ta = tile_ptr(poolL, L, J + d, d);
  const T *td = tile_ptr(poolL, L, J, 0);
  for (int e = threadIdx.x; e < 1024; e += 256) {
    Aa[e & 31][e >> 5] = ta[e];
    D[e & 31][e >> 5] = td[e];
  }
  __syncthreads();
  T *tu = tile_ptr(poolU, L, J, d);
  for (int e = threadIdx.x; e < 1024; e += 256) {
    int r = e & 31, c = e >> 5;
    T s = T(0);
    for (int k = 0; k <= c; ++k) s += Aa[r][k] * D[c][k];
    ta[e] = s;                 // (r, c) column-major
    tu[r * 32 + c] = s;        // transposed: U(J, d)(c, r) = L(J+d, J)(r, c)
  }
}

// A(J+d1, J+d2) -= L(J+d1, J) L(J+d2, J)^T, 1 <= d2 <= d1 <= w.
// part 0: every pair; part 1: the next tile column only (d2 = 1, blockIdx.y =
// d1 - 1); part 2: the rest (d2 >= 2).
template <typename T>
__global__ void __launch_bounds__(256) k_chol_update(const BandLayout *lay, int nsys, int J,
                                                     T *poolL, int part) {
  int j = blockIdx.x;
  BandLayout L = lay[j];
  int p = blockIdx.y;
  int d1, d2;
  if (part == 1) {
    d1 = p + 1;
    d2 = 1;
  } else if (part == 2) {
    d1 = 2;
    while (d1 * (d1 - 1) / 2 <= p) ++d1;
    d2 = p - (d1 - 1) * (d1 - 2) / 2 + 2;
  } else {
    d1 = 1;
    while ((d1 + 1) * d1 / 2 <= p) ++d1;
    d2 = p - d1 * (d1 - 1) / 2 + 1;
  }
  if (J >= L.nt || d1 > L.w || J + d1 >= L.nt) return;
  __shared__ T Aa[32][33];
  __shared__ T Bb[32][33];
  const T *ta = tile_ptr(poolL, L, J + d1, d1);
  const T *tb = tile_ptr(poolL, L, J + d2, d2);
  for (int e = threadIdx.x; e < 1024; e += 256) {
    Aa[e & 31][e >> 5] = ta[e];
    Bb[e & 31][e >> 5] = tb[e];
  }
  __syncthreads();
  T *tc = tile_ptr(poolL, L, J + d1, d1 - d2);
  for (int e = threadIdx.x; e < 1024; e += 256) {
    int r = e & 31, c = e >> 5;
    T s = T(0);
#pragma unroll 8
    for (int k = 0; k < 32; ++k) s += Aa[r][k] * Bb[c][k];
    tc[e] -= s;
  }
}

// ---- extraction of A_j from the global BSR ----------------------------------

template <typename T>
__global__ void k_extract_interior(const SubDesc *subs, const BandLayout *lay, int nnx,
                                   int nny, int nnz, const int32_t *__restrict__ rp,
                                   const double *__restrict__ val, T *pool) {
  const int j = blockIdx.y;
  const SubDesc &S = subs[j];
  const BandLayout L = lay[j];
  const int nn = S.ibox.count();
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)nn * 27) return;
  int l = (int)(t / 27), s = (int)(t % 27);
  int gi, gj, gk;
  S.ibox.global(l, gi, gj, gk);
  int di = s % 3 - 1, dj = (s / 3) % 3 - 1, dk = s / 9 - 1;
  int l2 = S.ibox.local(gi + di, gj + dj, gk + dk);
  if (l2 < 0 || l2 > l) return;
  int g = gi + nnx * (gj + nny * gk);
  // position of slot s in the global row: count valid slots before it
  int pos = rp[g];
  for (int q = 0; q < s; ++q) {
    int qi = gi + q % 3 - 1, qj = gj + (q / 3) % 3 - 1, qk = gk + q / 9 - 1;
    pos += ((unsigned)qi < (unsigned)nnx && (unsigned)qj < (unsigned)nny &&
            (unsigned)qk < (unsigned)nnz);
  }
  const int nc = S.nc;
  const double *blk = val + (size_t)nc * nc * pos;
  for (int rr = 0; rr < nc; ++rr)
    for (int cc = 0; cc < nc; ++cc) {
      int R = nc * l + rr, C = nc * l2 + cc;
      if (R < C) continue;
      int I = R >> 5, J = C >> 5;
      tile_ptr(pool, L, I, I - J)[(C & 31) * 32 + (R & 31)] = T(blk[nc * rr + cc]);
    }
}

}  // namespace

// ---- launchers ----------------------------------------------------------------

template <typename T>
int launch_band_clear(const BandLayout *d_lay, int nsys, T *pool, long long pool_elems,
                      cudaStream_t s) {
  GENEO_CUDA_TRY(cudaMemsetAsync(pool, 0, pool_elems * sizeof(T), s));
  k_band_pad<T><<<nsys, 32, 0, s>>>(d_lay, nsys, pool); GENEO_COUNT_LAUNCH();
  GENEO_CUDA_TRY(cudaGetLastError());
  return GENEO_OK;
}

// Trailing update of tile column J (part 0 all pairs, 1 the next tile column,
// 2 the rest): FP32 factors on the tensor cores (3xTF32), FP64 on the FMA units.
template <typename T>
int launch_update(const BandLayout *d_lay, int nsys, int J, int w_max, T *poolL, int part,
                  DevStatus *st, cudaStream_t s) {
  const int npairs = w_max * (w_max + 1) / 2;
  if constexpr (sizeof(T) == 4) {
    if (use_tensor_cores()) return launch_chol_update_tc(d_lay, nsys, J, w_max, poolL, part, st, s);
  }
  const int ny = part == 1 ? w_max : (part == 2 ? npairs - w_max : npairs);
  if (ny > 0) {
    k_chol_update<T><<<dim3(nsys, ny), 256, 0, s>>>(d_lay, nsys, J, poolL, part); GENEO_COUNT_LAUNCH();
  }
  return GENEO_OK;
}

template <typename T>
int launch_band_cholesky(const BandLayout *d_lay, int nsys, int nt_max, int w_max, T *poolL,
                         T *poolU, DevStatus *st, cudaStream_t s, cudaStream_t side) {
  int rc;
  if constexpr (sizeof(T) == 4) {
    if (use_tensor_cores() && (rc = prepare_chol_update_tc())) return rc;
  }
  if (!side || w_max == 0) {
    for (int J = 0; J < nt_max; ++J) {
      k_chol_diag<T><<<nsys, 1024, 0, s>>>(d_lay, nsys, J, poolL, poolU, st); GENEO_COUNT_LAUNCH();
      if (w_max > 0) {
        k_chol_trsm<T><<<dim3(nsys, w_max), 256, 0, s>>>(d_lay, nsys, J, poolL, poolU); GENEO_COUNT_LAUNCH();
        if ((rc = launch_update<T>(d_lay, nsys, J, w_max, poolL, 0, st, s))) return rc;
      }
    }
    GENEO_CUDA_TRY(cudaGetLastError());
    return GENEO_OK;
  }
  // Look-ahead: once tile column J+1 has received its update from column J
  // (part 1), its diagonal block and panel are factored on the side stream
  // while the main stream applies the rest of column J's trailing update.
  cudaEvent_t e_main, e_side;
  GENEO_CUDA_TRY(cudaEventCreateWithFlags(&e_main, cudaEventDisableTiming));
  GENEO_CUDA_TRY(cudaEventCreateWithFlags(&e_side, cudaEventDisableTiming));
  k_chol_diag<T><<<nsys, 1024, 0, s>>>(d_lay, nsys, 0, poolL, poolU, st); GENEO_COUNT_LAUNCH();
  k_chol_trsm<T><<<dim3(nsys, w_max), 256, 0, s>>>(d_lay, nsys, 0, poolL, poolU); GENEO_COUNT_LAUNCH();
  for (int J = 0; J + 1 < nt_max; ++J) {
    if ((rc = launch_update<T>(d_lay, nsys, J, w_max, poolL, 1, st, s))) return rc;
    GENEO_CUDA_TRY(cudaEventRecord(e_main, s));
    GENEO_CUDA_TRY(cudaStreamWaitEvent(side, e_main, 0));
    k_chol_diag<T><<<nsys, 1024, 0, side>>>(d_lay, nsys, J + 1, poolL, poolU, st); GENEO_COUNT_LAUNCH();
    k_chol_trsm<T><<<dim3(nsys, w_max), 256, 0, side>>>(d_lay, nsys, J + 1, poolL, poolU); GENEO_COUNT_LAUNCH();
    if ((rc = launch_update<T>(d_lay, nsys, J, w_max, poolL, 2, st, s))) return rc;
    GENEO_CUDA_TRY(cudaEventRecord(e_side, side));
    GENEO_CUDA_TRY(cudaStreamWaitEvent(s, e_side, 0));
  }
  cudaEventDestroy(e_main);
  cudaEventDestroy(e_side);
  GENEO_CUDA_TRY(cudaGetLastError());
  return GENEO_OK;
}

// The GenEO eigensolver's multi-right-hand-side solves run the one-CTA
// look-ahead sweep of the local solves (schwarz.cu), one CTA per (system,
// right-hand side), the column in shared memory, or streamed through a ring
// of tile rows when it does not fit.
int launch_band_solve_dense(const BandLayout *d_lay, int nsys, int npad_max, int w_max,
                            int ring, const double *poolL, const double *poolU, const double *in,
                            long long in_sys, int in_row, double *out, long long out_sys,
                            int out_row, int ncols, int mode, cudaStream_t s) {
  return launch_band_solve_la(d_lay, nsys, npad_max, w_max, ring, poolL, poolU, in, in_sys,
                              in_row, out, out_sys, out_row, ncols, mode, s);
}

template <typename T>
int launch_extract_interior(const SubDesc *d_subs, const BandLayout *d_lay, int nsub,
                            int max_nodes, int nnx, int nny, int nnz, const int32_t *rp,
                            const double *val, T *pool, cudaStream_t s) {
  long long tot = (long long)max_nodes * 27;
  dim3 grid((unsigned)((tot + 255) / 256), nsub);
  k_extract_interior<T><<<grid, 256, 0, s>>>(d_subs, d_lay, nnx, nny, nnz, rp, val, pool); GENEO_COUNT_LAUNCH();
  GENEO_CUDA_TRY(cudaGetLastError());
  return GENEO_OK;
}

template int launch_band_clear<double>(const BandLayout *, int, double *, long long, cudaStream_t);
template int launch_band_clear<float>(const BandLayout *, int, float *, long long, cudaStream_t);
template int launch_band_cholesky<double>(const BandLayout *, int, int, int, double *, double *,
                                          DevStatus *, cudaStream_t, cudaStream_t);
template int launch_band_cholesky<float>(const BandLayout *, int, int, int, float *, float *,
                                         DevStatus *, cudaStream_t, cudaStream_t);
template int launch_extract_interior<double>(const SubDesc *, const BandLayout *, int, int, int,
                                             int, int, const int32_t *, const double *,
                                             double *, cudaStream_t);
template int launch_extract_interior<float>(const SubDesc *, const BandLayout *, int, int, int,
                                            int, int, const int32_t *, const double *, float *,
                                            cudaStream_t);
}  // namespace geneo
