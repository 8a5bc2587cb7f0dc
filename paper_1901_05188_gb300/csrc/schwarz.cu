// One-level additive Schwarz local solves (Sec. 3.1, eqn:onelevelAS) with one
// thread-block cluster per subdomain.
//
// Each of the C CTAs of a cluster keeps a full copy of the local vector y_j in
// shared memory and owns the band tiles d = 1 + c + kC of every tile row.  A
// step of a sweep: every CTA multiplies its tiles with the already solved
// blocks of y, pushes its 32 partial sums into the partial buffer of every
// CTA of the cluster (distributed shared memory), one cluster barrier, then
// every CTA applies the inverted diagonal block to y_I - sum of partials
// itself, so y_I appears in all copies without a second exchange.  Tiles of
// the next step are loaded into registers during the barrier phase and the
// step after that is prefetched into L2.
#include <cooperative_groups.h>

#include "band.cuh"

namespace cg = cooperative_groups;

namespace geneo {

namespace {

constexpr int kClWarps = 16;        // warp 0: diagonal block; warps 1..15: off-diagonal tiles
constexpr int kGroups = 4;          // a tile is split into 4 units of 8 columns

template <typename T>
__device__ __forceinline__ const T *tile_at(const T *base, const BandLayout &L, int I, int d) {
  return base + L.off + (((long long)I * (L.w + 1) + d) << 10);
}

__device__ __forceinline__ void prefetch_l2(const void *p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// The unit u = (t, g) of CTA c in tile row I: tile d = 1 + c + t*C, columns 8g..8g+7.
template <int C>
__device__ __forceinline__ int unit_tile(int u, int c) {
  return 1 + c + (u / kGroups) * C;
}

template <typename T, int C>
__device__ void cluster_sweep(const cg::cluster_group &cluster, const T *__restrict__ pool,
                              const BandLayout &L, T *y, T *red, T *part, bool backward) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int c = (int)cluster.block_rank();
  const int nt = L.nt, w = L.w;
  const int cw = warp - 1;                      // compute-warp index (-1 for warp 0)
  constexpr int kLinesPerUnit = 8 * 32 * (int)sizeof(T) / 128;
  T nx[8];                                      // register copy of the next step's first unit
  auto dmax_of = [&](int I) { return backward ? min(w, nt - 1 - I) : min(w, I); };
  auto row_of = [&](int step) { return backward ? nt - 1 - step : step; };
  auto load_unit = [&](int I, int u, T *dst) {
    const int d = unit_tile<C>(u, c);
    if (cw < 0 || d > dmax_of(I)) return;
    const T *t = tile_at(pool, L, I, d) + (u % kGroups) * 8 * 32;
#pragma unroll
    for (int k = 0; k < 8; ++k) dst[k] = __ldg(t + k * 32 + lane);
  };
  if (nt > 0) load_unit(row_of(0), cw, nx);
  T dv[32];                                     // warp 0: inverted diagonal tile, lane's row
  if (warp == 0 && nt > 0) {
    const T *D = tile_at(pool, L, row_of(0), 0);
#pragma unroll
    for (int k = 0; k < 32; ++k) dv[k] = __ldg(D + k * 32 + lane);
  }
  for (int step = 0; step < nt; ++step) {
    const int I = row_of(step);
    const int dm = dmax_of(I);
    const int par = step & 1;
    if (step + 2 < nt && cw >= 0) {             // L2 prefetch two steps ahead
      const int I2 = row_of(step + 2);
      for (int u = cw; unit_tile<C>(u, c) <= dmax_of(I2); u += kClWarps - 1)
        if (lane < kLinesPerUnit)
          prefetch_l2(tile_at(pool, L, I2, unit_tile<C>(u, c)) + (u % kGroups) * 256 +
                      lane * (128 / sizeof(T)));
    }
    T a0 = T(0), a1 = T(0);
    if (cw >= 0) {
      for (int u = cw; unit_tile<C>(u, c) <= dm; u += kClWarps - 1) {
        const int d = unit_tile<C>(u, c);
        const T *yJ = y + (backward ? (I + d) : (I - d)) * 32 + (u % kGroups) * 8;
        T v[8];
        if (u == cw) {
#pragma unroll
          for (int k = 0; k < 8; ++k) v[k] = nx[k];
        } else {
          const T *t = tile_at(pool, L, I, d) + (u % kGroups) * 8 * 32;
#pragma unroll
          for (int k = 0; k < 8; ++k) v[k] = __ldg(t + k * 32 + lane);
        }
#pragma unroll
        for (int k = 0; k < 8; k += 2) {
          a0 += v[k] * yJ[k];
          a1 += v[k + 1] * yJ[k + 1];
        }
      }
      if (step + 1 < nt) load_unit(row_of(step + 1), cw, nx);   // in flight over the barrier
    }
    red[warp * 32 + lane] = a0 + a1;
    __syncthreads();
    if (warp == 0) {
      T s = T(0);
#pragma unroll
      for (int k = 1; k < kClWarps; ++k) s += red[k * 32 + lane];
#pragma unroll
      for (int q = 0; q < C; ++q) {
        T *dst = cluster.map_shared_rank(part, q);
        dst[(par * C + c) * 32 + lane] = s;
      }
    }
    cluster.sync();
    if (warp == 0) {
      T s = y[I * 32 + lane];
#pragma unroll
      for (int q = 0; q < C; ++q) s -= part[(par * C + q) * 32 + lane];
      red[lane] = s;
      __syncwarp();
      T o0 = T(0), o1 = T(0), o2 = T(0), o3 = T(0);
#pragma unroll
      for (int k = 0; k < 32; k += 4) {
        o0 += dv[k] * red[k];
        o1 += dv[k + 1] * red[k + 1];
        o2 += dv[k + 2] * red[k + 2];
        o3 += dv[k + 3] * red[k + 3];
      }
      y[I * 32 + lane] = (o0 + o1) + (o2 + o3);
      if (step + 1 < nt) {
        const T *D = tile_at(pool, L, row_of(step + 1), 0);
#pragma unroll
        for (int k = 0; k < 32; ++k) dv[k] = __ldg(D + k * 32 + lane);
      }
    }
    __syncthreads();
  }
}

template <typename T, int C>
__global__ void __launch_bounds__(kClWarps * 32)
    k_schwarz_cluster(const SubDesc *subs, const BandLayout *lay, int nnx, int nny,
                      const T *poolL, const T *poolU, const double *__restrict__ r,
                      T *__restrict__ xloc, const CGScalars *cgs) {
  if (cgs && cgs->done) return;           // the same for every CTA of the cluster
  cg::cluster_group cluster = cg::this_cluster();
  extern __shared__ __align__(16) unsigned char smraw[];
  T *red = reinterpret_cast<T *>(smraw);  // [kClWarps][32]
  T *part = red + kClWarps * 32;          // [2][C][32]
  T *y = part + 2 * C * 32;               // [npad]
  const int j = blockIdx.x / C;
  const SubDesc &S = subs[j];
  const BandLayout L = lay[j];
  const int n = S.n_int, npad = L.nt * 32;
  for (int l = threadIdx.x; l < npad; l += blockDim.x) {
    T v = T(0);
    if (l < n) {
      int node = l / 3, comp = l - 3 * node;
      int gi, gj, gk;
      S.ibox.global(node, gi, gj, gk);
      v = T(r[3 * (gi + nnx * (gj + nny * gk)) + comp]);
    }
    y[l] = v;
  }
  cluster.sync();                          // every CTA's shared memory is live
  cluster_sweep<T, C>(cluster, poolL, L, y, red, part, false);
  cluster_sweep<T, C>(cluster, poolU, L, y, red, part, true);
  if (cluster.block_rank() == 0) {
    T *out = xloc + S.v_int;
    for (int l = threadIdx.x; l < n; l += blockDim.x) out[l] = y[l];
  }
  cluster.sync();                          // no CTA leaves while others may still write to it
}

template <typename T>
int smem_bytes(int npad, int C) {
  return (kClWarps * 32 + 2 * C * 32 + npad) * (int)sizeof(T);
}

template <typename T, int C>
int launch_c(const SubDesc *d_subs, const BandLayout *d_lay, int nsub, int npad_max, int nnx,
             int nny, const T *poolL, const T *poolU, const double *r, T *xloc,
             const CGScalars *cgs, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(nsub * C);
  cfg.blockDim = dim3(kClWarps * 32);
  cfg.dynamicSmemBytes = smem_bytes<T>(npad_max, C);
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  GENEO_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_schwarz_cluster<T, C>, d_subs, d_lay, nnx, nny,
                                    poolL, poolU, r, xloc, cgs));
  GENEO_COUNT_LAUNCH();
  return GENEO_OK;
}

template <typename T, int C>
int prepare_c(int npad_max) {
  return ensure_smem(k_schwarz_cluster<T, C>, smem_bytes<T>(npad_max, C));
}

}  // namespace

int schwarz_cluster_size(int nsub, int sm_count) {
  // one CTA per SM; the largest power-of-two cluster that leaves half the
  // SMs' worth of headroom (measured best on the 32-subdomain workload: 4)
  int c = 1;
  while (c < 8 && nsub * (2 * c) <= sm_count) c *= 2;
  return c;
}

template <typename T>
int prepare_schwarz_solve(int npad_max) {
  if (smem_bytes<T>(npad_max, 8) > 227 * 1024) return GENEO_ERR_INVALID_ARG;
  int st;
  if ((st = prepare_c<T, 1>(npad_max))) return st;
  if ((st = prepare_c<T, 2>(npad_max))) return st;
  if ((st = prepare_c<T, 4>(npad_max))) return st;
  return prepare_c<T, 8>(npad_max);
}

template <typename T>
int launch_schwarz_solve(const SubDesc *d_subs, const BandLayout *d_lay, int nsub, int npad_max,
                         int nnx, int nny, const T *poolL, const T *poolU, const double *r,
                         T *xloc, const CGScalars *cgs, int cluster, DevStatus *status,
                         cudaStream_t s) {
  (void)status;
  switch (cluster) {
    case 8: return launch_c<T, 8>(d_subs, d_lay, nsub, npad_max, nnx, nny, poolL, poolU, r, xloc, cgs, s);
    case 4: return launch_c<T, 4>(d_subs, d_lay, nsub, npad_max, nnx, nny, poolL, poolU, r, xloc, cgs, s);
    case 2: return launch_c<T, 2>(d_subs, d_lay, nsub, npad_max, nnx, nny, poolL, poolU, r, xloc, cgs, s);
    default: return launch_c<T, 1>(d_subs, d_lay, nsub, npad_max, nnx, nny, poolL, poolU, r, xloc, cgs, s);
  }
}

template int prepare_schwarz_solve<double>(int);
template int prepare_schwarz_solve<float>(int);
template int launch_schwarz_solve<double>(const SubDesc *, const BandLayout *, int, int, int, int,
                                          const double *, const double *, const double *,
                                          double *, const CGScalars *, int, DevStatus *,
                                          cudaStream_t);
template int launch_schwarz_solve<float>(const SubDesc *, const BandLayout *, int, int, int, int,
                                         const float *, const float *, const double *, float *,
                                         const CGScalars *, int, DevStatus *, cudaStream_t);

}  // namespace geneo
