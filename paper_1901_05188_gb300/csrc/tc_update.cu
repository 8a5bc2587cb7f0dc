// Trailing update of the FP32 band tile Cholesky on the tensor cores
// (mixed-precision subdomain factors, Sec. 3.1 local solves; the paper factors
// A_j with a sparse direct solver in double precision).
//
// For tile column J the update is A(J+d1, J+d2) -= P_d1 P_d2^T with the panel
// tiles P_d = L(J+d, J), 1 <= d2 <= d1 <= w: the lower block triangle of the
// product of the (32 w x 32) panel with itself.  One CTA computes a block of
// 4 x 4 tiles (128 x 128) with tcgen05.mma kind::tf32 into tensor memory and
// subtracts it from the tiles in global memory.  Each FP32 operand is split
// into a TF32 head and a TF32 tail, x = hi + lo, and the product is formed as
// hi*hi + hi*lo + lo*hi (three MMAs per k-step, FP32 accumulation), which
// keeps single-precision accuracy ("3xTF32").
//
// Shared-memory operands are K-major without swizzle: core matrices of 8 rows
// x 16 bytes, the two K-adjacent cores of one k-step 128 B apart (leading
// byte offset) and successive 8-row groups 1024 B apart (stride byte offset).
// One thread issues the MMAs and commits them to an mbarrier; every wait is
// bounded and a time-out is recorded in the device status word.
#include <cstdlib>

#include "band.cuh"

namespace geneo {

namespace {

constexpr int kTcM = 128, kTcK = 32;
constexpr int kTcOp = kTcM * kTcK * 4;         // 16 KB per operand buffer
constexpr int kTcSmem = 4 * kTcOp;             // A hi/lo, B hi/lo
constexpr int kTcThreads = 128;
constexpr int kTcWaitLimit = 1 << 24;

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ int core_off(int m, int k) {
  return (m >> 3) * 1024 + (k >> 2) * 128 + (m & 7) * 16 + (k & 3) * 4;
}
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  uint64_t d = (uint64_t)((addr & 0x3FFFF) >> 4);
  d |= (uint64_t)(128 >> 4) << 16;              // leading byte offset: next K core
  d |= (uint64_t)(1024 >> 4) << 32;             // stride byte offset: next 8 rows
  d |= (uint64_t)1 << 46;                       // tcgen05 descriptor version
  return d;                                     // no swizzle, base offset 0
}
__device__ __forceinline__ float to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}
__device__ __forceinline__ const float *tile_c(const float *base, const BandLayout &L, int I, int d) {
  return base + L.off + (((long long)I * (L.w + 1) + d) << 10);
}
__device__ __forceinline__ float *tile_m(float *base, const BandLayout &L, int I, int d) {
  return base + L.off + (((long long)I * (L.w + 1) + d) << 10);
}

// Block (a, b), b <= a, of the lower block triangle for update part `part`
// (0: all blocks, 1: block column 0, 2: block columns >= 1).
__device__ __forceinline__ void tc_block(int q, int part, int &a, int &b) {
  if (part == 1) {
    a = q;
    b = 0;
  } else if (part == 2) {
    a = 1;
    while (a * (a + 1) / 2 <= q) ++a;
    b = q - a * (a - 1) / 2 + 1;
  } else {
    a = 0;
    while ((a + 1) * (a + 2) / 2 <= q) ++a;
    b = q - a * (a + 1) / 2;
  }
}

// Stage the four panel tiles of block row `blk` (d = 4 blk + 1 .. 4 blk + 4)
// as the K-major TF32 head and tail operands; missing tiles are zero.
__device__ __forceinline__ void stage_panel(const float *pool, const BandLayout &L, int J, int blk,
                                            unsigned char *hi, unsigned char *lo) {
  for (int e = threadIdx.x; e < kTcM * kTcK; e += kTcThreads) {
    const int t = e >> 10, idx = e & 1023;        // tile of the block, element of the tile
    const int r = idx & 31, k = idx >> 5;         // column-major tile: (r, k) at k * 32 + r
    const int d = 4 * blk + 1 + t;
    float v = 0.f;
    if (d <= L.w && J + d < L.nt) v = tile_c(pool, L, J + d, d)[idx];
    const float h = to_tf32(v);
    const int off = core_off(32 * t + r, k);
    *reinterpret_cast<float *>(hi + off) = h;
    *reinterpret_cast<float *>(lo + off) = to_tf32(v - h);
  }
}

__global__ void __launch_bounds__(kTcThreads)
    k_chol_update_tc(const BandLayout *lay, int J, float *poolL, int part, DevStatus *status) {
  extern __shared__ __align__(1024) unsigned char smraw[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_base;
  const int j = blockIdx.x;
  const BandLayout L = lay[j];
  int a, b;
  tc_block(blockIdx.y, part, a, b);
  // nothing to do for this system: every tile of the block row is outside
  if (J >= L.nt || 4 * a + 1 > L.w || J + 4 * a + 1 >= L.nt) return;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  unsigned char *sAh = smraw, *sAl = smraw + kTcOp, *sBh = smraw + 2 * kTcOp,
                *sBl = smraw + 3 * kTcOp;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 128;"
                 ::"r"(smem_u32(&tmem_base)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)));
  stage_panel(poolL, L, J, a, sAh, sAl);
  stage_panel(poolL, L, J, b, sBh, sBl);
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;
  if (tid == 0) {
    // kind::tf32, D f32, A and B tf32 K-major, N = 128, M = 128
    const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kTcM >> 3) << 17) |
                           ((uint32_t)(kTcM >> 4) << 24);
    const uint32_t ah = smem_u32(sAh), al = smem_u32(sAl), bh = smem_u32(sBh), bl = smem_u32(sBl);
#pragma unroll
    for (int kk = 0; kk < kTcK / 8; ++kk) {
      const uint32_t ko = kk * 256;
      const uint64_t da[3] = {smem_desc(ah + ko), smem_desc(ah + ko), smem_desc(al + ko)};
      const uint64_t db[3] = {smem_desc(bh + ko), smem_desc(bl + ko), smem_desc(bh + ko)};
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const uint32_t acc = (kk == 0 && q == 0) ? 0u : 1u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n"
            ::"r"(tmem), "l"(da[q]), "l"(db[q]), "r"(idesc), "r"(acc));
      }
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 ::"r"(smem_u32(&mbar)) : "memory");
  }
  uint32_t done = 0;
  for (int it = 0; it < kTcWaitLimit && !done; ++it)
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n"
                 " selp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(done) : "r"(smem_u32(&mbar)) : "memory");
  if (!done && lane == 0) {
    if (atomicCAS(&status->code, 0, GENEO_ERR_TIMEOUT) == 0) {
      status->where = j;
      status->detail = J;
    }
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (done) {
    // warp w holds rows of tile d1 = 4a + 1 + w (TMEM lanes 32 w ..), lane = row
    const int d1 = 4 * a + 1 + warp;
    const bool row_ok = d1 <= L.w && J + d1 < L.nt;
#pragma unroll 1
    for (int cb = 0; cb < 4; ++cb) {
      uint32_t r[32];
      const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + cb * 32;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
          "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
            "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
            "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
            "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
            "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
            "=r"(r[31])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      const int d2 = 4 * b + 1 + cb;
      if (row_ok && d2 <= d1) {
        float *tc = tile_m(poolL, L, J + d1, d1 - d2);
#pragma unroll
        for (int c = 0; c < 32; ++c) tc[c * 32 + lane] -= __uint_as_float(r[c]);
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 128;" ::"r"(tmem));
  }
}

}  // namespace

int prepare_chol_update_tc() { return ensure_smem(k_chol_update_tc, kTcSmem); }

bool use_tensor_cores() {
  static const bool on = [] {
    const char *e = std::getenv("GENEO_TENSOR_CORES");
    return !(e && e[0] == '0');
  }();
  return on;
}

int launch_chol_update_tc(const BandLayout *d_lay, int nsys, int J, int w_max, float *poolL,
                          int part, DevStatus *status, cudaStream_t s) {
  const int rb = (w_max + 3) / 4;                 // block rows of 4 tiles
  int nblk = part == 1 ? rb : (part == 2 ? rb * (rb - 1) / 2 : rb * (rb + 1) / 2);
  if (nblk <= 0) return GENEO_OK;
  k_chol_update_tc<<<dim3(nsys, nblk), kTcThreads, kTcSmem, s>>>(d_lay, J, poolL, part, status);
  GENEO_COUNT_LAUNCH();
  return GENEO_OK;
}

}  // namespace geneo
