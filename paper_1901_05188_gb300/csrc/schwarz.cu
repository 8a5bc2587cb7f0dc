// One-level additive Schwarz local solves (Sec. 3.1, eqn:onelevelAS) with one
// thread-block cluster per subdomain.
//
// Each of the C CTAs of a cluster keeps a full copy of the local vector y_j in
// shared memory and owns the band tiles d = 1 + c + kC of every tile row.  A
// step of a sweep solves R consecutive tile rows I_0..I_{R-1}.  All warps
// multiply their tiles with the already solved blocks of y (the "far" tiles:
// row I_r, distance d > r); per-CTA partial sums go into the partial buffer of
// every CTA of the cluster (distributed shared memory); one cluster barrier;
// then the chain warps of every CTA finish the R rows themselves: subtract the
// partials, the couplings inside the group (L(I_r, I_r-d), d <= r) and apply
// the inverted diagonal block, so each y_I appears in all copies without a
// second exchange.  The chain runs on four warps (one per SM sub-partition),
// each taking 8 of the 32 columns of every chain tile, because on this GPU a
// warp's dependent FP64 instructions are the critical path.  Tiles of the next
// step are loaded into registers during the barrier phase and the step after
// that is prefetched into L2.
//
// Three other forms of the same sweep follow, all chosen among by the set-up
// autotuner: the look-ahead sweep (far warps multiply row I+1 while the chain
// finishes row I, one split cluster barrier per row); and the staged forms,
// where one thread copies each step's tiles into shared memory a step ahead
// (cp.async.bulk completed on an mbarrier) and the per-CTA partials travel by
// st.async into every CTA's buffer, completing a transaction count on that
// CTA's mbarrier, so no cluster barrier remains inside a sweep (R rows per
// step, or the look-ahead order where the far warps push row I+1's partial
// while the chain finishes row I).
#include <cooperative_groups.h>

#include "band.cuh"
#include "batch.cuh"

namespace cg = cooperative_groups;

namespace geneo {

namespace {

constexpr int kClWarps = 16;        // all warps multiply far tiles
constexpr int kChain = 4;           // warps 0..3 also run the per-row chain
constexpr int kGroups = 4;          // a tile is split into 4 units of 8 columns

template <typename T>
__device__ __forceinline__ const T *tile_at(const T *base, const BandLayout &L, int I, int d) {
  return base + L.off + (((long long)I * (L.w + 1) + d) << 10);
}

__device__ __forceinline__ void prefetch_l2(const void *p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

__device__ __forceinline__ void chain_bar() {
  asm volatile("bar.sync 1, %0;" ::"n"(kChain * 32) : "memory");
}

// Far tiles of row r of a step owned by CTA c: d = 1 + c + t*C for t in
// [t0, t0 + n), with r + 1 <= d <= dmax.
template <int C>
__device__ __forceinline__ void far_tiles(int r, int dmax, int c, int &t0, int &n) {
  t0 = (r > c) ? (r - c + C - 1) / C : 0;
  const int d0 = 1 + c + t0 * C;
  n = (dmax >= d0) ? (dmax - d0) / C + 1 : 0;
}

template <typename T, int C, int R>
struct Sweep {
  static constexpr int kNearSlots = R > 1 ? R * (R - 1) / 2 : 1;
  const T *pool;
  BandLayout L;
  int c, nt, w;
  bool backward;

  __device__ __forceinline__ bool valid(int step, int r) const { return step * R + r < nt; }
  __device__ __forceinline__ int row(int step, int r) const {
    const int q = step * R + r;
    return backward ? nt - 1 - q : q;
  }
  __device__ __forceinline__ int dmax(int I) const {
    return backward ? min(w, nt - 1 - I) : min(w, I);
  }
  // unit u of a step -> (r, d, g); false if the step has fewer units
  __device__ __forceinline__ bool unit(int step, int u, int &r, int &d, int &g) const {
#pragma unroll
    for (int q = 0; q < R; ++q) {
      if (!valid(step, q)) return false;
      int t0, n;
      far_tiles<C>(q, dmax(row(step, q)), c, t0, n);
      if (u < kGroups * n) {
        r = q;
        d = 1 + c + (t0 + u / kGroups) * C;
        g = u % kGroups;
        return true;
      }
      u -= kGroups * n;
    }
    return false;
  }
  __device__ __forceinline__ const T *unit_ptr(int step, int r, int d, int g) const {
    return tile_at(pool, L, row(step, r), d) + g * 8 * 32;
  }
};

// Second half of a step, shared by the sweeps that load their tiles from
// global memory and from shared-memory stages: per-CTA partials of the far
// products to every CTA of the cluster, one cluster barrier, then the chain
// warps finish the R rows (partials, couplings inside the group, inverted
// diagonal block) and write y_I.
template <typename T, int C, int R>
__device__ __forceinline__ void step_tail(const cg::cluster_group &cluster,
                                          const Sweep<T, C, R> &S, int step, T (&acc)[R][2],
                                          const T (&dv)[R][8],
                                          const T (&nv)[Sweep<T, C, R>::kNearSlots][8], T *y,
                                          T *red, T *chn, T *part, int &buf) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int c = S.c, par = step & 1;
#pragma unroll
  for (int q = 0; q < R; ++q) red[(warp * R + q) * 32 + lane] = acc[q][0] + acc[q][1];
  __syncthreads();
  if (warp < kChain) {
    // CTA partial of each row: warps w, w+4, w+8, w+12, then the four sums
    T *cb = chn + (buf & 1) * (kChain * R * 32);
#pragma unroll
    for (int q = 0; q < R; ++q) {
      T s = red[(warp * R + q) * 32 + lane];
#pragma unroll
      for (int k = warp + kChain; k < kClWarps; k += kChain) s += red[(k * R + q) * 32 + lane];
      cb[(warp * R + q) * 32 + lane] = s;
    }
    chain_bar();
    ++buf;
    T tot[R];
#pragma unroll
    for (int q = 0; q < R; ++q) {
      tot[q] = cb[q * 32 + lane];
#pragma unroll
      for (int k = 1; k < kChain; ++k) tot[q] += cb[(k * R + q) * 32 + lane];
    }
    for (int dst = warp; dst < C; dst += kChain) {
      T *p = cluster.map_shared_rank(part, dst);
#pragma unroll
      for (int q = 0; q < R; ++q) p[((par * R + q) * C + c) * 32 + lane] = tot[q];
    }
  }
  cluster.sync();
  if (warp < kChain) {
    T yr[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if (!S.valid(step, r)) break;
      const int I = S.row(step, r);
      T s = y[I * 32 + lane];
#pragma unroll
      for (int q = 0; q < C; ++q) s -= part[((par * R + r) * C + q) * 32 + lane];
      if (r > 0) {                            // couplings to the rows solved in this step
        T pn0 = T(0), pn1 = T(0);
#pragma unroll
        for (int d = 1; d <= r; ++d)
#pragma unroll
          for (int k = 0; k < 8; k += 2) {
            pn0 += nv[r * (r - 1) / 2 + d - 1][k] * __shfl_sync(0xffffffffu, yr[r - d], warp * 8 + k);
            pn1 += nv[r * (r - 1) / 2 + d - 1][k + 1] *
                   __shfl_sync(0xffffffffu, yr[r - d], warp * 8 + k + 1);
          }
        T *cb = chn + (buf & 1) * (kChain * R * 32);
        cb[warp * 32 + lane] = pn0 + pn1;
        chain_bar();
        ++buf;
        s -= ((cb[lane] + cb[32 + lane]) + cb[64 + lane]) + cb[96 + lane];
      }
      T po0 = T(0), po1 = T(0);
#pragma unroll
      for (int k = 0; k < 8; k += 2) {
        po0 += dv[r][k] * __shfl_sync(0xffffffffu, s, warp * 8 + k);
        po1 += dv[r][k + 1] * __shfl_sync(0xffffffffu, s, warp * 8 + k + 1);
      }
      T *cb = chn + (buf & 1) * (kChain * R * 32);
      cb[warp * 32 + lane] = po0 + po1;
      chain_bar();
      ++buf;
      yr[r] = ((cb[lane] + cb[32 + lane]) + cb[64 + lane]) + cb[96 + lane];
      if (warp == 0) y[I * 32 + lane] = yr[r];
    }
  }
  __syncthreads();
}

template <typename T, int C, int R>
__device__ void cluster_sweep(const cg::cluster_group &cluster, const T *__restrict__ pool,
                              const BandLayout &L, T *y, T *red, T *chn, T *part,
                              bool backward) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  Sweep<T, C, R> S{pool, L, (int)cluster.block_rank(), L.nt, L.w, backward};
  const int nsteps = (S.nt + R - 1) / R;
  constexpr int kLinesPerUnit = 8 * 32 * (int)sizeof(T) / 128;
  T nx[8];                                      // register copy of this warp's next first unit
  bool have_nx = false;
  {
    int r, d, g;
    if (nsteps > 0 && S.unit(0, warp, r, d, g)) {
      const T *t = S.unit_ptr(0, r, d, g);
#pragma unroll
      for (int k = 0; k < 8; ++k) nx[k] = __ldg(t + k * 32 + lane);
      have_nx = true;
    }
  }
  int buf = 0;                                  // rotating chain buffer
  for (int step = 0; step < nsteps; ++step) {
    // chain tiles of this step: columns 8*warp..8*warp+7 of every inverted
    // diagonal block and every coupling inside the group
    T dv[R][8];
    T nv[Sweep<T, C, R>::kNearSlots][8];
    if (warp < kChain) {
#pragma unroll
      for (int r = 0; r < R; ++r) {
        if (!S.valid(step, r)) break;
        const int I = S.row(step, r);
        const T *D = tile_at(pool, L, I, 0) + warp * 8 * 32;
#pragma unroll
        for (int k = 0; k < 8; ++k) dv[r][k] = __ldg(D + k * 32 + lane);
#pragma unroll
        for (int d = 1; d <= r; ++d) {         // zero outside the band (d > w)
          const T *N = tile_at(pool, L, I, d) + warp * 8 * 32;
#pragma unroll
          for (int k = 0; k < 8; ++k)
            nv[r * (r - 1) / 2 + d - 1][k] = d <= S.w ? __ldg(N + k * 32 + lane) : T(0);
        }
      }
    }
    if (step + 2 < nsteps) {                    // L2 prefetch two steps ahead
      int r, d, g;
      for (int u = warp; S.unit(step + 2, u, r, d, g); u += kClWarps)
        if (lane < kLinesPerUnit)
          prefetch_l2(S.unit_ptr(step + 2, r, d, g) + lane * (128 / sizeof(T)));
      if (warp < kChain && lane < kLinesPerUnit) {
#pragma unroll
        for (int q = 0; q < R; ++q) {
          if (!S.valid(step + 2, q)) break;
          const int I = S.row(step + 2, q);
#pragma unroll
          for (int d = 0; d <= q; ++d)
            if (d <= S.w)
              prefetch_l2(tile_at(pool, L, I, d) + warp * 8 * 32 + lane * (128 / sizeof(T)));
        }
      }
    }
    // far tiles
    T acc[R][2];
#pragma unroll
    for (int q = 0; q < R; ++q) acc[q][0] = acc[q][1] = T(0);
    {
      // B units per warp in flight at once (their loads are issued before any FMA)
      constexpr int B = sizeof(T) == 8 ? 2 : 4;
      bool first = true;
      for (int u = warp;; u += B * kClWarps) {
        T v[B][8];
        int rb[B], db[B], gb[B];
        bool ok[B];
#pragma unroll
        for (int b = 0; b < B; ++b) {
          ok[b] = S.unit(step, u + b * kClWarps, rb[b], db[b], gb[b]);
          if (!ok[b]) continue;
          if (b == 0 && first && have_nx) {
#pragma unroll
            for (int e = 0; e < 8; ++e) v[b][e] = nx[e];
          } else {
            const T *t = S.unit_ptr(step, rb[b], db[b], gb[b]);
#pragma unroll
            for (int e = 0; e < 8; ++e) v[b][e] = __ldg(t + e * 32 + lane);
          }
        }
#pragma unroll
        for (int b = 0; b < B; ++b) {
          if (!ok[b]) continue;
          const int I = S.row(step, rb[b]);
          const T *yJ = y + (backward ? (I + db[b]) : (I - db[b])) * 32 + gb[b] * 8;
          T a0 = T(0), a1 = T(0);
#pragma unroll
          for (int e = 0; e < 8; e += 2) {
            a0 += v[b][e] * yJ[e];
            a1 += v[b][e + 1] * yJ[e + 1];
          }
#pragma unroll
          for (int q = 0; q < R; ++q)
            if (q == rb[b]) {
              acc[q][0] += a0;
              acc[q][1] += a1;
            }
        }
        first = false;
        if (!ok[B - 1]) break;
      }
      have_nx = false;
      int r, d, g;
      if (step + 1 < nsteps && S.unit(step + 1, warp, r, d, g)) {   // in flight over the barriers
        const T *t = S.unit_ptr(step + 1, r, d, g);
#pragma unroll
        for (int e = 0; e < 8; ++e) nx[e] = __ldg(t + e * 32 + lane);
        have_nx = true;
      }
    }
    step_tail<T, C, R>(cluster, S, step, acc, dv, nv, y, red, chn, part, buf);
  }
}

// ---- sweep with its tiles staged in shared memory ---------------------------
// The same step as above, but the tiles a CTA reads in a step (its R inverted
// diagonal blocks, the couplings inside the group and its far tiles) are
// copied into a shared-memory stage by bulk asynchronous copies
// (cp.async.bulk, completed on an mbarrier) that one thread issues a step
// ahead, so neither the far products nor the chain wait on L2 or HBM.  A
// stage holds R * (1 + ceil(w / C)) + R (R - 1) / 2 tiles; every tile of the
// pool is a contiguous, 4 KB aligned block, so each copy is one tile.
constexpr int kStages = 2;
constexpr int kXBuf = 4;                        // partial-exchange buffers (and mbarriers)
constexpr int kIssuer = kClWarps * 32 - 32;     // lane 0 of the last warp issues the copies

__device__ __forceinline__ uint32_t sm_addr(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Wait for phase `parity` of an mbarrier; false after about a second.
__device__ __forceinline__ bool mbar_wait(uint64_t *m, uint32_t parity) {
  const uint32_t a = sm_addr(m);
  uint32_t done = 0;
  const uint64_t t0 = global_ns();
  for (int it = 0; !done; ++it) {
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (!done && (it & 255) == 255 && global_ns() - t0 > 1000000000ull) break;
  }
  return done != 0;
}

__device__ __forceinline__ void bulk_tile(void *dst, const void *src, uint32_t bytes,
                                          uint64_t *m) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
      ::"r"(sm_addr(dst)), "l"(src), "r"(bytes), "r"(sm_addr(m))
      : "memory");
}

// Tiles per stage for half-bandwidth w (host and device).
__host__ __device__ __forceinline__ int stage_tiles(int w, int C, int R) {
  return R * (1 + (w + C - 1) / C) + R * (R - 1) / 2;
}

// Issue the copies of one step into stage `st` (one thread).
template <typename T, int C, int R>
__device__ void stage_step(const Sweep<T, C, R> &S, int step, T *st, uint64_t *m) {
  constexpr uint32_t kTile = 1024 * sizeof(T);
  constexpr int kFar0 = R + (R * (R - 1)) / 2;  // first far slot
  int ntiles = 0;
#pragma unroll
  for (int q = 0; q < R; ++q) {
    if (!S.valid(step, q)) break;
    int t0, n;
    far_tiles<C>(q, S.dmax(S.row(step, q)), S.c, t0, n);
    ntiles += 1 + min(q, S.w) + n;
  }
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
               ::"r"(sm_addr(m)), "r"(ntiles * kTile)
               : "memory");
  int slot = kFar0;
#pragma unroll
  for (int q = 0; q < R; ++q) {
    if (!S.valid(step, q)) break;
    const int I = S.row(step, q);
    bulk_tile(st + q * 1024, tile_at(S.pool, S.L, I, 0), kTile, m);
    for (int d = 1; d <= q && d <= S.w; ++d)
      bulk_tile(st + (R + q * (q - 1) / 2 + d - 1) * 1024, tile_at(S.pool, S.L, I, d), kTile, m);
    int t0, n;
    far_tiles<C>(q, S.dmax(I), S.c, t0, n);
    for (int t = 0; t < n; ++t, ++slot)
      bulk_tile(st + slot * 1024, tile_at(S.pool, S.L, I, 1 + S.c + (t0 + t) * C), kTile, m);
  }
}

// Exchange of the per-CTA far partials without a cluster barrier: the chain
// warps of every CTA store their partials straight into each CTA's buffer
// with st.async, whose bytes complete a transaction count on the receiving
// CTA's mbarrier (armed by its thread 0 for the step); the receiving chain
// warps wait on that barrier alone, and the far warps never wait on the
// cluster.  Buffer and barrier alternate with the step parity; a CTA cannot
// send the partials of step s + 2 before every CTA has consumed those of step
// s (it needs their step s + 1 partials first).
__device__ __forceinline__ uint32_t cluster_addr(const void *p, int rank) {
  uint32_t a;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(a) : "r"(sm_addr(p)), "r"(rank));
  return a;
}

__device__ __forceinline__ void st_async(uint32_t addr, float v, uint32_t bar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.b32 [%0], %1, [%2];"
               ::"r"(addr), "r"(__float_as_uint(v)), "r"(bar)
               : "memory");
}

__device__ __forceinline__ void st_async(uint32_t addr, double v, uint32_t bar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.b64 [%0], %1, [%2];"
               ::"r"(addr), "l"(__double_as_longlong(v)), "r"(bar)
               : "memory");
}

// Wait for phase `parity` with cluster-scope acquire (remote writes visible);
// false after about a second.
__device__ __forceinline__ bool mbar_wait_cluster(uint64_t *m, uint32_t parity) {
  const uint32_t a = sm_addr(m);
  uint32_t done = 0;
  const uint64_t t0 = global_ns();
  for (int it = 0; !done; ++it) {
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (!done && (it & 255) == 255 && global_ns() - t0 > 1000000000ull) break;
  }
  return done != 0;
}

// Second half of a staged step with FP64 factors, where the issue rate of
// FP64 instructions bounds a step.  Chain warp w owns rows 8w..8w+7 of the
// step's tile rows; lane 4i + k works on row 8w + i and column group k (8
// columns), so every sum over warps, CTAs or columns is a 4-term sum per lane
// and two butterfly shuffles, with no sum repeated by the four warps:
//   1. the CTA partial of each row from the 16 far-warp partials;
//   2. the partials to every CTA (st.async, lane k to CTAs k, k + 4), wait;
//   3. s = y_I - (sum of the C partials) - couplings inside the group;
//   4. s to shared memory, then y_I = D^-1 s from this warp's 8 rows of the
//      inverted diagonal block.
template <typename T, int C, int R>
__device__ __forceinline__ void step_tail_async(const Sweep<T, C, R> &S, int step, uint32_t gstep,
                                                const T (&acc)[R], const T (&dv)[R][8],
                                                const T (&nv)[Sweep<T, C, R>::kNearSlots][8],
                                                T *y, T *red, T *sb, T *part, uint64_t *mbx,
                                                bool &dead, DevStatus *status, int sys) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int c = S.c, par = gstep & 1;
#pragma unroll
  for (int q = 0; q < R; ++q) red[(warp * R + q) * 32 + lane] = acc[q];
  __syncthreads();
  if (warp < kChain) {
    const int i = lane >> 2, k = lane & 3, row = warp * 8 + i;
    T tot[R];
#pragma unroll
    for (int q = 0; q < R; ++q) {
      T p = ((red[((4 * k) * R + q) * 32 + row] + red[((4 * k + 1) * R + q) * 32 + row]) +
             red[((4 * k + 2) * R + q) * 32 + row]) +
            red[((4 * k + 3) * R + q) * 32 + row];
      p += __shfl_xor_sync(0xffffffffu, p, 1);
      p += __shfl_xor_sync(0xffffffffu, p, 2);
      tot[q] = p;
    }
    if constexpr (C > 1) {
      if (threadIdx.x == 0)
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                     ::"r"(sm_addr(mbx + par)), "r"((uint32_t)(C * R * 32 * sizeof(T)))
                     : "memory");
      for (int dst = k; dst < C; dst += 4) {
        const uint32_t bar = cluster_addr(mbx + par, dst);
#pragma unroll
        for (int q = 0; q < R; ++q)
          st_async(cluster_addr(part + ((par * R + q) * C + c) * 32 + row, dst), tot[q], bar);
      }
      if (!dead && !mbar_wait_cluster(mbx + par, (gstep >> 1) & 1u)) {
        dead = true;
        if (lane == 0 && atomicCAS(&status->code, 0, GENEO_ERR_TIMEOUT) == 0) {
          status->where = sys;
          status->detail = -1 - step;
        }
      }
#pragma unroll
      for (int q = 0; q < R; ++q) {
        T t = T(0);
#pragma unroll
        for (int src = k; src < C; src += 4) t += part[((par * R + q) * C + src) * 32 + row];
        t += __shfl_xor_sync(0xffffffffu, t, 1);
        t += __shfl_xor_sync(0xffffffffu, t, 2);
        tot[q] = t;
      }
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if (!S.valid(step, r)) break;
      const int I = S.row(step, r);
      T s = y[I * 32 + row] - tot[r];
      if (r > 0) {                            // couplings to the rows solved in this step
        chain_bar();                          // their y, written by every chain warp
        T pn = T(0);
#pragma unroll
        for (int d = 1; d <= r; ++d) {
          const T *yp = y + (S.backward ? I + d : I - d) * 32 + 8 * k;
#pragma unroll
          for (int e = 0; e < 8; ++e) pn = fma(nv[r * (r - 1) / 2 + d - 1][e], yp[e], pn);
        }
        pn += __shfl_xor_sync(0xffffffffu, pn, 1);
        pn += __shfl_xor_sync(0xffffffffu, pn, 2);
        s -= pn;
      }
      if (k == 0) sb[r * 32 + row] = s;
      chain_bar();
      T po = T(0);
#pragma unroll
      for (int e = 0; e < 8; ++e) po = fma(dv[r][e], sb[r * 32 + 8 * k + e], po);
      po += __shfl_xor_sync(0xffffffffu, po, 1);
      po += __shfl_xor_sync(0xffffffffu, po, 2);
      if (k == 0) y[I * 32 + row] = po;
    }
  }
  __syncthreads();
}

// FP32 variant of the chain: the four chain warps each take 8 columns of
// every chain tile for all 32 rows (the sums over warps are repeated in each
// of them), which keeps the dependent steps of a row short; with FP32 the
// row latency, not the arithmetic, bounds a step.
template <typename T, int C, int R>
__device__ __forceinline__ void step_tail_async_lat(const Sweep<T, C, R> &S, int step, uint32_t gstep,
                                                const T (&acc)[R], const T (&dv)[R][8],
                                                const T (&nv)[Sweep<T, C, R>::kNearSlots][8],
                                                T *y, T *red, T *chn, T *part, uint64_t *mbx,
                                                bool &dead, DevStatus *status, int sys) {
  int buf = 0;                                  // rotating chain buffer
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int c = S.c, par = gstep & 1;
#pragma unroll
  for (int q = 0; q < R; ++q) red[(warp * R + q) * 32 + lane] = acc[q];
  __syncthreads();
  if (warp < kChain) {
    // CTA partial of each row: warps w, w+4, w+8, w+12, then the four sums
    T *cb = chn + (buf & 1) * (kChain * R * 32);
#pragma unroll
    for (int q = 0; q < R; ++q) {
      T s = red[(warp * R + q) * 32 + lane];
#pragma unroll
      for (int k = warp + kChain; k < kClWarps; k += kChain) s += red[(k * R + q) * 32 + lane];
      cb[(warp * R + q) * 32 + lane] = s;
    }
    chain_bar();
    ++buf;
    T tot[R];
#pragma unroll
    for (int q = 0; q < R; ++q) {
      tot[q] = cb[q * 32 + lane];
#pragma unroll
      for (int k = 1; k < kChain; ++k) tot[q] += cb[(k * R + q) * 32 + lane];
    }
    if constexpr (C > 1) {
      if (threadIdx.x == 0)
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                     ::"r"(sm_addr(mbx + par)), "r"((uint32_t)(C * R * 32 * sizeof(T)))
                     : "memory");
      for (int dst = warp; dst < C; dst += kChain) {
        const uint32_t bar = cluster_addr(mbx + par, dst);
#pragma unroll
        for (int q = 0; q < R; ++q)
          st_async(cluster_addr(part + ((par * R + q) * C + c) * 32 + lane, dst), tot[q], bar);
      }
      if (!dead && !mbar_wait_cluster(mbx + par, (gstep >> 1) & 1u)) {
        dead = true;
        if (lane == 0 && atomicCAS(&status->code, 0, GENEO_ERR_TIMEOUT) == 0) {
          status->where = sys;
          status->detail = -1 - step;
        }
      }
    }
    T yr[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if (!S.valid(step, r)) break;
      const int I = S.row(step, r);
      T s = y[I * 32 + lane];
      if constexpr (C > 1) {
#pragma unroll
        for (int q = 0; q < C; ++q) s -= part[((par * R + r) * C + q) * 32 + lane];
      } else {
        s -= tot[r];
      }
      if (r > 0) {                            // couplings to the rows solved in this step
        T pn0 = T(0), pn1 = T(0);
#pragma unroll
        for (int d = 1; d <= r; ++d)
#pragma unroll
          for (int k = 0; k < 8; k += 2) {
            pn0 += nv[r * (r - 1) / 2 + d - 1][k] * __shfl_sync(0xffffffffu, yr[r - d], warp * 8 + k);
            pn1 += nv[r * (r - 1) / 2 + d - 1][k + 1] *
                   __shfl_sync(0xffffffffu, yr[r - d], warp * 8 + k + 1);
          }
        T *cb = chn + (buf & 1) * (kChain * R * 32);
        cb[warp * 32 + lane] = pn0 + pn1;
        chain_bar();
        ++buf;
        s -= ((cb[lane] + cb[32 + lane]) + cb[64 + lane]) + cb[96 + lane];
      }
      T po0 = T(0), po1 = T(0);
#pragma unroll
      for (int k = 0; k < 8; k += 2) {
        po0 += dv[r][k] * __shfl_sync(0xffffffffu, s, warp * 8 + k);
        po1 += dv[r][k + 1] * __shfl_sync(0xffffffffu, s, warp * 8 + k + 1);
      }
      T *cb = chn + (buf & 1) * (kChain * R * 32);
      cb[warp * 32 + lane] = po0 + po1;
      chain_bar();
      ++buf;
      yr[r] = ((cb[lane] + cb[32 + lane]) + cb[64 + lane]) + cb[96 + lane];
      if (warp == 0) y[I * 32 + lane] = yr[r];
    }
  }
  __syncthreads();
}

template <typename T, int C, int R>
__device__ void cluster_sweep_staged(const T *__restrict__ pool, int c, const BandLayout &L, T *y,
                                     T *red, T *chn, T *part, bool backward, T *stages,
                                     int stride, uint64_t *mbar, uint64_t *mbx, uint32_t &seq,
                                     bool &dead, DevStatus *status, int sys) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  Sweep<T, C, R> S{pool, L, c, L.nt, L.w, backward};
  const int nsteps = (S.nt + R - 1) / R;
  constexpr int kFar0 = R + (R * (R - 1)) / 2;
  int issued = 0;                               // steps staged (issuing thread)
  if (threadIdx.x == kIssuer && !dead)
    for (; issued < kStages - 1 && issued < nsteps; ++issued) {
      const uint32_t q = seq + issued;
      stage_step(S, issued, stages + (q % kStages) * stride, mbar + q % kStages);
    }
  for (int step = 0; step < nsteps; ++step) {
    const uint32_t q = seq + step;
    // the stage of step + kStages - 1 was last read in the previous step,
    // which every warp has left (block barrier at the end of a step)
    if (threadIdx.x == kIssuer && !dead && step + kStages - 1 < nsteps) {
      const uint32_t qn = q + kStages - 1;
      stage_step(S, step + kStages - 1, stages + (qn % kStages) * stride, mbar + qn % kStages);
      issued = step + kStages;
    }
    if (!dead && !mbar_wait(mbar + q % kStages, (q / kStages) & 1u)) {
      dead = true;
      if (lane == 0 && atomicCAS(&status->code, 0, GENEO_ERR_TIMEOUT) == 0) {
        status->where = sys;
        status->detail = step;
      }
    }
    const T *st = stages + (q % kStages) * stride;
    // chain tiles: FP64 row 8 * warp + lane / 4, columns 8 * (lane % 4) + e;
    // FP32 row lane, columns 8 * warp + e
    T dv[R][8];
    T nv[Sweep<T, C, R>::kNearSlots][8];
    if (warp < kChain) {
      const int el = sizeof(T) == 8 ? (8 * (lane & 3)) * 32 + warp * 8 + (lane >> 2)
                                    : (8 * warp) * 32 + lane;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        if (!S.valid(step, r)) break;
#pragma unroll
        for (int e = 0; e < 8; ++e) dv[r][e] = st[r * 1024 + el + e * 32];
#pragma unroll
        for (int d = 1; d <= r; ++d)            // zero outside the band (d > w)
#pragma unroll
          for (int e = 0; e < 8; ++e)
            nv[r * (r - 1) / 2 + d - 1][e] =
                d <= S.w ? st[(R + r * (r - 1) / 2 + d - 1) * 1024 + el + e * 32] : T(0);
      }
    }
    // far products, row by row: units u = warp, warp + 16, ... of the step,
    // accumulated straight into the row's accumulator
    T acc[R];
    int ubase = 0;                              // first unit of row r
#pragma unroll
    for (int r = 0; r < R; ++r) {
      acc[r] = T(0);
      if (!S.valid(step, r)) continue;
      const int I = S.row(step, r);
      int t0, n;
      far_tiles<C>(r, S.dmax(I), c, t0, n);
      const int uend = ubase + kGroups * n;
      for (int u = ubase + ((warp - ubase) % kClWarps + kClWarps) % kClWarps; u < uend;
           u += kClWarps) {
        const int lu = u - ubase, g = lu % kGroups;
        const int d = 1 + c + (t0 + lu / kGroups) * C;
        const T *t = st + (kFar0 + u / kGroups) * 1024 + g * 256;
        const T *yJ = y + (backward ? (I + d) : (I - d)) * 32 + g * 8;
#pragma unroll
        for (int e = 0; e < 8; ++e) acc[r] = fma(t[e * 32 + lane], yJ[e], acc[r]);
      }
      ubase = uend;
    }
    if constexpr (sizeof(T) == 8)
      step_tail_async<T, C, R>(S, step, q, acc, dv, nv, y, red, chn, part, mbx, dead, status, sys);
    else
      step_tail_async_lat<T, C, R>(S, step, q, acc, dv, nv, y, red, chn, part, mbx, dead, status,
                                   sys);
  }
  if (threadIdx.x == kIssuer && dead)           // copies still in flight land before the exit
    for (int s = max(0, issued - kStages); s < issued; ++s)
      mbar_wait(mbar + (seq + s) % kStages, ((seq + s) / kStages) & 1u);
  seq += nsteps;
}

// Staged look-ahead sweep (one tile row per step).  At step q the 12 far
// warps multiply the far tiles (distance >= 2, d = 2 + c + tC) of row I_{q+1},
// which need only rows solved before step q, sum their partials and push the
// CTA partial of row I_{q+1} into every CTA's exchange buffer (st.async,
// completed on that CTA's mbarrier); meanwhile the four chain warps finish row
// I_q: the coupling L(I_q, I_q - 1) y_{I_q - 1}, the wait for the C partials
// of row I_q (pushed during step q - 1), and the inverted diagonal block.  A
// step's stage holds the far tiles of I_{q+1} and, when shared memory allows
// (stage_chain), the chain's two tiles of I_q; otherwise the chain warps load
// those into registers at the end of the previous step, in flight over the
// block barrier.
// Exchange buffers rotate over four rows: a CTA can push the partials of row
// q + 3 while another still reads those of row q, but not of row q + 4.

__device__ __forceinline__ void far_bar() {
  asm volatile("bar.sync 2, %0;" ::"n"((kClWarps - kChain) * 32) : "memory");
}

__host__ __device__ __forceinline__ int stage_tiles_la(int w, int C) {
  return w > 1 ? (w - 1 + C - 1) / C : 1;
}

template <typename T, int C, bool kSC>
__device__ void cluster_sweep_staged_la(const T *__restrict__ pool, int c, const BandLayout &L,
                                        T *y, T *red, T *chn, T *part, bool backward, T *stages,
                                        int stride, uint64_t *mbar, uint64_t *mbx, uint32_t &seq,
                                        bool &dead, DevStatus *status, int sys) {
  constexpr int stage_chain = kSC ? 1 : 0;
  constexpr int kFarW = kClWarps - kChain;
  constexpr uint32_t kTile = 1024 * sizeof(T);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nt = L.nt, w = L.w;
  auto row = [&](int q) { return backward ? nt - 1 - q : q; };
  auto dmax = [&](int I) { return backward ? min(w, nt - 1 - I) : min(w, I); };
  auto nfar = [&](int I) {
    const int dm = dmax(I), d0 = 2 + c;
    return dm >= d0 ? (dm - d0) / C + 1 : 0;
  };
  auto stage = [&](int q) {                     // one thread: copies of step q
    const uint32_t g = seq + q;
    T *st = stages + (g % kStages) * stride;
    uint64_t *m = mbar + g % kStages;
    const int nf = q + 1 < nt ? nfar(row(q + 1)) : 0;
    const int I = row(q), has1 = stage_chain && dmax(I) >= 1 ? 1 : 0;
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                 ::"r"(sm_addr(m)), "r"((uint32_t)(nf + (stage_chain ? 1 + has1 : 0)) * kTile)
                 : "memory");
    if (stage_chain) {
      bulk_tile(st, tile_at(pool, L, I, 0), kTile, m);
      if (has1) bulk_tile(st + 1024, tile_at(pool, L, I, 1), kTile, m);
    }
    T *sf = st + (stage_chain ? 2 : 0) * 1024;
    for (int t = 0; t < nf; ++t)
      bulk_tile(sf + t * 1024, tile_at(pool, L, row(q + 1), 2 + c + t * C), kTile, m);
  };
  // chain tiles of row I_q, columns 8 * warp + e: D^-1 and L(I_q, I_q - 1)
  T dv[8], nv[8];
  auto chain_tiles = [&](int q) {
    const int I = row(q);
    const T *D = tile_at(pool, L, I, 0) + (8 * warp) * 32 + lane;
    const bool has1 = dmax(I) >= 1;
    const T *N = tile_at(pool, L, I, has1 ? 1 : 0) + (8 * warp) * 32 + lane;
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      dv[e] = __ldg(D + e * 32);
      nv[e] = has1 ? __ldg(N + e * 32) : T(0);
    }
  };
  if (!stage_chain && warp < kChain && nt > 0) chain_tiles(0);
  // push the CTA partial `v` of the row with sequence number g (far warps 0..C-1)
  auto push = [&](uint32_t g, int fw, T v) {
    if constexpr (C > 1) {
      st_async(cluster_addr(part + ((g % kXBuf) * C + c) * 32 + lane, fw), v,
               cluster_addr(mbx + g % kXBuf, fw));
    } else {
      part[(g % kXBuf) * 32 + lane] = v;
    }
  };
  int issued = 0;
  if (threadIdx.x == kIssuer && !dead && nt > 0) {
    stage(0);
    issued = 1;
  }
  // row 0 has no far tiles: its partials are zero
  if (warp >= kChain && warp - kChain < C && nt > 0) push(seq, warp - kChain, T(0));
  __syncthreads();
  int buf = 0;
  for (int q = 0; q < nt; ++q) {
    const uint32_t g = seq + q;
    if (threadIdx.x == kIssuer && !dead && q + 1 < nt) {   // the stage step q - 1 used is free
      stage(q + 1);
      issued = q + 2;
    }
    if ((warp >= kChain || stage_chain) && !dead &&
        !mbar_wait(mbar + g % kStages, (g / kStages) & 1u)) {
      dead = true;
      if (lane == 0 && atomicCAS(&status->code, 0, GENEO_ERR_TIMEOUT) == 0) {
        status->where = sys;
        status->detail = q;
      }
    }
    const T *st = stages + (g % kStages) * stride;
    const int I = row(q);
    if (warp < kChain) {
      if (C > 1 && threadIdx.x == 0)
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                     ::"r"(sm_addr(mbx + g % kXBuf)), "r"((uint32_t)(C * 32 * sizeof(T)))
                     : "memory");
      T p = T(0);
      if (dmax(I) >= 1) {
        const T *yp = y + (backward ? I + 1 : I - 1) * 32 + 8 * warp;
        const T *t1 = st + 1024 + (8 * warp) * 32 + lane;
#pragma unroll
        for (int e = 0; e < 8; ++e) p = fma(kSC ? t1[e * 32] : nv[e], yp[e], p);
      }
      T *cb = chn + (buf & 1) * (kChain * 32);
      cb[warp * 32 + lane] = p;
      chain_bar();
      ++buf;
      T s = y[I * 32 + lane] - (((cb[lane] + cb[32 + lane]) + cb[64 + lane]) + cb[96 + lane]);
      if constexpr (C > 1) {
        if (!dead && !mbar_wait_cluster(mbx + g % kXBuf, (g / kXBuf) & 1u)) {
          dead = true;
          if (lane == 0 && atomicCAS(&status->code, 0, GENEO_ERR_TIMEOUT) == 0) {
            status->where = sys;
            status->detail = -1 - q;
          }
        }
#pragma unroll
        for (int src = 0; src < C; ++src) s -= part[((g % kXBuf) * C + src) * 32 + lane];
      } else {
        s -= part[(g % kXBuf) * 32 + lane];
      }
      const T *t0 = st + (8 * warp) * 32 + lane;
      T po = T(0);
#pragma unroll
      for (int e = 0; e < 8; ++e)
        po = fma(kSC ? t0[e * 32] : dv[e], __shfl_sync(0xffffffffu, s, 8 * warp + e), po);
      cb = chn + (buf & 1) * (kChain * 32);
      cb[warp * 32 + lane] = po;
      chain_bar();
      ++buf;
      if (warp == 0) y[I * 32 + lane] = ((cb[lane] + cb[32 + lane]) + cb[64 + lane]) + cb[96 + lane];
      if (!stage_chain && q + 1 < nt) chain_tiles(q + 1);   // in flight over the block barrier
    } else if (q + 1 < nt) {
      const int fw = warp - kChain;
      const int In = row(q + 1), nu = kGroups * nfar(In);
      T a = T(0);
      for (int u = fw; u < nu; u += kFarW) {
        const int d = 2 + c + (u / kGroups) * C, gq = u % kGroups;
        const T *t = st + (u / kGroups + (stage_chain ? 2 : 0)) * 1024 + gq * 256 + lane;
        const T *yJ = y + (backward ? In + d : In - d) * 32 + gq * 8;
#pragma unroll
        for (int e = 0; e < 8; ++e) a = fma(t[e * 32], yJ[e], a);
      }
      red[fw * 32 + lane] = a;
      far_bar();
      if (fw < C) {
        T tot = red[lane];
#pragma unroll
        for (int k = 1; k < kFarW; ++k) tot += red[k * 32 + lane];
        push(g + 1, fw, tot);
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == kIssuer && dead)           // copies still in flight land before the exit
    for (int s = max(0, issued - kStages); s < issued; ++s)
      mbar_wait(mbar + (seq + s) % kStages, ((seq + s) / kStages) & 1u);
  seq += nt;
}

// Look-ahead sweep.  Warps 4..15 multiply the far tiles (distance >= 2) of row
// I+1, which need only rows <= I-1, while warps 0..3 finish row I: they reduce
// and exchange the far partials of row I (computed in the previous step),
// arrive at the cluster barrier, multiply the coupling tile L(I, I-1) (every
// CTA redundantly), wait, and apply the inverted diagonal block.  One split
// cluster barrier and one block barrier per row; the chain overlaps the far
// work.  Far tiles d = 2 + c + tC belong to CTA c.
__device__ __forceinline__ void cluster_arrive() {
  asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
}
__device__ __forceinline__ void cluster_wait() {
  asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// Where the look-ahead sweep keeps the local vector.  FullVec: all of it in
// shared memory, tile row I at y + 32 I, filled before and read after the
// sweep by the caller.  RingVec: only the tile rows the band can still touch,
// in a ring of `rows` slots (row I in slot I mod rows); one far warp reads the
// next row from `src` during each step and the chain writes each solved row to
// `dst`, so shared memory no longer bounds the subdomain size.  Step q (row I)
// reads rows I + 1 - w .. I and fills the slot of row I + 1, which last held
// row I + 1 - rows: with rows = max(w + 2, 3) that row is no longer read (the
// chain reads the previous row's slot even when w = 0 and its tile is zero).
__host__ __device__ constexpr int ring_rows(int w) { return w + 2 > 3 ? w + 2 : 3; }
struct FullVec {
  static constexpr bool kRing = false;
};

template <typename T, typename Src, typename Dst>
struct RingVec {
  static constexpr bool kRing = true;
  int rows;   // ring slots (tile rows)
  int n;      // unknowns: rows past n read as zero and are not written
  Src src;    // T operator()(int l): element l < n of the right-hand side
  Dst dst;    // void operator()(int l, T v): element l < n of the solution
};

// Contiguous vector (L2-coherent loads: the backward sweep reads what the
// forward sweep of the same launch wrote).
template <typename T>
struct ArraySrc {
  const T *p;
  __device__ T operator()(int l) const { return __ldcg(p + l); }
};
template <typename T>
struct ArrayDst {
  T *p;
  __device__ void operator()(int l, T v) const { p[l] = v; }
};
// Column of a row-major block of right-hand sides (row stride `ld`).
struct StridedSrc {
  const double *p;
  long long ld;
  __device__ double operator()(int l) const { return __ldcg(p + l * ld); }
};
struct StridedDst {
  double *p;
  long long ld;
  __device__ void operator()(int l, double v) const { p[l * ld] = v; }
};
// R_j r: the subdomain's interior unknowns gathered from the global vector.
template <typename T>
struct GatherSrc {
  const SubDesc *S;
  const double *r;
  int nnx, nny;
  __device__ T operator()(int l) const {
    const int nc = S->nc;
    const int node = l / nc, comp = l - nc * node;
    int gi, gj, gk;
    S->ibox.global(node, gi, gj, gk);
    return T(__ldcg(r + nc * (gi + nnx * (gj + nny * gk)) + comp));
  }
};

template <typename T, int C, typename V = FullVec>
__device__ void cluster_sweep_la(const cg::cluster_group &cluster, const T *__restrict__ pool,
                                 const BandLayout &L, T *y, T *red, T *chn, T *part,
                                 bool backward, const V &vec = V()) {
  constexpr int kFar = kClWarps - kChain;
  constexpr int B = sizeof(T) == 8 ? 2 : 4;
  constexpr int kLinesPerUnit = 8 * 32 * (int)sizeof(T) / 128;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int c = (int)cluster.block_rank();
  const int nt = L.nt, w = L.w;
  auto row = [&](int q) { return backward ? nt - 1 - q : q; };
  auto dmax = [&](int I) { return backward ? min(w, nt - 1 - I) : min(w, I); };
  // slot of tile row I, and of the row at distance d behind the row in slot s
  auto slot = [&](int I) {
    if constexpr (V::kRing) return I % vec.rows;
    else return I;
  };
  auto yrow = [&](int s, int d) {
    const int t = backward ? s + d : s - d;
    if constexpr (V::kRing) return t < 0 ? t + vec.rows : (t >= vec.rows ? t - vec.rows : t);
    else return t;
  };
  auto load_row = [&](int I) {                    // element `lane` of row I
    if constexpr (V::kRing) {
      const int l = I * 32 + lane;
      return l < vec.n ? vec.src(l) : T(0);
    } else {
      return T(0);
    }
  };
  // far units of row I for this CTA: d = 2 + c + t*C, 4 column groups per tile
  auto nfar = [&](int I) {
    const int dm = dmax(I), d0 = 2 + c;
    return dm >= d0 ? ((dm - d0) / C + 1) * kGroups : 0;
  };
  if constexpr (V::kRing) {
    if (warp == 0 && nt > 0) y[slot(row(0)) * 32 + lane] = load_row(row(0));
    __syncthreads();
  }
  int buf = 0;
  T dv[8], nv[8];                                 // chain: this warp's 8 columns
  if (warp < kChain && nt > 0) {
    const T *D = tile_at(pool, L, row(0), 0) + warp * 256;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      dv[k] = __ldg(D + k * 32 + lane);
      nv[k] = T(0);                               // row 0 has no coupling
    }
  }
  for (int q = 0; q < nt; ++q) {
    const int I = row(q);
    const int sI = slot(I);
    const int par = q & 1;
    if (warp >= kChain) {
      const int cw = warp - kChain;
      cluster_arrive();
      T a0 = T(0), a1 = T(0);
      if (q + 1 < nt) {
        const int In = row(q + 1), nu = nfar(In), sIn = slot(In);
        T next = T(0);                            // ring: row In, read by the chain in step q + 1
        if (V::kRing && cw == 0) next = load_row(In);
        if (q + 2 < nt) {                         // L2 prefetch of the next step's units
          const int I2 = row(q + 2), nu2 = nfar(I2);
          for (int u = cw; u < nu2; u += kFar)
            if (lane < kLinesPerUnit)
              prefetch_l2(tile_at(pool, L, I2, 2 + c + (u / kGroups) * C) + (u % kGroups) * 256 +
                          lane * (128 / sizeof(T)));
        }
        for (int u0 = cw; u0 < nu; u0 += B * kFar) {
          T v[B][8];
#pragma unroll
          for (int b = 0; b < B; ++b) {
            const int u = u0 + b * kFar;
            if (u < nu) {
              const T *t = tile_at(pool, L, In, 2 + c + (u / kGroups) * C) + (u % kGroups) * 256;
#pragma unroll
              for (int e = 0; e < 8; ++e) v[b][e] = __ldg(t + e * 32 + lane);
            }
          }
#pragma unroll
          for (int b = 0; b < B; ++b) {
            const int u = u0 + b * kFar;
            if (u < nu) {
              const int d = 2 + c + (u / kGroups) * C;
              const T *yJ = y + yrow(sIn, d) * 32 + (u % kGroups) * 8;
#pragma unroll
              for (int e = 0; e < 8; e += 2) {
                a0 += v[b][e] * yJ[e];
                a1 += v[b][e + 1] * yJ[e + 1];
              }
            }
          }
        }
        if (V::kRing && cw == 0) y[sIn * 32 + lane] = next;
      }
      red[(par ^ 1) * kFar * 32 + cw * 32 + lane] = a0 + a1;
      cluster_wait();
    } else {
      // far partials of row I: CTA sum, pushed to every CTA of the cluster
      if (q > 0) {
        T sp = T(0);
#pragma unroll
        for (int k = warp; k < kFar; k += kChain) sp += red[par * kFar * 32 + k * 32 + lane];
        T *cb = chn + (buf & 1) * (kChain * 32);
        cb[warp * 32 + lane] = sp;
        chain_bar();
        ++buf;
        const T tot = ((cb[lane] + cb[32 + lane]) + cb[64 + lane]) + cb[96 + lane];
        for (int dst = warp; dst < C; dst += kChain) {
          T *pp = cluster.map_shared_rank(part, dst);
          pp[(par * C + c) * 32 + lane] = tot;
        }
      }
      cluster_arrive();
      // coupling to the previous row, split by columns
      T p0 = T(0), p1 = T(0);
      if (q > 0) {
        const T *yJ = y + yrow(sI, 1) * 32 + warp * 8;
#pragma unroll
        for (int k = 0; k < 8; k += 2) {
          p0 += nv[k] * yJ[k];
          p1 += nv[k + 1] * yJ[k + 1];
        }
      }
      T *cb = chn + (buf & 1) * (kChain * 32);
      cb[warp * 32 + lane] = p0 + p1;
      chain_bar();
      ++buf;
      T sv = y[sI * 32 + lane] - (((cb[lane] + cb[32 + lane]) + cb[64 + lane]) + cb[96 + lane]);
      cluster_wait();
      if (q > 0) {
#pragma unroll
        for (int qq = 0; qq < C; ++qq) sv -= part[(par * C + qq) * 32 + lane];
      }
      T o0 = T(0), o1 = T(0);
#pragma unroll
      for (int k = 0; k < 8; k += 2) {
        o0 += dv[k] * __shfl_sync(0xffffffffu, sv, warp * 8 + k);
        o1 += dv[k + 1] * __shfl_sync(0xffffffffu, sv, warp * 8 + k + 1);
      }
      cb = chn + (buf & 1) * (kChain * 32);
      cb[warp * 32 + lane] = o0 + o1;
      chain_bar();
      ++buf;
      const T yI = ((cb[lane] + cb[32 + lane]) + cb[64 + lane]) + cb[96 + lane];
      if (warp == 0) {
        y[sI * 32 + lane] = yI;
        if constexpr (V::kRing) {
          if (c == 0 && I * 32 + lane < vec.n) vec.dst(I * 32 + lane, yI);
        }
      }
      if (q + 1 < nt) {                           // next row's chain tiles, in flight over the barrier
        const int In = row(q + 1);
        const T *D = tile_at(pool, L, In, 0) + warp * 256;
        const bool has1 = dmax(In) >= 1;
        const T *N = tile_at(pool, L, In, has1 ? 1 : 0) + warp * 256;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          dv[k] = __ldg(D + k * 32 + lane);
          nv[k] = has1 ? __ldg(N + k * 32 + lane) : T(0);
        }
      }
    }
    __syncthreads();
  }
}

template <typename T, int C>
__global__ void __launch_bounds__(kClWarps * 32)
    k_schwarz_cluster_la(const SubDesc *subs, const BandLayout *lay, int nnx, int nny,
                         const T *poolL, const T *poolU, const double *__restrict__ r,
                         T *__restrict__ xloc, const CGScalars *cgs) {
  if (cgs && cgs->done) return;           // the same for every CTA of the cluster
  cg::cluster_group cluster = cg::this_cluster();
  extern __shared__ __align__(16) unsigned char smraw[];
  T *red = reinterpret_cast<T *>(smraw);  // [2][kClWarps - kChain][32]
  T *chn = red + 2 * (kClWarps - kChain) * 32;   // [2][kChain][32]
  T *part = chn + 2 * kChain * 32;        // [2][C][32]
  T *y = part + 2 * C * 32;               // [npad]
  const int j = blockIdx.x / C;
  const SubDesc &S = subs[j];
  const BandLayout L = lay[j];
  const int n = S.n_int, npad = L.nt * 32;
  for (int l = threadIdx.x; l < npad; l += blockDim.x) {
    T v = T(0);
    if (l < n) {
      const int nc = S.nc;
      int node = l / nc, comp = l - nc * node;
      int gi, gj, gk;
      S.ibox.global(node, gi, gj, gk);
      v = T(r[nc * (gi + nnx * (gj + nny * gk)) + comp]);
    }
    y[l] = v;
  }
  cluster.sync();                          // every CTA's shared memory is live
  cluster_sweep_la<T, C>(cluster, poolL, L, y, red, chn, part, false);
  cluster.sync();                          // the partial buffers are reused by the second sweep
  cluster_sweep_la<T, C>(cluster, poolU, L, y, red, chn, part, true);
  if (cluster.block_rank() == 0) {
    T *out = xloc + S.v_int;
    for (int l = threadIdx.x; l < n; l += blockDim.x) out[l] = y[l];
  }
  cluster.sync();                          // no CTA leaves while others may still write to it
}

template <typename T, int C, int R>
__global__ void __launch_bounds__(kClWarps * 32)
    k_schwarz_cluster(const SubDesc *subs, const BandLayout *lay, int nnx, int nny,
                      const T *poolL, const T *poolU, const double *__restrict__ r,
                      T *__restrict__ xloc, const CGScalars *cgs) {
  if (cgs && cgs->done) return;           // the same for every CTA of the cluster
  cg::cluster_group cluster = cg::this_cluster();
  extern __shared__ __align__(16) unsigned char smraw[];
  T *red = reinterpret_cast<T *>(smraw);  // [kClWarps][R][32]
  T *chn = red + kClWarps * R * 32;       // [2][kChain][R][32]
  T *part = chn + 2 * kChain * R * 32;    // [2][R][C][32]
  T *y = part + 2 * R * C * 32;           // [npad]
  const int j = blockIdx.x / C;
  const SubDesc &S = subs[j];
  const BandLayout L = lay[j];
  const int n = S.n_int, npad = L.nt * 32;
  for (int l = threadIdx.x; l < npad; l += blockDim.x) {
    T v = T(0);
    if (l < n) {
      const int nc = S.nc;
      int node = l / nc, comp = l - nc * node;
      int gi, gj, gk;
      S.ibox.global(node, gi, gj, gk);
      v = T(r[nc * (gi + nnx * (gj + nny * gk)) + comp]);
    }
    y[l] = v;
  }
  cluster.sync();                          // every CTA's shared memory is live
  cluster_sweep<T, C, R>(cluster, poolL, L, y, red, chn, part, false);
  cluster_sweep<T, C, R>(cluster, poolU, L, y, red, chn, part, true);
  if (cluster.block_rank() == 0) {
    T *out = xloc + S.v_int;
    for (int l = threadIdx.x; l < n; l += blockDim.x) out[l] = y[l];
  }
  cluster.sync();                          // no CTA leaves while others may still write to it
}

template <typename T, int C, int R, bool kSC>
__global__ void __launch_bounds__(kClWarps * 32, 1)
    k_schwarz_cluster_staged(const SubDesc *subs, const BandLayout *lay, int nnx, int nny,
                             const T *poolL, const T *poolU, const double *__restrict__ r,
                             T *__restrict__ xloc, const CGScalars *cgs, int stride,
                             DevStatus *status) {
  if (cgs && cgs->done) return;           // the same for every CTA of the cluster
  cg::cluster_group cluster = cg::this_cluster();
  extern __shared__ __align__(16) unsigned char smraw[];
  constexpr int RR = R > 0 ? R : 1;
  T *stages = reinterpret_cast<T *>(smraw);                        // [kStages][stride]
  uint64_t *mbar = reinterpret_cast<uint64_t *>(stages + kStages * stride);   // [kStages]
  uint64_t *mbx = mbar + kStages;         // [kXBuf] partial exchange
  T *red = reinterpret_cast<T *>(mbx + kXBuf);   // [kClWarps][R][32] ([12][32] for R = 0)
  T *chn = red + kClWarps * RR * 32;      // [2][kChain][R][32]
  T *part = chn + 2 * kChain * RR * 32;   // [2][R][C][32] ([kXBuf][C][32] for R = 0)
  T *y = part + kXBuf * RR * C * 32;      // [npad]
  const int j = blockIdx.x / C;
  const SubDesc &S = subs[j];
  const BandLayout L = lay[j];
  const int n = S.n_int, npad = L.nt * 32;
  if (threadIdx.x == 0) {
    for (int b = 0; b < kStages + kXBuf; ++b)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(sm_addr(mbar + b)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  for (int l = threadIdx.x; l < npad; l += blockDim.x) {
    T v = T(0);
    if (l < n) {
      const int nc = S.nc;
      int node = l / nc, comp = l - nc * node;
      int gi, gj, gk;
      S.ibox.global(node, gi, gj, gk);
      v = T(r[nc * (gi + nnx * (gj + nny * gk)) + comp]);
    }
    y[l] = v;
  }
  cluster.sync();                          // shared memory and mbarriers live in every CTA
  uint32_t seq = 0;
  bool dead = false;
  const int c = (int)cluster.block_rank();
  if constexpr (R == 0) {
    cluster_sweep_staged_la<T, C, kSC>(poolL, c, L, y, red, chn, part, false, stages, stride,
                                       mbar, mbx, seq, dead, status, j);
    cluster_sweep_staged_la<T, C, kSC>(poolU, c, L, y, red, chn, part, true, stages, stride,
                                       mbar, mbx, seq, dead, status, j);
  } else {
    cluster_sweep_staged<T, C, R>(poolL, c, L, y, red, chn, part, false, stages, stride, mbar, mbx,
                                  seq, dead, status, j);
    cluster_sweep_staged<T, C, R>(poolU, c, L, y, red, chn, part, true, stages, stride, mbar, mbx,
                                  seq, dead, status, j);
  }
  if (cluster.block_rank() == 0) {
    T *out = xloc + S.v_int;
    for (int l = threadIdx.x; l < n; l += blockDim.x) out[l] = y[l];
  }
  cluster.sync();                          // no CTA leaves while others may still write to it
}

// ---- the GenEO eigensolver's band solves in the look-ahead form ------------------
// One CTA per (system, right-hand side): the column is loaded into shared
// memory (row stride in_row), swept forward and/or backward with the
// one-CTA look-ahead sweep above (far warps multiply row I+1 while the chain
// warps finish row I), and written back (row stride out_row).
__global__ void __launch_bounds__(kClWarps * 32)
    k_band_solve_la(const BandLayout *lay, const double *poolL, const double *poolU,
                    const double *__restrict__ in, long long in_sys, int in_row,
                    double *__restrict__ out, long long out_sys, int out_row, int mode) {
  cg::cluster_group cluster = cg::this_cluster();
  extern __shared__ __align__(16) unsigned char smraw[];
  double *red = reinterpret_cast<double *>(smraw);   // [2][kClWarps - kChain][32]
  double *chn = red + 2 * (kClWarps - kChain) * 32;   // [2][kChain][32]
  double *part = chn + 2 * kChain * 32;               // [2][1][32]
  double *y = part + 2 * 32;                          // [npad]
  const int j = blockIdx.x, c = blockIdx.y;
  const BandLayout L = lay[j];
  const int n = L.n, npad = L.nt * 32;
  const double *src = in + j * in_sys + c;
  for (int l = threadIdx.x; l < npad; l += blockDim.x) y[l] = l < n ? src[(long long)l * in_row] : 0.0;
  cluster.sync();
  if (mode & 1) cluster_sweep_la<double, 1>(cluster, poolL, L, y, red, chn, part, false);
  cluster.sync();
  if (mode & 2) cluster_sweep_la<double, 1>(cluster, poolU, L, y, red, chn, part, true);
  cluster.sync();
  double *dst = out + j * out_sys + c;
  for (int l = threadIdx.x; l < n; l += blockDim.x) dst[(long long)l * out_row] = y[l];
}

// ---- the same sweeps with the local vector streamed through a ring ----------
// For subdomains whose local vector does not fit in shared memory: the
// look-ahead sweep (one cluster of C CTAs per subdomain, or one CTA per
// (system, right-hand side)) with the vector in a ring of max(w + 2, 3) tile
// rows in every CTA.  The forward sweep writes y to a scratch vector as it
// goes (rank 0) and the backward sweep reads it back from there: two more
// passes over the n unknowns than the shared-memory form, beside the 32 (w + 1)
// factor elements per unknown that each sweep streams.  Reading y from a
// buffer the backward sweep does not write keeps a CTA that runs a step ahead
// from overwriting a row another CTA of the cluster has still to read.  The
// arithmetic and its order are those of the look-ahead launch with the same C
// (bit-identical results).
template <typename T, int C>
__global__ void __launch_bounds__(kClWarps * 32)
    k_schwarz_ring(const SubDesc *subs, const BandLayout *lay, int nnx, int nny, const T *poolL,
                   const T *poolU, const double *r, T *xloc, T *yscr, const CGScalars *cgs) {
  if (cgs && cgs->done) return;           // the same for every CTA of the cluster
  cg::cluster_group cluster = cg::this_cluster();
  extern __shared__ __align__(16) unsigned char smraw[];
  T *red = reinterpret_cast<T *>(smraw);   // [2][kClWarps - kChain][32]
  T *chn = red + 2 * (kClWarps - kChain) * 32;   // [2][kChain][32]
  T *part = chn + 2 * kChain * 32;        // [2][C][32]
  T *y = part + 2 * C * 32;               // [ring_rows(w)][32]
  const int j = blockIdx.x / C;
  const SubDesc *S = subs + j;
  const BandLayout L = lay[j];
  const int n = S->n_int;
  cluster.sync();                          // every CTA's shared memory is live
  const RingVec<T, GatherSrc<T>, ArrayDst<T>> fwd{ring_rows(L.w), n, {S, r, nnx, nny},
                                                  {yscr + S->v_int}};
  cluster_sweep_la<T, C>(cluster, poolL, L, y, red, chn, part, false, fwd);
  cluster.sync();                          // y complete in the scratch; the ring is reused
  const RingVec<T, ArraySrc<T>, ArrayDst<T>> bwd{ring_rows(L.w), n, {yscr + S->v_int},
                                                 {xloc + S->v_int}};
  cluster_sweep_la<T, C>(cluster, poolU, L, y, red, chn, part, true, bwd);
  cluster.sync();                          // no CTA leaves while others may still write to it
}

__global__ void __launch_bounds__(kClWarps * 32)
    k_band_solve_ring(const BandLayout *lay, const double *poolL, const double *poolU,
                      const double *in, long long in_sys, int in_row, double *out,
                      long long out_sys, int out_row, int mode) {
  cg::cluster_group cluster = cg::this_cluster();
  extern __shared__ __align__(16) unsigned char smraw[];
  double *red = reinterpret_cast<double *>(smraw);   // [2][kClWarps - kChain][32]
  double *chn = red + 2 * (kClWarps - kChain) * 32;   // [2][kChain][32]
  double *part = chn + 2 * kChain * 32;               // [2][1][32]
  double *y = part + 2 * 32;                          // [ring_rows(w)][32]
  const int j = blockIdx.x, c = blockIdx.y;
  const BandLayout L = lay[j];
  const double *src = in + j * in_sys + c;
  double *dst = out + j * out_sys + c;
  if (mode & 1) {
    const RingVec<double, StridedSrc, StridedDst> fwd{ring_rows(L.w), L.n, {src, in_row}, {dst, out_row}};
    cluster_sweep_la<double, 1>(cluster, poolL, L, y, red, chn, part, false, fwd);
    cluster.sync();
  }
  if (mode & 2) {
    const StridedSrc b = (mode & 1) ? StridedSrc{dst, out_row} : StridedSrc{src, in_row};
    const RingVec<double, StridedSrc, StridedDst> bwd{ring_rows(L.w), L.n, b, {dst, out_row}};
    cluster_sweep_la<double, 1>(cluster, poolU, L, y, red, chn, part, true, bwd);
  }
}

// ---- local solves of a batch of instances: one persistent launch ---------------
// Every CTA takes (instance, subdomain) items from a device work queue (the
// items are ordered largest local solve first, so the long ones start early
// and the short ones fill the tail) and runs the one-CTA form of the sweep the
// batch autotuner chose: look-ahead (R = 0) or one row per step (R = 1),
// tiles from global memory or staged in shared memory by bulk copies (St).
// The mbarriers of the staged forms are initialised once per CTA and their
// phase count carries over from item to item, as from the forward to the
// backward sweep.
template <typename T, int R, int St, bool kSC>
__global__ void __launch_bounds__(kClWarps * 32, 1)
    k_schwarz_batch(const BatchInst *inst, const CGScalars *cgs, const int2 *items, int nitems,
                    int *head, const double *__restrict__ r, int stride, DevStatus *status) {
  cg::cluster_group cluster = cg::this_cluster();
  extern __shared__ __align__(16) unsigned char smraw[];
  constexpr int RR = R > 0 ? R : 1;
  __shared__ int s_item;
  T *stages = nullptr, *red, *chn, *part, *y;
  uint64_t *mbar = nullptr, *mbx = nullptr;
  if constexpr (St) {
    stages = reinterpret_cast<T *>(smraw);
    mbar = reinterpret_cast<uint64_t *>(stages + kStages * stride);
    mbx = mbar + kStages;
    red = reinterpret_cast<T *>(mbx + kXBuf);
    chn = red + kClWarps * RR * 32;
    part = chn + 2 * kChain * RR * 32;
    y = part + kXBuf * RR * 32;
    if (threadIdx.x == 0) {
      for (int b = 0; b < kStages + kXBuf; ++b)
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(sm_addr(mbar + b)) : "memory");
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
  } else if constexpr (R == 0) {
    red = reinterpret_cast<T *>(smraw);   // [2][kClWarps - kChain][32]
    chn = red + 2 * (kClWarps - kChain) * 32;
    part = chn + 2 * kChain * 32;
    y = part + 2 * 32;
  } else {
    red = reinterpret_cast<T *>(smraw);   // [kClWarps][R][32]
    chn = red + kClWarps * R * 32;
    part = chn + 2 * kChain * R * 32;
    y = part + 2 * R * 32;
  }
  cluster.sync();
  uint32_t seq = 0;
  bool dead = false;
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(head, 1);
    __syncthreads();
    const int it = s_item;
    __syncthreads();                       // every thread has read the item before the next fetch
    if (it >= nitems) break;
    const int2 w = items[it];
    if (cgs[w.x].done) continue;
    const BatchInst &B = inst[w.x];
    const SubDesc &S = B.subs[w.y];
    const BandLayout L = B.lay[w.y];
    const T *poolL = static_cast<const T *>(B.facL), *poolU = static_cast<const T *>(B.facU);
    const double *rb = r + B.vbase;
    const int n = S.n_int, npad = L.nt * 32, nc = S.nc;
    for (int l = threadIdx.x; l < npad; l += blockDim.x) {
      T v = T(0);
      if (l < n) {
        const int node = l / nc, comp = l - nc * node;
        int gi, gj, gk;
        S.ibox.global(node, gi, gj, gk);
        v = T(rb[nc * (gi + B.nnx * (gj + B.nny * gk)) + comp]);
      }
      y[l] = v;
    }
    cluster.sync();
    if constexpr (St) {
      if constexpr (R == 0) {
        cluster_sweep_staged_la<T, 1, kSC>(poolL, 0, L, y, red, chn, part, false, stages, stride,
                                           mbar, mbx, seq, dead, status, w.y);
        cluster_sweep_staged_la<T, 1, kSC>(poolU, 0, L, y, red, chn, part, true, stages, stride,
                                           mbar, mbx, seq, dead, status, w.y);
      } else {
        cluster_sweep_staged<T, 1, R>(poolL, 0, L, y, red, chn, part, false, stages, stride, mbar,
                                      mbx, seq, dead, status, w.y);
        cluster_sweep_staged<T, 1, R>(poolU, 0, L, y, red, chn, part, true, stages, stride, mbar,
                                      mbx, seq, dead, status, w.y);
      }
    } else if constexpr (R == 0) {
      cluster_sweep_la<T, 1>(cluster, poolL, L, y, red, chn, part, false);
      cluster.sync();
      cluster_sweep_la<T, 1>(cluster, poolU, L, y, red, chn, part, true);
    } else {
      cluster_sweep<T, 1, R>(cluster, poolL, L, y, red, chn, part, false);
      cluster_sweep<T, 1, R>(cluster, poolU, L, y, red, chn, part, true);
    }
    T *out = static_cast<T *>(B.xloc) + S.v_int;
    for (int l = threadIdx.x; l < n; l += blockDim.x) out[l] = y[l];
    cluster.sync();                        // y and the buffers are reused by the next item
  }
}

template <typename T>
int smem_bytes(int npad, int C, int R) {
  if (R == 0) return ((2 * (kClWarps - kChain) + 2 * kChain + 2 * C) * 32 + npad) * (int)sizeof(T);
  return ((kClWarps + 2 * kChain + 2 * C) * R * 32 + npad) * (int)sizeof(T);
}

// The ring launches: the look-ahead buffers of C CTAs and the ring's tile rows.
template <typename T>
long long smem_bytes_ring(int w_max, int C = 1) {
  return ((2LL * (kClWarps - kChain) + 2 * kChain + 2 * C) * 32 +
          (long long)ring_rows(w_max) * 32) * sizeof(T);
}

// Tiles per stage of a staged launch; for the look-ahead sweep (R = 0) the two
// chain tiles are staged too when the whole launch then fits.
template <typename T>
long long smem_bytes_staged_t(int npad, int tiles, int C, int R) {
  const int RR = R > 0 ? R : 1;
  return (long long)kStages * tiles * 1024 * sizeof(T) + (kStages + kXBuf) * 8 +
         ((long long)(kClWarps + 2 * kChain + kXBuf * C) * RR * 32 + npad) * sizeof(T);
}

constexpr long long kSmemMax = 227 * 1024;

template <typename T>
int staged_tiles(int npad, int w, int C, int R, int *stage_chain) {
  *stage_chain = 0;
  if (R > 0) return stage_tiles(w, C, R);
  const int t = stage_tiles_la(w, C);
  if (smem_bytes_staged_t<T>(npad, t + 2, C, 0) <= kSmemMax) {
    *stage_chain = 1;
    return t + 2;
  }
  return t;
}

template <typename T>
long long smem_bytes_staged(int npad, int w, int C, int R) {
  int sc;
  return smem_bytes_staged_t<T>(npad, staged_tiles<T>(npad, w, C, R, &sc), C, R);
}

template <typename T, int C, int R>
int launch_cr(const SubDesc *d_subs, const BandLayout *d_lay, int nsub, int npad_max, int w_max,
              int staged, int nnx, int nny, const T *poolL, const T *poolU, const double *r,
              T *xloc, const CGScalars *cgs, DevStatus *status, cudaStream_t s) {
  if (!staged && smem_bytes<T>(npad_max, C, R) > kSmemMax) return GENEO_ERR_INVALID_ARG;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(nsub * C);
  cfg.blockDim = dim3(kClWarps * 32);
  cfg.dynamicSmemBytes = smem_bytes<T>(npad_max, C, R);
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  if constexpr (R <= 2) {
    if (staged) {
      const long long sm = smem_bytes_staged<T>(npad_max, w_max, C, R);
      if (sm > kSmemMax) return GENEO_ERR_INVALID_ARG;
      cfg.dynamicSmemBytes = (size_t)sm;
      int stage_chain;
      const int stride = staged_tiles<T>(npad_max, w_max, C, R, &stage_chain) * 1024;
      if (R == 0 && stage_chain) {
        GENEO_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_schwarz_cluster_staged<T, C, 0, true>, d_subs,
                                          d_lay, nnx, nny, poolL, poolU, r, xloc, cgs, stride,
                                          status));
      } else {
        GENEO_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_schwarz_cluster_staged<T, C, R, false>, d_subs,
                                          d_lay, nnx, nny, poolL, poolU, r, xloc, cgs, stride,
                                          status));
      }
    } else if constexpr (R == 0) {
      GENEO_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_schwarz_cluster_la<T, C>, d_subs, d_lay, nnx, nny,
                                        poolL, poolU, r, xloc, cgs));
    } else {
      GENEO_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_schwarz_cluster<T, C, R>, d_subs, d_lay, nnx, nny,
                                        poolL, poolU, r, xloc, cgs));
    }
  } else {
    if (staged) return GENEO_ERR_INVALID_ARG;
    GENEO_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_schwarz_cluster<T, C, R>, d_subs, d_lay, nnx, nny,
                                      poolL, poolU, r, xloc, cgs));
  }
  GENEO_COUNT_LAUNCH();
  return GENEO_OK;
}

template <typename T, int C>
int launch_c(int rows, int staged, const SubDesc *d_subs, const BandLayout *d_lay, int nsub,
             int npad_max, int w_max, int nnx, int nny, const T *poolL, const T *poolU,
             const double *r, T *xloc, const CGScalars *cgs, DevStatus *status, cudaStream_t s) {
  switch (rows) {
    case 0: return launch_cr<T, C, 0>(d_subs, d_lay, nsub, npad_max, w_max, staged, nnx, nny, poolL, poolU, r, xloc, cgs, status, s);
    case 4: return launch_cr<T, C, 4>(d_subs, d_lay, nsub, npad_max, w_max, staged, nnx, nny, poolL, poolU, r, xloc, cgs, status, s);
    case 2: return launch_cr<T, C, 2>(d_subs, d_lay, nsub, npad_max, w_max, staged, nnx, nny, poolL, poolU, r, xloc, cgs, status, s);
    default: return launch_cr<T, C, 1>(d_subs, d_lay, nsub, npad_max, w_max, staged, nnx, nny, poolL, poolU, r, xloc, cgs, status, s);
  }
}

// Opt in to the shared memory of every shape that fits (the others are never
// launched: the launchers refuse them).
template <typename T, int C>
int prepare_c(int npad_max, int w_max) {
  int st;
  auto fits = [&](int R) { return smem_bytes<T>(npad_max, C, R) <= kSmemMax; };
  if (fits(1) && (st = ensure_smem(k_schwarz_cluster<T, C, 1>, smem_bytes<T>(npad_max, C, 1)))) return st;
  if (fits(2) && (st = ensure_smem(k_schwarz_cluster<T, C, 2>, smem_bytes<T>(npad_max, C, 2)))) return st;
  if (fits(0) && (st = ensure_smem(k_schwarz_cluster_la<T, C>, smem_bytes<T>(npad_max, C, 0)))) return st;
  if (fits(4) && (st = ensure_smem(k_schwarz_cluster<T, C, 4>, smem_bytes<T>(npad_max, C, 4)))) return st;
  const long long s0 = smem_bytes_staged<T>(npad_max, w_max, C, 0);
  const long long s1 = smem_bytes_staged<T>(npad_max, w_max, C, 1);
  const long long s2 = smem_bytes_staged<T>(npad_max, w_max, C, 2);
  if (s0 <= kSmemMax) {
    if ((st = ensure_smem(k_schwarz_cluster_staged<T, C, 0, false>, (int)s0))) return st;
    if ((st = ensure_smem(k_schwarz_cluster_staged<T, C, 0, true>, (int)s0))) return st;
  }
  if (s1 <= kSmemMax && (st = ensure_smem(k_schwarz_cluster_staged<T, C, 1, false>, (int)s1))) return st;
  if (s2 <= kSmemMax && (st = ensure_smem(k_schwarz_cluster_staged<T, C, 2, false>, (int)s2))) return st;
  return GENEO_OK;
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
int prepare_schwarz_solve(int npad_max, int w_max) {
  if (smem_bytes_ring<T>(w_max, 8) > kSmemMax) return GENEO_ERR_INVALID_ARG;
  int st;
  if ((st = ensure_smem(k_schwarz_ring<T, 1>, (int)smem_bytes_ring<T>(w_max, 1)))) return st;
  if ((st = ensure_smem(k_schwarz_ring<T, 2>, (int)smem_bytes_ring<T>(w_max, 2)))) return st;
  if ((st = ensure_smem(k_schwarz_ring<T, 4>, (int)smem_bytes_ring<T>(w_max, 4)))) return st;
  if ((st = ensure_smem(k_schwarz_ring<T, 8>, (int)smem_bytes_ring<T>(w_max, 8)))) return st;
  if ((st = prepare_c<T, 1>(npad_max, w_max))) return st;
  if ((st = prepare_c<T, 2>(npad_max, w_max))) return st;
  if ((st = prepare_c<T, 4>(npad_max, w_max))) return st;
  return prepare_c<T, 8>(npad_max, w_max);
}

template <typename T>
bool schwarz_staged_fits(int npad_max, int w_max, int cluster, int rows) {
  return rows >= 0 && rows <= 2 && smem_bytes_staged<T>(npad_max, w_max, cluster, rows) <= kSmemMax;
}

template <typename T>
bool schwarz_shape_fits(int npad_max, int w_max, int cluster, int rows, int staged) {
  if (staged == 2)
    return (cluster == 1 || cluster == 2 || cluster == 4 || cluster == 8) && rows == 0 &&
           smem_bytes_ring<T>(w_max, cluster) <= kSmemMax;
  if (staged == 1) return schwarz_staged_fits<T>(npad_max, w_max, cluster, rows);
  return smem_bytes<T>(npad_max, cluster, rows) <= kSmemMax;
}

template <typename T, int C>
static int launch_ring(const SubDesc *d_subs, const BandLayout *d_lay, int nsub, int w_max,
                       int nnx, int nny, const T *poolL, const T *poolU, const double *r, T *xloc,
                       T *yscr, const CGScalars *cgs, cudaStream_t s) {
  const long long sm = smem_bytes_ring<T>(w_max, C);
  if (sm > kSmemMax || !yscr) return GENEO_ERR_INVALID_ARG;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(nsub * C);
  cfg.blockDim = dim3(kClWarps * 32);
  cfg.dynamicSmemBytes = (size_t)sm;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  GENEO_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_schwarz_ring<T, C>, d_subs, d_lay, nnx, nny, poolL,
                                    poolU, r, xloc, yscr, cgs));
  GENEO_COUNT_LAUNCH();
  return GENEO_OK;
}

template <typename T>
int launch_schwarz_solve(const SubDesc *d_subs, const BandLayout *d_lay, int nsub, int npad_max,
                         int w_max, int nnx, int nny, const T *poolL, const T *poolU,
                         const double *r, T *xloc, T *yscr, const CGScalars *cgs, int cluster,
                         int rows, int staged, DevStatus *status, cudaStream_t s) {
  if (staged == 2) {
    if (rows != 0) return GENEO_ERR_INVALID_ARG;
    switch (cluster) {
      case 1: return launch_ring<T, 1>(d_subs, d_lay, nsub, w_max, nnx, nny, poolL, poolU, r, xloc, yscr, cgs, s);
      case 2: return launch_ring<T, 2>(d_subs, d_lay, nsub, w_max, nnx, nny, poolL, poolU, r, xloc, yscr, cgs, s);
      case 4: return launch_ring<T, 4>(d_subs, d_lay, nsub, w_max, nnx, nny, poolL, poolU, r, xloc, yscr, cgs, s);
      case 8: return launch_ring<T, 8>(d_subs, d_lay, nsub, w_max, nnx, nny, poolL, poolU, r, xloc, yscr, cgs, s);
      default: return GENEO_ERR_INVALID_ARG;
    }
  }
  switch (cluster) {
    case 8: return launch_c<T, 8>(rows, staged, d_subs, d_lay, nsub, npad_max, w_max, nnx, nny, poolL, poolU, r, xloc, cgs, status, s);
    case 4: return launch_c<T, 4>(rows, staged, d_subs, d_lay, nsub, npad_max, w_max, nnx, nny, poolL, poolU, r, xloc, cgs, status, s);
    case 2: return launch_c<T, 2>(rows, staged, d_subs, d_lay, nsub, npad_max, w_max, nnx, nny, poolL, poolU, r, xloc, cgs, status, s);
    default: return launch_c<T, 1>(rows, staged, d_subs, d_lay, nsub, npad_max, w_max, nnx, nny, poolL, poolU, r, xloc, cgs, status, s);
  }
}

bool band_solve_fits(int w_max) { return smem_bytes_ring<double>(w_max) <= kSmemMax; }

int launch_band_solve_la(const BandLayout *d_lay, int nsys, int npad_max, int w_max, int ring,
                         const double *poolL, const double *poolU, const double *in,
                         long long in_sys, int in_row, double *out, long long out_sys,
                         int out_row, int ncols, int mode, cudaStream_t s) {
  const bool use_ring = ring || smem_bytes<double>(npad_max, 1, 0) > kSmemMax;
  const long long sm = use_ring ? smem_bytes_ring<double>(w_max) : smem_bytes<double>(npad_max, 1, 0);
  if (sm > kSmemMax) return GENEO_ERR_INVALID_ARG;
  if (int st = use_ring ? ensure_smem(k_band_solve_ring, (int)sm) : ensure_smem(k_band_solve_la, (int)sm))
    return st;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(nsys, ncols);
  cfg.blockDim = dim3(kClWarps * 32);
  cfg.dynamicSmemBytes = (size_t)sm;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = 1;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  if (use_ring) {
    GENEO_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_band_solve_ring, d_lay, poolL, poolU, in, in_sys,
                                      in_row, out, out_sys, out_row, mode));
  } else {
    GENEO_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_band_solve_la, d_lay, poolL, poolU, in, in_sys,
                                      in_row, out, out_sys, out_row, mode));
  }
  GENEO_COUNT_LAUNCH();
  return GENEO_OK;
}

// ---- batch launchers -----------------------------------------------------------
template <typename T>
static long long batch_smem(int npad_max, int w_max, int rows, int staged, int *stride,
                            int *stage_chain) {
  *stride = 0;
  *stage_chain = 0;
  if (!staged) return smem_bytes<T>(npad_max, 1, rows);
  const int tiles = staged_tiles<T>(npad_max, w_max, 1, rows, stage_chain);
  *stride = tiles * 1024;
  return smem_bytes_staged_t<T>(npad_max, tiles, 1, rows);
}

template <typename T>
bool batch_schwarz_fits(int npad_max, int w_max, int rows, int staged) {
  if (rows < 0 || rows > 1) return false;
  int st, sc;
  return batch_smem<T>(npad_max, w_max, rows, staged, &st, &sc) <= kSmemMax;
}

template <typename T>
int prepare_batch_schwarz(int npad_max, int w_max) {
  int st, stride, sc;
  long long b;
  if ((b = batch_smem<T>(npad_max, w_max, 0, 0, &stride, &sc)) <= kSmemMax &&
      (st = ensure_smem(k_schwarz_batch<T, 0, 0, false>, (int)b)))
    return st;
  if ((b = batch_smem<T>(npad_max, w_max, 1, 0, &stride, &sc)) <= kSmemMax &&
      (st = ensure_smem(k_schwarz_batch<T, 1, 0, false>, (int)b)))
    return st;
  if ((b = batch_smem<T>(npad_max, w_max, 0, 1, &stride, &sc)) <= kSmemMax) {
    if ((st = ensure_smem(k_schwarz_batch<T, 0, 1, false>, (int)b))) return st;
    if ((st = ensure_smem(k_schwarz_batch<T, 0, 1, true>, (int)b))) return st;
  }
  if ((b = batch_smem<T>(npad_max, w_max, 1, 1, &stride, &sc)) <= kSmemMax &&
      (st = ensure_smem(k_schwarz_batch<T, 1, 1, false>, (int)b)))
    return st;
  return GENEO_OK;
}

template <typename T>
int launch_batch_schwarz(const BatchInst *inst, const CGScalars *cg, const int2 *items,
                         int nitems, int *head, const double *r, int npad_max, int w_max,
                         int rows, int staged, int blocks, DevStatus *status, cudaStream_t s) {
  int stride, sc;
  const long long sm = batch_smem<T>(npad_max, w_max, rows, staged, &stride, &sc);
  if (sm > kSmemMax || rows < 0 || rows > 1) return GENEO_ERR_INVALID_ARG;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(blocks);
  cfg.blockDim = dim3(kClWarps * 32);
  cfg.dynamicSmemBytes = (size_t)sm;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = 1;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  if (staged) {
    if (rows == 0 && sc) {
      GENEO_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_schwarz_batch<T, 0, 1, true>, inst, cg, items,
                                        nitems, head, r, stride, status));
    } else if (rows == 0) {
      GENEO_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_schwarz_batch<T, 0, 1, false>, inst, cg, items,
                                        nitems, head, r, stride, status));
    } else {
      GENEO_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_schwarz_batch<T, 1, 1, false>, inst, cg, items,
                                        nitems, head, r, stride, status));
    }
  } else if (rows == 0) {
    GENEO_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_schwarz_batch<T, 0, 0, false>, inst, cg, items,
                                      nitems, head, r, stride, status));
  } else {
    GENEO_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_schwarz_batch<T, 1, 0, false>, inst, cg, items,
                                      nitems, head, r, stride, status));
  }
  GENEO_COUNT_LAUNCH();
  return GENEO_OK;
}

template bool batch_schwarz_fits<double>(int, int, int, int);
template bool batch_schwarz_fits<float>(int, int, int, int);
template int prepare_batch_schwarz<double>(int, int);
template int prepare_batch_schwarz<float>(int, int);
template int launch_batch_schwarz<double>(const BatchInst *, const CGScalars *, const int2 *, int,
                                          int *, const double *, int, int, int, int, int,
                                          DevStatus *, cudaStream_t);
template int launch_batch_schwarz<float>(const BatchInst *, const CGScalars *, const int2 *, int,
                                         int *, const double *, int, int, int, int, int,
                                         DevStatus *, cudaStream_t);

template int prepare_schwarz_solve<double>(int, int);
template int prepare_schwarz_solve<float>(int, int);
template bool schwarz_shape_fits<double>(int, int, int, int, int);
template bool schwarz_shape_fits<float>(int, int, int, int, int);
template bool schwarz_staged_fits<double>(int, int, int, int);
template bool schwarz_staged_fits<float>(int, int, int, int);
template int launch_schwarz_solve<double>(const SubDesc *, const BandLayout *, int, int, int, int,
                                          int, const double *, const double *, const double *,
                                          double *, double *, const CGScalars *, int, int, int,
                                          DevStatus *, cudaStream_t);
template int launch_schwarz_solve<float>(const SubDesc *, const BandLayout *, int, int, int, int,
                                         int, const float *, const float *, const double *,
                                         float *, float *, const CGScalars *, int, int, int,
                                         DevStatus *, cudaStream_t);

}  // namespace geneo
