// Shared definitions for the GenEO-PCG CUDA library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <stddef.h>

#include "../../include/geneo.h"

#define GENEO_CUDA_TRY(expr)                                   \
  do {                                                         \
    cudaError_t _e = (expr);                                   \
    if (_e != cudaSuccess) {                                   \
      geneo_set_last_cuda_error(_e, #expr, __FILE__, __LINE__); \
      return GENEO_ERR_CUDA;                                   \
    }                                                          \
  } while (0)

void geneo_set_last_cuda_error(cudaError_t e, const char *what, const char *file, int line);
void geneo_set_last_message(const char *msg);

namespace geneo {

// Kernel launches enqueued by this library (graph launches add their kernel
// nodes); a thread that is capturing a graph counts them only in its own
// thread-local counter, so the global count is not inflated by captures.
extern std::atomic<long long> g_launch_count;   // all threads, enqueued launches
extern thread_local bool g_counting;             // false while this thread captures a graph
extern thread_local long long g_thread_launches; // this thread's launches incl. captured ones
#define GENEO_COUNT_LAUNCH()                                                              \
  (++geneo::g_thread_launches,                                                            \
   geneo::g_launch_count.fetch_add(geneo::g_counting ? 1 : 0, std::memory_order_relaxed))

// Raise a kernel's dynamic shared memory limit to at least `bytes`.  The limit
// is a process-wide attribute of the function, so contexts on concurrent host
// threads only ever raise it (under a lock): a smaller problem set up on one
// thread cannot lower the limit under another thread's pending launch.
int ensure_smem_raw(const void *func, int bytes);
template <typename F>
inline int ensure_smem(F *func, int bytes) {
  return ensure_smem_raw(reinterpret_cast<const void *>(func), bytes);
}

constexpr int kTile = 32;          // band tile edge (rows = columns = one warp)
constexpr int kLanczosBlock = 8;   // block Lanczos block size p
constexpr int kMaxModes = 32;      // cap on modes kept per subdomain
constexpr int kMaxCand = 4;        // max subdomains containing a node, per axis
constexpr int kRedBlocks = 304;    // 2 x 152 SMs: grid of the reduction kernels
constexpr int kRedThreads = 256;

// ---------------------------------------------------------------------------
// Device status word: kernels never trap; they record the first error here.
struct DevStatus {
  int code;        // 0 = ok, else GENEO_ERR_*
  int where;       // subdomain / index of the failure
  int detail;      // e.g. the row of a failed pivot
};

// ---------------------------------------------------------------------------
// Bump allocator over one device workspace; a pass with base == nullptr only
// measures.
struct Arena {
  char *base = nullptr;
  size_t cap = 0;
  size_t off = 0;
  template <typename T>
  T *take(size_t n) {
    size_t a = (off + 255) & ~size_t(255);
    off = a + n * sizeof(T);
    return base ? reinterpret_cast<T *>(base + a) : nullptr;
  }
  bool fits() const { return off <= cap; }
};

// ---------------------------------------------------------------------------
// Axis-aligned node box with a local numbering whose fastest axis is perm[0]
// and slowest perm[2] (the band ordering: the longest axis goes slowest).
struct NodeBox {
  int lo[3];       // first global node coordinate per axis
  int n[3];        // number of nodes per axis
  int perm[3];     // local axis order, fastest first
  __host__ __device__ int count() const { return n[0] * n[1] * n[2]; }
  // local index of global node coordinates (i, j, k); -1 if outside
  __host__ __device__ int local(int i, int j, int k) const {
    int c[3] = {i - lo[0], j - lo[1], k - lo[2]};
    if (c[0] < 0 || c[1] < 0 || c[2] < 0 || c[0] >= n[0] || c[1] >= n[1] || c[2] >= n[2])
      return -1;
    return c[perm[0]] + n[perm[0]] * (c[perm[1]] + n[perm[1]] * c[perm[2]]);
  }
  // global node coordinates of local node l
  __host__ __device__ void global(int l, int &i, int &j, int &k) const {
    int c[3];
    int a = l % n[perm[0]];
    int r = l / n[perm[0]];
    int b = r % n[perm[1]];
    int d = r / n[perm[1]];
    c[perm[0]] = a;
    c[perm[1]] = b;
    c[perm[2]] = d;
    i = lo[0] + c[0];
    j = lo[1] + c[1];
    k = lo[2] + c[2];
  }
  // half bandwidth in dofs of a 27-point coupling in this numbering with nc
  // unknowns per node
  __host__ __device__ int half_band_dofs(int nc = 3) const {
    int nf = n[perm[0]], nm = n[perm[1]], ns = n[perm[2]];
    int dn = (nf > 1 ? 1 : 0) + (nm > 1 ? nf : 0) + (ns > 1 ? nf * nm : 0);
    return nc * dn + nc - 1;
  }
};

// Per-subdomain descriptor (host and device).
struct SubDesc {
  int nc;          // unknowns per node: 3 elasticity, 1 Darcy
  NodeBox ibox;    // nodes of V_{h,0}(Omega_j) (interior)
  NodeBox nbox;    // all nodes of Omega_j (Neumann set)
  int elo[3], ehi[3];   // element box of Omega_j, half-open
  // interior band factor (A_j)
  int n_int, nt_int, w_int;
  long long f_int;      // element offset of the tiles in the factor pool
  long long v_int;      // offset of the local vector buffer (n_pad entries)
  // Neumann band factor (S_j) and local BSR of B_j
  int n_neu, nt_neu, w_neu;
  long long f_neu;      // element offset (FP64) in the Neumann factor pool
  long long b_neu;      // block offset of B_j's 27-slot local BSR
  long long x_neu;      // offset of X_j on Neumann dofs
  // coarse space
  int m;                // modes kept
  int coff;             // first coarse index of this subdomain
  long long z_off;      // offset of Z_j (n_int x m, row-major) in the Z pool
};

// Distance of node (i, j, k) to the artificial boundary of Omega_j (the faces
// of its element box that lie inside the domain of nx x ny x nz elements),
// counted in element layers: the least distance to such a face's plane; 1
// when Omega_j has no artificial face (the whole domain).  The weight of the
// Sarkis partition of unity (Sec. 3.2, Sec. 3.3.1) is this distance over its
// sum across the subdomains whose interior holds the node.
__host__ __device__ __forceinline__ int artificial_distance(const SubDesc &S, int i, int j, int k,
                                                            int nx, int ny, int nz) {
  const int pos[3] = {i, j, k}, ne[3] = {nx, ny, nz};
  int d = 0x7fffffff;
  for (int a = 0; a < 3; ++a) {
    if (S.elo[a] > 0) d = min(d, pos[a] - S.elo[a]);
    if (S.ehi[a] < ne[a]) d = min(d, S.ehi[a] - pos[a]);
  }
  return d == 0x7fffffff ? 1 : d;
}

// ---------------------------------------------------------------------------
// Deterministic block reduction helpers.
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum over the block in a fixed order; result valid in thread 0.
template <int NT>
__device__ __forceinline__ double block_sum(double v, double *sh) {
  v = warp_sum(v);
  int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) sh[w] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x < 32) {
    r = (l < NT / 32) ? sh[l] : 0.0;
    r = warp_sum(r);
  }
  __syncthreads();
  return r;
}

}  // namespace geneo
