// Allocation-free variant of the fused SpMV + dot-product kernel.
//
// Some callers cannot allocate device memory at all: code that runs inside a
// fixed device-memory budget carved out by a host framework, a real-time
// control loop that must not enter the CUDA allocator, or a plug-in that only
// receives pointers to buffers owned by someone else.  For them
// geneo_spmv_dot_noalloc computes y = A x and x . y with no cudaMalloc, no
// cudaFree and no allocating library call: its only scratch (one partial sum
// per thread block and a ticket counter) lives in a file-scope __device__
// array below, which every GPU that loads this library holds until exit.
#include <mutex>

#include "kernels.cuh"

namespace geneo {

namespace {

constexpr int kNaRowsPerBlock = 8;            // one warp per block row, 8 warps
constexpr int kNaMaxPartials = 65536;         // scratch: 512 KiB of partial sums
constexpr int kNaMaxNodes = kNaRowsPerBlock * kNaMaxPartials;   // 524,288 block rows
constexpr int kNaMaxDevices = 64;

// Scratch: [0, kNaMaxPartials) partial sums, then the ticket counter.
static __device__ __align__(256) double g_noalloc_scratch[kNaMaxPartials + 32];

struct NaSetup {
  std::once_flag once;
  double *ptr = nullptr;
  cudaError_t err = cudaSuccess;
};
NaSetup g_na[kNaMaxDevices];

__global__ void __launch_bounds__(256)
    k_spmv_dot_noalloc(int nnode, const int32_t *__restrict__ rp, const int32_t *__restrict__ col,
                       const double *__restrict__ val, const double *__restrict__ x,
                       double *__restrict__ y, double *__restrict__ xy,
                       double *__restrict__ scratch) {
  __shared__ double sh[8];
  __shared__ bool is_last;
  unsigned int *counter = reinterpret_cast<unsigned int *>(scratch + kNaMaxPartials);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int row = blockIdx.x * kNaRowsPerBlock + warp;
  double acc = 0.0;
  if (row < nnode) {
    const int base = rp[row];
    const int ne = 9 * (rp[row + 1] - base);
    const double *v = val + 9 * (size_t)base;
    double a0 = 0.0, a1 = 0.0, a2 = 0.0;
    for (int e = lane; e < ne; e += 32) {
      const int blk = e / 9;        // exact for any row length
      const int rc = e - 9 * blk;
      const int r = rc / 3;
      double prod = v[e] * x[3 * col[base + blk] + rc - 3 * r];
      if (r == 0) a0 += prod;
      else if (r == 1) a1 += prod;
      else a2 += prod;
    }
    a0 = warp_sum(a0);
    a1 = warp_sum(a1);
    a2 = warp_sum(a2);
    if (lane == 0) {
      y[3 * row] = a0;
      y[3 * row + 1] = a1;
      y[3 * row + 2] = a2;
      acc = x[3 * row] * a0 + x[3 * row + 1] * a1 + x[3 * row + 2] * a2;
    }
  }
  if (lane == 0) sh[warp] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < 8; ++w) s += sh[w];
    scratch[blockIdx.x] = s;
    __threadfence();
    unsigned t = atomicAdd(counter, 1u);
    is_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!is_last) return;
  // last block: fixed-order sum of the partials (deterministic)
  __threadfence();
  double s = 0.0;
  for (int i = threadIdx.x; i < (int)gridDim.x; i += 256) s += ((volatile double *)scratch)[i];
  s = warp_sum(s);
  if (lane == 0) sh[warp] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += sh[w];
    *xy = t;
    *counter = 0;
  }
}

}  // namespace

}  // namespace geneo

using namespace geneo;

extern "C" int geneo_spmv_dot_noalloc(int n_nodes, const int32_t *row_ptr, const int32_t *col,
                                      const double *val, const double *x, double *y, double *xy,
                                      void *cuda_stream) {
  if (n_nodes < 1 || !row_ptr || !col || !val || !x || !y || !xy) {
    geneo_set_last_message("geneo_spmv_dot_noalloc: null pointer or n_nodes < 1");
    return GENEO_ERR_INVALID_ARG;
  }
  if (n_nodes > kNaMaxNodes) {
    geneo_set_last_message("geneo_spmv_dot_noalloc: n_nodes exceeds the static scratch limit of "
                           "524288 block rows");
    return GENEO_ERR_WORKSPACE_TOO_SMALL;
  }
  {
    // y is written while other warps still read x: the two must not overlap
    const char *xb = reinterpret_cast<const char *>(x);
    const char *yb = reinterpret_cast<const char *>(y);
    const size_t len = 3 * sizeof(double) * (size_t)n_nodes;
    if (xb < yb + len && yb < xb + len) {
      geneo_set_last_message("geneo_spmv_dot_noalloc: x and y overlap (in-place calls are not "
                             "supported)");
      return GENEO_ERR_INVALID_ARG;
    }
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    geneo_set_last_cuda_error(e, "cudaGetDevice", __FILE__, __LINE__);
    return GENEO_ERR_CUDA;
  }
  if (dev < 0 || dev >= kNaMaxDevices) {
    geneo_set_last_message("geneo_spmv_dot_noalloc: device ordinal above 63");
    return GENEO_ERR_INVALID_ARG;
  }
  // once per device, with that device current: device address of the scratch
  NaSetup &S = g_na[dev];
  std::call_once(S.once, [&S]() {
    S.err = cudaGetSymbolAddress(reinterpret_cast<void **>(&S.ptr), g_noalloc_scratch);
  });
  if (S.err != cudaSuccess || !S.ptr) {
    geneo_set_last_cuda_error(S.err, "cudaGetSymbolAddress(scratch)", __FILE__, __LINE__);
    return GENEO_ERR_CUDA;
  }
  cudaStream_t s = (cudaStream_t)cuda_stream;
  // the ticket counter must start at zero (a previous call may have been cut short)
  e = cudaMemsetAsync(S.ptr + kNaMaxPartials, 0, sizeof(unsigned int), s);
  if (e != cudaSuccess) {
    geneo_set_last_cuda_error(e, "cudaMemsetAsync(scratch counter)", __FILE__, __LINE__);
    return GENEO_ERR_CUDA;
  }
  const int blocks = (n_nodes + kNaRowsPerBlock - 1) / kNaRowsPerBlock;
  k_spmv_dot_noalloc<<<blocks, 256, 0, s>>>(n_nodes, row_ptr, col, val, x, y, xy, S.ptr);
  GENEO_COUNT_LAUNCH();
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    geneo_set_last_cuda_error(e, "k_spmv_dot_noalloc launch", __FILE__, __LINE__);
    return GENEO_ERR_CUDA;
  }
  return GENEO_OK;
}
