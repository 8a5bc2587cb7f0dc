// Assembly of A u = b (Sec. 2, eqn:fe_matrix_system) into 3x3-block BSR.
//
// Rather than scattering element matrices with atomics, each (node, neighbour)
// block is gathered from the (1, 2, 4 or 8) elements that contain both nodes:
// every block is written once, in order, with no atomics, so assembly is
// deterministic.  The element stiffness is integrated with 2x2x2 Gauss points.
#include "fem.cuh"
#include "kernels.cuh"

namespace geneo {

__global__ void k_material_base(int n_mat, const geneo_ortho *__restrict__ mats,
                                double *__restrict__ C0) {
  int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= n_mat) return;
  material_stiffness(mats[m], C0 + 36 * m);
}

__global__ void k_element_C(int nel, int n_mat, const double *__restrict__ C0,
                            const int32_t *__restrict__ emat, const double *__restrict__ th,
                            const double *__restrict__ ph, double *__restrict__ Cel,
                            DevStatus *st) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nel) return;
  int m = emat[e];
  if (m < 0 || m >= n_mat) {
    atomicCAS(&st->code, 0, GENEO_ERR_INVALID_ARG);
    m = 0;
  }
  double C[36];
  for (int i = 0; i < 36; ++i) C[i] = C0[36 * m + i];
  rotate_voigt(C, th[e], ph ? ph[e] : 0.0, Cel + 36 * (size_t)e);
}

__device__ __forceinline__ void node_ijk(int n, int nnx, int nny, int &i, int &j, int &k) {
  i = n % nnx;
  int r = n / nnx;
  j = r % nny;
  k = r / nny;
}

__device__ __forceinline__ bool slot_valid(int s, int i, int j, int k, int nnx, int nny, int nnz) {
  int di = s % 3 - 1, dj = (s / 3) % 3 - 1, dk = s / 9 - 1;
  return (unsigned)(i + di) < (unsigned)nnx && (unsigned)(j + dj) < (unsigned)nny &&
         (unsigned)(k + dk) < (unsigned)nnz;
}

__global__ void k_bsr_count(int nnx, int nny, int nnz, int32_t *__restrict__ cnt) {
  int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= nnx * nny * nnz) return;
  int i, j, k;
  node_ijk(n, nnx, nny, i, j, k);
  int cx = 1 + (i > 0) + (i < nnx - 1);
  int cy = 1 + (j > 0) + (j < nny - 1);
  int cz = 1 + (k > 0) + (k < nnz - 1);
  cnt[n] = cx * cy * cz;
}

// Exclusive scan of cnt[0..n) into out[0..n], one block (setup only).
__global__ void k_scan_single(int n, const int32_t *__restrict__ cnt, int32_t *__restrict__ out) {
  __shared__ int32_t sh[1024];
  __shared__ int32_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < n; base += 1024) {
    int idx = base + threadIdx.x;
    int v = idx < n ? cnt[idx] : 0;
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
      int t = threadIdx.x >= o ? sh[threadIdx.x - o] : 0;
      __syncthreads();
      sh[threadIdx.x] += t;
      __syncthreads();
    }
    if (idx < n) out[idx] = carry + sh[threadIdx.x] - v;
    __syncthreads();
    if (threadIdx.x == 1023) carry += sh[1023];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[n] = carry;
}

__global__ void k_bsr_fill(int nnx, int nny, int nnz, const int32_t *__restrict__ row_ptr,
                           int32_t *__restrict__ col) {
  int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= nnx * nny * nnz) return;
  int i, j, k;
  node_ijk(n, nnx, nny, i, j, k);
  int pos = row_ptr[n];
  for (int s = 0; s < 27; ++s) {
    if (!slot_valid(s, i, j, k, nnx, nny, nnz)) continue;
    int di = s % 3 - 1, dj = (s / 3) % 3 - 1, dk = s / 9 - 1;
    col[pos++] = (i + di) + nnx * ((j + dj) + nny * (k + dk));
  }
}

// One thread per (node, neighbour slot): sum the element blocks of the
// elements shared by the two nodes.
__global__ void k_assemble_values(int nx, int ny, int nz, const double *__restrict__ X,
                                  const double *__restrict__ Y, const double *__restrict__ Z,
                                  const double *__restrict__ Cel,
                                  const int32_t *__restrict__ row_ptr,
                                  double *__restrict__ val) {
  int nnx = nx + 1, nny = ny + 1, nnz = nz + 1;
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)nnx * nny * nnz * 27) return;
  int n = (int)(t / 27), s = (int)(t % 27);
  int i, j, k;
  node_ijk(n, nnx, nny, i, j, k);
  if (!slot_valid(s, i, j, k, nnx, nny, nnz)) return;
  int pos = row_ptr[n];
  for (int q = 0; q < s; ++q) pos += slot_valid(q, i, j, k, nnx, nny, nnz);
  int i2 = i + s % 3 - 1, j2 = j + (s / 3) % 3 - 1, k2 = k + s / 9 - 1;
  double acc[9];
  for (int q = 0; q < 9; ++q) acc[q] = 0.0;
  for (int ez = max(max(k, k2) - 1, 0); ez <= min(min(k, k2), nz - 1); ++ez)
    for (int ey = max(max(j, j2) - 1, 0); ey <= min(min(j, j2), ny - 1); ++ey)
      for (int ex = max(max(i, i2) - 1, 0); ex <= min(min(i, i2), nx - 1); ++ex) {
        int e = ex + nx * (ey + ny * ez);
        int a = (i - ex) + 2 * (j - ey) + 4 * (k - ez);
        int b = (i2 - ex) + 2 * (j2 - ey) + 4 * (k2 - ez);
        double Kb[9];
        element_block(Cel + 36 * (size_t)e, X[ex + 1] - X[ex], Y[ey + 1] - Y[ey],
                      Z[ez + 1] - Z[ez], a, b, Kb);
        for (int q = 0; q < 9; ++q) acc[q] += Kb[q];
      }
  double *out = val + 9 * (size_t)pos;
  for (int q = 0; q < 9; ++q) out[q] = acc[q];
}

// Consistent nodal load of the traction (0, 0, -q) on the face z = z_max
// (int over a bilinear face of N_a = area / 4) plus an optional nodal load.
__global__ void k_load(int nx, int ny, int nz, const double *__restrict__ X,
                       const double *__restrict__ Y, double q,
                       const double *__restrict__ nodal, double *__restrict__ b) {
  int nnx = nx + 1, nny = ny + 1;
  int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= nnx * nny * (nz + 1)) return;
  int i, j, k;
  node_ijk(n, nnx, nny, i, j, k);
  double f[3] = {0.0, 0.0, 0.0};
  if (k == nz && q != 0.0) {
    for (int ey = max(j - 1, 0); ey <= min(j, ny - 1); ++ey)
      for (int ex = max(i - 1, 0); ex <= min(i, nx - 1); ++ex)
        f[2] -= q * (X[ex + 1] - X[ex]) * (Y[ey + 1] - Y[ey]) * 0.25;
  }
  for (int c = 0; c < 3; ++c) b[3 * n + c] = f[c] + (nodal ? nodal[3 * n + c] : 0.0);
}

__global__ void k_dirichlet_mark(int nd, const int32_t *__restrict__ dofs,
                                 const double *__restrict__ vals, int ndof,
                                 uint8_t *__restrict__ mask, double *__restrict__ g,
                                 DevStatus *st) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nd) return;
  int d = dofs[t];
  if (d < 0 || d >= ndof) {
    atomicCAS(&st->code, 0, GENEO_ERR_INVALID_ARG);
    return;
  }
  mask[d] = 1;
  g[d] = vals ? vals[t] : 0.0;
}

// Lifting of the Dirichlet data (Sec. 2, u = g on the clamped face):
// lift_i = -sum_{c in D} A_ic g_c on free rows, lift_i = g_i on Dirichlet rows.
// It is kept so that a new load reuses it without the eliminated columns.
__global__ void k_dirichlet_lift(int nnode, int nc, const int32_t *__restrict__ row_ptr,
                                 const int32_t *__restrict__ col, const double *__restrict__ val,
                                 const uint8_t *__restrict__ mask, const double *__restrict__ g,
                                 double *__restrict__ lift) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nc * nnode) return;
  int n = t / nc, r = t % nc;
  if (mask[t]) {
    lift[t] = g[t];
    return;
  }
  double s = 0.0;
  for (int p = row_ptr[n]; p < row_ptr[n + 1]; ++p) {
    int cn = col[p];
    for (int c = 0; c < nc; ++c)
      if (mask[nc * cn + c]) s += val[(size_t)nc * nc * p + nc * r + c] * g[nc * cn + c];
  }
  lift[t] = -s;
}

// b_i = f_i + lift_i on free rows, b_i = g_i on Dirichlet rows.
__global__ void k_apply_lift(int n3, const uint8_t *__restrict__ mask,
                             const double *__restrict__ lift, double *__restrict__ b) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n3) return;
  b[t] = mask[t] ? lift[t] : b[t] + lift[t];
}

// Zero Dirichlet rows and columns, unit diagonal (nc unknowns per node).
__global__ void k_dirichlet_eliminate(int nnode, int nc, const int32_t *__restrict__ row_ptr,
                                      const int32_t *__restrict__ col,
                                      const uint8_t *__restrict__ mask,
                                      double *__restrict__ val) {
  int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= nnode) return;
  bool anyrow = false;
  for (int r = 0; r < nc; ++r) anyrow |= mask[nc * n + r] != 0;
  for (int p = row_ptr[n]; p < row_ptr[n + 1]; ++p) {
    int cn = col[p];
    bool anycol = false;
    for (int c = 0; c < nc; ++c) anycol |= mask[nc * cn + c] != 0;
    if (!anyrow && !anycol) continue;
    for (int r = 0; r < nc; ++r)
      for (int c = 0; c < nc; ++c)
        if (mask[nc * n + r] || mask[nc * cn + c])
          val[(size_t)nc * nc * p + nc * r + c] = (cn == n && r == c) ? 1.0 : 0.0;
  }
}

// ---- scalar Darcy problem (eqn:Darcy, eq-fe-darcy): one unknown per node ----

// One thread per (node, neighbour slot), gathered from the shared elements.
__global__ void k_assemble_values_darcy(int nx, int ny, int nz, const double *__restrict__ X,
                                        const double *__restrict__ Y,
                                        const double *__restrict__ Z,
                                        const double *__restrict__ perm,
                                        const int32_t *__restrict__ row_ptr,
                                        double *__restrict__ val) {
  int nnx = nx + 1, nny = ny + 1, nnz = nz + 1;
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)nnx * nny * nnz * 27) return;
  int n = (int)(t / 27), s = (int)(t % 27);
  int i, j, k;
  node_ijk(n, nnx, nny, i, j, k);
  if (!slot_valid(s, i, j, k, nnx, nny, nnz)) return;
  int pos = row_ptr[n];
  for (int q = 0; q < s; ++q) pos += slot_valid(q, i, j, k, nnx, nny, nnz);
  int i2 = i + s % 3 - 1, j2 = j + (s / 3) % 3 - 1, k2 = k + s / 9 - 1;
  double acc = 0.0;
  for (int ez = max(max(k, k2) - 1, 0); ez <= min(min(k, k2), nz - 1); ++ez)
    for (int ey = max(max(j, j2) - 1, 0); ey <= min(min(j, j2), ny - 1); ++ey)
      for (int ex = max(max(i, i2) - 1, 0); ex <= min(min(i, i2), nx - 1); ++ex) {
        int e = ex + nx * (ey + ny * ez);
        int a = (i - ex) + 2 * (j - ey) + 4 * (k - ez);
        int b = (i2 - ex) + 2 * (j2 - ey) + 4 * (k2 - ez);
        acc += darcy_entry(perm + 3 * (size_t)e, X[ex + 1] - X[ex], Y[ey + 1] - Y[ey],
                           Z[ez + 1] - Z[ez], a, b);
      }
  val[pos] = acc;
}

// b_n = int f N_n dx = sum over the elements of node n of f V_e / 8, plus nodal.
__global__ void k_load_darcy(int nx, int ny, int nz, const double *__restrict__ X,
                             const double *__restrict__ Y, const double *__restrict__ Z,
                             double f, const double *__restrict__ nodal, double *__restrict__ b) {
  int nnx = nx + 1, nny = ny + 1;
  int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= nnx * nny * (nz + 1)) return;
  int i, j, k;
  node_ijk(n, nnx, nny, i, j, k);
  double v = 0.0;
  if (f != 0.0)
    for (int ez = max(k - 1, 0); ez <= min(k, nz - 1); ++ez)
      for (int ey = max(j - 1, 0); ey <= min(j, ny - 1); ++ey)
        for (int ex = max(i - 1, 0); ex <= min(i, nx - 1); ++ex)
          v += f * (X[ex + 1] - X[ex]) * (Y[ey + 1] - Y[ey]) * (Z[ez + 1] - Z[ez]) * 0.125;
  b[n] = v + (nodal ? nodal[n] : 0.0);
}

// ---------------------------------------------------------------------------
int launch_assembly(const AssemblyArgs &a, cudaStream_t s) {
  const int T = 256;
  int nnx = a.nx + 1, nny = a.ny + 1, nnz = a.nz + 1;
  int nnode = nnx * nny * nnz;
  int nel = a.nx * a.ny * a.nz;
  k_material_base<<<(a.n_mat + 63) / 64, 64, 0, s>>>(a.n_mat, a.mats, a.C0); GENEO_COUNT_LAUNCH();
  k_element_C<<<(nel + T - 1) / T, T, 0, s>>>(nel, a.n_mat, a.C0, a.emat, a.theta, a.phi,
                                              a.Cel, a.status); GENEO_COUNT_LAUNCH();
  k_bsr_count<<<(nnode + T - 1) / T, T, 0, s>>>(nnx, nny, nnz, a.cnt); GENEO_COUNT_LAUNCH();
  k_scan_single<<<1, 1024, 0, s>>>(nnode, a.cnt, a.row_ptr); GENEO_COUNT_LAUNCH();
  k_bsr_fill<<<(nnode + T - 1) / T, T, 0, s>>>(nnx, nny, nnz, a.row_ptr, a.col); GENEO_COUNT_LAUNCH();
  long long nt = (long long)nnode * 27;
  k_assemble_values<<<(unsigned)((nt + 127) / 128), 128, 0, s>>>(
      a.nx, a.ny, a.nz, a.X, a.Y, a.Z, a.Cel, a.row_ptr, a.val); GENEO_COUNT_LAUNCH();
  k_load<<<(nnode + T - 1) / T, T, 0, s>>>(a.nx, a.ny, a.nz, a.X, a.Y, a.top_pressure,
                                           a.nodal, a.b); GENEO_COUNT_LAUNCH();
  GENEO_CUDA_TRY(cudaMemsetAsync(a.mask, 0, 3 * (size_t)nnode, s));
  GENEO_CUDA_TRY(cudaMemsetAsync(a.g, 0, 3 * (size_t)nnode * sizeof(double), s));
  if (a.n_dir > 0) {
    k_dirichlet_mark<<<(a.n_dir + T - 1) / T, T, 0, s>>>(a.n_dir, a.dir_dofs, a.dir_vals,
                                                         3 * nnode, a.mask, a.g, a.status); GENEO_COUNT_LAUNCH();
    k_dirichlet_lift<<<(3 * nnode + T - 1) / T, T, 0, s>>>(nnode, 3, a.row_ptr, a.col, a.val,
                                                           a.mask, a.g, a.lift); GENEO_COUNT_LAUNCH();
    k_apply_lift<<<(3 * nnode + T - 1) / T, T, 0, s>>>(3 * nnode, a.mask, a.lift, a.b); GENEO_COUNT_LAUNCH();
    k_dirichlet_eliminate<<<(nnode + T - 1) / T, T, 0, s>>>(nnode, 3, a.row_ptr, a.col, a.mask,
                                                            a.val); GENEO_COUNT_LAUNCH();
  }
  GENEO_CUDA_TRY(cudaGetLastError());
  return GENEO_OK;
}

// Stress recovery at the element centres: sigma_e = C_e B(0) u_e (Voigt order
// 11, 22, 33, 23, 13, 12; engineering shear strains).  At the centre of a box
// element dN_a/dx_d = s_d / (4 h_d) with the corner sign s_d = +-1.
__global__ void k_element_stress(int nx, int ny, int nz, const double *__restrict__ X,
                                 const double *__restrict__ Y, const double *__restrict__ Z,
                                 const double *__restrict__ Cel, const double *__restrict__ u,
                                 double *__restrict__ sig) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nx * ny * nz) return;
  const int ex = e % nx, ey = (e / nx) % ny, ez = e / (nx * ny);
  const int nnx = nx + 1, nny = ny + 1;
  const double ih[3] = {0.25 / (X[ex + 1] - X[ex]), 0.25 / (Y[ey + 1] - Y[ey]),
                        0.25 / (Z[ez + 1] - Z[ez])};
  double du[3][3] = {{0.0, 0.0, 0.0}, {0.0, 0.0, 0.0}, {0.0, 0.0, 0.0}};   // du_i / dx_d
  for (int a = 0; a < 8; ++a) {
    const int ia = a & 1, ja = (a >> 1) & 1, ka = (a >> 2) & 1;
    const long long n = (ex + ia) + (long long)nnx * ((ey + ja) + (long long)nny * (ez + ka));
    const double g[3] = {(2 * ia - 1) * ih[0], (2 * ja - 1) * ih[1], (2 * ka - 1) * ih[2]};
    for (int i = 0; i < 3; ++i) {
      const double ui = u[3 * n + i];
      for (int d = 0; d < 3; ++d) du[i][d] += g[d] * ui;
    }
  }
  const double eps[6] = {du[0][0], du[1][1], du[2][2], du[1][2] + du[2][1], du[0][2] + du[2][0],
                         du[0][1] + du[1][0]};
  const double *C = Cel + 36 * (size_t)e;
  for (int r = 0; r < 6; ++r) {
    double s = 0.0;
    for (int c = 0; c < 6; ++c) s += C[6 * r + c] * eps[c];
    sig[6 * (size_t)e + r] = s;
  }
}

int launch_element_stress(int nx, int ny, int nz, const double *X, const double *Y,
                          const double *Z, const double *Cel, const double *u, double *sig,
                          cudaStream_t s) {
  const int nel = nx * ny * nz, T = 256;
  k_element_stress<<<(nel + T - 1) / T, T, 0, s>>>(nx, ny, nz, X, Y, Z, Cel, u, sig); GENEO_COUNT_LAUNCH();
  GENEO_CUDA_TRY(cudaGetLastError());
  return GENEO_OK;
}

int launch_load(const AssemblyArgs &a, cudaStream_t s) {
  const int T = 256;
  int nnode = (a.nx + 1) * (a.ny + 1) * (a.nz + 1);
  const int nc = a.nc == 1 ? 1 : 3;
  if (nc == 1) {
    k_load_darcy<<<(nnode + T - 1) / T, T, 0, s>>>(a.nx, a.ny, a.nz, a.X, a.Y, a.Z, a.top_pressure,
                                                   a.nodal, a.b); GENEO_COUNT_LAUNCH();
  } else {
    k_load<<<(nnode + T - 1) / T, T, 0, s>>>(a.nx, a.ny, a.nz, a.X, a.Y, a.top_pressure,
                                             a.nodal, a.b); GENEO_COUNT_LAUNCH();
  }
  if (a.n_dir > 0) {
    k_apply_lift<<<(nc * nnode + T - 1) / T, T, 0, s>>>(nc * nnode, a.mask, a.lift, a.b); GENEO_COUNT_LAUNCH();
  }
  GENEO_CUDA_TRY(cudaGetLastError());
  return GENEO_OK;
}

int launch_assembly_darcy(const AssemblyArgs &a, cudaStream_t s) {
  const int T = 256;
  int nnx = a.nx + 1, nny = a.ny + 1, nnz = a.nz + 1;
  int nnode = nnx * nny * nnz;
  k_bsr_count<<<(nnode + T - 1) / T, T, 0, s>>>(nnx, nny, nnz, a.cnt); GENEO_COUNT_LAUNCH();
  k_scan_single<<<1, 1024, 0, s>>>(nnode, a.cnt, a.row_ptr); GENEO_COUNT_LAUNCH();
  k_bsr_fill<<<(nnode + T - 1) / T, T, 0, s>>>(nnx, nny, nnz, a.row_ptr, a.col); GENEO_COUNT_LAUNCH();
  long long nt = (long long)nnode * 27;
  k_assemble_values_darcy<<<(unsigned)((nt + 127) / 128), 128, 0, s>>>(
      a.nx, a.ny, a.nz, a.X, a.Y, a.Z, a.perm, a.row_ptr, a.val); GENEO_COUNT_LAUNCH();
  k_load_darcy<<<(nnode + T - 1) / T, T, 0, s>>>(a.nx, a.ny, a.nz, a.X, a.Y, a.Z, a.top_pressure,
                                                 a.nodal, a.b); GENEO_COUNT_LAUNCH();
  GENEO_CUDA_TRY(cudaMemsetAsync(a.mask, 0, (size_t)nnode, s));
  GENEO_CUDA_TRY(cudaMemsetAsync(a.g, 0, (size_t)nnode * sizeof(double), s));
  if (a.n_dir > 0) {
    k_dirichlet_mark<<<(a.n_dir + T - 1) / T, T, 0, s>>>(a.n_dir, a.dir_dofs, a.dir_vals, nnode,
                                                         a.mask, a.g, a.status); GENEO_COUNT_LAUNCH();
    k_dirichlet_lift<<<(nnode + T - 1) / T, T, 0, s>>>(nnode, 1, a.row_ptr, a.col, a.val, a.mask,
                                                       a.g, a.lift); GENEO_COUNT_LAUNCH();
    k_apply_lift<<<(nnode + T - 1) / T, T, 0, s>>>(nnode, a.mask, a.lift, a.b); GENEO_COUNT_LAUNCH();
    k_dirichlet_eliminate<<<(nnode + T - 1) / T, T, 0, s>>>(nnode, 1, a.row_ptr, a.col, a.mask,
                                                            a.val); GENEO_COUNT_LAUNCH();
  }
  GENEO_CUDA_TRY(cudaGetLastError());
  return GENEO_OK;
}

}  // namespace geneo
