// Band-tiled Cholesky factorisation and triangular sweeps (internal).
#pragma once

#include "kernels.cuh"
#include "precond.cuh"

namespace geneo {


// Zero a pool of tiles and put ones on the padded diagonal of every system.
template <typename T>
int launch_band_clear(const BandLayout *d_lay, int nsys, T *pool, long long pool_elems,
                      cudaStream_t s);

// Right-looking tile Cholesky of nsys band systems held in poolL (lower
// triangle of each tile row as input).  On exit poolL/poolU hold the forward
// and backward tile streams described in precond.cuh.  With a side stream the
// next tile column is factored there while `s` applies the trailing update
// (the work is ordered by events and complete on `s` at return).
template <typename T>
int launch_band_cholesky(const BandLayout *d_lay, int nsys, int nt_max, int w_max, T *poolL,
                         T *poolU, DevStatus *st, cudaStream_t s, cudaStream_t side = nullptr);

// Solve with ncols right-hand sides per system.  Column c of system j lives at
// in[j*in_sys + l*in_row + c] (l = 0..n-1); the result goes to
// out[j*out_sys + l*out_row + c] for l < n (padding rows are not written).
// In-place use (in == out with equal strides) is allowed.
// mode: 1 forward (L), 2 backward (L^T), 3 both.  w_max: the largest tile
// half-bandwidth; ring = 1 streams every column through a ring of max(w + 2, 3)
// tile rows in shared memory (chosen anyway when a whole column does not fit).
int launch_band_solve_dense(const BandLayout *d_lay, int nsys, int npad_max, int w_max,
                            int ring, const double *poolL, const double *poolU, const double *in,
                            long long in_sys, int in_row, double *out, long long out_sys,
                            int out_row, int ncols, int mode, cudaStream_t s);

// The same solve with the one-CTA look-ahead sweep of the local solves.
int launch_band_solve_la(const BandLayout *d_lay, int nsys, int npad_max, int w_max, int ring,
                         const double *poolL, const double *poolU, const double *in,
                         long long in_sys, int in_row, double *out, long long out_sys,
                         int out_row, int ncols, int mode, cudaStream_t s);
// Whether the ring form of the band solve fits for tile half-bandwidth w_max.
bool band_solve_fits(int w_max);

// FP32 trailing update of tile column J on the tensor cores (3xTF32 tcgen05
// MMAs, blocks of 4 x 4 tiles); part as for the band Cholesky's update
// (0 all, 1 the first block column, 2 the other block columns).
int prepare_chol_update_tc();
int launch_chol_update_tc(const BandLayout *d_lay, int nsys, int J, int w_max, float *poolL,
                          int part, DevStatus *status, cudaStream_t s);
// Tensor cores for the FP32 factor updates unless GENEO_TENSOR_CORES=0.
bool use_tensor_cores();

// Extract A_j = R_j A R_j^T (interior dofs) from the global BSR into band tiles.
template <typename T>
int launch_extract_interior(const SubDesc *d_subs, const BandLayout *d_lay, int nsub,
                            int max_nodes, int nnx, int nny, int nnz, const int32_t *rp,
                            const double *val, T *pool, cudaStream_t s);

// Opt in to the shared memory the Schwarz solve needs (call before capture);
// w_max is the largest tile half-bandwidth of the local factors.
template <typename T>
int prepare_schwarz_solve(int npad_max, int w_max);

// One-level Schwarz local solves: x_j = A_j^-1 R_j r for every subdomain, one
// thread-block cluster of `cluster` CTAs (1, 2, 4 or 8) per subdomain, `rows`
// tile rows (1, 2 or 4) per cluster barrier, or rows = 0 for the look-ahead
// sweep (the next row's far tiles overlap the current row's chain).  With
// staged = 1 (rows 0, 1 or 2) every step's tiles are copied into shared
// memory a step ahead by bulk asynchronous copies and the per-CTA partials
// are exchanged by st.async on mbarriers instead of cluster barriers; a copy
// or partial that does not land within about a second sets GENEO_ERR_TIMEOUT
// in *status.  staged = 2 (rows 0): the look-ahead sweep with the local
// vector streamed through a ring of max(w + 2, 3) tile rows, for subdomains
// whose local vector does not fit in shared memory; its forward sweep leaves
// y in yscr (same layout as xloc).
template <typename T>
int launch_schwarz_solve(const SubDesc *d_subs, const BandLayout *d_lay, int nsub,
                         int npad_max, int w_max, int nnx, int nny, const T *poolL,
                         const T *poolU, const double *r, T *xloc, T *yscr, const CGScalars *cg,
                         int cluster, int rows, int staged, DevStatus *status, cudaStream_t s);
// True when the staged launch (cluster, rows) fits in shared memory.
template <typename T>
bool schwarz_staged_fits(int npad_max, int w_max, int cluster, int rows);
// True when the launch shape (cluster, rows, staged 0, 1 or 2) fits.
template <typename T>
bool schwarz_shape_fits(int npad_max, int w_max, int cluster, int rows, int staged);
// Cluster size that fills the GPU: the largest power of two <= 8 with
// 2 * nsub * size <= number of SMs (at least 1).
int schwarz_cluster_size(int nsub, int sm_count);

// Per node: offsets into the local solutions of the subdomains whose interior
// holds it (8 slots, -1 padded) and the number of overlapping subdomains
// containing it (0xFF: more than 8 interior subdomains, visited directly).
void launch_gather_map(int nx, int ny, int nz, int px, int py, const int *cand,
                       const int cand_off[3], const SubDesc *d_subs, int *gmap, uint8_t *gcnt,
                       cudaStream_t s);

// z = sum_j R_j^T (D_j x_j + (Z y)_j): deterministic gather over subdomains
// through the gather map; zy holds Z_j y_j per interior dof (from
// launch_coarse_apply) or is null.  With pou, D_j = X_j: the weights wloc
// (laid out like the local solutions) when given, else 1 / multiplicity.
template <typename T>
void launch_schwarz_gather(int nx, int ny, int nz, int px, int py, const int *cand,
                           const int cand_off[3], const SubDesc *d_subs, const int *gmap,
                           const uint8_t *gcnt, const T *xloc, const double *zy, int pou,
                           const double *wloc, const uint8_t *mask, double *z,
                           const CGScalars *cg, cudaStream_t s);

// Coarse restriction w = Z^T r (partials over blocks of kZRows rows),
// reduction, y = A_H^-1 w and the prolongation zy_j = Z_j y_j per interior
// dof.  wpart holds nsub * restrict_chunks(max_nint) * mcap doubles.
constexpr int kZRows = 128;
inline int restrict_chunks(int max_nint) { return (max_nint + kZRows - 1) / kZRows; }
void launch_coarse_apply(const SubDesc *d_subs, int nsub, int max_nint, int nnx, int nny,
                         const double *Zp, const double *r, double *wpart, double *wH,
                         double *yH, double *zy, const double *AHinv, int nH, int mcap,
                         const CGScalars *cg, cudaStream_t s);

// Inexact coarse solve (Sec. 3.3.3): BJ[j] = inverse of subdomain j's
// diagonal block of A_H (m_j x m_j, stride mcap), then per application the
// restriction, block-Jacobi PCG on A_H y = w to ||w - A_H y|| <= tol ||w|| or
// maxit steps in one cooperative launch (work: 4 nH + 4 * coarse_pcg_blocks()
// doubles; bar: two barrier words, zero before the first launch), and the
// prolongation.  inner_its (or null) accumulates the inner steps taken.
void launch_coarse_bj_inverse(const SubDesc *d_subs, int nsub, int nH, const double *AH,
                              double *BJ, int mcap, cudaStream_t s);
int coarse_pcg_blocks();
int launch_coarse_apply_iterative(const SubDesc *d_subs, int nsub, int max_nint, int nnx,
                                  int nny, const double *Zp, const double *r, double *wpart,
                                  double *wH, double *yH, double *zy, const double *AH,
                                  const double *BJ, int nH, int mcap, double *work,
                                  unsigned int *bar, double tol, int maxit, const CGScalars *cg,
                                  DevStatus *st, int *inner_its, cudaStream_t s);

}  // namespace geneo
