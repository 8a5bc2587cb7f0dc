// GenEO eigenproblems, coarse basis and coarse matrix (internal).
#pragma once

#include "band.cuh"

namespace geneo {

// Partition of unity (kind 0: 1 / multiplicity, Sec. 3.3.1; kind 1: Sarkis's
// distance-weighted one, Sec. 3.2) on every subdomain's Neumann dofs (Xneu,
// offset x_neu), or on its interior dofs laid out like the local solutions
// (wloc, offset v_int); zero on global Dirichlet dofs.
void launch_pou_neumann(const SubDesc *d_subs, int nsub, int max_nodes, const int *cand,
                        const int cand_off[3], const uint8_t *mask, int nnx, int nny, int nnz,
                        int px, int py, int kind, double *Xneu, cudaStream_t s);
void launch_pou_interior(const SubDesc *d_subs, int nsub, int max_nodes, const int *cand,
                         const int cand_off[3], const uint8_t *mask, int nnx, int nny, int nnz,
                         int px, int py, int kind, double *wloc, cudaStream_t s);

// S_j = A_{Omega_j} - sigma X_j A_{Omega_j^o} X_j into band tiles (lower part)
// and B_j = X_j A_{Omega_j^o} X_j into a 27-slot local BSR.
void launch_neumann_assemble(const SubDesc *d_subs, const BandLayout *d_lay, int nsub,
                             int max_nodes, int nx, int ny, int nz, const double *X,
                             const double *Y, const double *Z, const double *Cel,
                             const double *perm,
                             const int *ecnt, const int ecnt_off[3], const uint8_t *mask,
                             const double *Xneu, double sigma, double *poolS, double *Bloc,
                             cudaStream_t s);

// W[:, 0:p] = B_j T[:, 0:p] on Neumann dofs (row-major blocks with ld p).
void launch_bloc_mv(const SubDesc *d_subs, int nsub, int max_nodes, const double *Bloc,
                    const double *T, double *W, long long sys_stride, int p,
                    cudaStream_t s);

// Random start block (counter-based hash), rows >= n_neu zero.
void launch_random_block(const SubDesc *d_subs, int nsub, int npad, double *V, int ld,
                         long long sys_stride, int p, unsigned long long seed,
                         cudaStream_t s);

// H[j] = A_j^T B_j over the first n rows (n = n_neu of subdomain j):
// A_j: n x na at lda, B_j: n x nb at ldb; H row-major na x nb (stride hs).
// Per-system flag: repeat the projection of W against V where the first pass
// removed more than half of some column's squared norm (G = W^T W after the
// pass, H the removed coefficients, na x p per system with stride hs).
void launch_reorth_gate(int nsub, const double *G, int p, const double *H, int na, long long hs,
                        int *gate, cudaStream_t s);
void launch_tsdots(const SubDesc *d_subs, int nsub, int npad, const double *A, int lda,
                   long long sa, int na, const double *B, int ldb, long long sb, int nb,
                   double *Hpart, int chunks, double *H, long long hs, cudaStream_t s,
                   const int *gate = nullptr);

// C_j = beta C_j + alpha A_j H_j (rows < n_neu).
// gate[j] == 0 (when gate is given) skips system j: the products leave C
// unchanged and the dot products return zeros.
void launch_tsgemm(const SubDesc *d_subs, int nsub, int npad, const double *A, int lda,
                   long long sa, int na, const double *H, int ldh, long long hs, double *C,
                   int ldc, long long sc, int nb, double alpha, double beta, cudaStream_t s,
                   const int *gate = nullptr);

// Cholesky-QR step on p x p Gram matrices: R = chol(G), W <- W R^-1 (columns
// with a vanishing pivot are zeroed); Racc <- R Racc.  Rinv: nsub p x p scratch.
void launch_cholqr(const SubDesc *d_subs, int nsub, int npad, const double *G, double *W,
                   int p, double *Racc, double *Rinv, int first, double abs_tiny, cudaStream_t s);
// Thick restart: Hm <- diag(theta_0..kk-1) with the coupling block R_s S[last p rows, :kk].
void launch_restart_hm(int nsub, double *Hm, int kdim, const double *Eval, const double *Evec,
                       const double *Rblk, int kk, int p, cudaStream_t s);

// Hm[:, col block k] += Hs (rows 0..(k+1)p-1); sub-diagonal block from Racc.
void launch_hm_accum(int nsub, double *Hm, int kdim, const double *Hs, int rows, int k, int p,
                     cudaStream_t s);
void launch_hm_subdiag(int nsub, double *Hm, int kdim, const double *Racc, int k, int p,
                       double *Rblk, cudaStream_t s);
void launch_copy_block(const SubDesc *d_subs, int nsub, int npad, const double *W, int ldw,
                       long long sw, double *V, int ldv, long long sv, int p,
                       cudaStream_t s);

// The nw largest Ritz pairs of the kdim x kdim projected matrices (Householder
// tridiagonalisation, bisection, inverse iteration); values descending;
// residual estimates from the last Lanczos block.
int launch_ritz_eig(int nsub, const double *Hm, int kdim, int nw, int p, const double *Rblk,
                    double *Eval, double *Evec, double *Eres, cudaStream_t s);

// Z_j = X_j P_j on interior dofs (row-major n_int x m_j).
void launch_build_Z(const SubDesc *d_subs, int nsub, int max_nint, const double *P, int ldp,
                    long long sp, const double *Xneu, double *Zp, cudaStream_t s);

// Y_j = A Z_j on the Neumann dofs of subdomain j (row-major n_neu x m_j).
void launch_AZ(const SubDesc *d_subs, int nsub, int max_nodes, int nnx, int nny, int nnz,
               const int32_t *rp, const int32_t *col, const double *val, const double *Zp,
               const long long *yoff, double *Yp, cudaStream_t s);

// A_H blocks for the listed subdomain pairs (j <= k), mirrored.
void launch_coarse_blocks(const SubDesc *d_subs, const int2 *pairs, int npairs,
                          const double *Zp, const double *Yp, const long long *yoff,
                          double *AH, int nH, cudaStream_t s);

// Dense nH x nH (row-major) -> lower band tiles of one system; symmetrise.
void launch_dense_to_tiles(const double *AH, int nH, const BandLayout *d_lay, double *pool,
                           cudaStream_t s);
void launch_symmetrize(double *M, int n, cudaStream_t s);
void launch_identity(double *M, int n, cudaStream_t s);
// scale columns of P_j (rows < n_neu) by 1/||col||; norms from the diagonal of G
// The six rigid displacements of each subdomain's Neumann nodes into P
// (row-major, leading dimension ld >= 6, system stride sp; other entries 0).
void launch_rigid_modes(const SubDesc *d_subs, int nsub, int npad, const double *X,
                        const double *Y, const double *Z, double *P, int ld, long long sp,
                        cudaStream_t s);
void launch_normalize_cols(const SubDesc *d_subs, int nsub, int npad, double *P, int ld,
                           long long sp, int ncol, const double *G, cudaStream_t s);

}  // namespace geneo
