// Two-level additive Schwarz preconditioner with GenEO coarse space (internal).
#pragma once

#include <vector>

#include "common.cuh"

namespace geneo {

// Band-tiled SPD system: tile row I holds tiles (I, d), d = 0..w, for block
// column J = I - d; each tile is 32 x 32, column-major (entry (r, c) at
// c*32 + r).  After factorisation the L copy holds L(I, I-d) for d >= 1 and
// inv(L(I,I)) at d = 0; the U copy holds L(I+d, I)^T for d >= 1 and
// inv(L(I,I))^T at d = 0, so the backward sweep streams tile rows exactly
// like the forward one.
struct BandLayout {
  int n, nt, w;        // dofs, tile rows, tile half-bandwidth
  long long off;       // element offset of tile (0, 0) in its pool
};

struct Precond {
  geneo_partition part{};
  geneo_modes modes{};
  geneo_precision prec = GENEO_FP64;
  geneo_schwarz schwarz = GENEO_AS;
  geneo_coarse coarse = GENEO_COARSE_GENEO;
  int nsub = 0;
  int cluster = 1;                // CTAs per subdomain in the Schwarz local solves
  int rows = 1;                   // tile rows per cluster barrier in the Schwarz local solves
  int staged = 0;                 // Schwarz tiles staged in shared memory by bulk copies (1),
                                  // or the local vector streamed through a ring of tile rows (2)
  int sms = 0;                    // SM count of the device
  std::vector<SubDesc> subs;
  SubDesc *d_subs = nullptr;
  BandLayout *d_lay_int = nullptr, *d_lay_neu = nullptr, *d_lay_H = nullptr;
  long long *d_yoff = nullptr;
  int2 *d_pairs = nullptr;
  double *Hs = nullptr, *G = nullptr, *Racc = nullptr;
  int *gmap = nullptr;            // gather map [nnode][8]: local-solution offsets, -1 padded
  uint8_t *gcnt = nullptr;        // [nnode] overlapping-subdomain count (0xFF: map full)
  int *d_cand = nullptr;          // [nnx + nny + nnz][kMaxCand] subdomain axis index or -1
  int *d_ecnt = nullptr;          // [nx + ny + nz] subdomains containing the element, per axis
  int cand_off[3] = {0, 0, 0}, ecnt_off[3] = {0, 0, 0};
  int nt_int_max = 0, w_int_max = 0, npad_int_max = 0;
  int nt_neu_max = 0, w_neu_max = 0, npad_neu_max = 0;
  int eig_ring = 0;               // the eigensolver's band solves stream their columns through a ring
  long long fac_int_elems = 0, xloc_elems = 0;
  long long fac_neu_elems = 0, bloc_blocks = 0, xneu_elems = 0;
  // interior factors (T = double or float), L and U copies
  void *facL = nullptr, *facU = nullptr;
  void *xloc = nullptr;           // per-subdomain local solutions
  void *yloc = nullptr;           // the ring form's forward-sweep results (layout of xloc)
  int pou = 0;                    // partition of unity: GENEO_POU_MULTIPLICITY or _SARKIS
  double *wloc = nullptr;         // Sarkis weights X_j on interior dofs (like xloc), or null
  // GenEO eigenproblem data (FP64)
  double *neuL = nullptr, *neuU = nullptr;   // factor of S = A - sigma B
  double *Bloc = nullptr;         // 27-slot local BSR of B (9 doubles per block)
  double *Xneu = nullptr;         // PoU on Neumann dofs
  int ksteps = 12;                // Lanczos block steps per cycle (basis size kdim = p * ksteps)
  int kdim = 0;                   // p * ksteps
  int kkeep = 0;                  // Ritz vectors kept at a thick restart
  int max_cycles = 12;            // restart cycles
  int lanczos_steps = 0;          // block steps of the last eigensolve (two band sweeps each)
  int eig_cycles = 0;
  double eig_tol = 1e-6;          // Ritz residual <= eig_tol * theta (bounds the eigenvalue error)
  double *Vt = nullptr;           // restart scratch [nsub][npad][kkeep]
  int *gate = nullptr;            // per subdomain: second re-orthogonalisation pass needed
  double *V = nullptr;            // Lanczos basis [nsub][npad_neu][kdim + p] row-major
  double *W = nullptr;            // [nsub][npad_neu][p]
  double *T1 = nullptr;           // work block [nsub][npad_neu][p]
  double *Hm = nullptr;           // projected matrix [nsub][kdim][kdim]
  double *Hpart = nullptr;        // partial dot products
  int hchunks = 0;
  double *Evec = nullptr;         // Ritz vectors of the projected matrix [nsub][kdim][kdim]
  double *Eval = nullptr;         // Ritz values [nsub][kdim]
  double *Eres = nullptr;         // Ritz residual estimates [nsub][kdim]
  double *Rblk = nullptr;         // [nsub][p][p] last QR factor
  double *P = nullptr;            // eigenvectors [nsub][npad_neu][mcap]
  int mcap = 0;                   // max_modes + 1
  // coarse space (FP64)
  int nH = 0, nH_cap = 0;
  long long z_elems = 0;
  double *Zp = nullptr;           // Z_j, row-major n_int x m_j per subdomain
  double *Yp = nullptr;           // A Z_j on Neumann dofs, [nsub] x n_neu x m_j
  double *AH = nullptr, *AHinv = nullptr;   // dense nH x nH
  double *AHL = nullptr, *AHU = nullptr;    // tiles of the coarse factor
  double *wpart = nullptr;        // restriction partials [nsub][row blocks][mcap]
  double *wH = nullptr, *yH = nullptr;
  double *zy = nullptr;           // coarse correction Z_j y_j per interior dof [sum n_int]
  int csolver = 0;                // GENEO_COARSE_DIRECT or GENEO_COARSE_ITERATIVE
  double ctol = 1e-2;             // inner relative residual of the iterative coarse solve
  int cmaxit = 200;               // its step limit
  double *BJ = nullptr;           // block-Jacobi inverses [nsub][mcap][mcap]
  double *cwork = nullptr;        // inner PCG vectors and partials
  unsigned int *cbar = nullptr;   // grid-barrier words of the inner PCG
  int *c_inner = nullptr;         // inner steps accumulated over the applications
  int max_nint = 0;               // largest interior dof count of a subdomain
  int max_nodes_int = 0, max_nodes_neu = 0;   // largest interior / Neumann node count
  std::vector<int> m;
  std::vector<double> lambdas;    // [nsub][mcap]
  double eig_max_res = 0.0;
  bool eig_done = false;          // eigenpairs selected and Z built
  float ms_eig = 0.f, ms_coarse = 0.f, ms_factor = 0.f;
  double bytes_per_apply = 0.0;
};


}  // namespace geneo
