// Internal launch interfaces between the kernel files and the C ABI layer.
#pragma once

#include "common.cuh"

namespace geneo {

struct AssemblyArgs {
  int nx, ny, nz, n_mat, n_dir;
  int nc;                           // unknowns per node: 3 elasticity, 1 Darcy
  const double *perm;               // Darcy: (Kx, Ky, Kz) per element (device)
  const double *X, *Y, *Z;          // node coordinates (device)
  const geneo_ortho *mats;          // device
  const int32_t *emat;              // device
  const double *theta, *phi;        // device (phi may be null)
  const int32_t *dir_dofs;          // device
  const double *dir_vals;           // device (may be null)
  const double *nodal;              // device (may be null)
  double top_pressure;              // elasticity: top traction; Darcy: the uniform source f
  double *C0, *Cel;                 // per-material / per-element Voigt stiffness
  int32_t *cnt, *row_ptr, *col;
  double *val, *b, *g;
  double *lift;                     // Dirichlet lifting: g on Dirichlet rows, -A_FD g on free rows
  uint8_t *mask;
  DevStatus *status;
};
int launch_assembly(const AssemblyArgs &a, cudaStream_t s);
// The scalar Darcy system (one unknown per node, 1x1 blocks in the same pattern).
int launch_assembly_darcy(const AssemblyArgs &a, cudaStream_t s);
// Right-hand side only (load kernel + stored lifting): b = mask ? lift : f + lift.
int launch_load(const AssemblyArgs &a, cudaStream_t s);
// Element stresses at the centres (6 per element, Voigt order) from u.
int launch_element_stress(int nx, int ny, int nz, const double *X, const double *Y,
                          const double *Z, const double *Cel, const double *u, double *sig,
                          cudaStream_t s);

// Scalars of one (F)PCG solve, resident on the device.
struct CGScalars {
  double bb, tol2;            // ||b||^2 and tol^2
  double rz, pq, alpha, beta, rr, zq;
  int it, maxit, done;        // done: 0 running, 1 converged, 2 breakdown, 3 max_it
  int flexible;
  unsigned int counter;       // last-block ticket
};

struct BSR {
  int nnode;
  const int32_t *row_ptr, *col;
  const double *val;
  int nc = 3;                        // block size: unknowns per node (3 or 1)
};

// y = A x (FP64, warp per block row).
void launch_spmv(const BSR &A, const double *x, double *y, cudaStream_t s);
// CG building blocks (each kernel returns at once when cg->done != 0).
void launch_cg_init(int n, const double *b, double *x, double *r, CGScalars *cg,
                    double *part, cudaStream_t s);
void launch_cg_init2(int n, const double *r, const double *z, double *p, CGScalars *cg,
                     double *part, cudaStream_t s);
void launch_cg_spmv_pq(const BSR &A, const double *p, double *q, CGScalars *cg, double *part,
                       cudaStream_t s);
void launch_cg_update_xr(int n, const double *p, const double *q, double *x, double *r,
                         CGScalars *cg, double *part, double *alphas, cudaStream_t s);
void launch_cg_dots(int n, const double *r, const double *z, const double *q, CGScalars *cg,
                    double *part, double *betas, cudaStream_t s);
void launch_cg_update_p(int n, const double *z, double *p, CGScalars *cg, cudaStream_t s);
void launch_copy_if_running(int n, const double *src, double *dst, const CGScalars *cg,
                            cudaStream_t s);
// ||v||^2 into *out (deterministic two-stage; part holds kRedBlocks doubles)
void launch_norm2(int n, const double *v, double *out, double *part, unsigned *counter,
                  cudaStream_t s);
// out = a - b
void launch_sub(int n, const double *a, const double *b, double *out, cudaStream_t s);

}  // namespace geneo
