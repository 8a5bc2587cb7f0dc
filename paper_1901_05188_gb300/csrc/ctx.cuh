// The library context (internal).
#pragma once

#include <vector>
#include <string>

#include "kernels.cuh"
#include "precond.cuh"

struct geneo_ctx {
  cudaStream_t stream = nullptr;
  cudaStream_t cap_stream = nullptr;        // private stream used only to capture graphs
  cudaStream_t eig_stream = nullptr;        // GenEO eigensolve and coarse space (highest priority)
  cudaStream_t eig_stream2 = nullptr;       // second group of the Lanczos iterations (same)
  cudaStream_t side_stream = nullptr;       // its look-ahead factorisation (highest priority)
  cudaStream_t fac_stream = nullptr;        // subdomain factorisation, overlapping the eigensolve
  cudaStream_t fac_side = nullptr;          // its look-ahead stream
  int device = 0;
  int pou_kind = 0;                          // partition of unity of the next geneo_setup
  int csolver = 0;                           // coarse solver of the next geneo_setup
  double ctol = 1e-2;                        // its inner tolerance (iterative)
  int cmaxit = 200;                          // its inner step limit (iterative)

  // ---- mesh / assembled system (phase 0)
  bool assembled = false;
  int nx = 0, ny = 0, nz = 0, nnode = 0, ndof = 0, nel = 0, nnzb = 0;
  int nc = 3;                              // unknowns per node: 3 elasticity, 1 Darcy
  std::vector<double> hx, hy, hz;          // host copies of node coordinates
  std::vector<uint8_t> hmask;              // host copy of the Dirichlet mask
  void *ws0 = nullptr;
  size_t ws0_bytes = 0;
  bool ws0_owned = false;
  void *ws0_bound = nullptr;
  size_t ws0_bound_bytes = 0;
  double *X = nullptr, *Y = nullptr, *Z = nullptr;
  double *Cel = nullptr, *C0 = nullptr;
  int32_t *row_ptr = nullptr, *col = nullptr, *cnt = nullptr;
  double *val = nullptr, *b = nullptr, *g = nullptr;
  double *lift = nullptr;                  // Dirichlet lifting (kept for new loads)
  double *sig = nullptr;                   // element stresses (6 per element), output staging
  int n_dir = 0;
  uint8_t *mask = nullptr;
  geneo::DevStatus *status = nullptr;
  // staging of caller inputs
  geneo_ortho *mats = nullptr;
  int32_t *emat = nullptr, *dir_dofs = nullptr;
  double *theta = nullptr, *phi = nullptr, *dir_vals = nullptr, *nodal = nullptr;
  double *perm = nullptr;                  // Darcy: (Kx, Ky, Kz) per element

  // ---- preconditioner + Krylov state (phase 1)
  bool setup_done = false;
  void *ws1 = nullptr;
  size_t ws1_bytes = 0;
  bool ws1_owned = false;
  void *ws1_bound = nullptr;
  size_t ws1_bound_bytes = 0;
  geneo::Precond pc;                        // subdomain factors, coarse space
  // Krylov vectors
  double *x = nullptr, *r = nullptr, *p = nullptr, *q = nullptr, *z = nullptr, *tmp = nullptr;
  double *part = nullptr, *alphas = nullptr, *betas = nullptr, *scal = nullptr;
  geneo::CGScalars *cg = nullptr;
  geneo::CGScalars *cg_host = nullptr;      // pinned mirror
  int maxit_cap = 0;
  cudaGraphExec_t graph = nullptr;          // K iterations
  int graph_iters = 0;
  long long graph_kernels = 0;              // kernel nodes in one graph launch
  double *graph_tol_key = nullptr;
  geneo_stats last_stats{};
  float ms_assemble = 0.f;
};

namespace geneo {
bool is_device_ptr(const void *p);
}
