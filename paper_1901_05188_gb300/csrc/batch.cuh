// Batched solves over many independent instances (internal).
//
// A batch advances the (F)PCG iterations of many assembled and set-up
// contexts together: every kernel launch of an iteration covers every
// instance, each instance keeps its own Krylov scalars and stops on its own,
// and the one-level local solves of all instances run in one persistent
// launch that takes (instance, subdomain) items from a device work queue,
// largest first.  The instances' matrices, factors and coarse spaces stay in
// their contexts' workspaces; the batch owns only the concatenated Krylov
// vectors, the per-instance scalars and the work tables.
#pragma once

#include "band.cuh"
#include "kernels.cuh"

namespace geneo {

// One instance as the batched kernels see it.
struct BatchInst {
  long long vbase;                 // first entry of this instance in the batch vectors
  int nnode, nc, ndof;
  const int32_t *row_ptr, *col;
  const double *val;
  const uint8_t *mask;
  int flexible;
  // subdomains and one-level term
  int nsub, nnx, nny, nnz, px, py;
  const SubDesc *subs;
  const BandLayout *lay;
  const void *facL, *facU;
  void *xloc;
  const int *cand;
  int co0, co1, co2;
  const int *gmap;
  const uint8_t *gcnt;
  int pou;                         // D_j = X_j
  const double *wloc;              // Sarkis weights, or null (multiplicity)
  // coarse space (nH = 0: none)
  int nH, mcap, nchunk;
  const double *Zp, *AHinv;
  double *wpart, *wH, *yH, *zy;
};

// Work tables of a batch (device arrays).
struct BatchTables {
  int n;                           // instances
  const long long *task_off;       // [n + 1] warp tasks of 32 scalar rows, per instance
  long long ntask;
  const long long *node_off;       // [n + 1] blocks of 256 nodes, per instance
  long long nnodeblk;
  const int2 *sub_items;           // (instance, subdomain), largest local solve first
  int nsub_items;
  const int4 *chunk_items;         // (instance, subdomain, row chunk of Z_j)
  int nchunk_items;
  const int2 *row_items;           // (instance, coarse row)
  int nrow_items;
};

// Krylov steps (one launch each over all instances; tpart holds 2 doubles per
// task, the per-instance sums are taken by launch_batch_reduce).
void launch_batch_init(const BatchInst *inst, const BatchTables &T, const double *b, double *x,
                       double *r, double *tpart, cudaStream_t s);
void launch_batch_init2(const BatchInst *inst, const BatchTables &T, const CGScalars *cg,
                        const double *r, const double *z, double *p, double *tpart,
                        cudaStream_t s);
void launch_batch_spmv_pq(const BatchInst *inst, const BatchTables &T, const CGScalars *cg,
                          const double *p, double *q, double *tpart, cudaStream_t s);
void launch_batch_update_xr(const BatchInst *inst, const BatchTables &T, const CGScalars *cg,
                            const double *p, const double *q, double *x, double *r,
                            double *tpart, cudaStream_t s);
void launch_batch_dots(const BatchInst *inst, const BatchTables &T, const CGScalars *cg,
                       const double *r, const double *z, const double *q, double *tpart,
                       cudaStream_t s);
void launch_batch_update_p(const BatchInst *inst, const BatchTables &T, const CGScalars *cg,
                           const double *z, double *p, cudaStream_t s);
// y = A x for every instance (no scalars); partial ||a - y||^2 per task when a
// is given (the true residual at the end)
void launch_batch_residual(const BatchInst *inst, const BatchTables &T, const double *x,
                           const double *a, double *tpart, cudaStream_t s);
// Per-instance sums of the task partials and the scalar update of a step:
// 0 init (||b||^2), 1 init2 (r.z), 2 after the SpMV (p.q -> alpha),
// 3 after the x, r update (||r||^2, iteration count, convergence),
// 4 after the dots (r.z, z.q -> beta), 5 true residual (into out[i]).
void launch_batch_reduce(const BatchInst *inst, const BatchTables &T, CGScalars *cg,
                         const double *tpart, int kind, double *alphas, double *betas,
                         int hist, double *out, cudaStream_t s);

// Preconditioner pieces over all instances.
void launch_batch_coarse(const BatchInst *inst, const BatchTables &T, const CGScalars *cg,
                         const double *r, cudaStream_t s);
void launch_batch_gather(const BatchInst *inst, const BatchTables &T, const CGScalars *cg,
                         bool precision_f32, double *z, cudaStream_t s);
// One-level local solves of every (instance, subdomain) item in one persistent
// launch of `blocks` CTAs pulling items from *head (zero it before).
template <typename T>
int launch_batch_schwarz(const BatchInst *inst, const CGScalars *cg, const int2 *items,
                         int nitems, int *head, const double *r, int npad_max, int w_max,
                         int rows, int staged, int blocks, DevStatus *status, cudaStream_t s);
template <typename T>
bool batch_schwarz_fits(int npad_max, int w_max, int rows, int staged);
template <typename T>
int prepare_batch_schwarz(int npad_max, int w_max);

}  // namespace geneo
