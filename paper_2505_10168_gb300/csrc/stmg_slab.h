// stmg_slab.h -- slab-parallel exact time stepping (stmg_slab.cu).
#pragma once
#include <cuda_runtime.h>

namespace stmg {

constexpr int kMaxNodesPerThread = 16;  // nodes per thread of a 512-thread block: N <= 8192

// Finest-level data the slab kernel needs (FP64 device arrays of N+2 values by node).
struct SlabView {
  int N, NT, pitch, K;  // K: time levels per slab
  double dx, dt, omega;
  const double* dw;     // D_i / omega (b' -> b)
  const double* pl;     // coupling to the previous time level (negated mass / dt)
  const double* pc;
  const double* pr;
  const double* inv;    // 1 / Thomas pivot
  const double* alpha;  // -lower / pivot
  const double* beta;   // -modified upper
};

// Rows n = jK+1 .. min((j+1)K, NT) of the exact forward solution from checkpoint rows
// ckpt[j] (dense rows of N+1 values), one block per slab j.  bs: scaled right-hand side
// (padded).  u_out (optional, padded): all rows, checkpoints included.  lam (optional,
// padded): with it, scratch[2 * nslabs * N] receives the sensitivity partial sums per slab
// in the layout of the per-chunk sensitivity reduction.
cudaError_t launch_slabs(const SlabView& sv, const double* bs, const double* ckpt, double* u_out, const double* lam,
                         double* scratch, cudaStream_t s);

// Exact solve of one whole level (J u = b, or J^T u = b) from its scaled right-hand side
// bs, one block: the coarsest-level solver for levels with more than a few dozen nodes.
template <typename T>
cudaError_t launch_exact_par(const SlabView& sv, bool adj, const T* bs, T* u, cudaStream_t s);

}  // namespace stmg
