// stmg_slab.cu -- exact implicit time stepping over independent time slabs, with the
// design sensitivity fused in: the forward states of a solve are kept only every K-th
// time level (checkpoints) and each slab of K levels is recomputed from its checkpoint
// when it is needed.
//
// J is block lower-bidiagonal (Sec. 2.2): row n of the solution follows from row n-1 by
// one solve with the tridiagonal (M/dt + K) restricted to nodes 1..N.  Its Thomas factors
// do not change from step to step, so each step is two first-order linear recurrences,
//   forward  y_i = a_i y_{i-1} + f_i / p_i  (a_i = -l_i / p_i),
//   backward x_i = c_i x_{i+1} + y_i        (c_i = -u_i / p_i),
// which one thread block evaluates as a parallel scan of affine maps (Blelloch 1990:
// composition (A2, C2) o (A1, C1) = (A2 A1, A2 C1 + C2) is associative).  One block per
// slab; slabs are independent, so all of them run at once.  FP64 throughout.
#include "stmg_internal.h"
#include "stmg_slab.h"

namespace stmg {
namespace {

constexpr int kSlabThreads = 512;
constexpr int kSlabWarps = kSlabThreads / 32;
constexpr unsigned kFull = 0xffffffffu;

struct Aff {
  double A, C;  // x -> A x + C
};

// g o f: first f, then g.
__device__ __forceinline__ Aff compose(const Aff& g, const Aff& f) { return Aff{g.A * f.A, fma(g.A, f.C, g.C)}; }

// Exclusive scan of affine maps across the block, in thread order (REV: in reverse thread
// order); returns the composition of the maps of all preceding threads.  sh: 2*kSlabWarps.
template <bool REV>
__device__ __forceinline__ Aff block_exclusive_scan(Aff v, double* sh) {
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int wl = REV ? 31 - lane : lane;       // position within the warp in scan order
  const int ww = REV ? kSlabWarps - 1 - warp : warp;
  // inclusive warp scan in scan order
  Aff inc = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const double pa = REV ? __shfl_down_sync(kFull, inc.A, d) : __shfl_up_sync(kFull, inc.A, d);
    const double pc = REV ? __shfl_down_sync(kFull, inc.C, d) : __shfl_up_sync(kFull, inc.C, d);
    if (wl >= d) inc = compose(inc, Aff{pa, pc});
  }
  // exclusive within the warp
  double ea = REV ? __shfl_down_sync(kFull, inc.A, 1) : __shfl_up_sync(kFull, inc.A, 1);
  double ec = REV ? __shfl_down_sync(kFull, inc.C, 1) : __shfl_up_sync(kFull, inc.C, 1);
  Aff ex = wl == 0 ? Aff{1.0, 0.0} : Aff{ea, ec};
  // warp totals
  if (wl == 31) {
    sh[2 * ww] = inc.A;
    sh[2 * ww + 1] = inc.C;
  }
  __syncthreads();
  Aff pre{1.0, 0.0};
  for (int w = 0; w < ww; ++w) pre = compose(Aff{sh[2 * w], sh[2 * w + 1]}, pre);
  __syncthreads();
  return compose(ex, pre);
}

// One slab per block: rows n = j K + 1 .. min((j+1) K, NT) from the checkpoint row j K.
// u_out (optional): the recomputed rows (padded layout).  SENS: accumulate the
// sensitivity partial sums of every element over the slab's rows into scratch.
template <bool SENS>
__global__ void __launch_bounds__(kSlabThreads) k_slabs(SlabView sv, const double* __restrict__ bs,
                                                        const double* __restrict__ ckpt, double* __restrict__ u_out,
                                                        const double* __restrict__ lam, double* __restrict__ scratch) {
  extern __shared__ double sm[];
  const int N = sv.N, P = sv.pitch;
  double* prev = sm;                 // N + 2 values: row n-1 (node 0 masked to 0)
  double* cur = sm + (N + 2);        // N + 2 values: row n
  double* sh = sm + 2 * (N + 2);     // scan scratch
  const int j = blockIdx.x;
  const int nfirst = j * sv.K + 1;
  const int nlast = min((j + 1) * sv.K, sv.NT);
  // nodes 1..N split into contiguous runs per thread
  const int per = (N + kSlabThreads - 1) / kSlabThreads;
  const int i0 = 1 + threadIdx.x * per;
  const int i1 = min(N, i0 + per - 1);
  // load the checkpoint row (dense, N+1 values per row)
  for (int i = threadIdx.x; i <= N + 1; i += kSlabThreads) {
    prev[i] = (i >= 1 && i <= N) ? ckpt[(size_t)j * (N + 1) + i] : 0.0;
    cur[i] = 0.0;
  }
  if (u_out) {
    double* u0 = u_out + (size_t)(j * sv.K) * P;
    for (int i = threadIdx.x; i <= N; i += kSlabThreads) u0[i] = ckpt[(size_t)j * (N + 1) + i];
  }
  double sk[kMaxNodesPerThread], sc[kMaxNodesPerThread];
#pragma unroll
  for (int q = 0; q < kMaxNodesPerThread; ++q) sk[q] = sc[q] = 0.0;
  __syncthreads();
  for (int n = nfirst; n <= nlast; ++n) {
    const bool has_prev = n > 1;
    const double* bn = bs + (size_t)n * P;
    // forward recurrence: local composition of the thread's run
    Aff loc{1.0, 0.0};
    for (int i = i0; i <= i1; ++i) {
      double f = bn[i] * sv.dw[i];
      if (has_prev) f -= sv.pl[i] * prev[i - 1] + sv.pc[i] * prev[i] + sv.pr[i] * prev[i + 1];
      cur[i] = f * sv.inv[i];  // c_i of the forward map
      loc = compose(Aff{sv.alpha[i], cur[i]}, loc);
    }
    Aff pre = block_exclusive_scan<false>(loc, sh);
    double y = pre.C;  // y_{i0-1} (y_0 = 0)
    for (int i = i0; i <= i1; ++i) {
      y = fma(sv.alpha[i], y, cur[i]);
      cur[i] = y;
    }
    __syncthreads();
    // backward recurrence x_i = c_i x_{i+1} + y_i from i = N down to 1 (x_{N+1} = 0)
    Aff locb{1.0, 0.0};
    for (int i = i1; i >= i0; --i) locb = compose(Aff{sv.beta[i], cur[i]}, locb);
    Aff preb = block_exclusive_scan<true>(locb, sh);
    double x = preb.C;  // x_{i1+1}
    for (int i = i1; i >= i0; --i) {
      x = fma(sv.beta[i], x, cur[i]);
      cur[i] = x;
    }
    __syncthreads();
    if (SENS) {
      // element e = i - 1 between nodes i-1 and i (node 0 masked): partial sums of
      // (lam_e - lam_{e+1})(u_e - u_{e+1}) and lam^T [[2,1],[1,2]] (u_n - u_{n-1})
      const double* ln = lam + (size_t)n * P;
#pragma unroll
      for (int q = 0; q < kMaxNodesPerThread; ++q) {
        const int i = i0 + q;
        if (i <= i1) {
          const double ue = i == 1 ? 0.0 : cur[i - 1], ue1 = cur[i];
          const double le = i == 1 ? 0.0 : ln[i - 1], le1 = ln[i];
          double de = ue, de1 = ue1;
          if (has_prev) {
            de -= i == 1 ? 0.0 : prev[i - 1];
            de1 -= prev[i];
          }
          sk[q] = fma(le - le1, ue - ue1, sk[q]);
          sc[q] = fma(le, 2.0 * de + de1, sc[q]);
          sc[q] = fma(le1, de + 2.0 * de1, sc[q]);
        }
      }
    }
    if (u_out) {
      double* un = u_out + (size_t)n * P;
      for (int i = threadIdx.x; i <= N; i += kSlabThreads) un[i] = i == 0 ? bn[0] / sv.omega : cur[i];
    }
    __syncthreads();
    for (int i = i0; i <= i1; ++i) prev[i] = cur[i];
    __syncthreads();
  }
  if (SENS) {
    const int chunks = gridDim.x;
#pragma unroll
    for (int q = 0; q < kMaxNodesPerThread; ++q) {
      const int i = i0 + q;
      if (i <= i1) {
        scratch[(size_t)j * N + (i - 1)] = sk[q] / sv.dx;
        scratch[(size_t)(chunks + j) * N + (i - 1)] = sc[q] * sv.dx / (6.0 * sv.dt);
      }
    }
  }
}

// Exact solve of J u = b (ADJ: J^T u = b) over a whole level in one block: Dirichlet
// DOFs u = b / W = b' / omega, then each time level from the previous (next for J^T) by
// the same two block-scanned Thomas recurrences.  T is the storage type; arithmetic and
// the carried row are FP64.  The coarsest-level solver of Alg. 1 for wide levels.
template <typename T, bool ADJ>
__global__ void __launch_bounds__(kSlabThreads) k_exact_par(SlabView sv, const T* __restrict__ bs,
                                                            T* __restrict__ u) {
  extern __shared__ double sm[];
  const int N = sv.N, NT = sv.NT, P = sv.pitch;
  double* prev = sm;
  double* cur = sm + (N + 2);
  double* sh = sm + 2 * (N + 2);
  for (int i = threadIdx.x; i <= N; i += kSlabThreads) u[i] = (T)((double)bs[i] / sv.omega);
  for (int n = 1 + threadIdx.x; n <= NT; n += kSlabThreads)
    u[(size_t)n * P] = (T)((double)bs[(size_t)n * P] / sv.omega);
  for (int i = threadIdx.x; i <= N + 1; i += kSlabThreads) prev[i] = cur[i] = 0.0;
  const int per = (N + kSlabThreads - 1) / kSlabThreads;
  const int i0 = 1 + threadIdx.x * per;
  const int i1 = min(N, i0 + per - 1);
  __syncthreads();
  for (int step = 1; step <= NT; ++step) {
    const int n = ADJ ? NT + 1 - step : step;
    const bool has_prev = ADJ ? (n < NT) : (n > 1);
    const T* bn = bs + (size_t)n * P;
    Aff loc{1.0, 0.0};
    for (int i = i0; i <= i1; ++i) {
      double f = (double)bn[i] * sv.dw[i];
      if (has_prev) f -= sv.pl[i] * prev[i - 1] + sv.pc[i] * prev[i] + sv.pr[i] * prev[i + 1];
      cur[i] = f * sv.inv[i];
      loc = compose(Aff{sv.alpha[i], cur[i]}, loc);
    }
    Aff pre = block_exclusive_scan<false>(loc, sh);
    double y = pre.C;
    for (int i = i0; i <= i1; ++i) {
      y = fma(sv.alpha[i], y, cur[i]);
      cur[i] = y;
    }
    __syncthreads();
    Aff locb{1.0, 0.0};
    for (int i = i1; i >= i0; --i) locb = compose(Aff{sv.beta[i], cur[i]}, locb);
    Aff preb = block_exclusive_scan<true>(locb, sh);
    double x = preb.C;
    for (int i = i1; i >= i0; --i) {
      x = fma(sv.beta[i], x, cur[i]);
      cur[i] = x;
    }
    __syncthreads();
    T* un = u + (size_t)n * P;
    for (int i = i0; i <= i1; ++i) {
      un[i] = (T)cur[i];
      prev[i] = cur[i];
    }
    __syncthreads();
  }
}

}  // namespace

cudaError_t launch_slabs(const SlabView& sv, const double* bs, const double* ckpt, double* u_out, const double* lam,
                         double* scratch, cudaStream_t s) {
  if ((sv.N + kSlabThreads - 1) / kSlabThreads > kMaxNodesPerThread) return cudaErrorInvalidValue;
  const int nslabs = (sv.NT + sv.K - 1) / sv.K;
  const size_t smem = sizeof(double) * (2 * (size_t)(sv.N + 2) + 2 * kSlabWarps);
  if (smem > 48 * 1024) {
    cudaError_t e = lam ? cudaFuncSetAttribute(k_slabs<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)
                        : cudaFuncSetAttribute(k_slabs<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  if (lam) k_slabs<true><<<nslabs, kSlabThreads, smem, s>>>(sv, bs, ckpt, u_out, lam, scratch);
  else k_slabs<false><<<nslabs, kSlabThreads, smem, s>>>(sv, bs, ckpt, u_out, nullptr, nullptr);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace stmg

namespace stmg {

template <typename T>
cudaError_t launch_exact_par(const SlabView& sv, bool adj, const T* bs, T* u, cudaStream_t s) {
  if ((sv.N + kSlabThreads - 1) / kSlabThreads > kMaxNodesPerThread) return cudaErrorInvalidValue;
  const size_t smem = sizeof(double) * (2 * (size_t)(sv.N + 2) + 2 * kSlabWarps);
  if (smem > 48 * 1024) {
    cudaError_t e = adj ? cudaFuncSetAttribute(k_exact_par<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)smem)
                        : cudaFuncSetAttribute(k_exact_par<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)smem);
    if (e != cudaSuccess) return e;
  }
  if (adj) k_exact_par<T, true><<<1, kSlabThreads, smem, s>>>(sv, bs, u);
  else k_exact_par<T, false><<<1, kSlabThreads, smem, s>>>(sv, bs, u);
  count_launches(1);
  return cudaGetLastError();
}

template cudaError_t launch_exact_par<double>(const SlabView&, bool, const double*, double*, cudaStream_t);
template cudaError_t launch_exact_par<float>(const SlabView&, bool, const float*, float*, cudaStream_t);

}  // namespace stmg
