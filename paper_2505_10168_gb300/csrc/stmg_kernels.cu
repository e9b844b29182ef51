// stmg_kernels.cu -- CUDA kernels of the STMG V-cycle for sm_103a: damped Jacobi,
// residual, restriction, prolongation, the exact time-stepping solve, deterministic
// norms, coefficient/material/load set-up and the adjoint sensitivity.
//
// These are the per-DOF kernels; every space-time vector uses the padded layout of
// stmg_internal.h.  Reductions are two-pass with a fixed grid and a fixed tree order,
// so results do not depend on scheduling.
#include <algorithm>
#include <atomic>
#include <type_traits>

#include "stmg_internal.h"

namespace stmg {

static std::atomic<unsigned long long> g_launches{0};
void count_launches(unsigned n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
unsigned long long launches_so_far() { return g_launches.load(std::memory_order_relaxed); }

namespace {

constexpr int kThreads = 256;

inline unsigned blocks_for(long long n, int threads = kThreads) {
  long long b = (n + threads - 1) / threads;
  return (unsigned)(b < 1 ? 1 : b);
}

// Grids of at most kPdlMaxBlocks blocks (the levels below ~300 k DOFs, where a launch costs
// more than the work) go out with programmatic dependent launch, so that a kernel's launch
// overlaps its predecessor's drain; each such kernel calls pdl_wait() before any access to
// memory.  Larger grids launch the ordinary way: launched early, their fixed grids of
// FP64-bound blocks land unevenly on the SMs (measured slower).
constexpr unsigned kPdlMaxBlocks = 1216;
template <typename... KArgs, typename... Args>
cudaError_t launch_small(void (*kernel)(KArgs...), unsigned blocks, cudaStream_t s, Args... args) {
  if (blocks <= kPdlMaxBlocks) return launch_pdl(kernel, dim3(blocks), dim3(kThreads), s, args...);
  kernel<<<blocks, kThreads, 0, s>>>(args...);
  return cudaGetLastError();
}

// Row and node of a flat DOF index idx = n (N+1) + i (idx < 2^31).
__device__ __forceinline__ void split_index(uint32_t idx, const FastDiv& fd, int& n, int& i) {
  const uint32_t q = (uint32_t)(((uint64_t)__umulhi(idx, fd.M) + idx) >> fd.s);
  n = (int)q;
  i = (int)(idx - q * fd.d);
}

// (J u) at DOF (n, i) of a level, p = n * pitch + i (Sec. 2.2 stencil, Appendix A).
template <typename T>
__device__ __forceinline__ T apply_at(const LevelView<T>& lv, bool adj, const T* __restrict__ u, int n, int i,
                                      size_t p) {
  if (n == 0 || i == 0) return lv.W * u[p];
  const T* cf = lv.coef;
  const int P = lv.pitch;
  T acc = cf[kL * P + i] * u[p - 1];
  acc = fma(cf[kD * P + i], u[p], acc);
  acc = fma(cf[kU * P + i], u[p + 1], acc);
  const bool has_prev = adj ? (n < lv.NT) : (n > 1);
  if (has_prev) {
    const size_t q = adj ? p + P : p - P;
    acc = fma(cf[kPL * P + i], u[q - 1], acc);
    acc = fma(cf[kPC * P + i], u[q], acc);
    acc = fma(cf[kPR * P + i], u[q + 1], acc);
  }
  return acc;
}

// acc + sum_k S_k u_k over the off-diagonal neighbours of a non-Dirichlet DOF.
template <typename T, bool ADJ>
__device__ __forceinline__ T add_neighbours(const LevelView<T>& lv, const T* __restrict__ u, int n, int i, size_t p,
                                            T acc) {
  const T* cf = lv.coef;
  const int P = lv.pitch;
  acc = fma(cf[kSL * P + i], u[p - 1], acc);
  acc = fma(cf[kSU * P + i], u[p + 1], acc);
  const bool has_prev = ADJ ? (n < lv.NT) : (n > 1);
  if (has_prev) {
    const size_t q = ADJ ? p + P : p - P;
    acc = fma(cf[kSPL * P + i], u[q - 1], acc);
    acc = fma(cf[kSPC * P + i], u[q], acc);
    acc = fma(cf[kSPR * P + i], u[q + 1], acc);
  }
  return acc;
}

// Damped Jacobi (Sec. 3.1) in the scaled form: uo = (1 - omega) u + b' + sum_k S_k u_k.
template <typename T, bool ADJ>
__global__ void __launch_bounds__(kThreads) k_sweep(LevelView<T> lv, uint32_t total, const T* __restrict__ u,
                                                    const T* __restrict__ bs, T* __restrict__ uo) {
  pdl_wait();  // a no-op unless launched dependent (small grids)
  const uint32_t idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= total) return;
  int n, i;
  split_index(idx, lv.fd, n, i);
  const size_t p = (size_t)n * lv.pitch + i;
  T acc = fma(lv.omc, u[p], bs[p]);
  if (n != 0 && i != 0) acc = add_neighbours<T, ADJ>(lv, u, n, i, p, acc);
  uo[p] = acc;
}

// Scaled residual y = b' - omega u + sum_k S_k u_k = (omega / D)(b - J u).
template <typename T, bool ADJ>
__device__ __forceinline__ T scaled_residual(const LevelView<T>& lv, const T* __restrict__ u,
                                             const T* __restrict__ bs, int n, int i, size_t p) {
  T y = fma(-lv.omega, u[p], bs[p]);
  if (n != 0 && i != 0) y = add_neighbours<T, ADJ>(lv, u, n, i, p, y);
  return y;
}

template <typename T>
__device__ __forceinline__ T unscale(const LevelView<T>& lv, int n, int i) {
  return (n == 0 || i == 0) ? lv.Wo : lv.coef[kDW * lv.pitch + i];
}

// Block-level deterministic sum of one double per thread; result valid in thread 0.
template <int BLOCK>
__device__ __forceinline__ double block_sum(double v) {
  __shared__ double red[BLOCK];
  red[threadIdx.x] = v;
  __syncthreads();
#pragma unroll
  for (int w = BLOCK / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  return red[0];
}

// Sweep that also accumulates ||b - J u||^2 of the input iterate (fixed grid, grid-stride).
// The sweep's increment y = uo - u is the scaled residual (omega / D)(b - J u), exact in T;
// the norm only decides termination, so 2^k r = (D / omega) 2^k y is formed and squared in
// FP32 per thread (y scaled and truncated by its bit fields, dw32 = the FP32 copy of
// D / omega; 2^k from scale_exp, undone in the final sum) and summed in FP64 across the
// block: in FP64 the kernel costs 7 operations per DOF, a plain sweep 6.
template <typename T, bool ADJ>
__global__ void __launch_bounds__(kThreads) k_sweep_norm(LevelView<T> lv, uint32_t total, const T* __restrict__ u,
                                                         const T* __restrict__ bs, T* __restrict__ uo,
                                                         const float* __restrict__ dw32,
                                                         const int* __restrict__ kexp,
                                                         double* __restrict__ partials) {
  float acc = 0.f;
  const float Wo32 = (float)lv.Wo;
  const int k = scale_exp(kexp);
  for (uint32_t idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += gridDim.x * blockDim.x) {
    int n, i;
    split_index(idx, lv.fd, n, i);
    const size_t p = (size_t)n * lv.pitch + i;
    const T y = scaled_residual<T, ADJ>(lv, u, bs, n, i, p);
    uo[p] = u[p] + y;
    float yf;
    if constexpr (std::is_same<T, double>::value) yf = to_f32_trunc(y, k);
    else yf = y;
    const float r = ((n == 0 || i == 0) ? Wo32 : dw32[i]) * yf;
    acc = fmaf(r, r, acc);
  }
  const double s = block_sum<kThreads>((double)acc);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// r = b - J u (MODE 0, from b') or y = J u (MODE 1, plain coefficients).
template <typename T, bool ADJ, int MODE>
__global__ void __launch_bounds__(kThreads) k_residual(LevelView<T> lv, uint32_t total, const T* __restrict__ u,
                                                       const T* __restrict__ bs, T* __restrict__ r) {
  pdl_wait();  // a no-op unless launched dependent (small grids)
  const uint32_t idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= total) return;
  int n, i;
  split_index(idx, lv.fd, n, i);
  const size_t p = (size_t)n * lv.pitch + i;
  if (MODE == 0) r[p] = unscale(lv, n, i) * scaled_residual<T, ADJ>(lv, u, bs, n, i, p);
  else if (MODE == 2) r[p] = scaled_residual<T, ADJ>(lv, u, bs, n, i, p);
  else r[p] = apply_at(lv, ADJ, u, n, i, p);
}

// Restriction from the scaled residual y = (omega/D) r with the weights of the fine level's
// kRW* slots, which fold D/omega of the fine node and omega/D_c of the coarse node into
// P^T (the operator of k_restrict applied to r): x, b_c = wl y_{2j-1} + wc y_{2j} +
// wr y_{2j+1}; t causal, b_c = a0 y_{2m} + a1 y_{2m+1}; t bilinear, b_c = a0 y_{2m} +
// a1 (y_{2m-1} + y_{2m+1}).  Coarse row 0 (Dirichlet) takes its weights from r0 = W_f/W_c,
// r0h = r0/2 and, for t, kRWL (fine row 1).  One arithmetic form per type with the weights
// selected: a branch between forms would be if-converted into both, and on this GPU every
// FP64 instruction costs 64 issue cycles of its unit.  The FP64 residual thereby drops its
// unscaling multiply (6 FMAs per DOF instead of 7).
template <typename T, int TYPE>
__global__ void __launch_bounds__(kThreads) k_restrict_scaled(int Nf, int NTf, int pf, const T* cf, T r0, T r0h,
                                                              const T* __restrict__ y, LevelView<T> cv,
                                                              uint32_t total, T* __restrict__ bc) {
  pdl_wait();  // a no-op unless launched dependent (small grids)
  const uint32_t idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= total) return;
  int m, j;
  split_index(idx, cv.fd, m, j);
  const bool dir = m == 0;
  T out;
  if (TYPE == 1) {
    const T* row = y + (size_t)m * pf + 2 * j;
    const T yc = row[0];
    const T yl = j >= 1 ? row[-1] : T(0);
    const T yr = 2 * j + 1 <= Nf ? row[1] : T(0);
    const T wl = dir ? r0h : cf[kRWL * pf + j];
    const T wc = dir ? r0 : cf[kRWC * pf + j];
    const T wr = dir ? r0h : cf[kRWR * pf + j];
    out = fma(wl, yl, fma(wr, yr, wc * yc));
  } else {
    const T* col = y + j;
    const T y0 = col[(size_t)(2 * m) * pf];
    const T y1 = 2 * m + 1 <= NTf ? col[(size_t)(2 * m + 1) * pf] : T(0);
    const T wc = cf[kRWC * pf + j];
    const T a0 = dir ? r0h : wc;
    if (TYPE == 2) {
      const T a1 = dir ? cf[kRWL * pf + j] : wc;
      out = fma(a1, y1, a0 * y0);
    } else {
      const T a1 = dir ? cf[kRWL * pf + j] : cf[kRWR * pf + j];
      const T am = dir ? T(0) : cf[kRWR * pf + j];
      const T ym = dir ? T(0) : col[(size_t)(2 * m - 1) * pf];
      out = fma(a1, y1, fma(am, ym, a0 * y0));
    }
  }
  bc[(size_t)m * cv.pitch + j] = out;
}

// The kRW* weights of a fine level toward its coarse level (one thread per coarse node j
// for x, per node i for t).  u_i = D_i/omega (W_f/omega at i = 0) is the fine kDW slot,
// s_j = omega/D_c (omega/W_c at j = 0) the coarse kW slot.
__global__ void k_build_rweights(int type, int Nf, int pf, int Nc, int pc, double Wf, double Wc, double omega,
                                 const double* __restrict__ cfc, double* cf64, float* cf32) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  double wl, wc, wr;
  if (type == 1) {
    if (j > Nc) return;
    const double sc = cfc[kW * pc + j];
    wc = sc * cf64[kDW * pf + 2 * j];
    wl = j >= 1 ? 0.5 * sc * cf64[kDW * pf + 2 * j - 1] : 0.0;
    wr = 2 * j + 1 <= Nf ? 0.5 * sc * cf64[kDW * pf + 2 * j + 1] : 0.0;
  } else {
    // t: kRWC interior coarse rows, kRWR half of it (bilinear outer rows), kRWL fine row 1
    // in coarse row 0 (fine row 0 there: W_f / (2 W_c), a kernel argument)
    if (j > Nf) return;
    const double ui = cf64[kDW * pf + j];
    wc = 0.5 * cfc[kW * pc + j] * ui;
    wr = 0.5 * wc;
    wl = (type == 2 ? 0.5 : 0.25) * (omega / Wc) * ui;
  }
  cf64[kRWL * pf + j] = wl;
  cf64[kRWC * pf + j] = wc;
  cf64[kRWR * pf + j] = wr;
  cf32[kRWL * pf + j] = (float)wl;
  cf32[kRWC * pf + j] = (float)wc;
  cf32[kRWR * pf + j] = (float)wr;
}

// Restriction b_c = s P^T r (Sec. 3.1), stored scaled by omega / D_c of the coarse level:
// type 1, x: 1/2 [1 2 1] within the row, s = 1; type 2, t causal: rows 2m and 2m+1, s = 1/2
// (row 2m+1 absent past the last fine row); type 3, t bilinear (Sec. 5.1): rows 2m-1, 2m,
// 2m+1 weighted 1/2, 1, 1/2, s = 1/2.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_restrict(int type, int Nf, int NTf, int pf, const T* __restrict__ r,
                                                       LevelView<T> cv, uint32_t total, T* __restrict__ bc) {
  const uint32_t idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= total) return;
  int m, j;
  split_index(idx, cv.fd, m, j);
  T acc;
  if (type == 1) {
    const T* row = r + (size_t)m * pf;
    acc = row[2 * j];
    if (2 * j - 1 >= 0) acc += T(0.5) * row[2 * j - 1];
    if (2 * j + 1 <= Nf) acc += T(0.5) * row[2 * j + 1];
  } else if (type == 2) {
    acc = r[(size_t)(2 * m) * pf + j];
    if (2 * m + 1 <= NTf) acc += r[(size_t)(2 * m + 1) * pf + j];
    acc *= T(0.5);
  } else {
    // bilinear in time (Sec. 5.1): P^T gathers rows 2m-1, 2m, 2m+1 with 1/2, 1, 1/2; s = 1/2
    acc = r[(size_t)(2 * m) * pf + j];
    if (2 * m - 1 >= 0) acc += T(0.5) * r[(size_t)(2 * m - 1) * pf + j];
    if (2 * m + 1 <= NTf) acc += T(0.5) * r[(size_t)(2 * m + 1) * pf + j];
    acc *= T(0.5);
  }
  const T sc = (m == 0 || j == 0) ? cv.wW : cv.coef[kW * cv.pitch + j];
  bc[(size_t)m * cv.pitch + j] = sc * acc;
}

// u += P z (Sec. 3.1): type 1, x: fine node 2j gets z_j, node 2j+1 gets (z_j + z_{j+1}) / 2;
// type 2, t causal: fine rows 2m and 2m+1 get coarse row m; type 3, t bilinear: fine row
// 2m gets z_m and row 2m+1 gets (z_m + z_{m+1}) / 2.  One thread per coarse DOF updates
// both fine DOFs it feeds (nodes 2j, 2j+1 of a row, as one 2-vector, or rows 2m, 2m+1 of a
// node), so each z is read once and an interpolated DOF costs one add and one FMA: on this
// GPU FP64 additions run at the FMA rate, 1/64 of FP32, and one per DOF already takes
// longer than the kernel's memory traffic.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_prolong_add(int type, int Nf, int NTf, FastDiv fdc, uint32_t total,
                                                          int pf, T* __restrict__ u, int pc, const T* __restrict__ z) {
  pdl_wait();  // a no-op unless launched dependent (small grids)
  const uint32_t idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= total) return;
  int a, c;
  split_index(idx, fdc, a, c);
  if (type == 1) {
    // a: row n, c: coarse node j; the last coarse node feeds fine node N alone (one
    // arithmetic form for both, so that no FP64 operation is duplicated by if-conversion)
    using V2 = typename std::conditional<std::is_same<T, double>::value, double2, float2>::type;
    const T* zr = z + (size_t)a * pc;
    T* ur = u + (size_t)a * pf + 2 * c;
    const bool pair = 2 * c + 1 <= Nf;
    const T z0 = zr[c];
    const T z1 = pair ? zr[c + 1] : T(0);
    V2 v;
    if (pair) v = *reinterpret_cast<const V2*>(ur);
    else v = V2{ur[0], T(0)};
    v.x = v.x + z0;
    v.y = fma(T(0.5), z0 + z1, v.y);
    if (pair) *reinterpret_cast<V2*>(ur) = v;
    else ur[0] = v.x;
  } else {
    // a: coarse row m, c: node i
    const T z0 = z[(size_t)a * pc + c];
    T* u0 = u + (size_t)(2 * a) * pf + c;
    u0[0] = u0[0] + z0;
    if (2 * a + 1 <= NTf) {
      T* u1 = u0 + pf;
      if (type == 2) u1[0] = u1[0] + z0;
      else u1[0] = fma(T(0.5), z0 + z[(size_t)(a + 1) * pc + c], u1[0]);
    }
  }
}

// x <- (omega/D) x or (D/omega) x at every DOF (padding untouched).
template <typename T>
__global__ void __launch_bounds__(kThreads) k_scale(LevelView<T> lv, uint32_t total, bool to_scaled,
                                                    T* __restrict__ x) {
  const uint32_t idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= total) return;
  int n, i;
  split_index(idx, lv.fd, n, i);
  const bool dir = n == 0 || i == 0;
  const T f = to_scaled ? (dir ? lv.wW : lv.coef[kW * lv.pitch + i]) : (dir ? lv.Wo : lv.coef[kDW * lv.pitch + i]);
  const size_t p = (size_t)n * lv.pitch + i;
  x[p] = f * x[p];
}

// Exact solve of J u = b (or J^T u = b) by implicit time stepping: Dirichlet DOFs
// u = b / W; then for each step a Thomas solve of (M/dt + K)_int T_n = f_n with
// f_n = b_n - (coupling to the previous step), forward in time for J and backward for
// J^T.  Arithmetic in FP64 whatever the storage type.  For levels of at most 64 elements:
// one warp, lane l owning nodes 2l+1 and 2l+2.  Both Thomas sweeps are first-order affine
// recurrences, x_i = a_i x_{i-1} + c_i (elimination) and y_i = e_i y_{i+1} + d_i (back
// substitution), evaluated as warp scans of affine maps: the multipliers are the same for
// every step, so their partial products are formed once, and a step costs one FMA and one
// shuffle per scan level.  Each lane reads the next step's right-hand side a step ahead.
// The right-hand side arrives scaled (b' = (omega/D) b): b = (D/omega) b' in the interior
// and u = b / W = b' / omega on the Dirichlet DOFs.
constexpr int kExactWarpMaxN = 64;

__device__ __forceinline__ double shfl_up_d(double v, int d) { return __shfl_up_sync(0xffffffffu, v, d); }
__device__ __forceinline__ double shfl_down_d(double v, int d) { return __shfl_down_sync(0xffffffffu, v, d); }

template <typename T>
__global__ void __launch_bounds__(32) k_exact(ThomasView tv, bool adj, const T* __restrict__ b, T* __restrict__ u) {
  const int N = tv.N, NT = tv.NT, P = tv.pitch;
  const int lane = threadIdx.x;
  pdl_wait();
  for (int i = lane; i <= N; i += 32) u[i] = (T)((double)b[i] / tv.omega);
  for (int n = 1 + lane; n <= NT; n += 32) u[(size_t)n * P] = (T)((double)b[(size_t)n * P] / tv.omega);
  const int i0 = 2 * lane + 1, i1 = 2 * lane + 2;
  const bool h0 = i0 <= N, h1 = i1 <= N;
  // elimination: dp_i = (f_i - lo_i dp_{i-1}) inv_i, i.e. a_i = -lo_i inv_i, c_i = f_i inv_i;
  // back substitution: y_i = d_i - cp_i y_{i+1}, i.e. e_i = -cp_i; absent nodes are identities
  const double inv0 = h0 ? tv.inv[i0] : 0.0, inv1 = h1 ? tv.inv[i1] : 0.0;
  const double a0 = h0 && i0 > 1 ? -tv.lo[i0] * inv0 : (h0 ? 0.0 : 1.0);
  const double a1 = h1 ? -tv.lo[i1] * inv1 : 1.0;
  const double e0 = h0 && i0 < N ? -tv.cp[i0] : (h0 ? 0.0 : 1.0);
  const double e1 = h1 && i1 < N ? -tv.cp[i1] : (h1 ? 0.0 : 1.0);
  const double dw0 = h0 ? tv.dw[i0] : 0.0, dw1 = h1 ? tv.dw[i1] : 0.0;
  const double pl0 = h0 ? tv.pl[i0] : 0.0, pc0 = h0 ? tv.pc[i0] : 0.0, pr0 = h0 ? tv.pr[i0] : 0.0;
  const double pl1 = h1 ? tv.pl[i1] : 0.0, pc1 = h1 ? tv.pc[i1] : 0.0, pr1 = h1 ? tv.pr[i1] : 0.0;
  // lane aggregates and the Kogge-Stone multipliers of both scans (step-invariant)
  const double A = a1 * a0, E = e0 * e1;
  double Af[5], Eb[5];
  {
    double x = A, y = E;
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      const int d = 1 << k;
      const double xu = shfl_up_d(x, d), yd = shfl_down_d(y, d);
      Af[k] = lane >= d ? x : 0.0;
      Eb[k] = lane + d < 32 ? y : 0.0;
      if (lane >= d) x *= xu;
      if (lane + d < 32) y *= yd;
    }
  }
  double p0 = 0.0, p1 = 0.0;  // previous step's solution at i0, i1 (node 0: eliminated column)
  auto load = [&](int step, double& f0, double& f1) {
    const int n = adj ? NT + 1 - step : step;
    const T* bn = b + (size_t)n * P;
    f0 = h0 ? (double)bn[i0] * dw0 : 0.0;
    f1 = h1 ? (double)bn[i1] * dw1 : 0.0;
  };
  double f0 = 0.0, f1 = 0.0;
  if (NT >= 1) load(1, f0, f1);
  for (int step = 1; step <= NT; ++step) {
    double g0 = 0.0, g1 = 0.0;
    if (step < NT) load(step + 1, g0, g1);
    const int n = adj ? NT + 1 - step : step;
    const bool has_prev = adj ? (n < NT) : (n > 1);
    if (has_prev) {
      const double pm = shfl_up_d(p1, 1);    // node i0 - 1
      const double pp = shfl_down_d(p0, 1);  // node i1 + 1
      const double pmm = lane == 0 ? 0.0 : pm;
      const double ppp = i1 + 1 <= N ? pp : 0.0;
      f0 -= pl0 * pmm + pc0 * p0 + pr0 * p1;
      f1 -= pl1 * p0 + pc1 * p1 + pr1 * ppp;
    }
    // elimination scan: lane value = dp at node i1 given dp = 0 before node 1
    const double c0 = f0 * inv0, c1 = f1 * inv1;
    double C = a1 * c0 + c1;
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      const double cu = shfl_up_d(C, 1 << k);
      if (lane >= (1 << k)) C = fma(Af[k], cu, C);
    }
    const double cb = shfl_up_d(C, 1);  // every lane shuffles; lane 0 then takes dp_0 = 0
    const double before = lane == 0 ? 0.0 : cb;
    const double d0 = h0 ? a0 * before + c0 : 0.0;
    const double d1 = h1 ? C : 0.0;
    // back-substitution scan from node N down: lane value = y at node i0
    double D = e0 * d1 + d0;
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      const double dd = shfl_down_d(D, 1 << k);
      if (lane + (1 << k) < 32) D = fma(Eb[k], dd, D);
    }
    const double da = shfl_down_d(D, 1);  // every lane shuffles; lane 31 then takes y_{N+1} = 0
    const double after = lane == 31 ? 0.0 : da;
    const double y1 = h1 ? e1 * after + d1 : 0.0;
    const double y0 = h0 ? D : 0.0;
    T* un = u + (size_t)n * P;
    if (h0) un[i0] = (T)y0;
    if (h1) un[i1] = (T)y1;
    p0 = y0;
    p1 = y1;
    f0 = g0;
    f1 = g1;
  }
}

// Exact solve of a narrow coarsest level by a scan in time.  With the Dirichlet columns
// eliminated, the interior rows of J u = b read A u_n = b_n - B u_{n-1} (n >= 2; row 1 has
// no coupling to the Dirichlet row 0), with A = (M/dt + K)_int and B = -(M/dt)_int, and
// those of J^T u = b read A u_n = b_n - B u_{n+1} (n <= NT - 1), B being symmetric.  So
// u_n = f_n + G u_{n-+1} with f_n = A^-1 b_n and G = -A^-1 B in both directions.  The f_n
// are independent tridiagonal solves (Thomas, one row per thread); the recurrence is a
// Kogge-Stone scan over n, whose step with distance 2^k multiplies by G^(2^k), precomputed
// on the host (pw: K row-major N x N matrices).  One block; the rows live in shared memory
// (two buffers of NT x N doubles).  Arithmetic in FP64 whatever the storage type.
template <typename T>
__global__ void __launch_bounds__(256) k_exact_scan(ThomasView tv, bool adj, int K, const double* __restrict__ pw,
                                                    const T* __restrict__ b, T* __restrict__ u) {
  extern __shared__ double sm[];
  const int N = tv.N, NT = tv.NT, P = tv.pitch;
  const int tid = threadIdx.x, nth = blockDim.x;
  pdl_wait();
  for (int i = tid; i <= N; i += nth) u[i] = (T)((double)b[i] / tv.omega);
  for (int n = 1 + tid; n <= NT; n += nth) u[(size_t)n * P] = (T)((double)b[(size_t)n * P] / tv.omega);
  double* g = sm;                    // row n (1..NT), node i (1..N) at (n - 1) * N + i - 1
  double* h = sm + (size_t)NT * N;
  for (int n = 1 + tid; n <= NT; n += nth) {
    double* f = g + (size_t)(n - 1) * N - 1;  // f[i], i = 1..N
    const T* bn = b + (size_t)n * P;
    double dp = 0.0;
    for (int i = 1; i <= N; ++i) {
      dp = ((double)bn[i] * tv.dw[i] - tv.lo[i] * dp) * tv.inv[i];
      f[i] = dp;
    }
    for (int i = N - 1; i >= 1; --i) f[i] -= tv.cp[i] * f[i + 1];
  }
  __syncthreads();
  for (int k = 0, d = 1; k < K; ++k, d <<= 1) {
    const double* Gk = pw + (size_t)k * N * N;
    for (int q = tid; q < NT * N; q += nth) {
      const int n = 1 + q / N, i = q - (n - 1) * N;
      const int m = adj ? n + d : n - d;
      double v = g[q];
      if (adj ? m <= NT : m >= 1) {
        const double* src = g + (size_t)(m - 1) * N;
        const double* row = Gk + (size_t)i * N;
        for (int j = 0; j < N; ++j) v = fma(row[j], src[j], v);
      }
      h[q] = v;
    }
    __syncthreads();
    double* t = g;
    g = h;
    h = t;
  }
  for (int q = tid; q < NT * N; q += nth) {
    const int n = 1 + q / N, i = q - (n - 1) * N;
    u[(size_t)n * P + 1 + i] = (T)g[q];
  }
}

// One projected-gradient design update, the stand-in for the MMA optimiser of the
// optimisation loop (Sec. 7.2): y = chi - move * (g / max|g|) and
// chi_new = clamp(y - mu, max(0, chi - move), min(1, chi + move)), mu >= 0 the smallest
// shift with mean(chi_new) <= vol (the volume constraint of Sec. 7.1), by 64 bisection
// steps on [0, 2].  One block of 1024 threads; every reduction is a fixed tree, and y, the
// bounds and the shift are rounded exactly as written (no FMA contraction).
constexpr int kDesignThreads = 1024;
constexpr int kDesignBisection = 64;

template <bool MAX>
__device__ double block_reduce(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) {
    const double w = __shfl_xor_sync(0xffffffffu, v, o);
    v = MAX ? fmax(v, w) : v + w;
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();  // red is reused by consecutive reductions
  if (lane == 0) red[wid] = v;
  __syncthreads();
  if (wid == 0) {
    v = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) {
      const double w = __shfl_xor_sync(0xffffffffu, v, o);
      v = MAX ? fmax(v, w) : v + w;
    }
    if (lane == 0) red[32] = v;
  }
  __syncthreads();
  return red[32];
}

__device__ __forceinline__ double design_value(double c, double gi, double gmax, double move, double mu) {
  const double step = gmax > 0.0 ? gi / gmax : 0.0;
  const double y = __dsub_rn(c, __dmul_rn(move, step));
  const double lo = fmax(0.0, __dsub_rn(c, move));
  const double hi = fmin(1.0, __dadd_rn(c, move));
  return fmin(fmax(__dsub_rn(y, mu), lo), hi);
}

__global__ void __launch_bounds__(kDesignThreads) k_design_update(int N, const double* chi, const double* g,
                                                                 double vol, double move, double* out) {
  __shared__ double red[33];
  double m = 0.0;
  for (int i = threadIdx.x; i < N; i += blockDim.x) m = fmax(m, fabs(g[i]));
  const double gmax = block_reduce<true>(m, red);
  auto mean_at = [&](double mu) {
    double s = 0.0;
    for (int i = threadIdx.x; i < N; i += blockDim.x) s += design_value(chi[i], g[i], gmax, move, mu);
    return block_reduce<false>(s, red) / N;
  };
  double mu = 0.0;
  if (mean_at(0.0) > vol) {
    double a = 0.0, b = 2.0;
    for (int it = 0; it < kDesignBisection; ++it) {
      const double mid = 0.5 * (a + b);
      if (mean_at(mid) > vol) a = mid;
      else b = mid;
    }
    mu = b;
  }
  // each element is read and written by the same thread: out may alias chi
  for (int i = threadIdx.x; i < N; i += blockDim.x) out[i] = design_value(chi[i], g[i], gmax, move, mu);
}

// ||r||^2 of r = b - J u from the stored b' (u null: r = b), optionally storing the
// scaled residual y = (omega/D) r as R.
template <typename T, typename R, bool ADJ>
__global__ void __launch_bounds__(kThreads) k_resnorm(LevelView<T> lv, uint32_t total, const T* __restrict__ u,
                                                      const T* __restrict__ bs, R* __restrict__ y_out,
                                                      double* __restrict__ partials) {
  double acc = 0.0;
  for (uint32_t idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += gridDim.x * blockDim.x) {
    int n, i;
    split_index(idx, lv.fd, n, i);
    const size_t p = (size_t)n * lv.pitch + i;
    const T y = u ? scaled_residual<T, ADJ>(lv, u, bs, n, i, p) : bs[p];
    if (y_out) y_out[p] = (R)y;
    const double r = (double)(unscale(lv, n, i) * y);
    acc = fma(r, r, acc);
  }
  const double s = block_sum<kThreads>(acc);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// Mixed-scheme defect on the finest level: y = (omega/D)(b - J u) in FP64 (the scaled
// residual of the FP64 iterate), stored as FP32 scaled by 2^k as the right-hand side of the
// next FP32 cycle.  The squared norm, which only feeds the termination test, is accumulated
// in FP32 per thread (2^k r = (D/omega) 2^k y with the FP32 coefficients) and summed in FP64
// across the block: 6 FP64 FMAs per DOF (the conversion to FP32 runs on the integer pipe).
template <bool ADJ>
__global__ void __launch_bounds__(kThreads) k_defect(LevelView<double> lv, uint32_t total, const float* __restrict__ dw32,
                                                     const double* __restrict__ u, const double* __restrict__ bs,
                                                     const int* __restrict__ kexp, float* __restrict__ ys32,
                                                     double* __restrict__ partials) {
  float acc = 0.f;
  const float Wo32 = (float)lv.Wo;
  const int k = scale_exp(kexp);
  for (uint32_t idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += gridDim.x * blockDim.x) {
    int n, i;
    split_index(idx, lv.fd, n, i);
    const size_t p = (size_t)n * lv.pitch + i;
    const float y = to_f32_trunc(scaled_residual<double, ADJ>(lv, u, bs, n, i, p), k);
    ys32[p] = y;
    const float r = ((n == 0 || i == 0) ? Wo32 : dw32[i]) * y;
    acc = fmaf(r, r, acc);
  }
  const double s = block_sum<kThreads>((double)acc);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// y = 2^k b' truncated to FP32 over a whole padded array, two values per thread: the
// mixed scheme's first defect from u = 0 (k from scale_exp).
__global__ void __launch_bounds__(kThreads) k_to_f32_pairs(size_t n2, const double2* __restrict__ b,
                                                           const int* __restrict__ kexp, float2* __restrict__ y) {
  const size_t j = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (j >= n2) return;
  const int k = scale_exp(kexp);
  const double2 v = b[j];
  y[j] = make_float2(to_f32_trunc(v.x, k), to_f32_trunc(v.y, k));
}

// Sum of the per-block partials into out[0].  kget: the partials are of 2^k r (k from
// scale_exp), so the sum is scaled by 2^-2k.  kset: the partials are ||b||^2 over `count`
// DOFs; sets k so that 2^k b has an RMS in [1, 2) (k = 0 for a zero or non-finite sum).
__global__ void k_final_sum(const double* __restrict__ partials, int n, double* __restrict__ out,
                            const int* __restrict__ kget, int* __restrict__ kset, double count) {
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) acc += partials[i];
  const double s = block_sum<1024>(acc);
  if (threadIdx.x == 0) {
    out[0] = kget ? ldexp(s, -2 * *kget) : s;
    if (kset) {
      const double ms = s / count;
      int k = 0;
      if (ms > 0.0 && isfinite(ms)) k = -(ilogb(ms) >> 1);
      kset[0] = max(-kMaxScaleExp, min(kMaxScaleExp, k));
    }
  }
}

__global__ void __launch_bounds__(kThreads) k_dot(size_t n, const double* __restrict__ a,
                                                  const double* __restrict__ b, double* __restrict__ partials) {
  double acc = 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    acc = fma(a[i], b[i], acc);
  const double s = block_sum<kThreads>(acc);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads) k_scaled_copy(size_t n, double alpha, const double* __restrict__ x,
                                                          double* __restrict__ y) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    y[i] = alpha * x[i];
}

__global__ void __launch_bounds__(kThreads) k_add_correction(size_t n, double* __restrict__ u,
                                                             const float* __restrict__ e,
                                                             const int* __restrict__ kexp) {
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i < n) u[i] += to_f64(e[i], -scale_exp(kexp));
}

// Stencil coefficients per node from element k, c (Sec. 2.2 element matrices, Appendix A).
// m_e = c_e dx / (6 dt) and s_e = k_e / dx; node i touches elements i-1 and i.  Also the
// smoother's scaled coefficients (see stmg_internal.h).
__global__ void k_build_coef(int N, int pitch, double dx, double dt, double W, double omega,
                             const double* __restrict__ k, const double* __restrict__ c, double* __restrict__ cf64,
                             float* __restrict__ cf32) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= pitch) return;
  double v[kNumCoef];
#pragma unroll
  for (int s = 0; s < kNumCoef; ++s) v[s] = 0.0;
  if (i == 0) {
    v[kD] = W;
    v[kW] = omega / W;
    v[kDW] = W / omega;
  } else if (i <= N) {
    const double ml = c[i - 1] * dx / (6.0 * dt), sl = k[i - 1] / dx;
    const double mr = i < N ? c[i] * dx / (6.0 * dt) : 0.0, sr = i < N ? k[i] / dx : 0.0;
    v[kL] = i >= 2 ? ml - sl : 0.0;
    v[kU] = i < N ? mr - sr : 0.0;
    v[kD] = 2.0 * ml + sl + 2.0 * mr + sr;
    v[kPL] = i >= 2 ? -ml : 0.0;
    v[kPC] = -2.0 * (ml + mr);
    v[kPR] = i < N ? -mr : 0.0;
    v[kW] = omega / v[kD];
    v[kDW] = v[kD] / omega;
    v[kSL] = -v[kW] * v[kL];
    v[kSU] = -v[kW] * v[kU];
    v[kSPL] = -v[kW] * v[kPL];
    v[kSPC] = -v[kW] * v[kPC];
    v[kSPR] = -v[kW] * v[kPR];
  }
#pragma unroll
  for (int s = 0; s < kNumCoef; ++s) {
    if (cf64) cf64[(size_t)s * pitch + i] = v[s];
    if (cf32) cf32[(size_t)s * pitch + i] = (float)v[s];
  }
}

// SIMP (Sec. 2.1).
__global__ void k_simp(int N, const double* __restrict__ chi, Simp6 sp, double* __restrict__ k,
                       double* __restrict__ c) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= N) return;
  const double x = chi[e];
  k[e] = sp.v[0] + (sp.v[1] - sp.v[0]) * pow(x, sp.v[4]);
  c[e] = sp.v[2] + (sp.v[3] - sp.v[2]) * pow(x, sp.v[5]);
}

// b = B b_Neu with b_Neu,i = dx/2 (q_{i-1} + q_i) for element-wise constant q, stored
// scaled as b' = mult (omega/D) b; q == nullptr: the same constant qconst on every element.
// Writes every value of the padded rows.  Threads own columns and loop over rows, so the
// column factor f (omega/D_i) with f = mult dx / 2 is formed once per thread and a DOF costs
// one FP64 add and one multiply (none for a constant load).  partials: also ||b||^2, as
// f^2 sum (q_{i-1} + q_i)^2 over the interior DOFs (b is zero on the Dirichlet DOFs), one
// FMA per DOF, one partial per block.
__global__ void __launch_bounds__(kThreads) k_assemble_load(LevelView<double> lv, const double* __restrict__ q,
                                                            double qconst, double f, double* __restrict__ b,
                                                            double* __restrict__ partials) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int N = lv.N;
  double acc = 0.0;
  if (i < lv.pitch) {
    const bool interior = i >= 1 && i <= N;
    const double g = interior ? f * lv.coef[kW * lv.pitch + i] : 0.0;
    const double qc = i < N ? 2.0 * qconst : qconst;
    const double vconst = g * qc;
    for (int n = blockIdx.y; n <= lv.NT; n += gridDim.y) {
      double v = 0.0;
      if (n >= 1 && interior) {
        double qs = qc;
        if (q) {
          const double* qn = q + (size_t)n * N;
          qs = qn[i - 1] + (i < N ? qn[i] : 0.0);
          v = g * qs;
        } else {
          v = vconst;
        }
        if (partials) acc = fma(qs, qs, acc);
      }
      b[(size_t)n * lv.pitch + i] = v;
    }
  }
  if (partials) {
    const double sum = block_sum<kThreads>(acc);
    if (threadIdx.x == 0) partials[blockIdx.y * gridDim.x + blockIdx.x] = f * f * sum;
  }
}

// Sensitivity partial sums over a chunk of time levels for element e (Sec. 7.2):
//   S_k = sum_n (lam_e - lam_{e+1}) (u_e - u_{e+1}) / dx
//   S_c = sum_n dx/(6 dt) [lam_e (2 d_e + d_{e+1}) + lam_{e+1} (d_e + 2 d_{e+1})],
// d_j = u[n][j] - u[n-1][j] (the n-1 term only for n >= 2); node 0 values are masked.
__global__ void k_sens_partial(int N, int NT, int pitch, double dx, double dt, const double* __restrict__ u,
                               const double* __restrict__ lam, double* __restrict__ scratch) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  const int chunk = blockIdx.y;
  if (e >= N) return;
  const int n0 = max(1, chunk * kSensRowsPerChunk), n1 = min(NT, (chunk + 1) * kSensRowsPerChunk - 1);
  double sk = 0.0, sc = 0.0;
  for (int n = n0; n <= n1; ++n) {
    const double* un = u + (size_t)n * pitch;
    const double* ln = lam + (size_t)n * pitch;
    const double ue = e == 0 ? 0.0 : un[e], ue1 = un[e + 1];
    const double le = e == 0 ? 0.0 : ln[e], le1 = ln[e + 1];
    double de = ue, de1 = ue1;
    if (n >= 2) {
      const double* up = un - pitch;
      de -= e == 0 ? 0.0 : up[e];
      de1 -= up[e + 1];
    }
    sk = fma(le - le1, ue - ue1, sk);
    sc = fma(le, 2.0 * de + de1, sc);
    sc = fma(le1, de + 2.0 * de1, sc);
  }
  const int chunks = gridDim.y;
  scratch[(size_t)chunk * N + e] = sk / dx;
  scratch[(size_t)(chunks + chunk) * N + e] = sc * dx / (6.0 * dt);
}

__global__ void k_sens_final(int N, int chunks, const double* __restrict__ chi, Simp6 sp,
                             const double* __restrict__ scratch, double* __restrict__ g) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= N) return;
  double sk = 0.0, sc = 0.0;
  for (int q = 0; q < chunks; ++q) {
    sk += scratch[(size_t)q * N + e];
    sc += scratch[(size_t)(chunks + q) * N + e];
  }
  const double x = chi[e];
  const double dk = sp.v[4] * (sp.v[1] - sp.v[0]) * pow(x, sp.v[4] - 1.0);
  const double dc = sp.v[5] * (sp.v[3] - sp.v[2]) * pow(x, sp.v[5] - 1.0);
  g[e] = -(dk * sk + dc * sc);
}

}  // namespace

// ------------------------------------------------------------------------------ launchers

template <typename T>
inline uint32_t dofs(const LevelView<T>& lv) {
  return (uint32_t)((uint64_t)(lv.NT + 1) * (uint64_t)(lv.N + 1));
}

template <typename T>
cudaError_t launch_sweep(const LevelView<T>& lv, bool adj, const T* u, const T* bs, T* uo, cudaStream_t s) {
  const uint32_t n = dofs(lv);
  const cudaError_t e = adj ? launch_small(k_sweep<T, true>, blocks_for(n), s, lv, n, u, bs, uo)
                            : launch_small(k_sweep<T, false>, blocks_for(n), s, lv, n, u, bs, uo);
  if (e != cudaSuccess) return e;
  count_launches(1);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_sweep_norm(const LevelView<T>& lv, bool adj, const T* u, const T* bs, T* uo, const float* dw32,
                              const int* kexp, double* partials, double* out, cudaStream_t s) {
  const uint32_t n = dofs(lv);
  if (!std::is_same<T, double>::value) kexp = nullptr;  // FP32 levels are not rescaled
  if (adj) k_sweep_norm<T, true><<<kNormBlocks, kThreads, 0, s>>>(lv, n, u, bs, uo, dw32, kexp, partials);
  else k_sweep_norm<T, false><<<kNormBlocks, kThreads, 0, s>>>(lv, n, u, bs, uo, dw32, kexp, partials);
  k_final_sum<<<1, 1024, 0, s>>>(partials, kNormBlocks, out, kexp, nullptr, 0.0);
  count_launches(2);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_residual(const LevelView<T>& lv, bool adj, const T* u, const T* bs, T* r, cudaStream_t s) {
  const uint32_t n = dofs(lv);
  if (adj) k_residual<T, true, 0><<<blocks_for(n), kThreads, 0, s>>>(lv, n, u, bs, r);
  else k_residual<T, false, 0><<<blocks_for(n), kThreads, 0, s>>>(lv, n, u, bs, r);
  count_launches(1);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_residual_scaled(const LevelView<T>& lv, bool adj, const T* u, const T* bs, T* y, cudaStream_t s) {
  const uint32_t n = dofs(lv);
  const cudaError_t e = adj ? launch_small(k_residual<T, true, 2>, blocks_for(n), s, lv, n, u, bs, y)
                            : launch_small(k_residual<T, false, 2>, blocks_for(n), s, lv, n, u, bs, y);
  if (e != cudaSuccess) return e;
  count_launches(1);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_restrict_scaled(int type, int Nf, int NTf, int pf, const T* coef, T r0, const T* y,
                                   const LevelView<T>& cv, T* bc, cudaStream_t s) {
  const uint32_t n = dofs(cv);
  const T r0h = T(0.5) * r0;
  const unsigned g = blocks_for(n);
  const cudaError_t e =
      type == 1   ? launch_small(k_restrict_scaled<T, 1>, g, s, Nf, NTf, pf, coef, r0, r0h, y, cv, n, bc)
      : type == 2 ? launch_small(k_restrict_scaled<T, 2>, g, s, Nf, NTf, pf, coef, r0, r0h, y, cv, n, bc)
                  : launch_small(k_restrict_scaled<T, 3>, g, s, Nf, NTf, pf, coef, r0, r0h, y, cv, n, bc);
  if (e != cudaSuccess) return e;
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_build_rweights(int type, int Nf, int pf, int Nc, int pc, double Wf, double Wc, double omega,
                                  const double* cfc, double* cf64, float* cf32, cudaStream_t s) {
  const int n = (type == 1 ? Nc : Nf) + 1;
  k_build_rweights<<<blocks_for(n), kThreads, 0, s>>>(type, Nf, pf, Nc, pc, Wf, Wc, omega, cfc, cf64, cf32);
  count_launches(1);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_apply(const LevelView<T>& lv, bool adj, const T* u, T* y, cudaStream_t s) {
  const uint32_t n = dofs(lv);
  if (adj) k_residual<T, true, 1><<<blocks_for(n), kThreads, 0, s>>>(lv, n, u, nullptr, y);
  else k_residual<T, false, 1><<<blocks_for(n), kThreads, 0, s>>>(lv, n, u, nullptr, y);
  count_launches(1);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_restrict(int type, int Nf, int NTf, int pf, const T* r, const LevelView<T>& cv, T* bc,
                            cudaStream_t s) {
  const uint32_t n = dofs(cv);
  k_restrict<T><<<blocks_for(n), kThreads, 0, s>>>(type, Nf, NTf, pf, r, cv, n, bc);
  count_launches(1);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_prolong_add(int type, int Nf, int NTf, int pf, T* u, int Nc, int NTc, int pc, const T* z,
                               cudaStream_t s) {
  // one thread per coarse DOF: (row, coarse node) for x, (coarse row, node) for t
  const int width = type == 1 ? Nc + 1 : Nf + 1;
  const int rows = type == 1 ? NTf + 1 : NTc + 1;
  const uint32_t n = (uint32_t)((uint64_t)rows * (uint64_t)width);
  const cudaError_t e = launch_small(k_prolong_add<T>, blocks_for(n), s, type, Nf, NTf, make_fastdiv(width), n, pf, u, pc, z);
  if (e != cudaSuccess) return e;
  count_launches(1);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_exact_scan(const ThomasView& tv, bool adj, int K, const double* pw, const T* b, T* u,
                              cudaStream_t s) {
  const size_t smem = 2 * sizeof(double) * (size_t)tv.NT * tv.N;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_exact_scan<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(1);
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  count_launches(1);
  return cudaLaunchKernelEx(&cfg, k_exact_scan<T>, tv, adj, K, pw, b, u);
}

template <typename T>
cudaError_t launch_exact(const ThomasView& tv, bool adj, const T* b, T* u, cudaStream_t s) {
  if (tv.N < 1 || tv.N > kExactWarpMaxN) return cudaErrorInvalidValue;
  count_launches(1);
  return launch_pdl(k_exact<T>, dim3(1), dim3(32), s, tv, adj, b, u);
}

cudaError_t launch_design_update(int N, const double* chi, const double* g, double vol, double move, double* out,
                                 cudaStream_t s) {
  k_design_update<<<1, kDesignThreads, 0, s>>>(N, chi, g, vol, move, out);
  count_launches(1);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_scale(const LevelView<T>& lv, bool to_scaled, T* x, cudaStream_t s) {
  const uint32_t n = dofs(lv);
  k_scale<T><<<blocks_for(n), kThreads, 0, s>>>(lv, n, to_scaled, x);
  count_launches(1);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_resnorm(const LevelView<T>& lv, bool adj, const T* u, const T* bs, double* partials, double* out,
                           cudaStream_t s, int* kset) {
  const uint32_t n = dofs(lv);
  if (adj) k_resnorm<T, T, true><<<kNormBlocks, kThreads, 0, s>>>(lv, n, u, bs, (T*)nullptr, partials);
  else k_resnorm<T, T, false><<<kNormBlocks, kThreads, 0, s>>>(lv, n, u, bs, (T*)nullptr, partials);
  k_final_sum<<<1, 1024, 0, s>>>(partials, kNormBlocks, out, nullptr, kset, (double)n);
  count_launches(2);
  return cudaGetLastError();
}

cudaError_t launch_defect(const LevelView<double>& lv, const float* coef32, bool adj, const double* u,
                          const double* bs, const int* kexp, float* ys32, double* partials, double* out,
                          cudaStream_t s) {
  const uint32_t n = dofs(lv);
  const float* dw32 = coef32 + (size_t)kDW * lv.pitch;
  if (adj) k_defect<true><<<kNormBlocks, kThreads, 0, s>>>(lv, n, dw32, u, bs, kexp, ys32, partials);
  else k_defect<false><<<kNormBlocks, kThreads, 0, s>>>(lv, n, dw32, u, bs, kexp, ys32, partials);
  k_final_sum<<<1, 1024, 0, s>>>(partials, kNormBlocks, out, kexp, nullptr, 0.0);
  count_launches(2);
  return cudaGetLastError();
}

cudaError_t launch_rhs32(const LevelView<double>& lv, const double* bs, const int* kexp, float* ys32,
                         cudaStream_t s) {
  // the whole padded array in pairs (the padding of b' is zero, and so becomes that of y)
  const size_t n2 = (size_t)(lv.NT + 1) * lv.pitch / 2;
  k_to_f32_pairs<<<blocks_for((long long)n2), kThreads, 0, s>>>(n2, reinterpret_cast<const double2*>(bs), kexp,
                                                                reinterpret_cast<float2*>(ys32));
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_add_correction(size_t n, double* u, const float* e, const int* kexp, cudaStream_t s) {
  k_add_correction<<<blocks_for((long long)n), kThreads, 0, s>>>(n, u, e, kexp);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_scaled_copy(size_t n, double alpha, const double* x, double* y, cudaStream_t s) {
  const long long blocks = std::min<long long>(blocks_for((long long)n), 8LL * kNormBlocks);
  k_scaled_copy<<<(unsigned)std::max<long long>(1, blocks), kThreads, 0, s>>>(n, alpha, x, y);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_dot(size_t n, const double* a, const double* b, double* partials, double* out, cudaStream_t s) {
  k_dot<<<kNormBlocks, kThreads, 0, s>>>(n, a, b, partials);
  k_final_sum<<<1, 1024, 0, s>>>(partials, kNormBlocks, out, nullptr, nullptr, 0.0);
  count_launches(2);
  return cudaGetLastError();
}

cudaError_t launch_build_coef(int N, int pitch, double dx, double dt, double W, double omega, const double* k,
                              const double* c, double* coef64, float* coef32, cudaStream_t s) {
  k_build_coef<<<blocks_for(pitch), kThreads, 0, s>>>(N, pitch, dx, dt, W, omega, k, c, coef64, coef32);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_simp(int N, const double* chi, Simp6 sp, double* k, double* c, cudaStream_t s) {
  k_simp<<<blocks_for(N), kThreads, 0, s>>>(N, chi, sp, k, c);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_assemble_load(const LevelView<double>& lv, double dx, const double* q, double* bs,
                                 cudaStream_t s, double qconst, double mult, double* partials, double* out,
                                 int* kset) {
  // about 8 blocks per SM of 152 (at most kNormBlocks with the norm), each thread looping
  // over its column's rows; the norm is fused while one partial per block fits the
  // kNormBlocks-entry buffer (rows of at most 155 k columns), else it is a pass of its own
  const unsigned gx = blocks_for(lv.pitch);
  const bool fuse = partials && gx <= (unsigned)kNormBlocks;
  const int cap = fuse ? kNormBlocks : 152 * 8;
  const unsigned gy = (unsigned)std::max(1, std::min(lv.NT + 1, (int)(cap / gx)));
  k_assemble_load<<<dim3(gx, gy), kThreads, 0, s>>>(lv, q, qconst, mult * 0.5 * dx, bs, fuse ? partials : nullptr);
  count_launches(1);
  if (fuse) {
    k_final_sum<<<1, 1024, 0, s>>>(partials, (int)(gx * gy), out, nullptr, kset, (double)dofs(lv));
    count_launches(1);
  } else if (partials) {
    return launch_resnorm<double>(lv, false, nullptr, bs, partials, out, s, kset);
  }
  return cudaGetLastError();
}

cudaError_t launch_sensitivity(int N, int NT, int pitch, double dx, double dt, const double* chi, Simp6 sp,
                               const double* u, const double* lam, double* scratch, double* g, cudaStream_t s) {
  const int chunks = sens_chunks(NT);
  dim3 grid(blocks_for(N, 128), chunks);
  k_sens_partial<<<grid, 128, 0, s>>>(N, NT, pitch, dx, dt, u, lam, scratch);
  k_sens_final<<<blocks_for(N), kThreads, 0, s>>>(N, chunks, chi, sp, scratch, g);
  count_launches(2);
  return cudaGetLastError();
}

cudaError_t launch_sens_final(int N, int chunks, const double* chi, Simp6 sp, const double* scratch, double* g,
                              cudaStream_t s) {
  k_sens_final<<<blocks_for(N), kThreads, 0, s>>>(N, chunks, chi, sp, scratch, g);
  count_launches(1);
  return cudaGetLastError();
}

#define STMG_INST(T)                                                                                              \
  template cudaError_t launch_sweep<T>(const LevelView<T>&, bool, const T*, const T*, T*, cudaStream_t);          \
  template cudaError_t launch_sweep_norm<T>(const LevelView<T>&, bool, const T*, const T*, T*, const float*,     \
                                            const int*, double*, double*,                                       \
                                            cudaStream_t);                                                        \
  template cudaError_t launch_residual<T>(const LevelView<T>&, bool, const T*, const T*, T*, cudaStream_t);       \
  template cudaError_t launch_residual_scaled<T>(const LevelView<T>&, bool, const T*, const T*, T*, cudaStream_t); \
  template cudaError_t launch_restrict_scaled<T>(int, int, int, int, const T*, T, const T*, const LevelView<T>&,  \
                                                 T*, cudaStream_t);                                               \
  template cudaError_t launch_apply<T>(const LevelView<T>&, bool, const T*, T*, cudaStream_t);                    \
  template cudaError_t launch_restrict<T>(int, int, int, int, const T*, const LevelView<T>&, T*, cudaStream_t);   \
  template cudaError_t launch_prolong_add<T>(int, int, int, int, T*, int, int, int, const T*, cudaStream_t);      \
  template cudaError_t launch_exact<T>(const ThomasView&, bool, const T*, T*, cudaStream_t);                      \
  template cudaError_t launch_exact_scan<T>(const ThomasView&, bool, int, const double*, const T*, T*, cudaStream_t); \
  template cudaError_t launch_scale<T>(const LevelView<T>&, bool, T*, cudaStream_t);                              \
  template cudaError_t launch_resnorm<T>(const LevelView<T>&, bool, const T*, const T*, double*, double*,         \
                                         cudaStream_t, int*);
STMG_INST(double)
STMG_INST(float)
#undef STMG_INST

}  // namespace stmg
