// stmg_internal.h -- shared declarations between the host driver and the CUDA kernels.
//
// Device layout of one level with N elements and NT steps: a space-time vector is
// (NT+1) rows of `pitch` values; columns 0..N hold the nodes, columns N+1..pitch-1 are
// zero padding that no kernel ever writes (pitch >= N+2, so the right neighbour of node
// N is always a zero padding value).
//
// Operator (Sec. 2.2 stencil with the Dirichlet treatment of Appendix A): for the
// non-Dirichlet DOFs (n >= 1, i >= 1)
//
//   (J u)[n][i] = L_i u[n][i-1] + D_i u[n][i] + U_i u[n][i+1]
//               + PL_i u[p][i-1] + PC_i u[p][i] + PR_i u[p][i+1],
//
// p = n-1 for J (present for n >= 2) and p = n+1 for J^T (present for n <= NT-1); the
// mass and stiffness blocks are symmetric, so J and J^T share the coefficients (Sec. 7.2).
// Dirichlet DOFs (row 0 and column 0) have (J u) = W u.  L_1 = PL_1 = 0 and
// U_N = PR_N = 0 remove the eliminated column 0 and the missing element past x = L.
//
// Scaled form used by the smoother (Sec. 3.1 damped Jacobi with D the diagonal of J):
// every level stores its right-hand side as b' = (omega / D) b, and the coefficients
// S_k = -omega c_k / D for the five off-diagonal neighbours, so that one sweep is
//
//   u <- (1 - omega) u + b' + sum_k S_k u_k          (6 fused multiply-adds),
//
// and the residual is r = b - J u = (D / omega) (b' - omega u + sum_k S_k u_k).
#pragma once
#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

#include <vector>

#include "stmg.h"

namespace stmg {

enum CoefSlot {
  kL = 0, kD = 1, kU = 2, kPL = 3, kPC = 4, kPR = 5,  // J entries
  kW = 6,                                             // omega / D (b -> b')
  kDW = 7,                                            // D / omega (b' -> b)
  kSL = 8, kSU = 9, kSPL = 10, kSPC = 11, kSPR = 12,  // -omega c_k / D
  // restriction toward the next level applied to the scaled residual y = (omega/D) r, with
  // the fine (D/omega) and the coarse (omega/D_c) scalings folded in (launch_build_rweights):
  // x, per coarse node j: weights of fine nodes 2j-1, 2j, 2j+1 (interior rows); t, per node
  // i: kRWC for interior coarse rows, kRWR = kRWC / 2, kRWL for fine row 1 in coarse row 0
  kRWL = 13, kRWC = 14, kRWR = 15,
  kNumCoef = 16
};

inline int level_pitch(int N) {
  int need = N + 2;
  int align = need > 64 ? 32 : 8;
  return (need + align - 1) / align * align;
}

// x / d for 0 <= x < 2^31 by a multiply-high (Granlund & Montgomery 1994, round-up
// variant): s = ceil(log2 d), M = floor(2^32 (2^s - d) / d) + 1, q = (mulhi(x, M) + x) >> s.
struct FastDiv {
  uint32_t d, M, s;
};
inline FastDiv make_fastdiv(uint32_t d) {
  uint32_t s = 0;
  while ((1ull << s) < d) ++s;
  const uint64_t M = ((1ull << 32) * ((1ull << s) - d)) / d + 1;
  return FastDiv{d, (uint32_t)M, s};
}

// Geometry and coefficients of a level as the kernels see it.
template <typename T>
struct LevelView {
  int N, NT, pitch;
  FastDiv fd;     // division by N + 1
  const T* coef;  // kNumCoef * pitch
  T W;            // W_Diri
  T omega;
  T omc;          // 1 - omega
  T wW;           // omega / W_Diri
  T Wo;           // W_Diri / omega
};

// Precomputed Thomas factors of the interior tridiagonal block (M/dt + K)_int and the
// mass coupling, FP64, arrays of N+2 values indexed by node (entry 0 unused), plus
// D / omega per node to turn the stored b' back into b.
struct ThomasView {
  int N, NT, pitch;
  const double* lo;   // sub-diagonal coefficient (of node i-1)
  const double* inv;  // 1 / pivot
  const double* cp;   // modified super-diagonal (upper / pivot)
  const double* pl;   // time-coupling coefficients PL, PC, PR (negated mass / dt)
  const double* pc;
  const double* pr;
  const double* dw;   // D_i / omega
  double W, omega;
};

// FP64 <-> FP32 conversions by IEEE-754 bit fields on the integer pipe (on this GPU the
// conversion instructions share the slow FP64 pipe), with an exact power-of-two scale:
// to_f32_trunc(d, k) = d 2^k with the mantissa truncated (relative error < 2^-23), signed
// zero below 2^-126 and infinity above the FP32 range; to_f64(f, k) = f 2^k exactly (FP32
// subnormals, which the FP32 kernels flush, become zero).  |k| <= kMaxScaleExp.
constexpr int kMaxScaleExp = 800;
__device__ __forceinline__ float to_f32_trunc(double d, int k = 0) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(d);
  const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
  const unsigned sign = hi & 0x80000000u;
  const int be = (int)((hi >> 20) & 0x7ffu);
  const int e = be - 1023 + 127 + k;
  const unsigned mant = ((hi & 0xfffffu) << 3) | (lo >> 29);
  unsigned r = sign | ((unsigned)e << 23) | mant;
  r = (e <= 0 || be == 0) ? sign : r;
  r = e >= 255 ? (sign | 0x7f800000u) : r;
  return __uint_as_float(r);
}
__device__ __forceinline__ double to_f64(float f, int k = 0) {
  const unsigned b = __float_as_uint(f);
  const unsigned sign = b & 0x80000000u, e = (b >> 23) & 0xffu, m = b & 0x7fffffu;
  const unsigned hi = e == 0 ? sign : (sign | ((unsigned)((int)e + 1023 - 127 + k) << 20) | (m >> 3));
  const unsigned lo = e == 0 ? 0u : (m << 29);
  return __hiloint2double((int)hi, (int)lo);
}

// The power-of-two scale 2^k of the FP32 arithmetic on the finest level (kept in device
// memory so that captured graphs read the current one): the FP32 copies of FP64 residuals
// are scaled by 2^k, FP32 corrections are scaled back by 2^-k, and the FP32 termination
// norms are taken of 2^k r and scaled back by 2^-2k.  k is chosen when ||b|| is summed,
// so that 2^k b has an RMS in [1, 2): magnitudes of b far outside the FP32 range neither
// flush to zero nor overflow.  In range, the result is independent of k (a power-of-two
// scale commutes with every rounding).
__device__ __forceinline__ int scale_exp(const int* kexp) { return kexp ? *kexp : 0; }

// Programmatic dependent launch (sm_90 and later): a kernel launched with launch_pdl may
// start while the previous kernel of its stream drains; it calls pdl_wait() before its first
// access to memory that earlier kernels write, which also lets the next such kernel launch.
// Launched the ordinary way, a kernel's pdl_wait() returns at once.
__device__ __forceinline__ void pdl_wait() {
  asm volatile("griddepcontrol.wait;\n" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
}
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// Sets the message returned by stmg_last_error(NULL) on this host thread.
void set_global_error(const char* msg);

// Process-wide count of kernels launched by the library (stmg_kernel_launches).
void count_launches(unsigned n);
unsigned long long launches_so_far();

constexpr int kNormBlocks = 608;  // 4 x 152 SMs: fixed grid of every reduction

// ---- launchers (stmg_kernels.cu); all return cudaGetLastError() after the launch ----
// One damped-Jacobi sweep uo <- u + omega D^-1 (b - J u) with b' = (omega/D) b stored.
template <typename T>
cudaError_t launch_sweep(const LevelView<T>& lv, bool adj, const T* u, const T* bs, T* uo, cudaStream_t s);
// The same sweep, also writing the partial sums of ||b - J u||^2 (u = the input iterate)
// into partials[kNormBlocks]; then out[0] = the total.  Deterministic.  dw32: the level's
// FP32 D / omega (the norm is accumulated in FP32 per thread).
template <typename T>
cudaError_t launch_sweep_norm(const LevelView<T>& lv, bool adj, const T* u, const T* bs, T* uo, const float* dw32,
                              const int* kexp, double* partials, double* out, cudaStream_t s);
// The scaled residual y = (omega/D)(b - J u) = b' - omega u + sum S u (no unscaling).
template <typename T>
cudaError_t launch_residual_scaled(const LevelView<T>& lv, bool adj, const T* u, const T* bs, T* y, cudaStream_t s);
// b'_c = R r from the scaled residual y with the fine level's kRW* weights (coef: the fine
// level's coefficient table; r0 = W_f / W_c for x-restriction's Dirichlet row).
template <typename T>
cudaError_t launch_restrict_scaled(int type, int Nf, int NTf, int pf, const T* coef, T r0, const T* y,
                                   const LevelView<T>& cv, T* bc, cudaStream_t s);
// Fills the fine level's kRW* slots (FP64 and FP32 tables) for restriction type 1/2/3 toward
// a coarse level with coefficient table cfc (pitch pc, Nc elements).
cudaError_t launch_build_rweights(int type, int Nf, int pf, int Nc, int pc, double Wf, double Wc, double omega,
                                  const double* cfc, double* cf64, float* cf32, cudaStream_t s);
// r = b - J u from the stored b'.
template <typename T>
cudaError_t launch_residual(const LevelView<T>& lv, bool adj, const T* u, const T* bs, T* r, cudaStream_t s);
// y = J u (plain coefficients).
template <typename T>
cudaError_t launch_apply(const LevelView<T>& lv, bool adj, const T* u, T* y, cudaStream_t s);
// b'_c = (omega / D_c) (s P^T r): restriction with the coarse scaling folded in.
template <typename T>
cudaError_t launch_restrict(int type, int Nf, int NTf, int pf, const T* r, const LevelView<T>& cv, T* bc,
                            cudaStream_t s);
template <typename T>
cudaError_t launch_prolong_add(int type, int Nf, int NTf, int pf, T* u, int Nc, int NTc, int pc, const T* z,
                               cudaStream_t s);
// Exact solve of J u = b from the stored b'.
template <typename T>
cudaError_t launch_exact(const ThomasView& tv, bool adj, const T* bs, T* u, cudaStream_t s);
// The same solve for narrow levels as a scan in time with the precomputed powers
// pw[k] = G^(2^k), k < K, of G = -A^-1 B (N x N, row-major); needs 2 NT N doubles of shared
// memory.
template <typename T>
cudaError_t launch_exact_scan(const ThomasView& tv, bool adj, int K, const double* pw, const T* bs, T* u,
                              cudaStream_t s);
// x <- (omega/D) x (to_scaled) or (D/omega) x over a level vector, in place.
template <typename T>
cudaError_t launch_scale(const LevelView<T>& lv, bool to_scaled, T* x, cudaStream_t s);

// ||b - J u||^2 (u == nullptr: ||b||^2) from the stored b' into out[0]; with kset, also the
// scale exponent of the FP32 arithmetic from this norm (see scale_exp).
template <typename T>
cudaError_t launch_resnorm(const LevelView<T>& lv, bool adj, const T* u, const T* bs, double* partials, double* out,
                           cudaStream_t s, int* kset = nullptr);
// Mixed scheme, FP64 level 0: y = (omega/D)(b - J u) stored as FP32 scaled by 2^k (it is the
// scaled right-hand side of the FP32 cycle), with ||b - J u||^2 (of 2^k r accumulated in
// FP32 per thread, scaled back; it only feeds the termination test) into out[0].
// coef32: the level's FP32 coefficients.
cudaError_t launch_defect(const LevelView<double>& lv, const float* coef32, bool adj, const double* u,
                          const double* bs, const int* kexp, float* ys32, double* partials, double* out,
                          cudaStream_t s);
// The same for u = 0: ys32 = b' 2^k (truncated to FP32) over the level's DOFs.
cudaError_t launch_rhs32(const LevelView<double>& lv, const double* bs, const int* kexp, float* ys32,
                         cudaStream_t s);
// u64 += double(e32) 2^-k over the whole padded array (kexp null: k = 0).
cudaError_t launch_add_correction(size_t n, double* u, const float* e, const int* kexp, cudaStream_t s);
// a . b over the padded arrays (padding is zero) into out[0]; deterministic.
cudaError_t launch_dot(size_t n, const double* a, const double* b, double* partials, double* out, cudaStream_t s);
// y[i] = alpha x[i] for i < n (y may equal x).
cudaError_t launch_scaled_copy(size_t n, double alpha, const double* x, double* y, cudaStream_t s);

// Coefficient arrays of a level from per-element k, c (device, FP64).
cudaError_t launch_build_coef(int N, int pitch, double dx, double dt, double W, double omega, const double* k,
                              const double* c, double* coef64, float* coef32, cudaStream_t s);
// SIMP parameters {k_ins, k_con, c_ins, c_con, p_k, p_c}, passed by value to kernels.
struct Simp6 {
  double v[6];
};
cudaError_t launch_simp(int N, const double* chi, Simp6 sp, double* k, double* c, cudaStream_t s);
// b' = mult (omega/D) B b_Neu from element loads q[(NT+1) x N] (dense; nullptr: the
// constant qconst on every element) into the padded layout; with partials (kNormBlocks
// entries), also ||b||^2 into out[0] and, with kset, the FP32 scale exponent from it.
cudaError_t launch_assemble_load(const LevelView<double>& lv, double dx, const double* q, double* bs, cudaStream_t s,
                                 double qconst = 0.0, double mult = 1.0, double* partials = nullptr,
                                 double* out = nullptr, int* kset = nullptr);
// ---- Galerkin reassembly (P-method, Sec. 5.1; stmg_galerkin.cu) ----
// Level operator in row-class form: time row n uses coefficient set cls[n];
// co[(c * 9 + (d + 1) * 3 + (e + 1)) * (N + 1) + i] is the coefficient of u(n + d, i + e) in
// row (n, i).
struct GalOp {
  int N = 0, NT = 0, ncls = 0;
  std::vector<int> cls;
  std::vector<double> co;
};
// Level 0 (the BE-FE operator of Sec. 2.2 with the Dirichlet rows of Appendix A) from its
// per-node J entries.
GalOp galop_level0(int N, int NT, double W, const double* L, const double* D, const double* U, const double* PL,
                   const double* PC, const double* PR);
// out = R f P for a transfer of type 1 (x), 2 (causal t) or 3 (bilinear t); false if the
// product would reach beyond three time rows.
bool galop_coarsen(const GalOp& f, int type, GalOp& out);
// Block-tridiagonal LU in time of J (adj: J^T): per row m, G_m = S_m^-1 and H_m = S_m^-1 U_m
// ((N+1)^2 each, row-major) and L_m as 3 x (N+1); false if a pivot vanishes.
bool galop_block_lu(const GalOp& op, bool adj, std::vector<double>& G, std::vector<double>& H,
                    std::vector<double>& Lsub);
// Device view of a row-class level: cls (NT+1), co (ncls * 9 * (N+1)), wd = omega / diagonal
// (ncls * (N+1)).
struct GalView {
  int N, NT, pitch;
  FastDiv fd;
  const int* cls;
  const double* co;
  const double* wd;
};
cudaError_t launch_gal_apply(const GalView& g, bool adj, const double* u, double* y, cudaStream_t s);
cudaError_t launch_gal_sweep(const GalView& g, bool adj, const double* u, const double* b, double* out,
                             cudaStream_t s);
cudaError_t launch_gal_residual(const GalView& g, bool adj, const double* u, const double* b, double* r,
                                cudaStream_t s);
cudaError_t launch_gal_exact(int n, int M, int pitch, const double* G, const double* H, const double* Lsub,
                             const double* b, double* u, cudaStream_t s);

// Projected-gradient design update of the optimisation loop (one block; out may alias chi).
cudaError_t launch_design_update(int N, const double* chi, const double* g, double vol, double move, double* out,
                                 cudaStream_t s);
// Sensitivity: partial sums over time chunks, then the per-element reduction.
constexpr int kSensRowsPerChunk = 256;
// scratch: 2 * sens_chunks(NT) * N doubles.
cudaError_t launch_sensitivity(int N, int NT, int pitch, double dx, double dt, const double* chi, Simp6 sp,
                               const double* u, const double* lam, double* scratch, double* g, cudaStream_t s);
// Per-element reduction of scratch[2 * chunks * N] partial sums into the gradient.
cudaError_t launch_sens_final(int N, int chunks, const double* chi, Simp6 sp, const double* scratch, double* g,
                              cudaStream_t s);
// Largest gridDim.y (and z) of a launch.
constexpr int kMaxGridY = 65535;
// Time levels 0..NT in chunks of kSensRowsPerChunk rows (the chunks are gridDim.y of the
// partial-sum launch).
inline int sens_chunks(int NT) { return (NT + kSensRowsPerChunk) / kSensRowsPerChunk; }

}  // namespace stmg

// Library-internal entry for the request server (stmg_host.cu): solves on the handle's
// finest level with the load assembled on the device from q_dev (element loads in device
// memory) or, when q_dev is null, the uniform load q_value; the right-hand side is
// multiplied by rhs_scale (dt for the compliance adjoint).  theta = b^T x dt of the result
// x with b the unscaled load vector; out (host or device, optional) receives x.
stmg_status stmg_solve_resident(stmg_t h, bool adjoint, const double* q_dev, double q_value, double rhs_scale,
                                double* out, int* cycles, double* relres, double* theta);
