// stmg_internal.h -- shared declarations between the host driver and the CUDA kernels.
//
// Device layout of one level with N elements and NT steps: a space-time vector is
// (NT+1) rows of `pitch` values; columns 0..N hold the nodes, columns N+1..pitch-1 are
// zero padding that no kernel ever writes (pitch >= N+2, so the right neighbour of node
// N is always a zero padding value).  The stencil coefficients of a level are 8 arrays of
// `pitch` values each (struct of arrays, see CoefSlot), built once per level:
//
//   (J u)[n][i] = L_i u[n][i-1] + D_i u[n][i] + U_i u[n][i+1]
//               + PL_i u[p][i-1] + PC_i u[p][i] + PR_i u[p][i+1]
//
// for the non-Dirichlet DOFs (n >= 1, i >= 1), where p = n-1 for J (present for n >= 2)
// and p = n+1 for J^T (present for n <= NT-1); the mass and stiffness blocks are
// symmetric, so J and J^T share the coefficients (Sec. 2.2, Sec. 7.2).  Dirichlet DOFs
// (row 0 and column 0) have (J u) = W_Diri u (Appendix A).  L_1 = PL_1 = 0 and
// U_N = PR_N = 0 remove the Dirichlet column and the missing element past x = L.
#pragma once
#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

namespace stmg {

enum CoefSlot { kL = 0, kD = 1, kU = 2, kPL = 3, kPC = 4, kPR = 5, kInvD = 6, kNumCoef = 8 };

inline int level_pitch(int N) {
  int need = N + 2;
  int align = need > 64 ? 32 : 4;
  return (need + align - 1) / align * align;
}

// Geometry of a level as the kernels see it.
template <typename T>
struct LevelView {
  int N, NT, pitch;
  const T* coef;  // kNumCoef * pitch
  T W;            // W_Diri
  T wW;           // omega / W_Diri
};

// Precomputed Thomas factors of the interior tridiagonal block (M/dt + K)_int and the
// mass coupling, FP64, arrays of N+1 values indexed by node (entry 0 unused).
struct ThomasView {
  int N, NT, pitch;
  const double* lo;   // sub-diagonal coefficient (of node i-1)
  const double* inv;  // 1 / pivot
  const double* cp;   // modified super-diagonal (upper / pivot)
  const double* pl;   // time-coupling coefficients PL, PC, PR (negated mass / dt)
  const double* pc;
  const double* pr;
  double W;
};

// Sets the message returned by stmg_last_error(NULL) on this host thread.
void set_global_error(const char* msg);

// Process-wide count of kernels launched by the library (stmg_kernel_launches).
void count_launches(unsigned n);
unsigned long long launches_so_far();

// ---- launchers (stmg_kernels.cu); all return cudaGetLastError() after the launch ----
template <typename T>
cudaError_t launch_jacobi(const LevelView<T>& lv, bool adj, const T* u, const T* b, T* uo, cudaStream_t s);
template <typename T>
cudaError_t launch_residual(const LevelView<T>& lv, bool adj, const T* u, const T* b, T* r, cudaStream_t s);
// y = J u
template <typename T>
cudaError_t launch_apply(const LevelView<T>& lv, bool adj, const T* u, T* y, cudaStream_t s);
template <typename T>
cudaError_t launch_restrict(int type, int Nf, int NTf, int pf, const T* r, int Nc, int NTc, int pc, T* bc,
                            cudaStream_t s);
template <typename T>
cudaError_t launch_prolong_add(int type, int Nf, int NTf, int pf, T* u, int Nc, int NTc, int pc, const T* z,
                               cudaStream_t s);
template <typename T>
cudaError_t launch_exact(const ThomasView& tv, bool adj, const T* b, T* u, cudaStream_t s);

// Sum of squares of (b - J u) over all DOFs (u == nullptr: of b) into partials[kNormBlocks];
// then a single-block pass writes the total to out[0].  Deterministic (fixed order).
constexpr int kNormBlocks = 608;  // 4 x 152 SMs
template <typename T, typename R>
cudaError_t launch_resnorm(const LevelView<T>& lv, bool adj, const T* u, const T* b, R* r_out, double* partials,
                           double* out, cudaStream_t s);
// FP64 residual for the mixed scheme: r32 = float(b - J u), with its squared norm.
cudaError_t launch_defect(const LevelView<double>& lv, bool adj, const double* u, const double* b, float* r32,
                          double* partials, double* out, cudaStream_t s);
// u64 += double(e32) over the whole padded array.
cudaError_t launch_add_correction(size_t n, double* u, const float* e, cudaStream_t s);
// a . b over the padded arrays (padding is zero) into out[0]; deterministic.
cudaError_t launch_dot(size_t n, const double* a, const double* b, double* partials, double* out, cudaStream_t s);

// Coefficient arrays of a level from per-element k, c (device, FP64).
cudaError_t launch_build_coef(int N, int pitch, double dx, double dt, double W, double omega, const double* k,
                              const double* c, double* coef64, float* coef32, cudaStream_t s);
// SIMP parameters {k_ins, k_con, c_ins, c_con, p_k, p_c}, passed by value to kernels.
struct Simp6 {
  double v[6];
};
cudaError_t launch_simp(int N, const double* chi, Simp6 sp, double* k, double* c, cudaStream_t s);
// Nodal load from element loads q[(NT+1) x N] (dense) into b (padded layout).
cudaError_t launch_assemble_load(int N, int NT, int pitch, double dx, const double* q, double* b, cudaStream_t s);
// Sensitivity: partial sums over time chunks, then the per-element reduction.
constexpr int kSensRowsPerChunk = 256;
// scratch: 2 * sens_chunks(NT) * N doubles.
cudaError_t launch_sensitivity(int N, int NT, int pitch, double dx, double dt, const double* chi, Simp6 sp,
                               const double* u, const double* lam, double* scratch, double* g, cudaStream_t s);
// Time levels 0..NT in chunks of kSensRowsPerChunk rows.
inline int sens_chunks(int NT) { return (NT + kSensRowsPerChunk) / kSensRowsPerChunk; }

}  // namespace stmg
