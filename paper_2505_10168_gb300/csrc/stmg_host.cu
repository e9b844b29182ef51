// stmg_host.cu -- host side of the STMG library: the C ABI of include/stmg.h, the
// coarsening planner (Alg. 3/4), the level hierarchy in device memory, and the
// V-cycle / solver loops that enqueue the kernels of stmg_kernels.cu on the handle's
// stream.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <unordered_map>
#include <string>
#include <utility>
#include <vector>

#include "stmg.h"
#include "stmg_internal.h"
#include "stmg_placement.h"
#include "stmg_slab.h"
#include "stmg_stream.h"

using namespace stmg;

namespace {

thread_local std::string g_global_error;

// Samples of chi in [0, 1] (both ends included: kDeffSamples + 1 points) over which the
// design-independent D_eff of Sec. 7.2 takes the extrema of D_SIMP = k_SIMP / c_SIMP.
constexpr int kDeffSamples = 10000;

// One level of the hierarchy.
struct Level {
  int N = 0, NT = 0, pitch = 0, next = STMG_COARSEST;
  double dx = 0, dt = 0, W = 0, lam = 0;
  std::vector<double> k, c;  // host copies of the level material
  std::vector<double> chi;   // design field of the level (D-reassembly only)
  size_t nvec = 0;           // (NT+1) * pitch
  // device
  double* dk = nullptr;      // k, c (N values each)
  double* dc = nullptr;
  double* cf64 = nullptr;    // kNumCoef * pitch
  float* cf32 = nullptr;
  double* th = nullptr;      // Thomas factors: 8 arrays of N+2 doubles
  double *u = nullptr, *b = nullptr, *t = nullptr;    // FP64 vectors
  float *u32 = nullptr, *b32 = nullptr, *t32 = nullptr;  // FP32 vectors (mixed precision)
  // P-reassembly (levels >= 1): J as a Galerkin product in row-class form, right-hand side
  // stored unscaled; on the coarsest level the block LU of J and of J^T
  bool gal = false;
  GalOp gop;
  int* dcls = nullptr;
  double* dgco = nullptr;
  double* dgwd = nullptr;
  double* dglu[2] = {nullptr, nullptr};
  // narrow coarsest level: powers G^(2^k), k < npw, of G = -A^-1 B for the scan in time
  double* dpw = nullptr;
  int npw = 0;
};

}  // namespace

struct stmg_handle {
  stmg_opts o{};
  cudaStream_t s = nullptr;
  int N = 0, NT = 0;
  double L = 0, tT = 0;
  std::vector<Level> lev;
  double* partials = nullptr;  // kNormBlocks
  double* scal = nullptr;      // device scalars
  double hscal[8] = {0};       // host copies of device scalars
  // device memory: cudaMalloc/cudaFree unless the creator supplied hooks
  stmg_alloc_fn alloc_fn = nullptr;
  stmg_free_fn free_fn = nullptr;
  void* actx = nullptr;
  std::unordered_map<void*, size_t> sizes;  // live allocations (bytes, for stmg_device_bytes)
  std::vector<double> chi;                  // design field (D-reassembly)
  double simp[6] = {0, 0, 0, 0, 0, 0};
  long long bytes = 0;
  double* qstage = nullptr;    // device staging for host element loads
  size_t qstage_n = 0;
  double* sens = nullptr;      // sensitivity scratch
  size_t sens_n = 0;
  double* gstage = nullptr;    // element-array staging (chi, gradient)
  // CUDA graphs of one solver iteration, per [precision][adjoint]; captured on cs.
  cudaStream_t cs = nullptr;
  cudaGraphExec_t gexec[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
  unsigned gkernels[2][2] = {{0, 0}, {0, 0}};  // kernels per graph (launch statistics)
  double* graph_u0 = nullptr;  // level-0 u buffer that the FP64 graphs expect to hold u
  std::string err;
};

namespace {

stmg_status fail(stmg_t h, stmg_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (h) h->err = buf;
  else g_global_error = buf;
  return st;
}

#define CK(call)                                                                                 \
  do {                                                                                           \
    cudaError_t e_ = (call);                                                                     \
    if (e_ != cudaSuccess) {                                                                     \
      return fail(h, e_ == cudaErrorMemoryAllocation ? STMG_ENOMEM : STMG_ECUDA, "%s: %s (%s:%d)", #call, \
                  cudaGetErrorString(e_), __FILE__, __LINE__);                                   \
    }                                                                                            \
  } while (0)

#define CKS_NULL(expr)                    \
  do {                                    \
    stmg_status st_ = (expr);             \
    if (st_ != STMG_OK) return st_;       \
  } while (0)

#define CKS(expr)                         \
  do {                                    \
    stmg_status st_ = (expr);             \
    if (st_ != STMG_OK) return st_;       \
  } while (0)

// Allocation sizes are rounded up to 256 bytes (the alignment every hook must provide).
inline size_t round256(size_t b) { return (b + 255) / 256 * 256; }

template <typename T>
stmg_status dalloc(stmg_t h, T** p, size_t n) {
  *p = nullptr;
  if (n == 0) n = 1;
  const size_t bytes = round256(n * sizeof(T));
  void* q = nullptr;
  if (h->alloc_fn) {
    q = h->alloc_fn(bytes, h->actx);
    if (!q) return fail(h, STMG_ENOMEM, "allocator hook returned no memory for %zu bytes", bytes);
  } else {
    cudaError_t e = cudaMalloc(&q, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(h, STMG_ENOMEM, "cudaMalloc of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
    }
  }
  h->sizes[q] = bytes;
  h->bytes += (long long)bytes;
  *p = static_cast<T*>(q);
  return STMG_OK;
}

template <typename T>
void dfree(stmg_t h, T*& p) {
  if (p) {
    auto it = h->sizes.find((void*)p);
    if (it != h->sizes.end()) {
      h->bytes -= (long long)it->second;
      h->sizes.erase(it);
    }
    if (h->free_fn) h->free_fn((void*)p, h->actx);
    else cudaFree(p);
  }
  p = nullptr;
}

void free_level(stmg_t h, Level& L) {
  dfree(h, L.dk); dfree(h, L.dc); dfree(h, L.cf64); dfree(h, L.cf32); dfree(h, L.th);
  dfree(h, L.u); dfree(h, L.b); dfree(h, L.t); dfree(h, L.u32); dfree(h, L.b32); dfree(h, L.t32);
  dfree(h, L.dcls); dfree(h, L.dgco); dfree(h, L.dgwd); dfree(h, L.dglu[0]); dfree(h, L.dglu[1]);
  dfree(h, L.dpw);
  L.npw = 0;
}

bool finite_pos(double v) { return std::isfinite(v) && v > 0.0; }

// --------------------------------------------------------------------------------------
// Planner: Alg. 3 (Alg. 4 with min_nel).  lambda_eff = D_eff dt / dx^2 with
// D_eff = sqrt(min_e k_e/c_e * max_e k_e/c_e) or the fixed design-independent D_eff of
// Sec. 7.2.  x-coarsening averages resistivity (R) or conductivity (K) and heat capacity
// over element pairs; t-coarsening keeps the material and doubles dt.
// --------------------------------------------------------------------------------------
double level_lambda(const stmg_opts& o, const Level& L) {
  double deff = o.deff_fixed;
  if (!(deff > 0.0)) {
    double lo = L.k[0] / L.c[0], hi = lo;
    for (int e = 1; e < L.N; ++e) {
      const double d = L.k[e] / L.c[e];
      lo = std::min(lo, d);
      hi = std::max(hi, d);
    }
    deff = std::sqrt(lo * hi);
  }
  return deff * L.dt / (L.dx * L.dx);
}

double level_wdiri(const Level& L) {
  const double cmax = *std::max_element(L.c.begin(), L.c.end());
  const double kmax = *std::max_element(L.k.begin(), L.k.end());
  return cmax * L.dx / L.dt + kmax / L.dx;
}

// SIMP interpolation (Sec. 2.1) on the host, for the D-reassembly of coarse levels.
double simp_k(const double* s, double chi) { return s[0] + (s[1] - s[0]) * std::pow(chi, s[4]); }
double simp_c(const double* s, double chi) { return s[2] + (s[3] - s[2]) * std::pow(chi, s[5]); }

std::vector<Level> plan_levels(const stmg_opts& o, int N, int NT, double Ldom, double tT, const double* k,
                               const double* c, const double* chi = nullptr, const double* simp = nullptr) {
  std::vector<Level> out;
  Level f;
  f.N = N; f.NT = NT; f.dx = Ldom / N; f.dt = tT / NT;
  f.k.assign(k, k + N);
  f.c.assign(c, c + N);
  const bool design = o.reassembly == STMG_REASM_D && chi && simp;
  if (design) f.chi.assign(chi, chi + N);
  out.push_back(std::move(f));
  const int cap = o.num_levels > 0 ? o.num_levels : std::max(1, o.max_levels);
  while (true) {
    Level& L = out.back();
    L.W = level_wdiri(L);
    L.lam = level_lambda(o, L);
    L.next = STMG_COARSEST;
    if ((int)out.size() >= cap) break;
    const long long dofs = (long long)(L.NT + 1) * (L.N + 1);
    if (o.num_levels <= 0 && dofs <= o.max_coarse_dofs) break;
    const bool can_x = L.N % 2 == 0 && L.N >= 2;
    const bool can_t = L.NT % 2 == 0 && L.NT >= 2;
    const bool want_t = L.lam < o.lambda_crit || (o.min_nel > 0 && L.N / 2 < o.min_nel);
    int type;
    if (want_t) type = can_t ? STMG_TCOARSEN : (can_x ? STMG_XCOARSEN : STMG_COARSEST);
    else type = can_x ? STMG_XCOARSEN : (can_t ? STMG_TCOARSEN : STMG_COARSEST);
    if (type == STMG_COARSEST) break;
    L.next = type;
    Level C;
    if (type == STMG_XCOARSEN) {
      C.N = L.N / 2; C.NT = L.NT; C.dx = 2.0 * L.dx; C.dt = L.dt;
      C.k.resize(C.N);
      C.c.resize(C.N);
      if (design) C.chi.resize(C.N);
      for (int e = 0; e < C.N; ++e) {
        const double ka = L.k[2 * e], kb = L.k[2 * e + 1];
        if (design) {  // Sec. 5.1 "D": average the design field, then the SIMP model
          C.chi[e] = (L.chi[2 * e] + L.chi[2 * e + 1]) / 2.0;
          C.k[e] = simp_k(simp, C.chi[e]);
          C.c[e] = simp_c(simp, C.chi[e]);
          continue;
        }
        if (o.reassembly == STMG_REASM_R) {
          const double rho = (1.0 / ka + 1.0 / kb) / 2.0;  // mean thermal resistivity
          C.k[e] = 1.0 / rho;
        } else {
          C.k[e] = (ka + kb) / 2.0;
        }
        C.c[e] = (L.c[2 * e] + L.c[2 * e + 1]) / 2.0;
      }
    } else {
      C.N = L.N; C.NT = L.NT / 2; C.dx = L.dx; C.dt = 2.0 * L.dt;
      C.k = L.k;
      C.c = L.c;
      C.chi = L.chi;
    }
    out.push_back(std::move(C));
  }
  for (Level& L : out) {
    L.pitch = level_pitch(L.N);
    L.nvec = (size_t)(L.NT + 1) * L.pitch;
  }
  return out;
}

// Thomas factors of (M/dt + K) restricted to nodes 1..N, from the host material.
void thomas_factors(const Level& L, std::vector<double>& out) {
  const int N = L.N;
  const size_t S = N + 2;
  out.assign(8 * S, 0.0);
  double* lo = &out[0];
  double* inv = &out[S];
  double* cp = &out[2 * S];
  double* pl = &out[3 * S];
  double* pc = &out[4 * S];
  double* pr = &out[5 * S];
  std::vector<double> up(S, 0.0), di(S, 0.0);
  for (int i = 1; i <= N; ++i) {
    const double ml = L.c[i - 1] * L.dx / (6.0 * L.dt), sl = L.k[i - 1] / L.dx;
    const double mr = i < N ? L.c[i] * L.dx / (6.0 * L.dt) : 0.0, sr = i < N ? L.k[i] / L.dx : 0.0;
    lo[i] = i >= 2 ? ml - sl : 0.0;
    up[i] = i < N ? mr - sr : 0.0;
    di[i] = 2.0 * ml + sl + 2.0 * mr + sr;
    pl[i] = i >= 2 ? -ml : 0.0;
    pc[i] = -2.0 * (ml + mr);
    pr[i] = i < N ? -mr : 0.0;
  }
  double cprev = 0.0;
  double* alpha = &out[6 * S];
  double* beta = &out[7 * S];
  for (int i = 1; i <= N; ++i) {
    const double den = di[i] - lo[i] * cprev;
    inv[i] = 1.0 / den;
    cp[i] = up[i] * inv[i];
    cprev = cp[i];
    alpha[i] = -lo[i] * inv[i];
    beta[i] = -cp[i];
  }
}

// Device set-up of one level (material, coefficients, Thomas factors); vectors are
// allocated by alloc_vectors.
stmg_status setup_level(stmg_t h, Level& L) {
  if (!L.dk) CKS(dalloc(h, &L.dk, L.N));
  if (!L.dc) CKS(dalloc(h, &L.dc, L.N));
  if (!L.cf64) CKS(dalloc(h, &L.cf64, (size_t)kNumCoef * L.pitch));
  if (!L.cf32) CKS(dalloc(h, &L.cf32, (size_t)kNumCoef * L.pitch));
  if (!L.th) CKS(dalloc(h, &L.th, 8 * (size_t)(L.N + 2)));
  CK(cudaMemcpyAsync(L.dk, L.k.data(), L.N * sizeof(double), cudaMemcpyHostToDevice, h->s));
  CK(cudaMemcpyAsync(L.dc, L.c.data(), L.N * sizeof(double), cudaMemcpyHostToDevice, h->s));
  CK(launch_build_coef(L.N, L.pitch, L.dx, L.dt, L.W, h->o.omega, L.dk, L.dc, L.cf64, L.cf32, h->s));
  std::vector<double> th;
  thomas_factors(L, th);
  CK(cudaMemcpyAsync(L.th, th.data(), th.size() * sizeof(double), cudaMemcpyHostToDevice, h->s));
  // the host vector must outlive the async copy
  CK(cudaStreamSynchronize(h->s));
  return STMG_OK;
}

template <typename T>
stmg_status zero_alloc(stmg_t h, T** p, size_t n) {
  CKS(dalloc(h, p, n));
  CK(cudaMemsetAsync(*p, 0, n * sizeof(T), h->s));
  return STMG_OK;
}

stmg_status ensure_fp64(stmg_t h, Level& L) {
  if (!L.u) CKS(zero_alloc(h, &L.u, L.nvec));
  if (!L.b) CKS(zero_alloc(h, &L.b, L.nvec));
  if (!L.t) CKS(zero_alloc(h, &L.t, L.nvec));
  return STMG_OK;
}

stmg_status ensure_fp32(stmg_t h, Level& L) {
  if (!L.u32) CKS(zero_alloc(h, &L.u32, L.nvec));
  if (!L.b32) CKS(zero_alloc(h, &L.b32, L.nvec));
  if (!L.t32) CKS(zero_alloc(h, &L.t32, L.nvec));
  return STMG_OK;
}

stmg_status alloc_vectors(stmg_t h) {
  for (size_t l = 0; l < h->lev.size(); ++l) {
    Level& L = h->lev[l];
    if (l == 0 || h->o.precision == STMG_FP64) CKS(ensure_fp64(h, L));
    if (h->o.precision == STMG_MIXED) CKS(ensure_fp32(h, L));
  }
  return STMG_OK;
}

template <typename T>
LevelView<T> view(const Level& L, double omega);
template <>
LevelView<double> view<double>(const Level& L, double omega) {
  // Galerkin levels store b unscaled: their scalings are the identity (the coefficient
  // slots kW and kDW hold 1 as well)
  return LevelView<double>{L.N, L.NT, L.pitch, make_fastdiv(L.N + 1), L.cf64, L.W, omega, 1.0 - omega,
                           L.gal ? 1.0 : omega / L.W, L.gal ? 1.0 : L.W / omega};
}

GalView gal_view(const Level& L) {
  return GalView{L.N, L.NT, L.pitch, make_fastdiv(L.N + 1), L.dcls, L.dgco, L.dgwd};
}

// Galerkin-level operations exist in FP64 only (the P-reassembly is an FP64 option).
template <typename T>
cudaError_t gal_sweep(const Level&, bool, const T*, const T*, T*, cudaStream_t) {
  return cudaErrorNotSupported;
}
template <>
cudaError_t gal_sweep<double>(const Level& L, bool adj, const double* u, const double* b, double* out,
                              cudaStream_t s) {
  return launch_gal_sweep(gal_view(L), adj, u, b, out, s);
}
template <typename T>
cudaError_t gal_residual(const Level&, bool, const T*, const T*, T*, cudaStream_t) {
  return cudaErrorNotSupported;
}
template <>
cudaError_t gal_residual<double>(const Level& L, bool adj, const double* u, const double* b, double* r,
                                 cudaStream_t s) {
  return launch_gal_residual(gal_view(L), adj, u, b, r, s);
}
template <typename T>
cudaError_t gal_exact(const Level&, bool, const T*, T*, cudaStream_t) {
  return cudaErrorNotSupported;
}
template <>
cudaError_t gal_exact<double>(const Level& L, bool adj, const double* b, double* u, cudaStream_t s) {
  const int n = L.N + 1, M = L.NT + 1;
  const double* G = L.dglu[adj ? 1 : 0];
  if (!G) return cudaErrorInvalidValue;
  const size_t nn = (size_t)M * n * n;
  return launch_gal_exact(n, M, L.pitch, G, G + nn, G + 2 * nn, b, u, s);
}
template <>
LevelView<float> view<float>(const Level& L, double omega) {
  return LevelView<float>{L.N,          L.NT,           L.pitch,
                          make_fastdiv(L.N + 1), L.cf32, (float)L.W,
                          (float)omega, (float)(1.0 - omega), (float)(omega / L.W),
                          (float)(L.W / omega)};
}

ThomasView thomas_view(const Level& L, double omega) {
  const size_t S = L.N + 2;
  return ThomasView{L.N,         L.NT,        L.pitch,     L.th, L.th + S, L.th + 2 * S, L.th + 3 * S,
                    L.th + 4 * S, L.th + 5 * S, L.cf64 + (size_t)kDW * L.pitch, L.W, omega};
}

SlabView slab_view(const Level& L, double omega, int K) {
  const size_t S = L.N + 2;
  return SlabView{L.N,          L.NT,         L.pitch,      K,           L.dx,        L.dt,
                  omega,        L.cf64 + (size_t)kDW * L.pitch, L.th + 3 * S, L.th + 4 * S, L.th + 5 * S,
                  L.th + S,     L.th + 6 * S, L.th + 7 * S};
}

// Level vectors for precision T.
template <typename T>
struct Vecs {
  T *u, *b, *t;
};
template <typename T>
Vecs<T> vecs(Level& L);
template <>
Vecs<double> vecs<double>(Level& L) { return {L.u, L.b, L.t}; }
template <>
Vecs<float> vecs<float>(Level& L) { return {L.u32, L.b32, L.t32}; }
template <typename T>
const T* coef(const Level& L);
template <>
const double* coef<double>(const Level& L) { return L.cf64; }
template <>
const float* coef<float>(const Level& L) { return L.cf32; }
template <typename T>
void set_u(Level& L, T* u);
template <>
void set_u<double>(Level& L, double* u) { L.u = u; }
template <>
void set_u<float>(Level& L, float* u) { L.u32 = u; }
template <typename T>
void set_t(Level& L, T* t);
template <>
void set_t<double>(Level& L, double* t) { L.t = t; }
template <>
void set_t<float>(Level& L, float* t) { L.t32 = t; }

// Transfer kernel type of the coarsening below level L: 1 x, 2 causal t, 3 bilinear t.
inline int transfer_type(const stmg_opts& o, const Level& L) {
  return L.next == STMG_TCOARSEN && o.interp == STMG_INTERP_BILINEAR ? 3 : L.next;
}

// Exact solve on one level: the block LU of a Galerkin level; a scan over the time rows for
// a narrow, short coarsest level; one warp per step (the Thomas recurrences as warp scans)
// for other narrow levels; block-wide scans per step for wider ones.
template <typename T>
cudaError_t exact_level(stmg_t h, const Level& L, bool adj, const T* bs, T* u) {
  if (L.gal) return gal_exact<T>(L, adj, bs, u, h->s);
  if (L.dpw) return launch_exact_scan<T>(thomas_view(L, h->o.omega), adj, L.npw, L.dpw, bs, u, h->s);
  if (L.N > 64) return launch_exact_par<T>(slab_view(L, h->o.omega, L.NT), adj, bs, u, h->s);
  return launch_exact<T>(thomas_view(L, h->o.omega), adj, bs, u, h->s);
}

// nsweeps Jacobi steps on level L ping-ponging u and t (the level's u pointer follows
// the current iterate).
template <typename T>
stmg_status smooth_level(stmg_t h, Level& L, bool adj, int nsweeps) {
  const LevelView<T> lv = view<T>(L, h->o.omega);
  for (int s = 0; s < nsweeps; ++s) {
    Vecs<T> v = vecs<T>(L);
    if (L.gal) CK(gal_sweep<T>(L, adj, v.u, v.b, v.t, h->s));
    else CK(launch_sweep<T>(lv, adj, v.u, v.b, v.t, h->s));
    set_u<T>(L, v.t);
    set_t<T>(L, v.u);
  }
  return STMG_OK;
}

// Alg. 1, VCycle(l, u, b), in precision T on the level's own u and (scaled) b.
// zero_init: u starts at 0, so the first pre-smoothing step is exactly u = b' (a copy).
// first_done: the caller already ran the first pre-smoothing step.
template <typename T>
stmg_status vcycle(stmg_t h, int l, bool adj, bool zero_init, bool first_done) {
  Level& L = h->lev[l];
  if (l == (int)h->lev.size() - 1) {
    Vecs<T> v = vecs<T>(L);
    CK(exact_level<T>(h, L, adj, v.b, v.u));
    return STMG_OK;
  }
  Level& C = h->lev[l + 1];
  int pre = h->o.nu;
  if (zero_init && !first_done) {
    Vecs<T> v = vecs<T>(L);
    if (pre >= 2 && !L.gal) {
      // the first sweep from 0 is exactly b'; the second reads b' in its place
      CK(launch_sweep<T>(view<T>(L, h->o.omega), adj, v.b, v.b, v.u, h->s));
      pre -= 2;
    } else if (pre > 0 && !L.gal) {  // (a Galerkin level keeps b unscaled: it sweeps from 0 instead)
      CK(cudaMemcpyAsync(v.u, v.b, L.nvec * sizeof(T), cudaMemcpyDeviceToDevice, h->s));
      --pre;
    } else {
      CK(cudaMemsetAsync(v.u, 0, L.nvec * sizeof(T), h->s));
    }
  } else if (first_done) {
    --pre;
  }
  CKS(smooth_level<T>(h, L, adj, pre));
  {
    Vecs<T> v = vecs<T>(L);
    Vecs<T> vc = vecs<T>(C);
    if (!L.gal && !C.gal) {
      // scaled residual, restricted with the folded scalings (kRW* slots)
      CK(launch_residual_scaled<T>(view<T>(L, h->o.omega), adj, v.u, v.b, v.t, h->s));
      CK(launch_restrict_scaled<T>(transfer_type(h->o, L), L.N, L.NT, L.pitch, coef<T>(L), (T)(L.W / C.W), v.t,
                                   view<T>(C, h->o.omega), vc.b, h->s));
    } else {
      if (L.gal) CK(gal_residual<T>(L, adj, v.u, v.b, v.t, h->s));
      else CK(launch_residual<T>(view<T>(L, h->o.omega), adj, v.u, v.b, v.t, h->s));
      CK(launch_restrict<T>(transfer_type(h->o, L), L.N, L.NT, L.pitch, v.t, view<T>(C, h->o.omega), vc.b, h->s));
    }
  }
  CKS(vcycle<T>(h, l + 1, adj, true, false));
  {
    Vecs<T> v = vecs<T>(L);
    Vecs<T> vc = vecs<T>(C);
    CK(launch_prolong_add<T>(transfer_type(h->o, L), L.N, L.NT, L.pitch, v.u, C.N, C.NT, C.pitch, vc.u, h->s));
  }
  CKS(smooth_level<T>(h, L, adj, h->o.nu));
  return STMG_OK;
}

// Split n sweeps into the fewest passes of at most `most` fused sweeps, of near-equal size.
std::vector<int> split_sweeps(int n, int most) {
  std::vector<int> p;
  const int k = (n + most - 1) / most;
  for (int i = 0; i < k; ++i) p.push_back(n / k + (i < n % k ? 1 : 0));
  return p;
}

// Passes of a level's DOWN half: plain passes of at most 8 sweeps, then the pass that adds
// the residual and the restriction, with at most 5 (a DOWN pass's window halo covers the
// 5 sweeps, the residual and the restriction).  Every pass reads and writes the level's
// vectors once, so fewer, deeper passes move fewer bytes (nu = 60: 8 passes instead of 12).
std::vector<int> down_passes(int nu) {
  if (nu <= 5) return {nu};
  const int last = 5;
  std::vector<int> p = split_sweeps(nu - last, 8);
  p.push_back(last);
  return p;
}

// Passes of a level's UP half: the prolongation and at most 8 sweeps, then plain passes of
// at most 8.
std::vector<int> up_passes(int nu) { return split_sweeps(nu, 8); }

int* kexp(stmg_t h);

StreamArgs stream_args(const Level& L, double omega) {
  StreamArgs a{};
  a.N = L.N;
  a.NT = L.NT;
  a.pitch = L.pitch;
  a.omega = (float)omega;
  a.omc = (float)(1.0 - omega);
  a.Wo = (float)(L.W / omega);
  a.coef = L.cf32;
  return a;
}

// The DOWN half of level l < last in FP32 fused passes: the nu pre-smoothing sweeps (from
// zero, or on the finest level from the current FP32 iterate when an inner iteration
// continues), the residual and the restriction into level l+1's b' (one pass, or several
// when nu > 5).  Returns the buffer holding the level's smoothed iterate in *cur.
stmg_status down32(stmg_t h, int l, bool adj, bool zero_start, float** cur) {
  Level& L = h->lev[l];
  Level& C = h->lev[l + 1];
  const std::vector<int> passes = down_passes(h->o.nu);
  const bool xc = L.next == STMG_XCOARSEN;
  float* in = zero_start ? nullptr : L.u32;
  float* out = zero_start ? L.u32 : L.t32;
  for (size_t p = 0; p < passes.size(); ++p) {
    StreamArgs a = stream_args(L, h->o.omega);
    a.u_in = in;
    a.zero_init = p == 0 && zero_start;
    a.bs = L.b32;
    a.u_out = out;
    int mode = kStreamPlain;
    if (p + 1 == passes.size()) {
      mode = xc ? kStreamDownX : (h->o.interp == STMG_INTERP_BILINEAR ? kStreamDownTB : kStreamDownT);
      a.pc = C.pitch;
      a.ccoef = C.cf32;
      a.cwW = (float)(h->o.omega / C.W);
      a.bc = C.b32;
    }
    CK(launch_stream(mode, adj, passes[p], a, h->s));
    in = out;
    out = (out == L.u32) ? L.t32 : L.u32;
  }
  *cur = in;
  return STMG_OK;
}

// The UP half of level l < last: prolongation of level l+1's correction added to the
// iterate in `in`, then the nu post-smoothing sweeps; the result is added to the FP64
// iterate u64 (scaled back by 2^-k) when u64 is set, else stored in a level buffer.  The
// level's FP32 u pointer ends on the level's result.
stmg_status up32(stmg_t h, int l, bool adj, float* in, double* u64) {
  Level& L = h->lev[l];
  Level& C = h->lev[l + 1];
  const std::vector<int> passes = up_passes(h->o.nu);
  const bool xc = L.next == STMG_XCOARSEN;
  float* out = (in == L.u32) ? L.t32 : L.u32;
  for (size_t p = 0; p < passes.size(); ++p) {
    StreamArgs a = stream_args(L, h->o.omega);
    a.u_in = in;
    a.zero_init = 0;
    a.bs = L.b32;
    const bool last = p + 1 == passes.size();
    a.u_out = (last && u64) ? nullptr : out;
    a.u64 = (last && u64) ? u64 : nullptr;
    a.kexp = kexp(h);
    int mode = kStreamPlain;
    if (p == 0) {
      mode = xc ? kStreamUpX : (h->o.interp == STMG_INTERP_BILINEAR ? kStreamUpTB : kStreamUpT);
      a.pc = C.pitch;
      a.z = C.u32;
    }
    CK(launch_stream(mode, adj, passes[p], a, h->s));
    if (!(last && u64)) {
      in = out;
      out = (out == L.u32) ? L.t32 : L.u32;
    }
  }
  float* other = (in == L.u32) ? L.t32 : L.u32;
  L.u32 = in;
  L.t32 = other;
  return STMG_OK;
}

// Alg. 1 in FP32 with fused passes: on every level the nu pre-smoothing sweeps from a
// zero start, the residual and the restriction run as one DOWN pass (or several when
// nu > 5), and the prolongation plus the nu post-smoothing sweeps as one UP pass.  On the
// finest level the result is added to the FP64 iterate u64 (mixed scheme) instead of
// being stored.  The level's FP32 u pointer ends on the level's result.
stmg_status vcycle32_fused(stmg_t h, int l, bool adj, double* u64, bool zero_start = true) {
  Level& L = h->lev[l];
  if (l == (int)h->lev.size() - 1) {
    CK(exact_level<float>(h, L, adj, L.b32, L.u32));
    if (u64) CK(launch_add_correction(L.nvec, u64, L.u32, kexp(h), h->s));
    return STMG_OK;
  }
  float* cur = nullptr;
  CKS(down32(h, l, adj, zero_start, &cur));
  CKS(vcycle32_fused(h, l + 1, adj, nullptr));
  return up32(h, l, adj, cur, u64);
}

// Read one device double (after the stream's pending work).
stmg_status read_scalar(stmg_t h, const double* d, double* out) {
  CK(cudaMemcpyAsync(h->hscal, d, sizeof(double), cudaMemcpyDeviceToHost, h->s));
  CK(cudaStreamSynchronize(h->s));
  *out = h->hscal[0];
  return STMG_OK;
}

// Copy a dense (rows x cols) user array into a padded level buffer (or back).
stmg_status copy_in(stmg_t h, double* dst, int pitch, const double* src, int rows, int cols) {
  CK(cudaMemcpy2DAsync(dst, (size_t)pitch * sizeof(double), src, (size_t)cols * sizeof(double),
                       (size_t)cols * sizeof(double), rows, cudaMemcpyDefault, h->s));
  return STMG_OK;
}
stmg_status copy_out(stmg_t h, double* dst, const double* src, int pitch, int rows, int cols) {
  CK(cudaMemcpy2DAsync(dst, (size_t)cols * sizeof(double), src, (size_t)pitch * sizeof(double),
                       (size_t)cols * sizeof(double), rows, cudaMemcpyDefault, h->s));
  return STMG_OK;
}

// Memory the current device's kernels can read directly: its own device memory or managed
// memory.  Host memory and device memory of another GPU are not (calls stage them through
// their own buffers, or refuse them where a call takes device arrays only).
bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return noalloc_placement(static_cast<int>(a.type), a.device, dev) == kPlaceUsable;
}

// Element loads -> nodal b on level 0.
// with_norm: also ||b||^2 into the handle's first device scalar and the FP32 scale exponent.
stmg_status assemble_into(stmg_t h, const double* q, double* b, bool with_norm = false) {
  Level& L = h->lev[0];
  const double* qd = q;
  if (!is_device_ptr(q)) {
    const size_t n = (size_t)(L.NT + 1) * L.N;
    if (h->qstage_n < n) {
      dfree(h, h->qstage);
      h->qstage_n = 0;
      CKS(dalloc(h, &h->qstage, n));
      h->qstage_n = n;
    }
    CK(cudaMemcpyAsync(h->qstage, q, n * sizeof(double), cudaMemcpyDefault, h->s));
    qd = h->qstage;
  }
  if (with_norm)
    CK(launch_assemble_load(view<double>(L, h->o.omega), L.dx, qd, b, h->s, 0.0, 1.0, h->partials, h->scal, kexp(h)));
  else
    CK(launch_assemble_load(view<double>(L, h->o.omega), L.dx, qd, b, h->s));
  return STMG_OK;
}

// The device int holding the scale exponent k of the finest level's FP32 arithmetic (see
// scale_exp): the last of the handle's device scalars.
int* kexp(stmg_t h) { return reinterpret_cast<int*>(h->scal + 7); }

// ||b - J u||^2 on level 0; set_scale: u is null and k is chosen from ||b||.
stmg_status resnorm2(stmg_t h, bool adj, const double* u, const double* b, double* out, bool set_scale = false) {
  Level& L = h->lev[0];
  CK(launch_resnorm<double>(view<double>(L, h->o.omega), adj, u, b, h->partials, h->scal, h->s,
                            set_scale ? kexp(h) : nullptr));
  return read_scalar(h, h->scal, out);
}

void reset_graphs(stmg_t h) {
  for (auto& row : h->gexec)
    for (auto& g : row)
      if (g) {
        cudaGraphExecDestroy(g);
        g = nullptr;
      }
  h->graph_u0 = nullptr;
}

// Records what body() enqueues as a CUDA graph (captured on the handle's private stream;
// the graph itself is launched on the handle's stream).
template <typename F>
stmg_status capture_graph(stmg_t h, cudaGraphExec_t* out, unsigned* nkernels, F body) {
  cudaStream_t user = h->s;
  const unsigned long long before = launches_so_far();
  h->s = h->cs;
  cudaError_t e = cudaStreamBeginCapture(h->cs, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    h->s = user;
    return fail(h, STMG_ECUDA, "cudaStreamBeginCapture: %s", cudaGetErrorString(e));
  }
  stmg_status st = body();
  *nkernels = (unsigned)(launches_so_far() - before);
  count_launches(0u - *nkernels);  // capture only records; launches are counted per replay
  cudaGraph_t g = nullptr;
  e = cudaStreamEndCapture(h->cs, &g);
  h->s = user;
  if (st != STMG_OK) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return st;
  }
  if (e != cudaSuccess) return fail(h, STMG_ECUDA, "cudaStreamEndCapture: %s", cudaGetErrorString(e));
  e = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    *out = nullptr;
    return fail(h, STMG_ECUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(e));
  }
  return STMG_OK;
}

// The FP64 graphs were captured with level-0 u in one particular ping-pong buffer; a
// solve starts by putting u back there (before anything is written to it).
void normalize_level0(stmg_t h) {
  Level& L = h->lev[0];
  if (h->graph_u0 && L.u != h->graph_u0) std::swap(L.u, L.t);
}

// The solver loop of Sec. 3.1 on level 0's u and scaled b (already in place).
//
// FP64: the residual norm of the iterate u_n is accumulated by the first pre-smoothing
// sweep of cycle n+1 (that sweep evaluates b - J u_n anyway); the termination test is
// taken on it before the rest of that cycle runs, and if the solve stops, u_n is the
// sweep's input, still intact in the other ping-pong buffer.
// Mixed: r = b - J u in FP64 (also the scaled FP32 right-hand side), one FP32 V-cycle
// from zero on J e = r, u += e.
stmg_status solve_loop(stmg_t h, bool adj, bool warm, int* cycles_out, double* relres_out, bool nb2_ready = false) {
  Level& L = h->lev[0];
  const stmg_opts& o = h->o;
  const LevelView<double> lv = view<double>(L, o.omega);
  if (!warm) CK(cudaMemsetAsync(L.u, 0, L.nvec * sizeof(double), h->s));
  double nb2 = 0.0;
  // ||b||^2 and the FP32 scale exponent: already on the device when the load assembly
  // formed them (nb2_ready), else from the stored b'
  if (nb2_ready) CKS(read_scalar(h, h->scal, &nb2));
  else CKS(resnorm2(h, adj, nullptr, L.b, &nb2, true));
  int cycles = 0;
  double rel = 0.0;
  stmg_status st = STMG_EMAXITER;
  if (nb2 == 0.0) {
    CK(cudaMemsetAsync(L.u, 0, L.nvec * sizeof(double), h->s));
    st = STMG_OK;
  } else if (!std::isfinite(nb2)) {
    return fail(h, STMG_EINVAL, "right-hand side contains NaN or Inf");
  } else if (o.precision == STMG_MIXED) {
    const double nb = std::sqrt(nb2);
    double r2 = nb2;
    if (warm) {
      CK(launch_defect(lv, L.cf32, adj, L.u, L.b, kexp(h), L.b32, h->partials, h->scal, h->s));
      CKS(read_scalar(h, h->scal, &r2));
    } else {
      CK(launch_rhs32(lv, L.b, kexp(h), L.b32, h->s));  // u = 0: the defect is b itself
    }
    rel = std::sqrt(r2) / nb;
    if (rel < o.tol) st = STMG_OK;
    // the first defect is solved by several FP32 cycles (an inner iteration far above the
    // FP32 rounding floor) before the first FP64 correction
    const int first = std::max(1, o.mixed_first_cycles);
    if (st != STMG_OK && first > 1 && o.nu > 0 && o.max_cycles >= first) {
      for (int j = 1; j <= first; ++j) CKS(vcycle32_fused(h, 0, adj, j == first ? L.u : nullptr, j == 1));
      CK(launch_defect(lv, L.cf32, adj, L.u, L.b, kexp(h), L.b32, h->partials, h->scal, h->s));
      CKS(read_scalar(h, h->scal, &r2));
      rel = std::sqrt(r2) / nb;
      cycles = first;
      if (!(rel <= o.div_tol)) st = STMG_EDIVERGED;
      else if (rel < o.tol) st = STMG_OK;
    }
    cudaGraphExec_t& gx = h->gexec[1][adj ? 1 : 0];
    unsigned& gk = h->gkernels[1][adj ? 1 : 0];
    // later defects: mixed_inner_cycles FP32 cycles each (the first from zero, the others
    // continuing the FP32 iterate), then the FP64 correction and the next defect
    const int inner = o.nu > 0 ? o.mixed_inner_cycles : 1;
    while (st == STMG_EMAXITER && cycles + inner <= o.max_cycles) {
      if (!gx) {
        CKS(capture_graph(h, &gx, &gk, [&]() -> stmg_status {
          if (o.nu > 0) {
            for (int j = 1; j <= inner; ++j) CKS(vcycle32_fused(h, 0, adj, j == inner ? L.u : nullptr, j == 1));
          } else {
            CKS(vcycle<float>(h, 0, adj, true, false));
            CK(launch_add_correction(L.nvec, L.u, L.u32, kexp(h), h->s));
          }
          CK(launch_defect(lv, L.cf32, adj, L.u, L.b, kexp(h), L.b32, h->partials, h->scal, h->s));
          return STMG_OK;
        }));
      }
      CK(cudaGraphLaunch(gx, h->s));
      count_launches(gk);
      CKS(read_scalar(h, h->scal, &r2));
      rel = std::sqrt(r2) / nb;
      cycles += inner;
      if (!(rel <= o.div_tol)) {  // also catches NaN
        st = STMG_EDIVERGED;
        break;
      }
      if (rel < o.tol) st = STMG_OK;
    }
  } else {
    const double nb = std::sqrt(nb2);
    double r2 = nb2;
    const bool one_level = h->lev.size() == 1;
    // the first sweep of cycle 1 (with the norm of the starting iterate if it is not 0)
    if (!one_level && o.nu > 0) {
      if (warm) {
        CK(launch_sweep_norm<double>(lv, adj, L.u, L.b, L.t, L.cf32 + (size_t)kDW * L.pitch, kexp(h), h->partials,
                                            h->scal, h->s));
        CKS(read_scalar(h, h->scal, &r2));
      } else {
        CK(cudaMemcpyAsync(L.t, L.b, L.nvec * sizeof(double), cudaMemcpyDeviceToDevice, h->s));
      }
    } else if (warm) {
      CKS(resnorm2(h, adj, L.u, L.b, &r2));
    }
    rel = std::sqrt(r2) / nb;
    bool pending = !one_level && o.nu > 0;  // u -> t holds the first sweep of the next cycle
    if (rel < o.tol) st = STMG_OK;
    cudaGraphExec_t& gx = h->gexec[0][adj ? 1 : 0];
    unsigned& gk = h->gkernels[0][adj ? 1 : 0];
    for (int cyc = 1; cyc <= o.max_cycles && st != STMG_OK; ++cyc) {
      if (pending) {
        // one graph: the rest of this cycle and the first sweep of the next, whose
        // norm is that of this cycle's result (2 nu buffer swaps on level 0: even)
        if (!gx) {
          double* u_before = L.u;
          CKS(capture_graph(h, &gx, &gk, [&]() -> stmg_status {
            std::swap(L.u, L.t);
            CKS(vcycle<double>(h, 0, adj, false, true));
            CK(launch_sweep_norm<double>(lv, adj, L.u, L.b, L.t, L.cf32 + (size_t)kDW * L.pitch, kexp(h), h->partials,
                                            h->scal, h->s));
            return STMG_OK;
          }));
          if (L.u != u_before) return fail(h, STMG_ECUDA, "internal: odd number of level-0 swaps in a cycle");
          h->graph_u0 = L.u;
        }
        CK(cudaGraphLaunch(gx, h->s));
        count_launches(gk);
      } else {
        CKS(vcycle<double>(h, 0, adj, false, false));
        CK(launch_resnorm<double>(lv, adj, L.u, L.b, h->partials, h->scal, h->s));
      }
      CKS(read_scalar(h, h->scal, &r2));
      rel = std::sqrt(r2) / nb;
      cycles = cyc;
      if (!(rel <= o.div_tol)) {  // also catches NaN
        st = STMG_EDIVERGED;
        break;
      }
      if (rel < o.tol) st = STMG_OK;
    }
  }
  if (cycles_out) *cycles_out = cycles;
  if (relres_out) *relres_out = rel;
  return st;
}

stmg_status check_opts(stmg_t h, const stmg_opts& o) {
  if (o.nu < 0 || !(o.omega > 0) || !std::isfinite(o.lambda_crit) || (o.interp != STMG_INTERP_CAUSAL && o.interp != STMG_INTERP_BILINEAR) ||
      (o.reassembly != STMG_REASM_K && o.reassembly != STMG_REASM_R && o.reassembly != STMG_REASM_D &&
       o.reassembly != STMG_REASM_P) || o.min_nel < 0 || o.num_levels < 0 ||
      o.num_levels > 60 || o.max_levels < 1 || o.max_levels > 60 || o.max_coarse_dofs < 1 ||
      (o.precision != STMG_FP64 && o.precision != STMG_MIXED) || !(o.tol >= 0) || !(o.div_tol > 0) ||
      o.max_cycles < 0 || !(o.deff_fixed >= 0) || o.mixed_first_cycles < 0 || o.mixed_first_cycles > 20 ||
      o.mixed_inner_cycles < 1 || o.mixed_inner_cycles > 8)
    return fail(h, STMG_EINVAL, "invalid stmg_opts");
  if (o.reassembly == STMG_REASM_P && o.precision != STMG_FP64)
    return fail(h, STMG_EINVAL, "the Galerkin reassembly (STMG_REASM_P) runs in FP64 only");
  return STMG_OK;
}

stmg_status read_material(stmg_t h, int n, const double* k, const double* c, std::vector<double>& hk,
                          std::vector<double>& hc) {
  if (!k || !c) return fail(h, STMG_EINVAL, "k_el and c_el must be non-NULL");
  hk.resize(n);
  hc.resize(n);
  cudaStream_t s = h ? h->s : nullptr;
  cudaError_t e1 = cudaMemcpyAsync(hk.data(), k, n * sizeof(double), cudaMemcpyDefault, s);
  cudaError_t e2 = cudaMemcpyAsync(hc.data(), c, n * sizeof(double), cudaMemcpyDefault, s);
  cudaError_t e3 = cudaStreamSynchronize(s);
  if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess)
    return fail(h, STMG_ECUDA, "reading k/c failed: %s", cudaGetErrorString(cudaGetLastError()));
  for (int e = 0; e < n; ++e)
    if (!finite_pos(hk[e]) || !finite_pos(hc[e]))
      return fail(h, STMG_EINVAL, "k and c must be finite and > 0 (element %d: k=%g c=%g)", e, hk[e], hc[e]);
  return STMG_OK;
}

// P-reassembly (Sec. 5.1): every coarse operator is the Galerkin product of the level above,
// built on the host in row-class form from level 0's per-node J entries, plus the block LU
// of the coarsest one in both directions.  Levels >= 1 then keep their right-hand sides
// unscaled (identity in the kW and kDW coefficient slots).
stmg_status build_galerkin(stmg_t h) {
  if (h->o.reassembly != STMG_REASM_P || h->lev.size() < 2) return STMG_OK;
  Level& F = h->lev[0];
  const size_t P0 = F.pitch;
  std::vector<double> c0(6 * P0);
  CK(cudaMemcpyAsync(c0.data(), F.cf64, c0.size() * sizeof(double), cudaMemcpyDeviceToHost, h->s));
  CK(cudaStreamSynchronize(h->s));
  GalOp op = galop_level0(F.N, F.NT, F.W, &c0[kL * P0], &c0[kD * P0], &c0[kU * P0], &c0[kPL * P0], &c0[kPC * P0],
                          &c0[kPR * P0]);
  for (size_t l = 1; l < h->lev.size(); ++l) {
    Level& C = h->lev[l];
    GalOp next;
    if (!galop_coarsen(op, transfer_type(h->o, h->lev[l - 1]), next))
      return fail(h, STMG_EINVAL, "Galerkin product on level %zu reaches beyond three time rows", l);
    if (next.N != C.N || next.NT != C.NT) return fail(h, STMG_ECUDA, "internal: Galerkin level shape mismatch");
    const size_t w = (size_t)C.N + 1;
    std::vector<double> wd((size_t)next.ncls * w);
    for (int c = 0; c < next.ncls; ++c)
      for (size_t i = 0; i < w; ++i) {
        const double d = next.co[((size_t)c * 9 + 4) * w + i];
        if (!(d > 0.0) || !std::isfinite(d))
          return fail(h, STMG_EINVAL, "Galerkin level %zu has a non-positive diagonal (node %zu)", l, i);
        wd[(size_t)c * w + i] = h->o.omega / d;
      }
    std::vector<double> ones(C.pitch, 1.0);
    dfree(h, C.dcls); dfree(h, C.dgco); dfree(h, C.dgwd);
    CKS(dalloc(h, &C.dcls, next.cls.size()));
    CKS(dalloc(h, &C.dgco, next.co.size()));
    CKS(dalloc(h, &C.dgwd, wd.size()));
    CK(cudaMemcpyAsync(C.dcls, next.cls.data(), next.cls.size() * sizeof(int), cudaMemcpyHostToDevice, h->s));
    CK(cudaMemcpyAsync(C.dgco, next.co.data(), next.co.size() * sizeof(double), cudaMemcpyHostToDevice, h->s));
    CK(cudaMemcpyAsync(C.dgwd, wd.data(), wd.size() * sizeof(double), cudaMemcpyHostToDevice, h->s));
    CK(cudaMemcpyAsync(C.cf64 + (size_t)kW * C.pitch, ones.data(), C.pitch * sizeof(double), cudaMemcpyHostToDevice,
                       h->s));
    CK(cudaMemcpyAsync(C.cf64 + (size_t)kDW * C.pitch, ones.data(), C.pitch * sizeof(double),
                       cudaMemcpyHostToDevice, h->s));
    CK(cudaStreamSynchronize(h->s));  // the host vectors must outlive the copies
    C.gal = true;
    C.gop = std::move(next);
    op = C.gop;
  }
  Level& Z = h->lev.back();
  const size_t n = (size_t)Z.N + 1, M = (size_t)Z.NT + 1;
  if (M * n * n > ((size_t)1 << 24))
    return fail(h, STMG_EINVAL, "coarsest Galerkin level too large for its direct solver ((nt+1)(nel+1)^2 = %zu > 2^24)",
                M * n * n);
  for (int adj = 0; adj < 2; ++adj) {
    std::vector<double> G, H, Ls;
    if (!galop_block_lu(Z.gop, adj != 0, G, H, Ls))
      return fail(h, STMG_EINVAL, "coarsest Galerkin level is singular");
    dfree(h, Z.dglu[adj]);
    CKS(dalloc(h, &Z.dglu[adj], G.size() + H.size() + Ls.size()));
    CK(cudaMemcpyAsync(Z.dglu[adj], G.data(), G.size() * sizeof(double), cudaMemcpyHostToDevice, h->s));
    CK(cudaMemcpyAsync(Z.dglu[adj] + G.size(), H.data(), H.size() * sizeof(double), cudaMemcpyHostToDevice, h->s));
    CK(cudaMemcpyAsync(Z.dglu[adj] + G.size() + H.size(), Ls.data(), Ls.size() * sizeof(double),
                       cudaMemcpyHostToDevice, h->s));
    CK(cudaStreamSynchronize(h->s));
  }
  return STMG_OK;
}

// The coarsest level, when narrow and short enough, is solved by a scan in time (see
// k_exact_scan): G = -A^-1 B from its Thomas factors and G^(2^k) for 2^K >= NT.
stmg_status build_scan_powers(stmg_t h) {
  Level& Z = h->lev.back();
  dfree(h, Z.dpw);
  Z.npw = 0;
  const int N = Z.N, NT = Z.NT;
  if (Z.gal || N < 1 || N > 64 || NT < 2 || (long long)NT * N > 8192) return STMG_OK;
  int K = 0;
  while ((1 << K) < NT) ++K;
  if ((long long)K * NT * N * N > (1LL << 20)) return STMG_OK;
  std::vector<double> th;
  thomas_factors(Z, th);
  const size_t S = N + 2;
  const double *lo = &th[0], *inv = &th[S], *cp = &th[2 * S], *pl = &th[3 * S], *pc = &th[4 * S], *pr = &th[5 * S];
  std::vector<double> pw((size_t)K * N * N), x(S);
  double* G = pw.data();
  for (int J = 1; J <= N; ++J) {  // column J of B: rows J-1 (pr), J (pc), J+1 (pl)
    double dp = 0.0;
    for (int i = 1; i <= N; ++i) {
      const double bij = i == J ? pc[i] : (i == J + 1 ? pl[i] : (i + 1 == J ? pr[i] : 0.0));
      dp = (bij - lo[i] * dp) * inv[i];
      x[i] = dp;
    }
    for (int i = N - 1; i >= 1; --i) x[i] -= cp[i] * x[i + 1];
    for (int i = 1; i <= N; ++i) G[(size_t)(i - 1) * N + (J - 1)] = -x[i];
  }
  for (int k = 1; k < K; ++k) {
    const double* A = pw.data() + (size_t)(k - 1) * N * N;
    double* C = pw.data() + (size_t)k * N * N;
    for (int i = 0; i < N; ++i)
      for (int j = 0; j < N; ++j) {
        double acc = 0.0;
        for (int m = 0; m < N; ++m) acc += A[(size_t)i * N + m] * A[(size_t)m * N + j];
        C[(size_t)i * N + j] = acc;
      }
  }
  CKS(dalloc(h, &Z.dpw, pw.size()));
  CK(cudaMemcpyAsync(Z.dpw, pw.data(), pw.size() * sizeof(double), cudaMemcpyHostToDevice, h->s));
  CK(cudaStreamSynchronize(h->s));  // pw must outlive the copy
  Z.npw = K;
  return STMG_OK;
}

stmg_status build_hierarchy(stmg_t h, const std::vector<double>& hk, const std::vector<double>& hc) {
  reset_graphs(h);
  std::vector<Level> nl = plan_levels(h->o, h->N, h->NT, h->L, h->tT, hk.data(), hc.data(),
                                      h->chi.empty() ? nullptr : h->chi.data(), h->simp);
  // keep device buffers of levels whose shape is unchanged
  for (size_t l = 0; l < nl.size(); ++l) {
    if (l < h->lev.size() && h->lev[l].N == nl[l].N && h->lev[l].NT == nl[l].NT) {
      Level& old = h->lev[l];
      std::swap(nl[l].dk, old.dk); std::swap(nl[l].dc, old.dc); std::swap(nl[l].cf64, old.cf64);
      std::swap(nl[l].cf32, old.cf32); std::swap(nl[l].th, old.th); std::swap(nl[l].u, old.u);
      std::swap(nl[l].b, old.b); std::swap(nl[l].t, old.t); std::swap(nl[l].u32, old.u32);
      std::swap(nl[l].b32, old.b32); std::swap(nl[l].t32, old.t32);
    }
  }
  for (Level& old : h->lev) free_level(h, old);
  h->lev = std::move(nl);
  for (Level& L : h->lev) CKS(setup_level(h, L));
  CKS(alloc_vectors(h));
  CKS(build_galerkin(h));
  for (size_t l = 0; l + 1 < h->lev.size(); ++l) {
    Level& L = h->lev[l];
    const Level& C = h->lev[l + 1];
    if (L.gal || C.gal) continue;
    CK(launch_build_rweights(transfer_type(h->o, L), L.N, L.pitch, C.N, C.pitch, L.W, C.W, h->o.omega, C.cf64,
                             L.cf64, L.cf32, h->s));
  }
  CKS(build_scan_powers(h));
  CK(cudaStreamSynchronize(h->s));
  return STMG_OK;
}

stmg_status check_level(stmg_t h, int level) {
  if (!h) return fail(nullptr, STMG_EINVAL, "NULL handle");
  if (level < 0 || level >= (int)h->lev.size()) return fail(h, STMG_EINVAL, "level %d out of range", level);
  return STMG_OK;
}

}  // namespace

// ======================================================================================
// C ABI
// ======================================================================================
extern "C" {

void stmg_default_opts(stmg_opts* o) {
  if (!o) return;
  o->nu = 5;
  o->omega = 0.5;
  o->lambda_crit = 0.25;
  o->interp = STMG_INTERP_CAUSAL;
  o->reassembly = STMG_REASM_R;
  o->min_nel = 0;
  o->num_levels = 0;
  o->max_levels = 30;
  o->max_coarse_dofs = 512;
  o->deff_fixed = 0.0;
  o->precision = STMG_FP64;
  o->tol = 1e-10;
  o->div_tol = 1e9;
  o->max_cycles = 100;
  o->mixed_first_cycles = 4;
  o->mixed_inner_cycles = 4;
}

const char* stmg_last_error(stmg_t h) { return h ? h->err.c_str() : g_global_error.c_str(); }

// Common body of the create calls; chi/simp are given for D-reassembly (k_el, c_el then
// hold the SIMP material of chi).
static stmg_status create_common(stmg_t* out, int nel, int nt, double L, double t_end, const double* k_el,
                                 const double* c_el, const std::vector<double>* chi, const double* simp,
                                 const stmg_opts* opts, void* stream, stmg_alloc_fn alloc, stmg_free_fn free_fn,
                                 void* ctx) {
  stmg_t h = nullptr;
  if (!out) return fail(nullptr, STMG_EINVAL, "NULL output handle pointer");
  *out = nullptr;
  if (nel < 1 || nt < 1 || !finite_pos(L) || !finite_pos(t_end))
    return fail(nullptr, STMG_EINVAL, "need nel >= 1, nt >= 1, L > 0, t_end > 0");
  if ((long long)(nel + 1) * (long long)(nt + 1) >= (1LL << 31))
    return fail(nullptr, STMG_EINVAL, "grid too large: (nel+1)(nt+1) must stay below 2^31 DOFs");
  if ((alloc == nullptr) != (free_fn == nullptr))
    return fail(nullptr, STMG_EINVAL, "give both allocator hooks or neither");
  h = new (std::nothrow) stmg_handle();
  if (!h) return fail(nullptr, STMG_ENOMEM, "host allocation failed");
  h->alloc_fn = alloc;
  h->free_fn = free_fn;
  h->actx = ctx;
  if (opts) h->o = *opts;
  else stmg_default_opts(&h->o);
  h->s = (cudaStream_t)stream;
  h->N = nel; h->NT = nt; h->L = L; h->tT = t_end;
  std::vector<double> hk, hc;
  stmg_status st = check_opts(h, h->o);
  if (st == STMG_OK && (h->o.reassembly == STMG_REASM_D) != (chi != nullptr))
    st = fail(h, STMG_EINVAL, "D-reassembly needs the design field: use stmg_create_design (and only it)");
  if (st == STMG_OK && chi) {
    h->chi = *chi;
    for (int i = 0; i < 6; ++i) h->simp[i] = simp[i];
  }
  if (st == STMG_OK) st = read_material(h, nel, k_el, c_el, hk, hc);
  if (st == STMG_OK) st = dalloc(h, &h->partials, kNormBlocks);
  if (st == STMG_OK) st = dalloc(h, &h->scal, 8);
  if (st == STMG_OK && cudaMemset(h->scal, 0, 8 * sizeof(double)) != cudaSuccess)
    st = fail(h, STMG_ECUDA, "cudaMemset of the device scalars failed");
  if (st == STMG_OK) {
    cudaError_t e = cudaStreamCreateWithFlags(&h->cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) st = fail(h, STMG_ECUDA, "cudaStreamCreateWithFlags: %s", cudaGetErrorString(e));
  }
  if (st == STMG_OK) st = build_hierarchy(h, hk, hc);
  if (st != STMG_OK) {
    g_global_error = h->err;
    stmg_destroy(h);
    return st;
  }
  *out = h;
  return STMG_OK;
}

stmg_status stmg_create_with_allocator(stmg_t* out, int nel, int nt, double L, double t_end, const double* k_el,
                                       const double* c_el, const stmg_opts* opts, void* stream, stmg_alloc_fn alloc,
                                       stmg_free_fn free_fn, void* ctx) {
  return create_common(out, nel, nt, L, t_end, k_el, c_el, nullptr, nullptr, opts, stream, alloc, free_fn, ctx);
}

stmg_status stmg_create(stmg_t* out, int nel, int nt, double L, double t_end, const double* k_el,
                        const double* c_el, const stmg_opts* opts, void* stream) {
  return create_common(out, nel, nt, L, t_end, k_el, c_el, nullptr, nullptr, opts, stream, nullptr, nullptr, nullptr);
}

// Design field chi (host or device) -> host copy and its SIMP material.
static stmg_status read_design(stmg_t h, int nel, const double* chi, const double* simp6, std::vector<double>& hx,
                               std::vector<double>& hk, std::vector<double>& hc) {
  if (!chi || !simp6) return fail(h, STMG_EINVAL, "NULL design field or SIMP parameters");
  hx.resize(nel);
  cudaStream_t s = h ? h->s : nullptr;
  if (cudaMemcpyAsync(hx.data(), chi, nel * sizeof(double), cudaMemcpyDefault, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return fail(h, STMG_ECUDA, "reading chi failed: %s", cudaGetErrorString(cudaGetLastError()));
  hk.resize(nel);
  hc.resize(nel);
  for (int e = 0; e < nel; ++e) {
    if (!std::isfinite(hx[e])) return fail(h, STMG_EINVAL, "chi must be finite (element %d)", e);
    hk[e] = simp_k(simp6, hx[e]);
    hc[e] = simp_c(simp6, hx[e]);
  }
  return STMG_OK;
}

stmg_status stmg_create_design(stmg_t* out, int nel, int nt, double L, double t_end, const double* chi,
                               const double* simp6, const stmg_opts* opts, void* stream) {
  if (!out) return fail(nullptr, STMG_EINVAL, "NULL output handle pointer");
  *out = nullptr;
  if (nel < 1) return fail(nullptr, STMG_EINVAL, "need nel >= 1");
  stmg_opts o;
  if (opts) o = *opts;
  else stmg_default_opts(&o);
  o.reassembly = STMG_REASM_D;
  std::vector<double> hx, hk, hc;
  CKS_NULL(read_design(nullptr, nel, chi, simp6, hx, hk, hc));
  return create_common(out, nel, nt, L, t_end, hk.data(), hc.data(), &hx, simp6, &o, stream, nullptr, nullptr,
                       nullptr);
}

stmg_status stmg_update_design(stmg_t h, const double* chi) {
  if (!h) return fail(nullptr, STMG_EINVAL, "NULL handle");
  if (h->o.reassembly != STMG_REASM_D) return fail(h, STMG_EINVAL, "handle was not created with a design field");
  std::vector<double> hx, hk, hc;
  CKS(read_design(h, h->N, chi, h->simp, hx, hk, hc));
  h->chi = hx;
  return build_hierarchy(h, hk, hc);
}

long long stmg_device_bytes(stmg_t h) { return h ? h->bytes : 0; }

stmg_status stmg_set_stream(stmg_t h, void* stream) {
  if (!h) return fail(nullptr, STMG_EINVAL, "NULL handle");
  h->s = (cudaStream_t)stream;  // every call returns with its work complete: nothing is pending
  return STMG_OK;
}

long long stmg_footprint(int nel, int nt, double L, double t_end, const double* k_el, const double* c_el,
                         const stmg_opts* opts) {
  if (nel < 1 || nt < 1 || !finite_pos(L) || !finite_pos(t_end) || !k_el || !c_el) return -1;
  if ((long long)(nel + 1) * (long long)(nt + 1) >= (1LL << 31)) return -1;
  stmg_opts o;
  if (opts) o = *opts;
  else stmg_default_opts(&o);
  if (o.reassembly == STMG_REASM_D) o.reassembly = STMG_REASM_R;  // same level sizes for the same path
  for (int e = 0; e < nel; ++e)
    if (!finite_pos(k_el[e]) || !finite_pos(c_el[e])) return -1;
  const std::vector<Level> lev = plan_levels(o, nel, nt, L, t_end, k_el, c_el);
  long long b = (long long)round256(kNormBlocks * sizeof(double)) + (long long)round256(8 * sizeof(double));
  for (size_t l = 0; l < lev.size(); ++l) {
    const Level& v = lev[l];
    b += 2 * (long long)round256(v.N * sizeof(double));
    b += (long long)round256((size_t)kNumCoef * v.pitch * sizeof(double));
    b += (long long)round256((size_t)kNumCoef * v.pitch * sizeof(float));
    b += (long long)round256(8 * (size_t)(v.N + 2) * sizeof(double));
    if (l == 0 || o.precision == STMG_FP64) b += 3 * (long long)round256(v.nvec * sizeof(double));
    if (o.precision == STMG_MIXED) b += 3 * (long long)round256(v.nvec * sizeof(float));
  }
  return b;
}

void stmg_destroy(stmg_t h) {
  if (!h) return;
  if (h->s) cudaStreamSynchronize(h->s);
  else cudaDeviceSynchronize();
  reset_graphs(h);
  if (h->cs) cudaStreamDestroy(h->cs);
  for (Level& L : h->lev) free_level(h, L);
  dfree(h, h->partials);
  dfree(h, h->scal);
  dfree(h, h->qstage);
  dfree(h, h->sens);
  dfree(h, h->gstage);
  delete h;
}

stmg_status stmg_update_material(stmg_t h, const double* k_el, const double* c_el) {
  if (!h) return fail(nullptr, STMG_EINVAL, "NULL handle");
  std::vector<double> hk, hc;
  CKS(read_material(h, h->N, k_el, c_el, hk, hc));
  return build_hierarchy(h, hk, hc);
}

stmg_status stmg_simp(int nel, const double* chi, const double* simp6, double* k_el, double* c_el, void* stream) {
  stmg_t h = nullptr;
  if (nel < 1 || !chi || !simp6 || !k_el || !c_el) return fail(nullptr, STMG_EINVAL, "bad stmg_simp arguments");
  if (!is_device_ptr(chi) || !is_device_ptr(k_el) || !is_device_ptr(c_el))
    return fail(nullptr, STMG_EINVAL, "stmg_simp takes arrays on the current device");
  Simp6 sp;
  for (int i = 0; i < 6; ++i) sp.v[i] = simp6[i];
  CK(launch_simp(nel, chi, sp, k_el, c_el, (cudaStream_t)stream));
  CK(cudaStreamSynchronize((cudaStream_t)stream));
  return STMG_OK;
}

stmg_status stmg_design_update(int nel, const double* chi, const double* dtheta, double vol_frac, double move,
                               double* chi_new, void* stream) {
  if (nel < 1 || !chi || !dtheta || !chi_new || !(vol_frac > 0.0 && vol_frac <= 1.0) || !(move > 0.0 && move <= 1.0))
    return fail(nullptr, STMG_EINVAL, "bad stmg_design_update arguments");
  if (!is_device_ptr(chi) || !is_device_ptr(dtheta) || !is_device_ptr(chi_new))
    return fail(nullptr, STMG_EINVAL, "stmg_design_update takes device arrays");
  stmg_t h = nullptr;  // errors go to stmg_last_error(NULL)
  CK(launch_design_update(nel, chi, dtheta, vol_frac, move, chi_new, (cudaStream_t)stream));
  CK(cudaStreamSynchronize((cudaStream_t)stream));
  return STMG_OK;
}

stmg_status stmg_assemble_load(stmg_t h, const double* q_el, double* b) {
  if (!h) return fail(nullptr, STMG_EINVAL, "NULL handle");
  if (!q_el || !b) return fail(h, STMG_EINVAL, "NULL array");
  Level& L = h->lev[0];
  CKS(assemble_into(h, q_el, L.t));
  CK(launch_scale<double>(view<double>(L, h->o.omega), false, L.t, h->s));
  CKS(copy_out(h, b, L.t, L.pitch, L.NT + 1, L.N + 1));
  CK(cudaStreamSynchronize(h->s));
  return STMG_OK;
}

static stmg_status solve_common(stmg_t h, bool adj, const double* q_el, const double* b_nodal, double* u, int warm,
                                int* cycles, double* relres) {
  if (!h) return fail(nullptr, STMG_EINVAL, "NULL handle");
  if (!u || ((q_el == nullptr) == (b_nodal == nullptr)))
    return fail(h, STMG_EINVAL, "need u and exactly one of q_el / b_nodal");
  Level& L = h->lev[0];
  normalize_level0(h);
  if (q_el) {
    CKS(assemble_into(h, q_el, L.b, true));
  } else {
    CKS(copy_in(h, L.b, L.pitch, b_nodal, L.NT + 1, L.N + 1));
    CK(launch_scale<double>(view<double>(L, h->o.omega), true, L.b, h->s));
  }
  if (warm) CKS(copy_in(h, L.u, L.pitch, u, L.NT + 1, L.N + 1));
  stmg_status st = solve_loop(h, adj, warm != 0, cycles, relres, q_el != nullptr);
  if (st != STMG_OK && st != STMG_EDIVERGED && st != STMG_EMAXITER) return st;
  CKS(copy_out(h, u, L.u, L.pitch, L.NT + 1, L.N + 1));
  CK(cudaStreamSynchronize(h->s));
  if (st == STMG_EDIVERGED) fail(h, st, "relative residual exceeded div_tol");
  if (st == STMG_EMAXITER) fail(h, st, "max_cycles reached before tol");
  return st;
}

stmg_status stmg_solve(stmg_t h, const double* q_el, const double* b_nodal, double* u, int warm, int* cycles,
                       double* relres) {
  return solve_common(h, false, q_el, b_nodal, u, warm, cycles, relres);
}

stmg_status stmg_solve_adjoint(stmg_t h, const double* rhs, double* lam, int warm, int* cycles, double* relres) {
  if (!rhs) return fail(h, STMG_EINVAL, "NULL rhs");
  return solve_common(h, true, nullptr, rhs, lam, warm, cycles, relres);
}

stmg_status stmg_sensitivity(stmg_t h, const double* chi, const double* simp6, const double* u, const double* lam,
                             double* g) {
  if (!h) return fail(nullptr, STMG_EINVAL, "NULL handle");
  if (!chi || !simp6 || !u || !lam || !g) return fail(h, STMG_EINVAL, "NULL array");
  Level& L = h->lev[0];
  const size_t need = 2 * (size_t)sens_chunks(L.NT) * L.N;
  if (h->sens_n < need) {
    dfree(h, h->sens);
    h->sens_n = 0;
    CKS(dalloc(h, &h->sens, need));
    h->sens_n = need;
  }
  if (!h->gstage) CKS(dalloc(h, &h->gstage, 2 * (size_t)L.N));
  CKS(copy_in(h, L.u, L.pitch, u, L.NT + 1, L.N + 1));
  CKS(copy_in(h, L.t, L.pitch, lam, L.NT + 1, L.N + 1));
  CK(cudaMemcpyAsync(h->gstage, chi, L.N * sizeof(double), cudaMemcpyDefault, h->s));
  Simp6 sp;
  for (int i = 0; i < 6; ++i) sp.v[i] = simp6[i];
  CK(launch_sensitivity(L.N, L.NT, L.pitch, L.dx, L.dt, h->gstage, sp, L.u, L.t, h->sens, h->gstage + L.N, h->s));
  CK(cudaMemcpyAsync(g, h->gstage + L.N, L.N * sizeof(double), cudaMemcpyDefault, h->s));
  CK(cudaStreamSynchronize(h->s));
  return STMG_OK;
}

stmg_status stmg_objective(stmg_t h, const double* b, const double* u, double theta_ref, double* theta) {
  if (!h) return fail(nullptr, STMG_EINVAL, "NULL handle");
  if (!b || !u || !theta || !(theta_ref != 0.0)) return fail(h, STMG_EINVAL, "bad stmg_objective arguments");
  Level& L = h->lev[0];
  CKS(copy_in(h, L.u, L.pitch, u, L.NT + 1, L.N + 1));
  CKS(copy_in(h, L.t, L.pitch, b, L.NT + 1, L.N + 1));
  CK(launch_dot(L.nvec, L.t, L.u, h->partials, h->scal, h->s));
  double s = 0.0;
  CKS(read_scalar(h, h->scal, &s));
  *theta = s * L.dt / theta_ref;
  return STMG_OK;
}

stmg_status stmg_objective_gradient(stmg_t h, const double* b, double theta_ref, double seed, double* grad_u) {
  if (!h) return fail(nullptr, STMG_EINVAL, "NULL handle");
  if (!b || !grad_u || !(theta_ref != 0.0) || !std::isfinite(seed))
    return fail(h, STMG_EINVAL, "bad stmg_objective_gradient arguments");
  if (!is_device_ptr(b) || !is_device_ptr(grad_u))
    return fail(h, STMG_EINVAL, "stmg_objective_gradient takes device arrays");
  const Level& L = h->lev[0];
  const size_t n = (size_t)(L.NT + 1) * (size_t)(L.N + 1);
  CK(launch_scaled_copy(n, seed * L.dt / theta_ref, b, grad_u, h->s));
  CK(cudaStreamSynchronize(h->s));
  return STMG_OK;
}

stmg_status stmg_deff_simp(const double* simp6, double* deff) {
  if (!simp6 || !deff) return fail(nullptr, STMG_EINVAL, "bad stmg_deff_simp arguments");
  for (int i = 0; i < 6; ++i)
    if (!std::isfinite(simp6[i])) return fail(nullptr, STMG_EINVAL, "stmg_deff_simp: non-finite SIMP parameter");
  const double kins = simp6[0], kcon = simp6[1], cins = simp6[2], ccon = simp6[3], pk = simp6[4], pc = simp6[5];
  if (!(kins > 0.0 && kcon > 0.0 && cins > 0.0 && ccon > 0.0 && pk >= 0.0 && pc >= 0.0))
    return fail(nullptr, STMG_EINVAL, "stmg_deff_simp: need positive k_ins, k_con, c_ins, c_con and p_k, p_c >= 0");
  double dmin = INFINITY, dmax = 0.0;
  for (int j = 0; j <= kDeffSamples; ++j) {
    const double x = (double)j / kDeffSamples;
    const double d = (kins + std::pow(x, pk) * (kcon - kins)) / (cins + std::pow(x, pc) * (ccon - cins));
    dmin = std::min(dmin, d);
    dmax = std::max(dmax, d);
  }
  *deff = std::sqrt(dmin * dmax);
  return STMG_OK;
}

int stmg_num_levels(stmg_t h) { return h ? (int)h->lev.size() : 0; }

stmg_status stmg_level_info(stmg_t h, int level, int* nel, int* nt, int* next, double* dx, double* dt,
                            double* w_diri, double* lambda_eff) {
  CKS(check_level(h, level));
  const Level& L = h->lev[level];
  if (nel) *nel = L.N;
  if (nt) *nt = L.NT;
  if (next) *next = L.next;
  if (dx) *dx = L.dx;
  if (dt) *dt = L.dt;
  if (w_diri) *w_diri = L.W;
  if (lambda_eff) *lambda_eff = L.lam;
  return STMG_OK;
}

stmg_status stmg_level_material(stmg_t h, int level, double* k, double* c) {
  CKS(check_level(h, level));
  const Level& L = h->lev[level];
  if (k) std::memcpy(k, L.k.data(), L.N * sizeof(double));
  if (c) std::memcpy(c, L.c.data(), L.N * sizeof(double));
  return STMG_OK;
}

stmg_status stmg_apply(stmg_t h, int level, int adjoint, const double* u, double* y) {
  CKS(check_level(h, level));
  if (!u || !y) return fail(h, STMG_EINVAL, "NULL array");
  Level& L = h->lev[level];
  CKS(ensure_fp64(h, L));
  CKS(copy_in(h, L.u, L.pitch, u, L.NT + 1, L.N + 1));
  if (L.gal) CK(launch_gal_apply(gal_view(L), adjoint != 0, L.u, L.t, h->s));
  else CK(launch_apply<double>(view<double>(L, h->o.omega), adjoint != 0, L.u, L.t, h->s));
  CKS(copy_out(h, y, L.t, L.pitch, L.NT + 1, L.N + 1));
  CK(cudaStreamSynchronize(h->s));
  return STMG_OK;
}

stmg_status stmg_smooth(stmg_t h, int level, int adjoint, int nsweeps, double* u, const double* b) {
  CKS(check_level(h, level));
  if (!u || !b || nsweeps < 0) return fail(h, STMG_EINVAL, "bad stmg_smooth arguments");
  Level& L = h->lev[level];
  CKS(ensure_fp64(h, L));
  CKS(copy_in(h, L.u, L.pitch, u, L.NT + 1, L.N + 1));
  CKS(copy_in(h, L.b, L.pitch, b, L.NT + 1, L.N + 1));
  CK(launch_scale<double>(view<double>(L, h->o.omega), true, L.b, h->s));
  CKS(smooth_level<double>(h, L, adjoint != 0, nsweeps));
  CKS(copy_out(h, u, L.u, L.pitch, L.NT + 1, L.N + 1));
  CK(cudaStreamSynchronize(h->s));
  return STMG_OK;
}

stmg_status stmg_restrict(stmg_t h, int level, const double* r, double* bc) {
  CKS(check_level(h, level));
  if (level + 1 >= (int)h->lev.size()) return fail(h, STMG_EINVAL, "level %d is the coarsest", level);
  if (!r || !bc) return fail(h, STMG_EINVAL, "NULL array");
  Level& L = h->lev[level];
  Level& C = h->lev[level + 1];
  CKS(ensure_fp64(h, L));
  CKS(ensure_fp64(h, C));
  CKS(copy_in(h, L.t, L.pitch, r, L.NT + 1, L.N + 1));
  CK(launch_restrict<double>(transfer_type(h->o, L), L.N, L.NT, L.pitch, L.t, view<double>(C, h->o.omega), C.b,
                             h->s));
  CK(launch_scale<double>(view<double>(C, h->o.omega), false, C.b, h->s));
  CKS(copy_out(h, bc, C.b, C.pitch, C.NT + 1, C.N + 1));
  CK(cudaStreamSynchronize(h->s));
  return STMG_OK;
}

stmg_status stmg_prolong_add(stmg_t h, int level, const double* z, double* u) {
  CKS(check_level(h, level));
  if (level + 1 >= (int)h->lev.size()) return fail(h, STMG_EINVAL, "level %d is the coarsest", level);
  if (!z || !u) return fail(h, STMG_EINVAL, "NULL array");
  Level& L = h->lev[level];
  Level& C = h->lev[level + 1];
  CKS(ensure_fp64(h, L));
  CKS(ensure_fp64(h, C));
  CKS(copy_in(h, C.u, C.pitch, z, C.NT + 1, C.N + 1));
  CKS(copy_in(h, L.u, L.pitch, u, L.NT + 1, L.N + 1));
  CK(launch_prolong_add<double>(transfer_type(h->o, L), L.N, L.NT, L.pitch, L.u, C.N, C.NT, C.pitch, C.u,
                                h->s));
  CKS(copy_out(h, u, L.u, L.pitch, L.NT + 1, L.N + 1));
  CK(cudaStreamSynchronize(h->s));
  return STMG_OK;
}

stmg_status stmg_exact_solve(stmg_t h, int level, int adjoint, const double* b, double* u) {
  CKS(check_level(h, level));
  if (!b || !u) return fail(h, STMG_EINVAL, "NULL array");
  Level& L = h->lev[level];
  if (L.N > 512 * kMaxNodesPerThread) return fail(h, STMG_EINVAL, "level too wide for the exact solver");
  if (L.gal && level + 1 != (int)h->lev.size())
    return fail(h, STMG_EINVAL, "Galerkin levels have a direct solver on the coarsest level only");
  CKS(ensure_fp64(h, L));
  CKS(copy_in(h, L.b, L.pitch, b, L.NT + 1, L.N + 1));
  CK(launch_scale<double>(view<double>(L, h->o.omega), true, L.b, h->s));
  CK(exact_level<double>(h, L, adjoint != 0, L.b, L.u));
  CKS(copy_out(h, u, L.u, L.pitch, L.NT + 1, L.N + 1));
  CK(cudaStreamSynchronize(h->s));
  return STMG_OK;
}

static stmg_status slabs_common(stmg_t h, const double* b_nodal, const double* ckpt, int slab_rows,
                                const double** ckpt_dev) {
  if (!b_nodal || !ckpt || slab_rows < 1) return fail(h, STMG_EINVAL, "need b_nodal, ckpt and slab_rows >= 1");
  Level& L = h->lev[0];
  if ((L.N + 511) / 512 > kMaxNodesPerThread) return fail(h, STMG_EINVAL, "nel too large for the slab solver");
  normalize_level0(h);
  CKS(copy_in(h, L.b, L.pitch, b_nodal, L.NT + 1, L.N + 1));
  CK(launch_scale<double>(view<double>(L, h->o.omega), true, L.b, h->s));
  const int nslabs = (L.NT + slab_rows - 1) / slab_rows;
  const size_t n = (size_t)nslabs * (L.N + 1);
  *ckpt_dev = ckpt;
  if (!is_device_ptr(ckpt)) {
    if (h->qstage_n < n) {
      dfree(h, h->qstage);
      h->qstage_n = 0;
      CKS(dalloc(h, &h->qstage, std::max(n, (size_t)(L.NT + 1) * L.N)));
      h->qstage_n = std::max(n, (size_t)(L.NT + 1) * L.N);
    }
    CK(cudaMemcpyAsync(h->qstage, ckpt, n * sizeof(double), cudaMemcpyDefault, h->s));
    *ckpt_dev = h->qstage;
  }
  return STMG_OK;
}

stmg_status stmg_recompute_slabs(stmg_t h, const double* b_nodal, const double* ckpt, int slab_rows, double* u) {
  if (!h) return fail(nullptr, STMG_EINVAL, "NULL handle");
  if (!u) return fail(h, STMG_EINVAL, "NULL u");
  const double* cd = nullptr;
  CKS(slabs_common(h, b_nodal, ckpt, slab_rows, &cd));
  Level& L = h->lev[0];
  CK(launch_slabs(slab_view(L, h->o.omega, slab_rows), L.b, cd, L.u, nullptr, nullptr, h->s));
  CKS(copy_out(h, u, L.u, L.pitch, L.NT + 1, L.N + 1));
  CK(cudaStreamSynchronize(h->s));
  return STMG_OK;
}

stmg_status stmg_sensitivity_slabs(stmg_t h, const double* chi, const double* simp6, const double* b_nodal,
                                   const double* ckpt, int slab_rows, const double* lam, double* g) {
  if (!h) return fail(nullptr, STMG_EINVAL, "NULL handle");
  if (!chi || !simp6 || !lam || !g) return fail(h, STMG_EINVAL, "NULL array");
  const double* cd = nullptr;
  CKS(slabs_common(h, b_nodal, ckpt, slab_rows, &cd));
  Level& L = h->lev[0];
  const int nslabs = (L.NT + slab_rows - 1) / slab_rows;
  const size_t need = 2 * (size_t)nslabs * L.N;
  if (h->sens_n < need) {
    dfree(h, h->sens);
    h->sens_n = 0;
    CKS(dalloc(h, &h->sens, need));
    h->sens_n = need;
  }
  if (!h->gstage) CKS(dalloc(h, &h->gstage, 2 * (size_t)L.N));
  CKS(copy_in(h, L.t, L.pitch, lam, L.NT + 1, L.N + 1));
  CK(cudaMemcpyAsync(h->gstage, chi, L.N * sizeof(double), cudaMemcpyDefault, h->s));
  CK(launch_slabs(slab_view(L, h->o.omega, slab_rows), L.b, cd, nullptr, L.t, h->sens, h->s));
  Simp6 sp;
  for (int i = 0; i < 6; ++i) sp.v[i] = simp6[i];
  CK(launch_sens_final(L.N, nslabs, h->gstage, sp, h->sens, h->gstage + L.N, h->s));
  CK(cudaMemcpyAsync(g, h->gstage + L.N, L.N * sizeof(double), cudaMemcpyDefault, h->s));
  CK(cudaStreamSynchronize(h->s));
  return STMG_OK;
}

stmg_status stmg_vcycle(stmg_t h, int adjoint, double* u, const double* b) {
  if (!h) return fail(nullptr, STMG_EINVAL, "NULL handle");
  if (!u || !b) return fail(h, STMG_EINVAL, "NULL array");
  Level& L = h->lev[0];
  CKS(copy_in(h, L.u, L.pitch, u, L.NT + 1, L.N + 1));
  CKS(copy_in(h, L.b, L.pitch, b, L.NT + 1, L.N + 1));
  CK(launch_scale<double>(view<double>(L, h->o.omega), true, L.b, h->s));
  if (h->o.precision == STMG_MIXED) {
    CK(cudaMemsetAsync(kexp(h), 0, sizeof(int), h->s));  // one cycle: FP32 arithmetic unscaled
    CK(launch_defect(view<double>(L, h->o.omega), L.cf32, adjoint != 0, L.u, L.b, kexp(h), L.b32, h->partials,
                     h->scal, h->s));
    if (h->o.nu > 0) {
      CKS(vcycle32_fused(h, 0, adjoint != 0, L.u));
    } else {
      CKS(vcycle<float>(h, 0, adjoint != 0, true, false));
      CK(launch_add_correction(L.nvec, L.u, L.u32, kexp(h), h->s));
    }
  } else {
    CKS(vcycle<double>(h, 0, adjoint != 0, false, false));
  }
  CKS(copy_out(h, u, L.u, L.pitch, L.NT + 1, L.N + 1));
  CK(cudaStreamSynchronize(h->s));
  return STMG_OK;
}

stmg_status stmg_mixed_pass(stmg_t h, int level, int adjoint, int kind) {
  if (!h) return fail(nullptr, STMG_EINVAL, "NULL handle");
  if (h->o.precision != STMG_MIXED || h->o.nu <= 0)
    return fail(h, STMG_EINVAL, "stmg_mixed_pass needs the mixed scheme with nu > 0");
  const int nl = (int)h->lev.size();
  if (kind < 0 || kind > 3 || level < 0 || level >= nl - 1 || (kind == 2 && level != 0))
    return fail(h, STMG_EINVAL, "stmg_mixed_pass: bad level %d or kind %d", level, kind);
  Level& L = h->lev[level];
  if (kind == 0) {
    float* cur = nullptr;
    return down32(h, level, adjoint != 0, true, &cur);
  }
  if (kind == 1) return up32(h, level, adjoint != 0, L.u32, level == 0 ? L.u : nullptr);
  if (kind == 3) return up32(h, level, adjoint != 0, L.u32, nullptr);
  CK(launch_defect(view<double>(L, h->o.omega), L.cf32, adjoint != 0, L.u, L.b, kexp(h), L.b32, h->partials, h->scal,
                   h->s));
  return STMG_OK;
}

}  // extern "C"

extern "C" unsigned long long stmg_kernel_launches(void) { return launches_so_far(); }

stmg_status stmg_solve_resident(stmg_t h, bool adj, const double* q_dev, double q_value, double rhs_scale, double* out,
                                int* cycles, double* relres, double* theta) {
  if (!h) return fail(nullptr, STMG_EINVAL, "NULL handle");
  Level& L = h->lev[0];
  const LevelView<double> lv = view<double>(L, h->o.omega);
  normalize_level0(h);
  CK(launch_assemble_load(lv, L.dx, q_dev, L.b, h->s, q_value, rhs_scale, h->partials, h->scal, kexp(h)));
  stmg_status st = solve_loop(h, adj, false, cycles, relres, true);
  if (st != STMG_OK && st != STMG_EDIVERGED && st != STMG_EMAXITER) return st;
  if (theta) {
    CK(cudaMemcpyAsync(L.t, L.b, L.nvec * sizeof(double), cudaMemcpyDeviceToDevice, h->s));
    CK(launch_scale<double>(lv, false, L.t, h->s));
    CK(launch_dot(L.nvec, L.t, L.u, h->partials, h->scal, h->s));
    double d = 0.0;
    CKS(read_scalar(h, h->scal, &d));
    *theta = d * L.dt / rhs_scale;
  }
  if (out) CKS(copy_out(h, out, L.u, L.pitch, L.NT + 1, L.N + 1));
  CK(cudaStreamSynchronize(h->s));
  return st;
}

namespace stmg {
void set_global_error(const char* msg) { g_global_error = msg; }
}  // namespace stmg
