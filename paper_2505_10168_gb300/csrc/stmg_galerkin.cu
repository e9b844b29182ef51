// stmg_galerkin.cu -- Galerkin reassembly of the coarse operators (P-method, Sec. 5.1):
// J_{l+1} = R_l J_l P_l.
//
// A product of the space-time operator with the transfer operators keeps the stencil inside
// three time rows and three nodes, but it is no longer the BE-FE stencil: with bilinear
// interpolation a row couples to the next time row too, the time-boundary rows differ from
// the interior ones, and the Dirichlet rows mix with their neighbours.  A level operator is
// therefore kept in row-class form: every time row n uses one of a few coefficient sets,
// cls[n], each holding the 9 coefficients of u(n + d, i + e), d, e in {-1, 0, 1}, for every
// node i.  Interior rows of a level share one set, so the storage is O(N) per level.
//
// The host forms each coarse row of R J P from the fine rows it gathers (at most three for
// bilinear R) and merges rows whose coefficients are equal.  FP64 kernels apply, smooth
// (damped Jacobi with D = diag(J_l)) and evaluate residuals on such a level; the coarsest
// level is solved exactly by a block-tridiagonal LU in time (dense blocks of N + 1 nodes,
// factored on the host once per hierarchy and direction).
#include <cmath>
#include <cstring>
#include <unordered_map>

#include "stmg_internal.h"

namespace stmg {

namespace {

inline size_t co_at(const GalOp& op, int c, int d, int e, int i) {
  return ((size_t)c * 9 + (size_t)(d + 1) * 3 + (size_t)(e + 1)) * (size_t)(op.N + 1) + (size_t)i;
}

// Weight of coarse node / row j in fine node / row i of the 1D prolongations (Sec. 3.1,
// 5.1): linear (x, and t bilinear) 1 at i = 2j, 1/2 at i = 2j +- 1; causal (t) 1 at
// i = 2j and i = 2j + 1.
inline double p_lin(int i, int j) {
  const int r = i - 2 * j;
  return r == 0 ? 1.0 : (r == 1 || r == -1 ? 0.5 : 0.0);
}
inline double p_causal(int i, int j) { return (i == 2 * j || i == 2 * j + 1) ? 1.0 : 0.0; }

uint64_t fnv(const double* p, size_t n) {
  const unsigned char* b = reinterpret_cast<const unsigned char*>(p);
  uint64_t h = 1469598103934665603ull;
  for (size_t k = 0; k < n * sizeof(double); ++k) h = (h ^ b[k]) * 1099511628211ull;
  return h;
}

// Appends row coefficients `row` (9 * (N + 1) values) as a class, or finds an equal one.
int intern(GalOp& op, std::unordered_map<uint64_t, std::vector<int>>& index, const std::vector<double>& row) {
  const size_t w = 9 * (size_t)(op.N + 1);
  const uint64_t key = fnv(row.data(), w);
  auto& bucket = index[key];
  for (int c : bucket)
    if (std::memcmp(op.co.data() + (size_t)c * w, row.data(), w * sizeof(double)) == 0) return c;
  const int c = op.ncls++;
  op.co.insert(op.co.end(), row.begin(), row.end());
  bucket.push_back(c);
  return c;
}

}  // namespace

GalOp galop_level0(int N, int NT, double W, const double* Lc, const double* Dc, const double* Uc, const double* PLc,
                   const double* PCc, const double* PRc) {
  GalOp op;
  op.N = N;
  op.NT = NT;
  std::unordered_map<uint64_t, std::vector<int>> index;
  const size_t w = 9 * (size_t)(N + 1);
  // row 0: the Dirichlet rows W_Diri I; row 1: no coupling to the eliminated row 0;
  // rows n >= 2: the BE-FE stencil (Sec. 2.2, Appendix A)
  for (int kind = 0; kind < 3; ++kind) {
    std::vector<double> row(w, 0.0);
    auto at = [&](int d, int e, int i) -> double& { return row[((size_t)(d + 1) * 3 + (e + 1)) * (N + 1) + i]; };
    for (int i = 0; i <= N; ++i) {
      if (kind == 0 || i == 0) {  // Dirichlet rows: W_Diri on the diagonal only
        at(0, 0, i) = W;
        continue;
      }
      at(0, -1, i) = Lc[i];
      at(0, 0, i) = Dc[i];
      at(0, 1, i) = Uc[i];
      if (kind == 2) {
        at(-1, -1, i) = PLc[i];
        at(-1, 0, i) = PCc[i];
        at(-1, 1, i) = PRc[i];
      }
    }
    intern(op, index, row);
  }
  op.cls.resize(NT + 1);
  for (int n = 0; n <= NT; ++n) op.cls[n] = n == 0 ? 0 : (n == 1 ? 1 : 2);
  return op;
}

bool galop_coarsen(const GalOp& f, int type, GalOp& out) {
  const bool xc = type == 1;
  GalOp c;
  c.N = xc ? f.N / 2 : f.N;
  c.NT = xc ? f.NT : f.NT / 2;
  const int Nf = f.N, NTf = f.NT, Nc = c.N, NTc = c.NT;
  const size_t w = 9 * (size_t)(Nc + 1);
  std::unordered_map<uint64_t, std::vector<int>> index;
  std::vector<double> row(w);
  auto at = [&](int d, int e, int i) -> double& { return row[((size_t)(d + 1) * 3 + (e + 1)) * (Nc + 1) + i]; };
  if (xc) {
    // rows keep their time index; every block is transformed as R_x B P_x with R_x = P_x^T
    std::vector<int> map(f.ncls);
    for (int k = 0; k < f.ncls; ++k) {
      std::fill(row.begin(), row.end(), 0.0);
      for (int d = -1; d <= 1; ++d)
        for (int j = 0; j <= Nc; ++j)
          for (int i = 2 * j - 1; i <= 2 * j + 1; ++i) {
            if (i < 0 || i > Nf) continue;
            const double r = p_lin(i, j);
            for (int e = -1; e <= 1; ++e) {
              const int ii = i + e;
              if (ii < 0 || ii > Nf) continue;
              const double a = f.co[co_at(f, k, d, e, i)];
              if (a == 0.0) continue;
              for (int jj = j - 1; jj <= j + 1; ++jj) {
                if (jj < 0 || jj > Nc) continue;
                const double p = p_lin(ii, jj);
                if (p != 0.0) at(d, jj - j, j) += r * a * p;
              }
            }
          }
      map[k] = intern(c, index, row);
    }
    c.cls.resize(NTc + 1);
    for (int n = 0; n <= NTc; ++n) c.cls[n] = map[f.cls[n]];
  } else {
    // coarse row m gathers fine rows n with R(m, n) = P(n, m) / 2; the fine column rows
    // n + d map back to coarse rows m' with P(n + d, m')
    const bool bil = type == 3;
    auto pt = [&](int n, int m) { return bil ? p_lin(n, m) : p_causal(n, m); };
    c.cls.resize(NTc + 1);
    for (int m = 0; m <= NTc; ++m) {
      std::fill(row.begin(), row.end(), 0.0);
      for (int n = 2 * m - 1; n <= 2 * m + 1; ++n) {
        if (n < 0 || n > NTf) continue;
        const double r = 0.5 * pt(n, m);
        if (r == 0.0) continue;
        const int k = f.cls[n];
        for (int d = -1; d <= 1; ++d) {
          const int nn = n + d;
          if (nn < 0 || nn > NTf) continue;
          // the coarse rows that fine row nn interpolates from lie within nn/2 -+ 1; one
          // outside m - 1 .. m + 1 would widen the stencil beyond three time rows
          for (int mm = (nn >> 1) - 1; mm <= (nn >> 1) + 1; ++mm) {
            if (mm < 0 || mm > NTc) continue;
            const double p = pt(nn, mm);
            if (p == 0.0) continue;
            if (mm < m - 1 || mm > m + 1) return false;
            for (int e = -1; e <= 1; ++e)
              for (int i = 0; i <= Nc; ++i) at(mm - m, e, i) += r * p * f.co[co_at(f, k, d, e, i)];
          }
        }
      }
      c.cls[m] = intern(c, index, row);
    }
  }
  out = std::move(c);
  return true;
}

namespace {

// In-place inverse of the n x n row-major matrix a by Gauss-Jordan elimination with
// partial pivoting; false if a pivot vanishes.
bool invert(std::vector<double>& a, int n) {
  std::vector<double> inv((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) inv[(size_t)i * n + i] = 1.0;
  for (int col = 0; col < n; ++col) {
    int piv = col;
    for (int r = col + 1; r < n; ++r)
      if (std::fabs(a[(size_t)r * n + col]) > std::fabs(a[(size_t)piv * n + col])) piv = r;
    const double pv = a[(size_t)piv * n + col];
    if (!(std::fabs(pv) > 0.0) || !std::isfinite(pv)) return false;
    if (piv != col)
      for (int k = 0; k < n; ++k) {
        std::swap(a[(size_t)piv * n + k], a[(size_t)col * n + k]);
        std::swap(inv[(size_t)piv * n + k], inv[(size_t)col * n + k]);
      }
    const double s = 1.0 / pv;
    for (int k = 0; k < n; ++k) {
      a[(size_t)col * n + k] *= s;
      inv[(size_t)col * n + k] *= s;
    }
    for (int r = 0; r < n; ++r) {
      if (r == col) continue;
      const double f = a[(size_t)r * n + col];
      if (f == 0.0) continue;
      for (int k = 0; k < n; ++k) {
        a[(size_t)r * n + k] -= f * a[(size_t)col * n + k];
        inv[(size_t)r * n + k] -= f * inv[(size_t)col * n + k];
      }
    }
  }
  a.swap(inv);
  return true;
}

}  // namespace

bool galop_block_lu(const GalOp& op, bool adj, std::vector<double>& G, std::vector<double>& H,
                    std::vector<double>& Lsub) {
  const int n = op.N + 1, M = op.NT + 1;
  const size_t nn = (size_t)n * n;
  G.assign((size_t)M * nn, 0.0);
  H.assign((size_t)M * nn, 0.0);
  Lsub.assign((size_t)M * 3 * n, 0.0);
  // block of time row m coupling to row m + d, as a dense n x n matrix (J or J^T)
  auto block = [&](int m, int d, std::vector<double>& B) {
    B.assign(nn, 0.0);
    if (m + d < 0 || m + d >= M) return;
    for (int i = 0; i < n; ++i)
      for (int e = -1; e <= 1; ++e) {
        const int j = i + e;
        if (j < 0 || j >= n) continue;
        // J: row (m, i), column (m + d, j); J^T: the entry of J at row (m + d, j), column (m, i)
        B[(size_t)i * n + j] = adj ? op.co[co_at(op, op.cls[m + d], -d, -e, j)] : op.co[co_at(op, op.cls[m], d, e, i)];
      }
  };
  std::vector<double> A, Lb, Ub, T((size_t)nn), S;
  for (int m = 0; m < M; ++m) {
    block(m, 0, S);
    if (m > 0) {
      // S_m = A_m - L_m G_{m-1} U_{m-1}, with H_{m-1} = G_{m-1} U_{m-1} already formed
      block(m, -1, Lb);
      const double* Hp = H.data() + (size_t)(m - 1) * nn;
      for (int i = 0; i < n; ++i)
        for (int k = 0; k < n; ++k) {
          double s = 0.0;
          for (int j = 0; j < n; ++j) s += Lb[(size_t)i * n + j] * Hp[(size_t)j * n + k];
          S[(size_t)i * n + k] -= s;
        }
      for (int i = 0; i < n; ++i)
        for (int e = -1; e <= 1; ++e) {
          const int j = i + e;
          if (j >= 0 && j < n) Lsub[((size_t)m * 3 + (e + 1)) * n + i] = Lb[(size_t)i * n + j];
        }
    }
    if (!invert(S, n)) return false;
    std::memcpy(G.data() + (size_t)m * nn, S.data(), nn * sizeof(double));
    if (m + 1 < M) {
      block(m, 1, Ub);
      double* Hm = H.data() + (size_t)m * nn;
      for (int i = 0; i < n; ++i)
        for (int k = 0; k < n; ++k) {
          double s = 0.0;
          for (int j = 0; j < n; ++j) s += S[(size_t)i * n + j] * Ub[(size_t)j * n + k];
          Hm[(size_t)i * n + k] = s;
        }
    }
  }
  return true;
}

namespace {

constexpr int kGalThreads = 256;

__device__ __forceinline__ void gsplit(uint32_t idx, const FastDiv& fd, int& n, int& i) {
  const uint32_t q = (uint32_t)(((uint64_t)__umulhi(idx, fd.M) + idx) >> fd.s);
  n = (int)q;
  i = (int)(idx - q * fd.d);
}

// (J u)(n, i) on a row-class level; ADJ: (J^T u)(n, i) = sum over the rows (n + d, i + e)
// whose stencil reaches (n, i).
template <bool ADJ>
__device__ __forceinline__ double gapply_at(const GalView& g, const double* __restrict__ u, int n, int i) {
  const size_t w = (size_t)(g.N + 1);
  double acc = 0.0;
#pragma unroll
  for (int d = -1; d <= 1; ++d) {
    const int nn = n + d;
    if (nn < 0 || nn > g.NT) continue;
    const int cn = ADJ ? g.cls[nn] : g.cls[n];
#pragma unroll
    for (int e = -1; e <= 1; ++e) {
      const int ii = i + e;
      if (ii < 0 || ii > g.N) continue;
      const double a = ADJ ? g.co[((size_t)cn * 9 + (size_t)(1 - d) * 3 + (size_t)(1 - e)) * w + ii]
                           : g.co[((size_t)cn * 9 + (size_t)(d + 1) * 3 + (size_t)(e + 1)) * w + i];
      acc = fma(a, u[(size_t)nn * g.pitch + ii], acc);
    }
  }
  return acc;
}

// MODE 0: y = J u; 1: y = u + (omega / D)(b - J u) (one damped-Jacobi step); 2: y = b - J u.
template <bool ADJ, int MODE>
__global__ void __launch_bounds__(kGalThreads) k_gal(GalView g, uint32_t total, const double* __restrict__ u,
                                                     const double* __restrict__ b, double* __restrict__ y) {
  const uint32_t idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= total) return;
  int n, i;
  gsplit(idx, g.fd, n, i);
  const size_t p = (size_t)n * g.pitch + i;
  const double ju = gapply_at<ADJ>(g, u, n, i);
  if (MODE == 0) {
    y[p] = ju;
  } else if (MODE == 1) {
    y[p] = fma(g.wd[(size_t)g.cls[n] * (g.N + 1) + i], b[p] - ju, u[p]);
  } else {
    y[p] = b[p] - ju;
  }
}

// Coarsest level: block-tridiagonal LU in time (G_m = S_m^-1, H_m = S_m^-1 U_m, L_m
// tridiagonal).  Forward: y_m = G_m (b_m - L_m y_{m-1}); backward: x_m = y_m - H_m x_{m+1}.
// One block; node i of every row is owned by thread i (strided).
__global__ void __launch_bounds__(kGalThreads) k_gal_exact(int n, int M, int pitch, const double* __restrict__ G,
                                                           const double* __restrict__ H,
                                                           const double* __restrict__ Lsub,
                                                           const double* __restrict__ b, double* __restrict__ u) {
  extern __shared__ double sm[];
  double* t = sm;      // right-hand side of the current row
  double* prev = sm + n;  // y_{m-1}, then x_{m+1}
  const size_t nn = (size_t)n * n;
  for (int m = 0; m < M; ++m) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      double s = b[(size_t)m * pitch + i];
      if (m > 0) {
        const double* l = Lsub + (size_t)m * 3 * n;
        if (i > 0) s -= l[i] * prev[i - 1];
        s -= l[n + i] * prev[i];
        if (i + 1 < n) s -= l[2 * n + i] * prev[i + 1];
      }
      t[i] = s;
    }
    __syncthreads();
    const double* Gm = G + (size_t)m * nn;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      double s = 0.0;
      for (int j = 0; j < n; ++j) s = fma(Gm[(size_t)i * n + j], t[j], s);
      u[(size_t)m * pitch + i] = s;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) prev[i] = u[(size_t)m * pitch + i];
    __syncthreads();
  }
  // prev holds x_{M-1} = y_{M-1}
  for (int m = M - 2; m >= 0; --m) {
    const double* Hm = H + (size_t)m * nn;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      double s = u[(size_t)m * pitch + i];
      for (int j = 0; j < n; ++j) s = fma(-Hm[(size_t)i * n + j], prev[j], s);
      t[i] = s;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      u[(size_t)m * pitch + i] = t[i];
      prev[i] = t[i];
    }
    __syncthreads();
  }
}

template <int MODE>
cudaError_t launch_gal(const GalView& g, bool adj, const double* u, const double* b, double* y, cudaStream_t s) {
  const uint32_t total = (uint32_t)((uint64_t)(g.NT + 1) * (uint64_t)(g.N + 1));
  const unsigned grid = (total + kGalThreads - 1) / kGalThreads;
  if (adj) k_gal<true, MODE><<<grid, kGalThreads, 0, s>>>(g, total, u, b, y);
  else k_gal<false, MODE><<<grid, kGalThreads, 0, s>>>(g, total, u, b, y);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_gal_apply(const GalView& g, bool adj, const double* u, double* y, cudaStream_t s) {
  return launch_gal<0>(g, adj, u, nullptr, y, s);
}
cudaError_t launch_gal_sweep(const GalView& g, bool adj, const double* u, const double* b, double* out,
                             cudaStream_t s) {
  return launch_gal<1>(g, adj, u, b, out, s);
}
cudaError_t launch_gal_residual(const GalView& g, bool adj, const double* u, const double* b, double* r,
                                cudaStream_t s) {
  return launch_gal<2>(g, adj, u, b, r, s);
}
cudaError_t launch_gal_exact(int n, int M, int pitch, const double* G, const double* H, const double* Lsub,
                             const double* b, double* u, cudaStream_t s) {
  const size_t smem = 2 * (size_t)n * sizeof(double);
  k_gal_exact<<<1, kGalThreads, smem, s>>>(n, M, pitch, G, H, Lsub, b, u);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace stmg
