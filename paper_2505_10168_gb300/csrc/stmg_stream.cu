// stmg_stream.cu -- fused FP32 passes of the V-cycle for the mixed-precision scheme.
//
// One warp owns a window of 128 columns (4 per lane, float4) of one level and marches
// through a chunk of time rows.  Because the space-time stencil couples row n only to
// rows n and n-1 (n+1 for the adjoint), S damped-Jacobi sweeps (Sec. 3.1) are a pipeline
// over rows: sweep k of row n needs sweep k-1 of rows n and n-1, so a warp keeps the
// previous row of every stage in registers and produces all S sweeps of a row as soon as
// the row is read.  The same pipeline then evaluates the residual and restricts it
// (Sec. 3.1, R = s P^T) to the coarse level (DOWN pass), or adds the prolongated coarse
// correction before sweeping (UP pass).  x-neighbours come from warp shuffles; the window
// carries an 8-column halo on each side and a chunk starts S(+1) rows early, so every
// output value is computed from exact inputs with no block-level synchronisation.
//
// A row's inputs (b', the starting iterate, the coarse correction, the FP64 iterate) are
// staged through a per-warp ring of rows in shared memory, filled by asynchronous copies
// several rows ahead, so the loads in flight cost no registers.  The row loop has no
// data-dependent branches: the Dirichlet row 0 is peeled off, rows alternate between two
// register sets of pipeline state, and every row-dependent choice is a select or a
// predicated store.
//
// HBM traffic per DOF of a level (x-coarsening, zero start): DOWN reads b' and writes u
// and b'_c (10 B); UP reads u, b', z and writes u (14 B); the finest-level UP of the
// mixed scheme adds its result straight into the FP64 iterate instead (26 B).
#include <atomic>
#include <type_traits>

#include "stmg_internal.h"
#include "stmg_stream.h"

namespace stmg {
namespace {

constexpr int kVec = 4;
constexpr int kWin = 32 * kVec;            // columns per warp window
constexpr int kHalo = 8;                   // halo columns on each side
constexpr int kOwn = kWin - 2 * kHalo;     // 112 columns owned per window
constexpr int kWarpsPerBlock = 4;
constexpr int kThreads = 32 * kWarpsPerBlock;
constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ float4 f4zero() { return make_float4(0.f, 0.f, 0.f, 0.f); }

__device__ __forceinline__ float4 ld4(const float* __restrict__ p, size_t off, bool ok) {
  return ok ? __ldg(reinterpret_cast<const float4*>(p + off)) : f4zero();
}

// Asynchronous global -> shared copies of base[off ...]; when ok is false nothing is read
// (base may then be null) and the destination is filled with zeros (src-size 0).
// fallback is any valid global address.
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
template <int BYTES, typename T>
__device__ __forceinline__ void cp_async(void* dst, const T* base, size_t off, const void* fallback, bool ok) {
  const void* src = ok ? static_cast<const void*>(base + off) : fallback;
  if (BYTES == 16) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem_u32(dst)), "l"(src), "r"(ok ? 16 : 0)
                 : "memory");
  } else {
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;\n" ::"r"(smem_u32(dst)), "l"(src), "n"(BYTES),
                 "r"(ok ? BYTES : 0)
                 : "memory");
  }
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// One stage of the pipeline on a lane's 4 columns: out = a*x + b' + sum_k S_k x_k, with
// a = 1 - omega for a sweep and a = -omega for the scaled residual.  DIR: a Dirichlet row
// (time level 0), whose row of J is W_Diri I.  px is the stage input of the previous row
// (the next row for J^T), zero where the stencil has no such coupling; pl, pr are its
// x-neighbours across the lane boundary, which that row's own stage shuffled and handed on.
// hl, hr receive this row's shuffled neighbours of x for the next row.
template <bool DIR>
__device__ __forceinline__ float4 stage(float a, const float4& x, const float4& px, float pl, float pr, float& hl,
                                        float& hr, const float4& b, const float4& sl, const float4& su,
                                        const float4& spl, const float4& spc, const float4& spr) {
  float4 o;
  o.x = fmaf(a, x.x, b.x);
  o.y = fmaf(a, x.y, b.y);
  o.z = fmaf(a, x.z, b.z);
  o.w = fmaf(a, x.w, b.w);
  if (DIR) {
    hl = 0.f;
    hr = 0.f;
    return o;
  }
  // At the window edges (lanes 0 and 31) the shuffles return the lane's own values: those
  // columns are halo, whose results are never used, and every value stays finite.
  const float xl = __shfl_up_sync(kFull, x.w, 1);
  const float xr = __shfl_down_sync(kFull, x.x, 1);
  hl = xl;
  hr = xr;
  o.x = fmaf(sl.x, xl, o.x);
  o.x = fmaf(su.x, x.y, o.x);
  o.y = fmaf(sl.y, x.x, o.y);
  o.y = fmaf(su.y, x.z, o.y);
  o.z = fmaf(sl.z, x.y, o.z);
  o.z = fmaf(su.z, x.w, o.z);
  o.w = fmaf(sl.w, x.z, o.w);
  o.w = fmaf(su.w, xr, o.w);
  o.x = fmaf(spl.x, pl, o.x);
  o.x = fmaf(spc.x, px.x, o.x);
  o.x = fmaf(spr.x, px.y, o.x);
  o.y = fmaf(spl.y, px.x, o.y);
  o.y = fmaf(spc.y, px.y, o.y);
  o.y = fmaf(spr.y, px.z, o.y);
  o.z = fmaf(spl.z, px.y, o.z);
  o.z = fmaf(spc.z, px.z, o.z);
  o.z = fmaf(spr.z, px.w, o.z);
  o.w = fmaf(spl.w, px.z, o.w);
  o.w = fmaf(spc.w, px.w, o.w);
  o.w = fmaf(spr.w, pr, o.w);
  return o;
}

__device__ __forceinline__ float4 mul4(const float4& s, const float4& v) {
  return make_float4(s.x * v.x, s.y * v.y, s.z * v.z, s.w * v.w);
}
__device__ __forceinline__ float4 sel4(bool c, const float4& p, const float4& q) {
  return make_float4(c ? p.x : q.x, c ? p.y : q.y, c ? p.z : q.z, c ? p.w : q.w);
}

// Fields of one ring slot, 16 bytes per lane each: b', the starting iterate, the coarse
// correction rows (UP), the FP64 iterate (two fields; UP and plain passes).
template <int MODE>
struct Ring {
  static constexpr bool kDown = MODE == 1 || MODE == 2 || MODE == 5;
  static constexpr bool kHasZ = MODE == 3 || MODE == 4 || MODE == 6;
  static constexpr int kB = 0, kU = 1, kZ = 2, kZB = 3;
  static constexpr int k64 = kDown ? 0 : (MODE == 6 ? 4 : (kHasZ ? 3 : 2));
  static constexpr int kFields = kDown ? 2 : k64 + 2;
  static constexpr int kDepth = kDown ? 8 : 4;  // rows in flight per warp (a power of two)
};

// Pipeline state after one row: v[0] the row's starting iterate (plus the prolongated
// correction), v[k] the row after sweep k; hl[k], hr[k] the neighbours of v[k-1] across the
// lane boundary that stage k shuffled (k = S + 1: the residual stage); r, rp the residuals
// of this row and the one before it (restriction modes).
template <int S>
struct Pipe {
  float4 v[S + 1];
  float hl[S + 2], hr[S + 2];
  float4 r, rp;
};

// MODE: 0 plain sweeps, 1 sweeps + residual + x-restriction, 2 sweeps + residual +
// causal t-restriction, 3 x-prolongation + sweeps, 4 causal t-prolongation + sweeps,
// 5 sweeps + residual + bilinear t-restriction, 6 bilinear t-prolongation + sweeps.
template <bool ADJ, int S, int MODE>
__global__ void __launch_bounds__(kThreads, 4) k_stream(StreamArgs a) {
  using R = Ring<MODE>;
  constexpr bool DOWN = R::kDown;
  constexpr int kD = R::kDepth;
  __shared__ float4 ring[kWarpsPerBlock][kD][R::kFields][32];

  const int lane = threadIdx.x & 31;
  const int w = threadIdx.x >> 5;
  const int wid = blockIdx.x * kWarpsPerBlock + w;
  if (wid >= a.strips * a.chunks) return;  // the whole warp leaves together
  const int strip = wid % a.strips;
  const int chunk = wid / a.strips;
  const int c0 = strip * kOwn - kHalo;
  const int col = c0 + kVec * lane;  // multiple of 4; either fully inside [0, pitch) or fully outside
  const bool inside = col >= 0 && col + kVec <= a.pitch;
  const bool owner = lane >= kHalo / kVec && lane < (kHalo + kOwn) / kVec && inside;
  const int P = a.pitch;

  const float4 sl = ld4(a.coef, (size_t)kSL * P + col, inside);
  const float4 su = ld4(a.coef, (size_t)kSU * P + col, inside);
  const float4 spl = ld4(a.coef, (size_t)kSPL * P + col, inside);
  const float4 spc = ld4(a.coef, (size_t)kSPC * P + col, inside);
  const float4 spr = ld4(a.coef, (size_t)kSPR * P + col, inside);
  float4 dw = f4zero();
  if (DOWN) dw = ld4(a.coef, (size_t)kDW * P + col, inside);
  // coarse scaling of the restricted residual: x: coarse nodes col/2 and col/2 + 1;
  // t: coarse node = fine node
  float2 cwx = make_float2(0.f, 0.f);
  float4 cwt = f4zero();
  if (MODE == 1 && inside && col / 2 + 1 < a.pc) {
    cwx.x = a.ccoef[(size_t)kW * a.pc + col / 2];
    cwx.y = a.ccoef[(size_t)kW * a.pc + col / 2 + 1];
  }
  if (MODE == 2 || MODE == 5) cwt = ld4(a.ccoef, (size_t)kW * a.pc + col, inside);
  const float4 cwW4 = make_float4(a.cwW, a.cwW, a.cwW, a.cwW);
  // prolongation only touches nodes 0..N
  const float4 pm = make_float4(col >= 0 && col <= a.N ? 1.f : 0.f, col + 1 >= 0 && col + 1 <= a.N ? 1.f : 0.f,
                                col + 2 >= 0 && col + 2 <= a.N ? 1.f : 0.f, col + 3 >= 0 && col + 3 <= a.N ? 1.f : 0.f);
  // x-restriction: coarse nodes col/2 and col/2 + 1 of this lane
  const bool own0 = owner && col <= a.N;
  const bool own1 = owner && col + 2 <= a.N;
  const float sx0 = col / 2 == 0 ? a.cwW : cwx.x;

  const int n0 = chunk * a.rows;
  const int n1 = min(a.NT + 1, n0 + a.rows);
  // rows before the chunk (after it, for J^T) that make every emitted value exact; the
  // bilinear restriction of the chunk's first coarse row also needs fine row n0 - 1
  constexpr int WARM = MODE == 5 ? S + 2 : (DOWN ? S + 1 : S);
  const int first = ADJ ? min(a.NT, n1 - 1 + WARM) : max(0, n0 - WARM);
  const int last = ADJ ? (MODE == 5 ? max(0, n0 - 1) : n0) : n1 - 1;
  const int step = ADJ ? -1 : 1;
  const int count = ADJ ? first - last + 1 : last - first + 1;

  // Row j of the chunk (row first + j * step) goes to ring slot j % kD.
  auto fetch = [&](const int j) {
    const bool ok = j < count;
    const int n = first + j * step;
    float4* slot = &ring[w][j % kD][0][0];
    const size_t ro = (size_t)n * P + col;
    cp_async<16>(slot + R::kB * 32 + lane, a.bs, ro, a.bs, ok && inside);
    if (!a.zero_init) cp_async<16>(slot + R::kU * 32 + lane, a.u_in, ro, a.bs, ok && inside);
    if (MODE == 3) {
      const int ca = col / 2;
      const size_t zo = (size_t)n * a.pc + ca;
      cp_async<8>(slot + R::kZ * 32 + lane, a.z, zo, a.bs, ok && col >= 0 && ca + 1 < a.pc);
      if (lane == 31) cp_async<4>(&slot[R::kZ * 32 + lane].z, a.z, zo + 2, a.bs, ok && col >= 0 && ca + 2 < a.pc);
    } else if (MODE == 4 || MODE == 6) {
      cp_async<16>(slot + R::kZ * 32 + lane, a.z, (size_t)(n >> 1) * a.pc + col, a.bs, ok && inside);
    }
    if (MODE == 6)
      cp_async<16>(slot + R::kZB * 32 + lane, a.z, (size_t)((n >> 1) + 1) * a.pc + col, a.bs, ok && inside && (n & 1));
    if (!DOWN && a.u64 != nullptr) {
      cp_async<16>(slot + R::k64 * 32 + lane, a.u64, ro, a.bs, ok && inside);
      cp_async<16>(slot + (R::k64 + 1) * 32 + lane, a.u64, ro + 2, a.bs, ok && inside);
    }
    cp_commit();
  };

  // One row: consume its ring slot, sweep, store, restrict.
  auto row = [&](auto dir_tag, const int j, const Pipe<S>& in, Pipe<S>& out) {
    constexpr bool DIR = decltype(dir_tag)::value;
    const int n = first + j * step;
    const bool emit = n >= n0 && n < n1;
    const float4* slot = &ring[w][j % kD][0][0];
    cp_wait<kD - 1>();
    const float4 b = slot[R::kB * 32 + lane];
    float4 x = a.zero_init ? f4zero() : slot[R::kU * 32 + lane];
    if (MODE == 3) {
      // x-prolongation: fine 2j <- z_j, fine 2j+1 <- (z_j + z_{j+1}) / 2
      const float4 zs = slot[R::kZ * 32 + lane];
      float z2 = __shfl_down_sync(kFull, zs.x, 1);
      if (lane == 31) z2 = zs.z;
      x.x = fmaf(pm.x, zs.x, x.x);
      x.y = fmaf(pm.y, 0.5f * (zs.x + zs.y), x.y);
      x.z = fmaf(pm.z, zs.y, x.z);
      x.w = fmaf(pm.w, 0.5f * (zs.y + z2), x.w);
    } else if (MODE == 4 || MODE == 6) {
      // causal t-prolongation: fine rows 2m and 2m+1 <- coarse row m; bilinear: fine row
      // 2m+1 <- (z_m + z_{m+1}) / 2
      float4 zz = slot[R::kZ * 32 + lane];
      if (MODE == 6) {
        const float4 zb = slot[R::kZB * 32 + lane];
        const float4 zh = make_float4(0.5f * (zz.x + zb.x), 0.5f * (zz.y + zb.y), 0.5f * (zz.z + zb.z),
                                      0.5f * (zz.w + zb.w));
        zz = sel4(n & 1, zh, zz);
      }
      x.x = fmaf(pm.x, zz.x, x.x);
      x.y = fmaf(pm.y, zz.y, x.y);
      x.z = fmaf(pm.z, zz.z, x.z);
      x.w = fmaf(pm.w, zz.w, x.w);
    }
    out.v[0] = x;
#pragma unroll
    for (int k = 1; k <= S; ++k) {
      if (k == 1 && a.zero_init) out.v[1] = b;  // a sweep from zero is exactly b'
      else
        out.v[k] = stage<DIR>(a.omc, out.v[k - 1], in.v[k - 1], in.hl[k], in.hr[k], out.hl[k], out.hr[k], b, sl, su,
                              spl, spc, spr);
    }
    if (!DOWN && a.u64 != nullptr) {
      double2 lo = *reinterpret_cast<const double2*>(slot + R::k64 * 32 + lane);
      double2 hi = *reinterpret_cast<const double2*>(slot + (R::k64 + 1) * 32 + lane);
      lo.x += to_f64(out.v[S].x);
      lo.y += to_f64(out.v[S].y);
      hi.x += to_f64(out.v[S].z);
      hi.y += to_f64(out.v[S].w);
      if (emit && owner) {
        double2* q = reinterpret_cast<double2*>(a.u64 + (size_t)n * P + col);
        q[0] = lo;
        q[1] = hi;
      }
    } else if (emit && owner) {
      *reinterpret_cast<float4*>(a.u_out + (size_t)n * P + col) = out.v[S];
    }
    if (DOWN) {
      // scaled residual y = b' - omega u + sum S_k u_k, r = (D / omega) y
      const float4 y = stage<DIR>(-a.omega, out.v[S], in.v[S], in.hl[S + 1], in.hr[S + 1], out.hl[S + 1], out.hr[S + 1], b,
                                  sl, su, spl, spc, spr);
      const float4 r = DIR ? make_float4(a.Wo * y.x, a.Wo * y.y, a.Wo * y.z, a.Wo * y.w) : mul4(dw, y);
      out.r = r;
      if (MODE == 5) out.rp = in.r;
      if (MODE == 1) {
        // b_c[j] = r[2j] + (r[2j-1] + r[2j+1]) / 2, scaled by omega / D_c
        const float rl = __shfl_up_sync(kFull, r.w, 1);
        const float s0 = DIR ? a.cwW : sx0;
        const float s1 = DIR ? a.cwW : cwx.y;
        const float2 o = make_float2(s0 * (r.x + 0.5f * (rl + r.y)), s1 * (r.z + 0.5f * (r.y + r.w)));
        float* dst = a.bc + (size_t)n * a.pc + col / 2;
        if (emit && own0) dst[0] = o.x;
        if (emit && own1) dst[1] = o.y;
      } else {
        float4 sum;
        int m;
        bool put;
        const bool odd = n & 1;
        if (MODE == 2) {
          // b_c[m] = (r[2m] + r[2m+1]) / 2 (causal P^T with s = 1/2); forward: emitted at
          // row 2m+1 (row NT alone when NT is even); J^T: emitted at row 2m
          if (!ADJ) {
            sum = odd ? make_float4(r.x + in.r.x, r.y + in.r.y, r.z + in.r.z, r.w + in.r.w) : r;
            put = emit && (odd || n == a.NT);
          } else {
            sum = make_float4(r.x + in.r.x, r.y + in.r.y, r.z + in.r.z, r.w + in.r.w);
            put = emit && !odd;
          }
          m = n >> 1;
        } else {
          // b_c[m] = (r[2m] + (r[2m-1] + r[2m+1]) / 2) / 2 (bilinear P^T with s = 1/2),
          // emitted when the last of its three fine rows has been processed
          const float4 so = make_float4(in.r.x + 0.5f * (in.rp.x + r.x), in.r.y + 0.5f * (in.rp.y + r.y),
                                        in.r.z + 0.5f * (in.rp.z + r.z), in.r.w + 0.5f * (in.rp.w + r.w));
          const float4 se = make_float4(r.x + 0.5f * in.r.x, r.y + 0.5f * in.r.y, r.z + 0.5f * in.r.z,
                                        r.w + 0.5f * in.r.w);
          sum = sel4(odd, so, se);
          if (!ADJ) {
            const int nm = n - 1;
            m = odd ? nm >> 1 : n >> 1;
            put = odd ? (nm >= n0 && nm < n1) : (emit && n == a.NT);
          } else {
            const int np = n + 1;
            m = odd ? np >> 1 : 0;
            put = odd ? (np >= n0 && np < n1) : (emit && n == 0);
          }
        }
        const float4 sc = sel4(m == 0, cwW4, cwt);
        const float4 o = make_float4(0.5f * sc.x * sum.x, 0.5f * sc.y * sum.y, 0.5f * sc.z * sum.z, 0.5f * sc.w * sum.w);
        if (put && owner) *reinterpret_cast<float4*>(a.bc + (size_t)m * a.pc + col) = o;
      }
    }
  };

  Pipe<S> A, B;
#pragma unroll
  for (int k = 0; k <= S; ++k) A.v[k] = f4zero();
#pragma unroll
  for (int k = 0; k <= S + 1; ++k) A.hl[k] = A.hr[k] = 0.f;
  A.r = f4zero();
  A.rp = f4zero();
#pragma unroll
  for (int j = 0; j < kD; ++j) fetch(j);
  int j = 0;
  if (!ADJ && first == 0) {
    // row 0 is a Dirichlet row; row 1 has no coupling to it (its columns are eliminated),
    // so the stage state handed on (values and cached neighbours) stays zero and only the
    // residuals carry over
    row(std::true_type{}, 0, A, B);
    fetch(kD);
    A.r = B.r;
    A.rp = B.rp;
    j = 1;
  }
  const int jend = (ADJ && last == 0) ? count - 1 : count;
  for (; j + 2 <= jend; j += 2) {
    row(std::false_type{}, j, A, B);
    fetch(j + kD);
    row(std::false_type{}, j + 1, B, A);
    fetch(j + 1 + kD);
  }
  if (j < jend) {
    row(std::false_type{}, j, A, B);
    fetch(j + kD);
    A = B;
    ++j;
  }
  if (ADJ && last == 0) row(std::true_type{}, j, A, B);
  cp_wait<0>();
}

template <bool ADJ, int S, int MODE>
cudaError_t launch_k(const StreamArgs& a0, cudaStream_t s) {
  // resident blocks per SM of this instantiation (the same on every device of a process)
  static std::atomic<int> resident{0};
  int nb = resident.load(std::memory_order_relaxed);
  if (nb == 0) {
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_stream<ADJ, S, MODE>, kThreads, 0);
    if (e != cudaSuccess) return e;
    nb = nb < 1 ? 1 : nb;
    resident.store(nb, std::memory_order_relaxed);
  }
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  StreamArgs a = a0;
  stream_layout(a.N, a.NT, (long long)nb * kWarpsPerBlock * sms, a);
  const long long warps = (long long)a.strips * a.chunks;
  const unsigned grid = (unsigned)((warps + kWarpsPerBlock - 1) / kWarpsPerBlock);
  k_stream<ADJ, S, MODE><<<grid, kThreads, 0, s>>>(a);
  return cudaGetLastError();
}

template <bool ADJ, int MODE>
cudaError_t launch_mode(const StreamArgs& a, int S, cudaStream_t s) {
  switch (S) {
    case 1: return launch_k<ADJ, 1, MODE>(a, s);
    case 2: return launch_k<ADJ, 2, MODE>(a, s);
    case 3: return launch_k<ADJ, 3, MODE>(a, s);
    case 4: return launch_k<ADJ, 4, MODE>(a, s);
    case 5: return launch_k<ADJ, 5, MODE>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

void stream_layout(int N, int NT, long long resident_warps, StreamArgs& a) {
  a.strips = (N + 1 + kOwn - 1) / kOwn;
  // one wave: about one chunk per resident warp, chunks of an even number of rows in
  // [4, 1024].  A chunk re-computes S + 1 warm-up rows, which costs little on the large
  // levels (hundreds of rows per chunk) and nothing on the small ones, where short chunks
  // put more of the idle warps to work and shorten the row pipeline each warp runs.
  const long long target = resident_warps < 1 ? 1 : resident_warps;
  long long rows = ((long long)(NT + 1) * a.strips + target - 1) / target;
  rows = rows < 4 ? 4 : (rows > 1024 ? 1024 : rows);
  rows += rows & 1;
  a.rows = (int)rows;
  a.chunks = (NT + 1 + a.rows - 1) / a.rows;
}

cudaError_t launch_stream(int mode, bool adj, int S, const StreamArgs& a, cudaStream_t s) {
  cudaError_t e = cudaErrorInvalidValue;
  switch (mode * 2 + (adj ? 1 : 0)) {
    case 0: e = launch_mode<false, 0>(a, S, s); break;
    case 1: e = launch_mode<true, 0>(a, S, s); break;
    case 2: e = launch_mode<false, 1>(a, S, s); break;
    case 3: e = launch_mode<true, 1>(a, S, s); break;
    case 4: e = launch_mode<false, 2>(a, S, s); break;
    case 5: e = launch_mode<true, 2>(a, S, s); break;
    case 6: e = launch_mode<false, 3>(a, S, s); break;
    case 7: e = launch_mode<true, 3>(a, S, s); break;
    case 8: e = launch_mode<false, 4>(a, S, s); break;
    case 9: e = launch_mode<true, 4>(a, S, s); break;
    case 10: e = launch_mode<false, 5>(a, S, s); break;
    case 11: e = launch_mode<true, 5>(a, S, s); break;
    case 12: e = launch_mode<false, 6>(a, S, s); break;
    case 13: e = launch_mode<true, 6>(a, S, s); break;
    default: break;
  }
  count_launches(1);
  return e;
}

}  // namespace stmg
