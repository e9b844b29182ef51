// stmg_stream_impl.cuh -- fused FP32 passes of the V-cycle for the mixed-precision scheme:
// the pass kernel and its launcher, instantiated by stmg_stream.cu (plain and UP passes) and
// stmg_stream_down.cu (DOWN passes).
//
// One warp owns a window of 32 * kVec columns (kVec per lane: 8 in the DOWN passes, 4 in
// the others) of one level and marches
// through a chunk of time rows.  Because the space-time stencil couples row n only to
// rows n and n-1 (n+1 for the adjoint), S damped-Jacobi sweeps (Sec. 3.1) are a pipeline
// over rows: sweep k of row n needs sweep k-1 of rows n and n-1, so a warp keeps the
// previous row of every stage in registers and produces all S sweeps of a row as soon as
// the row is read.  The same pipeline then evaluates the residual and restricts it
// (Sec. 3.1, R = s P^T) to the coarse level (DOWN pass), or adds the prolongated coarse
// correction before sweeping (UP pass).  x-neighbours come from warp shuffles; the window
// carries an 8-column halo on each side and a chunk starts S(+1) rows early, so every output
// value is computed from exact inputs with no block-level synchronisation.
//
// A row's inputs (b', the starting iterate, the coarse correction, the FP64 iterate) are
// staged through a per-warp ring of rows in shared memory, filled by asynchronous copies
// several rows ahead, so the loads in flight cost no registers.  The row loop has no
// data-dependent branches: the Dirichlet row 0 is peeled off, rows alternate between two
// register sets of pipeline state, and every row-dependent choice is a select or a
// predicated store.  Each lane holds kVec consecutive columns, so the per-row bookkeeping
// (ring, predicates, addresses, shuffles) is spread over that many DOFs.
//
// A pass runs S sweeps: up to 5 in a DOWN pass (plus the residual and the restriction) and
// up to 8 in a plain or UP pass, as far as the 8-column halo keeps the owned columns exact;
// more smoothing steps take several passes, each reading and writing the level once.
//
// HBM traffic per DOF of a level (x-coarsening, zero start): DOWN reads b' and writes u
// and b'_c (10 B); UP reads u, b', z and writes u (14 B); the finest-level UP of the
// mixed scheme adds its result straight into the FP64 iterate instead (26 B).
#pragma once
#include <atomic>
#include <type_traits>

#include "stmg_internal.h"
#include "stmg_stream.h"

namespace stmg {
namespace {


constexpr unsigned kFull = 0xffffffffu;

// Columns per lane by pass: the DOWN passes (issue-bound) hold 8, which halves their
// per-DOF bookkeeping and halo overhead; the UP and plain passes (latency-bound, with more
// streams and the FP64 accumulate) hold 4, which keeps twice as many warps resident.
template <int MODE>
struct Width {
  static constexpr bool kDown = MODE == 1 || MODE == 2 || MODE == 5;
  static constexpr int kVec = kDown ? 8 : 4;          // columns per lane
  static constexpr int kWarpsPerBlock = kDown ? 2 : 4;
  static constexpr int kThreads = 32 * kWarpsPerBlock;
  static constexpr int kMinBlocks = kDown ? 1 : 4;    // 4-column passes: <= 128 registers
  static constexpr int kHalo = 8;                     // halo columns on each side
  static constexpr int kOwn = 32 * kVec - 2 * kHalo;  // columns owned per window
  // A DOWN pass's S <= 5 sweeps and the residual spoil at most 6 columns from each window
  // edge, and the x-restriction reads one more; the S sweeps of a plain or UP pass spoil S
  // columns (the prolongation is exact across the whole window).  The halo must cover 7
  // and 8, and be whole lanes.
  static constexpr int kMaxS = kDown ? 5 : 8;
  static_assert(kHalo >= 7 && kHalo >= kMaxS && kHalo % kVec == 0, "halo must cover the spoiled columns in whole lanes");
};

// Resident blocks per SM the compiler plans registers for: more than 5 sweeps in a 4-column
// pass hold more pipeline state than 128 registers.
template <int MODE, int S>
struct MinBlocks {
  static constexpr int value = Width<MODE>::kDown ? Width<MODE>::kMinBlocks : (S <= 5 ? Width<MODE>::kMinBlocks : 3);
};

template <int V>
struct Vf {
  static_assert(V % 4 == 0, "lanes hold whole float4");
  float e[V];
};

template <int V>
__device__ __forceinline__ Vf<V> vzero() {
  Vf<V> v;
#pragma unroll
  for (int j = 0; j < V; ++j) v.e[j] = 0.f;
  return v;
}

template <int V>
__device__ __forceinline__ Vf<V> ldv(const float* __restrict__ p, size_t off, bool ok) {
  Vf<V> v;
#pragma unroll
  for (int q = 0; q < V / 4; ++q) {
    const float4 t = ok ? __ldg(reinterpret_cast<const float4*>(p + off) + q) : make_float4(0.f, 0.f, 0.f, 0.f);
    v.e[4 * q] = t.x;
    v.e[4 * q + 1] = t.y;
    v.e[4 * q + 2] = t.z;
    v.e[4 * q + 3] = t.w;
  }
  return v;
}

// V floats of lane `lane` from field `f` (V / 4 float4 wide) of a ring slot.
template <int V>
__device__ __forceinline__ Vf<V> lds_v(const float4* slot, int f, int lane) {
  Vf<V> v;
#pragma unroll
  for (int q = 0; q < V / 4; ++q) {
    const float4 t = slot[(f + q) * 32 + lane];
    v.e[4 * q] = t.x;
    v.e[4 * q + 1] = t.y;
    v.e[4 * q + 2] = t.z;
    v.e[4 * q + 3] = t.w;
  }
  return v;
}

template <int V>
__device__ __forceinline__ void stg_v(float* p, const Vf<V>& v) {
#pragma unroll
  for (int q = 0; q < V / 4; ++q)
    reinterpret_cast<float4*>(p)[q] = make_float4(v.e[4 * q], v.e[4 * q + 1], v.e[4 * q + 2], v.e[4 * q + 3]);
}

// Columns 2q, 2q+1 of a lane's vector as a pair (for packed FP32 arithmetic) and back.
template <int V>
__device__ __forceinline__ float2 pair(const Vf<V>& v, int q) {
  return make_float2(v.e[2 * q], v.e[2 * q + 1]);
}
template <int V>
__device__ __forceinline__ void set_pair(Vf<V>& v, int q, float2 t) {
  v.e[2 * q] = t.x;
  v.e[2 * q + 1] = t.y;
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

// The lane's columns of the five scaled neighbour coefficients -omega c_k / D.
template <int V>
struct Coefs {
  Vf<V> sl, su, spl, spc, spr;
};

// One stage of the pipeline on a lane's columns: out = a*x + b' + sum_k S_k x_k, with
// a = 1 - omega for a sweep and a = -omega for the scaled residual.  DIR: a Dirichlet row
// (time level 0), whose row of J is W_Diri I.  px is the stage input of the previous row
// (the next row for J^T), zero where the stencil has no such coupling; pl, pr are its
// x-neighbours across the lane boundary, which that row's own stage shuffled and handed on.
// hl, hr receive this row's shuffled neighbours of x for the next row.  The two terms whose
// operands are column-aligned (a x + b' and the previous row's centre) run as packed FP32
// pairs, one instruction for two columns; the four shifted-neighbour terms stay scalar.
template <bool DIR, int V>
__device__ __forceinline__ Vf<V> stage(float a, const Vf<V>& x, const Vf<V>& px, float pl, float pr, float& hl,
                                       float& hr, const Vf<V>& b, const Coefs<V>& cf) {
  Vf<V> o;
  const float2 a2 = make_float2(a, a);
#pragma unroll
  for (int q = 0; q < V / 2; ++q) {
    const float2 t = __ffma2_rn(a2, make_float2(x.e[2 * q], x.e[2 * q + 1]), make_float2(b.e[2 * q], b.e[2 * q + 1]));
    o.e[2 * q] = t.x;
    o.e[2 * q + 1] = t.y;
  }
  if (DIR) {
    hl = 0.f;
    hr = 0.f;
    return o;
  }
  // At the window edges (lanes 0 and 31) the shuffles return the lane's own values: those
  // columns are halo, whose results are never used, and every value stays finite.
  const float xl = __shfl_up_sync(kFull, x.e[V - 1], 1);
  const float xr = __shfl_down_sync(kFull, x.e[0], 1);
  hl = xl;
  hr = xr;
#pragma unroll
  for (int q = 0; q < V / 2; ++q) {
    const float2 c = __ffma2_rn(make_float2(cf.spc.e[2 * q], cf.spc.e[2 * q + 1]),
                                make_float2(px.e[2 * q], px.e[2 * q + 1]), make_float2(o.e[2 * q], o.e[2 * q + 1]));
    o.e[2 * q] = c.x;
    o.e[2 * q + 1] = c.y;
  }
#pragma unroll
  for (int j = 0; j < V; ++j) {
    const float left = j == 0 ? xl : x.e[j - 1];
    const float right = j == V - 1 ? xr : x.e[j + 1];
    const float pleft = j == 0 ? pl : px.e[j - 1];
    const float pright = j == V - 1 ? pr : px.e[j + 1];
    float t = fmaf(cf.sl.e[j], left, o.e[j]);
    t = fmaf(cf.su.e[j], right, t);
    t = fmaf(cf.spl.e[j], pleft, t);
    o.e[j] = fmaf(cf.spr.e[j], pright, t);
  }
  return o;
}

// Fields of one ring slot, kQ float4 per lane each (the FP64 iterate: 2 kQ): b', the
// starting iterate, the coarse correction rows (UP), the FP64 iterate (UP and plain passes
// that add into it; NO64: none of them does, and the slot ends before that field).
template <int MODE, bool NO64>
struct Ring {
  static constexpr bool kDown = Width<MODE>::kDown;
  static constexpr int kQ = Width<MODE>::kVec / 4;
  static constexpr bool kHasZ = MODE == 3 || MODE == 4 || MODE == 6;
  static constexpr int kB = 0, kU = kQ, kZ = 2 * kQ, kZB = 3 * kQ;
  static constexpr int k64 = kDown ? 0 : (MODE == 6 ? 4 * kQ : (kHasZ ? 3 * kQ : 2 * kQ));
  static constexpr int kWidth = kDown ? 2 * kQ : (NO64 ? k64 : k64 + 2 * kQ);  // float4 per lane and slot
  static constexpr int kDepth = 4;                               // rows in flight per warp
};

// Pipeline state after one row: v[0] the row's starting iterate (plus the prolongated
// correction), v[k] the row after sweep k; hl[k], hr[k] the neighbours of v[k-1] across the
// lane boundary that stage k shuffled (k = S + 1: the residual stage); r, rp the residuals
// of this row and the one before it (restriction modes).
template <int S, int V>
struct Pipe {
  Vf<V> v[S + 1];
  float hl[S + 2], hr[S + 2];
  Vf<V> r, rp;
};

// MODE: 0 plain sweeps, 1 sweeps + residual + x-restriction, 2 sweeps + residual +
// causal t-restriction, 3 x-prolongation + sweeps, 4 causal t-prolongation + sweeps,
// 5 sweeps + residual + bilinear t-restriction, 6 bilinear t-prolongation + sweeps.
// FORM: which of the pass's run-time choices are fixed when it is compiled, so that the row
// loop carries no branch on them.
//   kGeneral  both choices at run time (zero start, FP64 accumulate);
//   kLean     one input stream fewer: a DOWN pass from a zero iterate (stages no iterate
//             rows, holds less state: 166 registers instead of 196, 12 warps per SM instead
//             of 8), or a plain or UP pass that does not add into the FP64 iterate (stages
//             no FP64 rows, a ring slot of 3 fields instead of 5; mixed 4096 x 16384 solve
//             14.75 -> 14.53 ms);
//   kContinue a DOWN pass from the iterate in memory (14.50 -> 14.41 ms).
enum { kGeneral = 0, kLean = 1, kContinue = 2 };
template <bool ADJ, int S, int MODE, int FORM>
__global__ void __launch_bounds__(Width<MODE>::kThreads, MinBlocks<MODE, S>::value) k_stream(StreamArgs a) {
  static_assert(S >= 1 && S <= Width<MODE>::kMaxS, "sweeps per pass");
  using R = Ring<MODE, !Width<MODE>::kDown && FORM == kLean>;
  using Wd = Width<MODE>;
  constexpr int kVec = Wd::kVec;
  constexpr int kQ = kVec / 4;
  constexpr int kHalo = Wd::kHalo;
  constexpr int kOwn = Wd::kOwn;
  constexpr int kWarpsPerBlock = Wd::kWarpsPerBlock;
  using V = Vf<kVec>;
  constexpr bool DOWN = R::kDown;
  const bool zero_init = (DOWN && FORM == kLean) || (FORM != kContinue && a.zero_init != 0);
  const bool add64 = !DOWN && FORM == kGeneral && a.u64 != nullptr;  // add the result into the FP64 iterate
  constexpr int kD = R::kDepth;
  constexpr int kSlot = R::kWidth * 32;  // float4 per slot
  __shared__ float4 ring[kWarpsPerBlock * kD * kSlot];

  const int lane = threadIdx.x & 31;
  const int w = threadIdx.x >> 5;
  const int wid = blockIdx.x * kWarpsPerBlock + w;
  if (wid >= a.strips * a.chunks) return;  // the whole warp leaves together
  const int strip = wid % a.strips;
  const int chunk = wid / a.strips;
  const int c0 = strip * kOwn - kHalo;
  const int col = c0 + kVec * lane;  // multiple of kVec; either fully inside [0, pitch) or fully outside
  const bool inside = col >= 0 && col + kVec <= a.pitch;
  const bool owner = lane >= kHalo / kVec && lane < (kHalo + kOwn) / kVec && inside;
  const int P = a.pitch;
  float4* wring = ring + (size_t)w * kD * kSlot;

  Coefs<kVec> cf;
  cf.sl = ldv<kVec>(a.coef, (size_t)kSL * P + col, inside);
  cf.su = ldv<kVec>(a.coef, (size_t)kSU * P + col, inside);
  cf.spl = ldv<kVec>(a.coef, (size_t)kSPL * P + col, inside);
  cf.spc = ldv<kVec>(a.coef, (size_t)kSPC * P + col, inside);
  cf.spr = ldv<kVec>(a.coef, (size_t)kSPR * P + col, inside);
  V dw = vzero<kVec>();
  if (DOWN) dw = ldv<kVec>(a.coef, (size_t)kDW * P + col, inside);
  // coarse scaling of the restricted residual: x: coarse nodes col/2 .. col/2 + kVec/2 - 1
  // (node 0 is a Dirichlet node); t: coarse node = fine node (row 0: Dirichlet rows)
  constexpr int kH = kVec / 2;
  float cwx[kH];
  const int ca = col / 2;
#pragma unroll
  for (int q = 0; q < kH; ++q) {
    cwx[q] = 0.f;
    if (MODE == 1 && inside && ca + q < a.pc) cwx[q] = ca + q == 0 ? a.cwW : a.ccoef[(size_t)kW * a.pc + ca + q];
  }
  V cwt = vzero<kVec>();
  if (MODE == 2 || MODE == 5) cwt = ldv<kVec>(a.ccoef, (size_t)kW * a.pc + col, inside);
  // prolongation only touches nodes 0..N
  V pm;
#pragma unroll
  for (int j = 0; j < kVec; ++j) pm.e[j] = col + j >= 0 && col + j <= a.N ? 1.f : 0.f;

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
    float4* slot = wring + (j % kD) * kSlot;
    const size_t ro = (size_t)n * P + col;
#pragma unroll
    for (int q = 0; q < kQ; ++q) cp_async<16>(slot + (R::kB + q) * 32 + lane, a.bs, ro + 4 * q, a.bs, ok && inside);
    if (!zero_init) {
#pragma unroll
      for (int q = 0; q < kQ; ++q)
        cp_async<16>(slot + (R::kU + q) * 32 + lane, a.u_in, ro + 4 * q, a.bs, ok && inside);
    }
    if (MODE == 3) {
      // coarse nodes ca .. ca + kVec/2 - 1 of row n; lane 31 also takes node ca + kVec/2
      const size_t zo = (size_t)n * a.pc + ca;
      const bool zok = ok && col >= 0 && ca + kH <= a.pc;
      if (kH == 4) cp_async<16>(slot + R::kZ * 32 + lane, a.z, zo, a.bs, zok);
      else cp_async<8>(slot + R::kZ * 32 + lane, a.z, zo, a.bs, zok);
      if (lane == 31) {
        float* extra = reinterpret_cast<float*>(slot + (R::kZ + kH / 4) * 32 + lane) + kH % 4;
        cp_async<4>(extra, a.z, zo + kH, a.bs, ok && col >= 0 && ca + kH < a.pc);
      }
    } else if (MODE == 4 || MODE == 6) {
#pragma unroll
      for (int q = 0; q < kQ; ++q)
        cp_async<16>(slot + (R::kZ + q) * 32 + lane, a.z, (size_t)(n >> 1) * a.pc + col + 4 * q, a.bs, ok && inside);
    }
    if (MODE == 6) {
#pragma unroll
      for (int q = 0; q < kQ; ++q)
        cp_async<16>(slot + (R::kZB + q) * 32 + lane, a.z, (size_t)((n >> 1) + 1) * a.pc + col + 4 * q, a.bs,
                     ok && inside && (n & 1));
    }
    if (add64) {
#pragma unroll
      for (int q = 0; q < 2 * kQ; ++q) cp_async<16>(slot + (R::k64 + q) * 32 + lane, a.u64, ro + 2 * q, a.bs, ok && inside);
    }
    cp_commit();
  };

  // One row: consume its ring slot, sweep, store, restrict.
  int ku = 0;  // exponent of the scale of the FP64 accumulate (set after pdl_wait)
  auto row = [&](auto dir_tag, const int j, const Pipe<S, kVec>& in, Pipe<S, kVec>& out) {
    constexpr bool DIR = decltype(dir_tag)::value;
    const int n = first + j * step;
    const bool emit = n >= n0 && n < n1;
    const float4* slot = wring + (j % kD) * kSlot;
    cp_wait<kD - 1>();
    const V b = lds_v<kVec>(slot, R::kB, lane);
    V x = zero_init ? vzero<kVec>() : lds_v<kVec>(slot, R::kU, lane);
    if (MODE == 3) {
      // x-prolongation: fine 2q <- z_q, fine 2q+1 <- (z_q + z_{q+1}) / 2 (coarse node q of the lane)
      const float* zs = reinterpret_cast<const float*>(slot + R::kZ * 32 + lane);
      float zc[kH + 1];
#pragma unroll
      for (int q = 0; q < kH; ++q) zc[q] = zs[q];
      const float* zx = reinterpret_cast<const float*>(slot + (R::kZ + kH / 4) * 32 + lane) + kH % 4;
      const float zn = __shfl_down_sync(kFull, zc[0], 1);
      zc[kH] = lane == 31 ? *zx : zn;
#pragma unroll
      for (int q = 0; q < kH; ++q) {
        x.e[2 * q] = fmaf(pm.e[2 * q], zc[q], x.e[2 * q]);
        x.e[2 * q + 1] = fmaf(pm.e[2 * q + 1], 0.5f * (zc[q] + zc[q + 1]), x.e[2 * q + 1]);
      }
    } else if (MODE == 4 || MODE == 6) {
      // causal t-prolongation: fine rows 2m and 2m+1 <- coarse row m; bilinear: fine row
      // 2m+1 <- (z_m + z_{m+1}) / 2
      V zz = lds_v<kVec>(slot, R::kZ, lane);
      if (MODE == 6) {
        const V zb = lds_v<kVec>(slot, R::kZB, lane);
        const bool odd = n & 1;
#pragma unroll
        for (int q = 0; q < kVec / 2; ++q)
          set_pair(zz, q, odd ? __fmul2_rn(make_float2(0.5f, 0.5f), __fadd2_rn(pair(zz, q), pair(zb, q))) : pair(zz, q));
      }
#pragma unroll
      for (int q = 0; q < kVec / 2; ++q) set_pair(x, q, __ffma2_rn(pair(pm, q), pair(zz, q), pair(x, q)));
    }
    out.v[0] = x;
#pragma unroll
    for (int k = 1; k <= S; ++k) {
      if (k == 1 && zero_init) out.v[1] = b;  // a sweep from zero is exactly b'
      else
        out.v[k] = stage<DIR>(a.omc, out.v[k - 1], in.v[k - 1], in.hl[k], in.hr[k], out.hl[k], out.hr[k], b, cf);
    }
    if (add64) {
      double2 acc[kVec / 2];
#pragma unroll
      for (int q = 0; q < kVec / 2; ++q) {
        acc[q] = *reinterpret_cast<const double2*>(slot + (R::k64 + q) * 32 + lane);
        acc[q].x += to_f64(out.v[S].e[2 * q], ku);
        acc[q].y += to_f64(out.v[S].e[2 * q + 1], ku);
      }
      if (emit && owner) {
        double2* dst = reinterpret_cast<double2*>(a.u64 + (size_t)n * P + col);
#pragma unroll
        for (int q = 0; q < kVec / 2; ++q) dst[q] = acc[q];
      }
    } else if (emit && owner) {
      stg_v(a.u_out + (size_t)n * P + col, out.v[S]);
    }
    if (DOWN) {
      // scaled residual y = b' - omega u + sum S_k u_k, r = (D / omega) y
      const V y =
          stage<DIR>(-a.omega, out.v[S], in.v[S], in.hl[S + 1], in.hr[S + 1], out.hl[S + 1], out.hr[S + 1], b, cf);
      V r;
#pragma unroll
      for (int q = 0; q < kVec / 2; ++q)
        set_pair(r, q, __fmul2_rn(DIR ? make_float2(a.Wo, a.Wo) : pair(dw, q), pair(y, q)));
      out.r = r;
      if (MODE == 5) out.rp = in.r;
      if (MODE == 1) {
        // b_c[j] = r[2j] + (r[2j-1] + r[2j+1]) / 2, scaled by omega / D_c
        const float rl = __shfl_up_sync(kFull, r.e[kVec - 1], 1);
        float* dst = a.bc + (size_t)n * a.pc + ca;
#pragma unroll
        for (int q = 0; q < kH; ++q) {
          const float left = q == 0 ? rl : r.e[2 * q - 1];
          const float s = DIR ? a.cwW : cwx[q];
          const float o = s * (r.e[2 * q] + 0.5f * (left + r.e[2 * q + 1]));
          if (emit && owner && col + 2 * q <= a.N) dst[q] = o;
        }
      } else {
        V sum;
        int m;
        bool put;
        const bool odd = n & 1;
        if (MODE == 2) {
          // b_c[m] = (r[2m] + r[2m+1]) / 2 (causal P^T with s = 1/2); forward: emitted at
          // row 2m+1 (row NT alone when NT is even); J^T: emitted at row 2m
#pragma unroll
          for (int q = 0; q < kVec / 2; ++q)
            set_pair(sum, q, (ADJ || odd) ? __fadd2_rn(pair(r, q), pair(in.r, q)) : pair(r, q));
          put = ADJ ? (emit && !odd) : (emit && (odd || n == a.NT));
          m = n >> 1;
        } else {
          // b_c[m] = (r[2m] + (r[2m-1] + r[2m+1]) / 2) / 2 (bilinear P^T with s = 1/2),
          // emitted when the last of its three fine rows has been processed
#pragma unroll
          for (int q = 0; q < kVec / 2; ++q)
            set_pair(sum, q, odd ? __ffma2_rn(make_float2(0.5f, 0.5f), __fadd2_rn(pair(in.rp, q), pair(r, q)), pair(in.r, q))
                            : __ffma2_rn(make_float2(0.5f, 0.5f), pair(in.r, q), pair(r, q)));
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
        V o;
#pragma unroll
        for (int q = 0; q < kVec / 2; ++q)
          set_pair(o, q, __fmul2_rn(__fmul2_rn(make_float2(0.5f, 0.5f), m == 0 ? make_float2(a.cwW, a.cwW) : pair(cwt, q)),
                               pair(sum, q)));
        if (put && owner) stg_v(a.bc + (size_t)m * a.pc + col, o);
      }
    }
  };

  Pipe<S, kVec> A, B;
#pragma unroll
  for (int k = 0; k <= S; ++k) A.v[k] = vzero<kVec>();
#pragma unroll
  for (int k = 0; k <= S + 1; ++k) A.hl[k] = A.hr[k] = 0.f;
  A.r = vzero<kVec>();
  A.rp = vzero<kVec>();
  // Everything above reads only the level's coefficients, fixed since the hierarchy was
  // built.  The rows come from the kernels before this one: wait for them (a no-op unless
  // this grid was launched ahead of its predecessor's end) and let the next pass launch.
  pdl_wait();
  if (add64) ku = -scale_exp(a.kexp);
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

template <bool ADJ, int S, int MODE, int FORM>
cudaError_t launch_form(const StreamArgs& a0, cudaStream_t s) {
  // resident blocks per SM of this instantiation (the same on every device of a process)
  static std::atomic<int> resident{0};
  int nb = resident.load(std::memory_order_relaxed);
  if (nb == 0) {
    cudaError_t e =
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_stream<ADJ, S, MODE, FORM>, Width<MODE>::kThreads, 0);
    if (e != cudaSuccess) return e;
    nb = nb < 1 ? 1 : nb;
    resident.store(nb, std::memory_order_relaxed);
  }
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  StreamArgs a = a0;
  constexpr int wpb = Width<MODE>::kWarpsPerBlock;
  stream_layout(a.N, a.NT, Width<MODE>::kOwn, (long long)nb * wpb * sms, a);
  const long long warps = (long long)a.strips * a.chunks;
  const unsigned grid = (unsigned)((warps + wpb - 1) / wpb);
  // programmatic dependent launch: the pass may start (and load its coefficients) while the
  // previous kernel of the stream drains; it waits for that kernel before touching any row
  return launch_pdl(k_stream<ADJ, S, MODE, FORM>, dim3(grid), dim3(Width<MODE>::kThreads), s, a);
}

// Levels of at least this many DOFs take the DOWN kernel that holds the iterate state even
// from a zero start: they stream best at its 8 warps per SM (the zero-start kernel's 12 took
// the finest level of the 4096 x 16384 workload 155 us instead of 145), while the passes of
// the smaller levels gain from the zero-start kernel's fewer instructions and more warps.
constexpr long long kZeroStartMaxDofs = 1ll << 23;

template <bool ADJ, int S, int MODE>
cudaError_t launch_k(const StreamArgs& a, cudaStream_t s) {
  if constexpr (Width<MODE>::kDown) {
    if (!a.zero_init) return launch_form<ADJ, S, MODE, kContinue>(a, s);
    if ((long long)(a.N + 1) * (a.NT + 1) < kZeroStartMaxDofs) return launch_form<ADJ, S, MODE, kLean>(a, s);
  } else {
    if (a.u64 == nullptr) return launch_form<ADJ, S, MODE, kLean>(a, s);
  }
  return launch_form<ADJ, S, MODE, kGeneral>(a, s);
}

template <bool ADJ, int MODE>
cudaError_t launch_mode(const StreamArgs& a, int S, cudaStream_t s) {
  switch (S) {
    case 1: return launch_k<ADJ, 1, MODE>(a, s);
    case 2: return launch_k<ADJ, 2, MODE>(a, s);
    case 3: return launch_k<ADJ, 3, MODE>(a, s);
    case 4: return launch_k<ADJ, 4, MODE>(a, s);
    case 5: return launch_k<ADJ, 5, MODE>(a, s);
    default: break;
  }
  if constexpr (!Width<MODE>::kDown) {
    switch (S) {
      case 6: return launch_k<ADJ, 6, MODE>(a, s);
      case 7: return launch_k<ADJ, 7, MODE>(a, s);
      case 8: return launch_k<ADJ, 8, MODE>(a, s);
      default: break;
    }
  }
  return cudaErrorInvalidValue;
}

}  // namespace
}  // namespace stmg
