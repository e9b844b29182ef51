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
// HBM traffic per DOF of a level (x-coarsening, zero start): DOWN reads b' and writes u
// and b'_c (10 B); UP reads u, b', z and writes u (14 B); the finest-level UP of the
// mixed scheme adds its result straight into the FP64 iterate instead (26 B).
#include "stmg_internal.h"
#include "stmg_stream.h"

namespace stmg {
namespace {

constexpr int kVec = 4;
constexpr int kWin = 32 * kVec;            // columns per warp window
constexpr int kHalo = 8;                   // halo columns on each side
constexpr int kOwn = kWin - 2 * kHalo;     // 112 columns owned per window
constexpr int kWarpsPerBlock = 4;
constexpr int kPF = 3;                     // rows prefetched ahead
constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ float4 f4zero() { return make_float4(0.f, 0.f, 0.f, 0.f); }

__device__ __forceinline__ float4 ld4(const float* __restrict__ p, size_t off, bool ok) {
  return ok ? __ldg(reinterpret_cast<const float4*>(p + off)) : f4zero();
}

// One stage of the pipeline on a lane's 4 columns: out = a*x + b' + sum_k S_k x_k, with
// a = 1 - omega for a sweep and a = -omega for the scaled residual.
__device__ __forceinline__ float4 stage(float a, const float4& x, const float4& px, const float4& b, bool dir_row,
                                        bool has_prev, const float4& sl, const float4& su, const float4& spl,
                                        const float4& spc, const float4& spr) {
  // At the window edges (lanes 0 and 31) the shuffles return the lane's own values: those
  // columns are halo, whose results are never used, and every value stays finite.
  const float xl = __shfl_up_sync(kFull, x.w, 1);
  const float xr = __shfl_down_sync(kFull, x.x, 1);
  const float pl = __shfl_up_sync(kFull, px.w, 1);
  const float pr = __shfl_down_sync(kFull, px.x, 1);
  float4 o;
  o.x = fmaf(a, x.x, b.x);
  o.y = fmaf(a, x.y, b.y);
  o.z = fmaf(a, x.z, b.z);
  o.w = fmaf(a, x.w, b.w);
  if (!dir_row) {
    o.x = fmaf(sl.x, xl, o.x);
    o.x = fmaf(su.x, x.y, o.x);
    o.y = fmaf(sl.y, x.x, o.y);
    o.y = fmaf(su.y, x.z, o.y);
    o.z = fmaf(sl.z, x.y, o.z);
    o.z = fmaf(su.z, x.w, o.z);
    o.w = fmaf(sl.w, x.z, o.w);
    o.w = fmaf(su.w, xr, o.w);
    if (has_prev) {
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
    }
  }
  return o;
}

// MODE: 0 plain sweeps, 1 sweeps + residual + x-restriction, 2 sweeps + residual +
// causal t-restriction, 3 x-prolongation + sweeps, 4 causal t-prolongation + sweeps,
// 5 sweeps + residual + bilinear t-restriction, 6 bilinear t-prolongation + sweeps.
template <bool ADJ, int S, int MODE>
__global__ void __launch_bounds__(32 * kWarpsPerBlock) k_stream(StreamArgs a) {
  const int lane = threadIdx.x & 31;
  const int wid = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
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
  constexpr bool DOWN = MODE == 1 || MODE == 2 || MODE == 5;
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

  const int n0 = chunk * a.rows;
  const int n1 = min(a.NT + 1, n0 + a.rows);
  // rows before the chunk (after it, for J^T) that make every emitted value exact; the
  // bilinear restriction of the chunk's first coarse row also needs fine row n0 - 1
  constexpr int WARM = MODE == 5 ? S + 2 : (DOWN ? S + 1 : S);
  const int first = ADJ ? min(a.NT, n1 - 1 + WARM) : max(0, n0 - WARM);
  const int last = ADJ ? (MODE == 5 ? max(0, n0 - 1) : n0) : n1 - 1;
  const int step = ADJ ? -1 : 1;

  float4 prev[S + 1];
#pragma unroll
  for (int k = 0; k <= S; ++k) prev[k] = f4zero();
  float4 held = f4zero();  // t-restriction: residual of the first row of a pair
  float4 r1 = f4zero(), r2 = f4zero();  // bilinear t-restriction: residuals of the last two rows

  // Loads of the next kPF rows are issued before the current row is computed, so every
  // warp keeps several rows of HBM traffic in flight.
  const int count = ADJ ? first - last + 1 : last - first + 1;
  float4 qb[kPF], qu[kPF], qz[kPF], qzb[kPF];
  float qz2[kPF];
  auto load_row = [&](int k, float4& xb, float4& xu, float4& xz, float& xz2, float4& xzb) {
    const bool ok = k < count;
    const int n = first + k * step;
    const size_t ro = (size_t)n * P;
    xb = ld4(a.bs, ro + col, ok && inside);
    xu = ld4(a.u_in, ro + col, ok && inside && !a.zero_init);
    xz = f4zero();
    xz2 = 0.f;
    if (MODE == 3) {
      const int ca = col / 2;
      if (ok && col >= 0 && ca + 1 < a.pc) {
        const float2 t = __ldg(reinterpret_cast<const float2*>(a.z + (size_t)n * a.pc + ca));
        xz.x = t.x;
        xz.y = t.y;
      }
      if (ok && lane == 31 && col >= 0 && ca + 2 < a.pc) xz2 = a.z[(size_t)n * a.pc + ca + 2];
    } else if (MODE == 4 || MODE == 6) {
      xz = ld4(a.z, (size_t)(n >> 1) * a.pc + col, ok && inside);
    }
    xzb = f4zero();
    if (MODE == 6) xzb = ld4(a.z, (size_t)((n >> 1) + 1) * a.pc + col, ok && inside && (n & 1));
  };
#pragma unroll
  for (int p = 0; p < kPF; ++p) load_row(p, qb[p], qu[p], qz[p], qz2[p], qzb[p]);

  // one row: its loads come from ring slot p, which is then refilled kPF rows ahead
  auto process = [&](const int it, float4& sb, float4& su_, float4& sz, float& sz2, float4& szb) {
    const int n = first + it * step;
    const bool emit = n >= n0 && n < n1;
    const bool dir_row = n == 0;
    const bool has_prev = ADJ ? (n < a.NT) : (n > 1);
    const size_t rowoff = (size_t)n * P;
    const float4 b = sb;
    float4 cur[S + 1];
    cur[0] = su_;
    const float4 zr = sz;
    const float zr2 = sz2;
    const float4 zrb = szb;
    load_row(it + kPF, sb, su_, sz, sz2, szb);
    if (MODE == 3) {
      // x-prolongation: fine 2j <- z_j, fine 2j+1 <- (z_j + z_{j+1}) / 2
      float z2 = __shfl_down_sync(kFull, zr.x, 1);
      if (lane == 31) z2 = zr2;
      if (col + 0 >= 0 && col + 0 <= a.N) cur[0].x += zr.x;
      if (col + 1 >= 0 && col + 1 <= a.N) cur[0].y += 0.5f * (zr.x + zr.y);
      if (col + 2 >= 0 && col + 2 <= a.N) cur[0].z += zr.y;
      if (col + 3 >= 0 && col + 3 <= a.N) cur[0].w += 0.5f * (zr.y + z2);
    } else if (MODE == 4 || MODE == 6) {
      // causal t-prolongation: fine rows 2m and 2m+1 <- coarse row m; bilinear: fine row
      // 2m+1 <- (z_m + z_{m+1}) / 2
      float4 zz = zr;
      if (MODE == 6 && (n & 1))
        zz = make_float4(0.5f * (zr.x + zrb.x), 0.5f * (zr.y + zrb.y), 0.5f * (zr.z + zrb.z), 0.5f * (zr.w + zrb.w));
      if (col + 0 <= a.N) cur[0].x += zz.x;
      if (col + 1 <= a.N) cur[0].y += zz.y;
      if (col + 2 <= a.N) cur[0].z += zz.z;
      if (col + 3 <= a.N) cur[0].w += zz.w;
    }
#pragma unroll
    for (int k = 1; k <= S; ++k) {
      if (k == 1 && a.zero_init) cur[1] = b;  // a sweep from zero is exactly b'
      else cur[k] = stage(a.omc, cur[k - 1], prev[k - 1], b, dir_row, has_prev, sl, su, spl, spc, spr);
    }
    if (emit && owner) {
      if (a.u64) {
        double2* q = reinterpret_cast<double2*>(a.u64 + rowoff + col);
        double2 lo = q[0], hi = q[1];
        lo.x += to_f64(cur[S].x);
        lo.y += to_f64(cur[S].y);
        hi.x += to_f64(cur[S].z);
        hi.y += to_f64(cur[S].w);
        q[0] = lo;
        q[1] = hi;
      } else {
        *reinterpret_cast<float4*>(a.u_out + rowoff + col) = cur[S];
      }
    }
    if (DOWN) {
      // scaled residual y = b' - omega u + sum S_k u_k, r = (D / omega) y
      const float4 y = stage(-a.omega, cur[S], prev[S], b, dir_row, has_prev, sl, su, spl, spc, spr);
      float4 r;
      if (dir_row) {
        r = make_float4(a.Wo * y.x, a.Wo * y.y, a.Wo * y.z, a.Wo * y.w);
      } else {
        r = make_float4(dw.x * y.x, dw.y * y.y, dw.z * y.z, dw.w * y.w);
      }
      if (MODE == 1) {
        float rl = __shfl_up_sync(kFull, r.w, 1);
        if (lane == 0) rl = 0.f;
        if (emit && owner) {
          // b_c[j] = r[2j] + (r[2j-1] + r[2j+1]) / 2, scaled by omega / D_c
          const int j0 = col / 2;
          const float s0 = (n == 0 || j0 == 0) ? a.cwW : cwx.x;
          const float s1 = (n == 0) ? a.cwW : cwx.y;
          float* out = a.bc + (size_t)n * a.pc;
          if (col <= a.N) out[j0] = s0 * (r.x + 0.5f * (rl + r.y));
          if (col + 2 <= a.N) out[j0 + 1] = s1 * (r.z + 0.5f * (r.y + r.w));
        }
      } else if (MODE == 5) {
        // b_c[m] = (r[2m] + (r[2m-1] + r[2m+1]) / 2) / 2 (bilinear P^T with s = 1/2), emitted
        // when the last of the three rows arrives; r1, r2: the two rows before this one
        int m = -1;
        float4 sum = f4zero();
        if (!ADJ) {
          if ((n & 1) && n - 1 >= n0 && n - 1 < n1) {
            m = (n - 1) >> 1;
            const float4 lo = m >= 1 ? r2 : f4zero();
            sum = make_float4(r1.x + 0.5f * (lo.x + r.x), r1.y + 0.5f * (lo.y + r.y), r1.z + 0.5f * (lo.z + r.z),
                              r1.w + 0.5f * (lo.w + r.w));
          } else if (n == a.NT && !(n & 1) && emit) {
            m = n >> 1;
            sum = make_float4(r.x + 0.5f * r1.x, r.y + 0.5f * r1.y, r.z + 0.5f * r1.z, r.w + 0.5f * r1.w);
          }
        } else {
          if ((n & 1) && n + 1 >= n0 && n + 1 < n1) {
            m = (n + 1) >> 1;
            const float4 hi = n + 2 <= a.NT ? r2 : f4zero();
            sum = make_float4(r1.x + 0.5f * (hi.x + r.x), r1.y + 0.5f * (hi.y + r.y), r1.z + 0.5f * (hi.z + r.z),
                              r1.w + 0.5f * (hi.w + r.w));
          } else if (n == 0 && emit) {
            m = 0;
            sum = make_float4(r.x + 0.5f * r1.x, r.y + 0.5f * r1.y, r.z + 0.5f * r1.z, r.w + 0.5f * r1.w);
          }
        }
        if (m >= 0 && owner) {
          float4 sc = cwt;
          if (m == 0) sc = make_float4(a.cwW, a.cwW, a.cwW, a.cwW);
          *reinterpret_cast<float4*>(a.bc + (size_t)m * a.pc + col) =
              make_float4(0.5f * sc.x * sum.x, 0.5f * sc.y * sum.y, 0.5f * sc.z * sum.z, 0.5f * sc.w * sum.w);
        }
        r2 = r1;
        r1 = r;
      } else {
        // b_c[m] = (r[2m] + r[2m+1]) / 2 (causal P^T with s = 1/2), scaled by omega / D_c
        const bool second = ADJ ? (n % 2 == 0) : (n % 2 == 1 || n == a.NT);
        if (second) {
          float4 sum = r;
          if (ADJ ? (n + 1 <= a.NT) : (n % 2 == 1)) {
            sum.x += held.x;
            sum.y += held.y;
            sum.z += held.z;
            sum.w += held.w;
          }
          if (emit && owner) {
            const int m = n >> 1;
            float4 sc = cwt;
            if (m == 0) sc = make_float4(a.cwW, a.cwW, a.cwW, a.cwW);
            float4 o = make_float4(0.5f * sc.x * sum.x, 0.5f * sc.y * sum.y, 0.5f * sc.z * sum.z,
                                   0.5f * sc.w * sum.w);
            *reinterpret_cast<float4*>(a.bc + (size_t)m * a.pc + col) = o;
          }
          held = f4zero();
        } else {
          held = r;
        }
      }
    }
#pragma unroll
    for (int k = 0; k <= S; ++k) prev[k] = cur[k];
  };
  for (int it = 0; it < count; it += kPF) {
#pragma unroll
    for (int p = 0; p < kPF; ++p)
      if (it + p < count) process(it + p, qb[p], qu[p], qz[p], qz2[p], qzb[p]);
  }
}

template <bool ADJ, int MODE>
cudaError_t launch_mode(const StreamArgs& a, int S, unsigned grid, cudaStream_t s) {
  switch (S) {
    case 1: k_stream<ADJ, 1, MODE><<<grid, 32 * kWarpsPerBlock, 0, s>>>(a); break;
    case 2: k_stream<ADJ, 2, MODE><<<grid, 32 * kWarpsPerBlock, 0, s>>>(a); break;
    case 3: k_stream<ADJ, 3, MODE><<<grid, 32 * kWarpsPerBlock, 0, s>>>(a); break;
    case 4: k_stream<ADJ, 4, MODE><<<grid, 32 * kWarpsPerBlock, 0, s>>>(a); break;
    case 5: k_stream<ADJ, 5, MODE><<<grid, 32 * kWarpsPerBlock, 0, s>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace

void stream_layout(int N, int NT, StreamArgs& a) {
  a.strips = (N + 1 + kOwn - 1) / kOwn;
  // about 24 warps per SM on 152 SMs, chunks of an even number of rows in [16, 256]
  const long long target = 152LL * 24;
  long long rows = ((long long)(NT + 1) * a.strips + target - 1) / target;
  rows = rows < 16 ? 16 : (rows > 256 ? 256 : rows);
  rows += rows & 1;
  a.rows = (int)rows;
  a.chunks = (NT + 1 + a.rows - 1) / a.rows;
}

cudaError_t launch_stream(int mode, bool adj, int S, const StreamArgs& a, cudaStream_t s) {
  const long long warps = (long long)a.strips * a.chunks;
  const unsigned grid = (unsigned)((warps + kWarpsPerBlock - 1) / kWarpsPerBlock);
  cudaError_t e = cudaErrorInvalidValue;
  switch (mode * 2 + (adj ? 1 : 0)) {
    case 0: e = launch_mode<false, 0>(a, S, grid, s); break;
    case 1: e = launch_mode<true, 0>(a, S, grid, s); break;
    case 2: e = launch_mode<false, 1>(a, S, grid, s); break;
    case 3: e = launch_mode<true, 1>(a, S, grid, s); break;
    case 4: e = launch_mode<false, 2>(a, S, grid, s); break;
    case 5: e = launch_mode<true, 2>(a, S, grid, s); break;
    case 6: e = launch_mode<false, 3>(a, S, grid, s); break;
    case 7: e = launch_mode<true, 3>(a, S, grid, s); break;
    case 8: e = launch_mode<false, 4>(a, S, grid, s); break;
    case 9: e = launch_mode<true, 4>(a, S, grid, s); break;
    case 10: e = launch_mode<false, 5>(a, S, grid, s); break;
    case 11: e = launch_mode<true, 5>(a, S, grid, s); break;
    case 12: e = launch_mode<false, 6>(a, S, grid, s); break;
    case 13: e = launch_mode<true, 6>(a, S, grid, s); break;
    default: break;
  }
  count_launches(1);
  return e;
}

}  // namespace stmg
