// stmg_stream.cu -- the fused FP32 passes (kernel in stmg_stream_impl.cuh): work layout,
// the mode dispatch, and the plain and UP passes.  The DOWN passes are instantiated in
// stmg_stream_down.cu, so that the two halves compile in parallel.
#include "stmg_stream_impl.cuh"

namespace stmg {

void stream_layout(int N, int NT, int own, long long resident_warps, StreamArgs& a) {
  a.strips = (N + 1 + own - 1) / own;
  // one wave: about one chunk per resident warp, chunks of an even number of rows in
  // [2, 1024] (even: a t-restriction pairs rows 2m and 2m + 1 within one chunk).  A chunk
  // re-computes S + 1 warm-up rows, which costs little on the large levels (hundreds of
  // rows per chunk) and nothing on the small ones, where short chunks put more of the idle
  // warps to work and shorten the row pipeline each warp runs (2-row chunks: 0.4 % off the
  // mixed 4096 x 16384 solve against 4-row ones).
  const long long target = resident_warps < 1 ? 1 : resident_warps;
  long long rows = ((long long)(NT + 1) * a.strips + target - 1) / target;
  rows = rows < 2 ? 2 : (rows > 1024 ? 1024 : rows);
  rows += rows & 1;
  a.rows = (int)rows;
  a.chunks = (NT + 1 + a.rows - 1) / a.rows;
}

cudaError_t launch_stream(int mode, bool adj, int S, const StreamArgs& a, cudaStream_t s) {
  cudaError_t e = cudaErrorInvalidValue;
  switch (mode * 2 + (adj ? 1 : 0)) {
    case 0: e = launch_mode<false, 0>(a, S, s); break;
    case 1: e = launch_mode<true, 0>(a, S, s); break;
    case 2:
    case 3:
    case 4:
    case 5:
    case 10:
    case 11: e = launch_stream_down(mode, adj, S, a, s); break;  // the DOWN modes
    case 6: e = launch_mode<false, 3>(a, S, s); break;
    case 7: e = launch_mode<true, 3>(a, S, s); break;
    case 8: e = launch_mode<false, 4>(a, S, s); break;
    case 9: e = launch_mode<true, 4>(a, S, s); break;
    case 12: e = launch_mode<false, 6>(a, S, s); break;
    case 13: e = launch_mode<true, 6>(a, S, s); break;
    default: break;
  }
  count_launches(1);
  return e;
}

}  // namespace stmg
