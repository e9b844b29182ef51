// stmg_stream_down.cu -- the DOWN passes (sweeps + residual + restriction) of the fused
// FP32 V-cycle; kernel in stmg_stream_impl.cuh, dispatch in stmg_stream.cu.
#include "stmg_stream_impl.cuh"

namespace stmg {

cudaError_t launch_stream_down(int mode, bool adj, int S, const StreamArgs& a, cudaStream_t s) {
  switch (mode * 2 + (adj ? 1 : 0)) {
    case 2: return launch_mode<false, kStreamDownX>(a, S, s);
    case 3: return launch_mode<true, kStreamDownX>(a, S, s);
    case 4: return launch_mode<false, kStreamDownT>(a, S, s);
    case 5: return launch_mode<true, kStreamDownT>(a, S, s);
    case 10: return launch_mode<false, kStreamDownTB>(a, S, s);
    case 11: return launch_mode<true, kStreamDownTB>(a, S, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace stmg
