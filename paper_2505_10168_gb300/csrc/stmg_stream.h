// stmg_stream.h -- fused FP32 V-cycle passes (stmg_stream.cu).
#pragma once
#include <cuda_runtime.h>

namespace stmg {

enum StreamMode {
  kStreamPlain = 0,
  kStreamDownX = 1,   // + residual + x-restriction
  kStreamDownT = 2,   // + residual + causal t-restriction
  kStreamUpX = 3,     // x-prolongation first
  kStreamUpT = 4,     // causal t-prolongation first
  kStreamDownTB = 5,  // + residual + bilinear t-restriction
  kStreamUpTB = 6     // bilinear t-prolongation first
};

struct StreamArgs {
  // this level (FP32 arrays in the padded layout of stmg_internal.h)
  int N, NT, pitch;
  float omega, omc, Wo;    // omega, 1 - omega, W_Diri / omega
  const float* coef;       // kNumCoef * pitch
  const float* u_in;       // starting iterate (ignored when zero_init)
  const float* bs;         // scaled right-hand side b'
  float* u_out;            // result, or nullptr when u64 is set
  double* u64;             // finest level of the mixed scheme: u64 += result 2^-k
  const int* kexp;         // k (see scale_exp), read with u64
  int zero_init;           // the starting iterate is 0
  // coarse level: restriction target (DOWN) or correction source (UP)
  int pc;                  // coarse pitch
  const float* ccoef;      // coarse coefficients (DOWN)
  float cwW;               // coarse omega / W_Diri (DOWN)
  float* bc;               // coarse scaled right-hand side (DOWN)
  const float* z;          // coarse correction (UP)
  // work decomposition (filled by launch_stream)
  int rows, strips, chunks;
};

// Fills rows / strips / chunks for a level of N elements and NT steps, windows owning `own`
// columns, so that one wave of resident_warps warps covers it.
void stream_layout(int N, int NT, int own, long long resident_warps, StreamArgs& a);
// S sweeps in one pass of the given mode (1..5 for the DOWN modes, 1..8 for the plain and
// UP modes); adj selects J^T.
cudaError_t launch_stream(int mode, bool adj, int S, const StreamArgs& a, cudaStream_t s);
// The DOWN modes of launch_stream (kStreamDownX, kStreamDownT, kStreamDownTB), in their own
// translation unit; launch_stream counts the launch.
cudaError_t launch_stream_down(int mode, bool adj, int S, const StreamArgs& a, cudaStream_t s);

}  // namespace stmg
