// mlp.cuh -- the threshold network on one warp: lane j is hidden unit j of
// both layers.  Shared by the training kernels and the GEMM epilogue, which
// evaluates it once per tile.
//
// The paper compares each checksum residual with a predetermined threshold
// (Section 2.2).  The learned threshold scales the analytic one by
// 2^f(x_tile), f a 5 -> 32 -> 32 -> 1 ReLU network; the parameter vector is
// W1 [32][5], b1 [32], W2 [32][32], b2 [32], W3 [32], b3 (1281 floats).
#pragma once
#include <cuda_runtime.h>

namespace ftg {

constexpr int MLP_IN = 5, MLP_H = 32;
constexpr int MLP_W1 = 0, MLP_B1 = MLP_W1 + MLP_H * MLP_IN, MLP_W2 = MLP_B1 + MLP_H,
              MLP_B2 = MLP_W2 + MLP_H * MLP_H, MLP_W3 = MLP_B2 + MLP_H, MLP_B3 = MLP_W3 + MLP_H,
              MLP_PARAMS = MLP_B3 + 1;  // 1281

// Activations of one sample on one warp (this lane's unit).
struct MlpAct {
  float z1, z2, h2;
  float h1[MLP_H];  // every unit of the first layer, after ReLU
  float y;          // the output, the same on all lanes
};

// Forward pass of sample x (the same on all lanes) with parameters theta
// (global or shared memory).
__device__ __forceinline__ void mlp_forward_warp(const float* theta, const float* x, int lane, MlpAct& a) {
  float z1 = theta[MLP_B1 + lane];
#pragma unroll
  for (int k = 0; k < MLP_IN; ++k) z1 = fmaf(theta[MLP_W1 + lane * MLP_IN + k], x[k], z1);
  a.z1 = z1;
  const float h1 = fmaxf(z1, 0.f);
  float z2 = theta[MLP_B2 + lane];
#pragma unroll
  for (int i = 0; i < MLP_H; ++i) {
    a.h1[i] = __shfl_sync(0xffffffffu, h1, i);
    z2 = fmaf(theta[MLP_W2 + lane * MLP_H + i], a.h1[i], z2);
  }
  a.z2 = z2;
  a.h2 = fmaxf(z2, 0.f);
  float y = theta[MLP_W3 + lane] * a.h2;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) y += __shfl_xor_sync(0xffffffffu, y, o);
  a.y = y + theta[MLP_B3];
}

}  // namespace ftg
