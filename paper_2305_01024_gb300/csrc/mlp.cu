// mlp.cu -- training and standalone inference of the threshold network
// (mlp.cuh): forward, mean-squared-error gradient by backprop, Adam.  The
// paper leaves the detection threshold open (Section 2.2); this network has
// no counterpart there.
//
// Gradient: each warp runs samples one at a time with lane j holding unit j
// (forward, then the chain rule back through both ReLU layers), keeping its
// share of the gradient in registers; a block sums its warps in shared
// memory and writes one partial vector; a second kernel sums the partials of
// all blocks in a fixed order (in double) and applies Adam -- so a gradient
// is reproducible bit for bit.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "internal.cuh"
#include "mlp.cuh"

namespace ftg {

static_assert(MLP_PARAMS == FTGEMM_MLP_PARAMS, "parameter layout of the C ABI");
static_assert(MLP_IN == FTGEMM_MLP_INPUTS, "feature count of the C ABI");

constexpr int MLP_WARPS = 8;
constexpr int MLP_SLOT = MLP_PARAMS + 1;  // gradient, then the loss sum

// Partial sums over this block's samples of [d loss / d theta, sum (y - t)^2]
// for the samples s0 .. s0 + nb - 1 of X (n x 5) and t; the loss is
// inv_n * sum (y - t)^2.
__global__ void __launch_bounds__(MLP_WARPS * 32)
    mlp_grad_kernel(const float* __restrict__ X, const float* __restrict__ t, long long s0, int nb,
                    const float* __restrict__ theta, float inv_n, float* __restrict__ part) {
  __shared__ float sth[MLP_PARAMS];
  __shared__ float red[MLP_WARPS][MLP_SLOT];
  for (int i = threadIdx.x; i < MLP_PARAMS; i += blockDim.x) sth[i] = theta[i];
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float gw1[MLP_IN] = {0.f, 0.f, 0.f, 0.f, 0.f}, gb1 = 0.f, gw2[MLP_H], gb2 = 0.f, gw3 = 0.f, gb3 = 0.f, L = 0.f;
#pragma unroll
  for (int i = 0; i < MLP_H; ++i) gw2[i] = 0.f;
  for (int s = blockIdx.x * MLP_WARPS + warp; s < nb; s += gridDim.x * MLP_WARPS) {
    float x[MLP_IN];
#pragma unroll
    for (int k = 0; k < MLP_IN; ++k) x[k] = X[(s0 + s) * MLP_IN + k];
    MlpAct a;
    mlp_forward_warp(sth, x, lane, a);
    const float e = a.y - t[s0 + s];
    const float dy = 2.f * e * inv_n;  // d loss / d y
    L = fmaf(e, e, L);
    gb3 += dy;
    gw3 = fmaf(dy, a.h2, gw3);
    const float dz2 = a.z2 > 0.f ? dy * sth[MLP_W3 + lane] : 0.f;
    gb2 += dz2;
#pragma unroll
    for (int i = 0; i < MLP_H; ++i) gw2[i] = fmaf(dz2, a.h1[i], gw2[i]);
    float dh1 = 0.f;  // sum_j W2[j][lane] dz2_j
#pragma unroll
    for (int j = 0; j < MLP_H; ++j) dh1 = fmaf(sth[MLP_W2 + j * MLP_H + lane], __shfl_sync(0xffffffffu, dz2, j), dh1);
    const float dz1 = a.z1 > 0.f ? dh1 : 0.f;
    gb1 += dz1;
#pragma unroll
    for (int k = 0; k < MLP_IN; ++k) gw1[k] = fmaf(dz1, x[k], gw1[k]);
  }
  float* r = red[warp];
#pragma unroll
  for (int k = 0; k < MLP_IN; ++k) r[MLP_W1 + lane * MLP_IN + k] = gw1[k];
  r[MLP_B1 + lane] = gb1;
#pragma unroll
  for (int i = 0; i < MLP_H; ++i) r[MLP_W2 + lane * MLP_H + i] = gw2[i];
  r[MLP_B2 + lane] = gb2;
  r[MLP_W3 + lane] = gw3;
  if (lane == 0) {
    r[MLP_B3] = gb3;  // the same on every lane
    r[MLP_PARAMS] = L;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < MLP_SLOT; i += blockDim.x) {
    float s = 0.f;
#pragma unroll
    for (int w = 0; w < MLP_WARPS; ++w) s += red[w][i];
    part[(long long)blockIdx.x * MLP_SLOT + i] = s;
  }
}

// Sum the partials of nblk blocks (in block order, in double).  grad_out
// (optional) receives the gradient; with lr > 0 Adam updates theta, m, v
// (c1 = 1 / (1 - beta1^step), c2 = 1 / (1 - beta2^step)); loss_out
// (optional) receives inv_n * sum (y - t)^2.
__global__ void mlp_reduce_kernel(const float* __restrict__ part, int nblk, float* __restrict__ grad_out,
                                  float* __restrict__ theta, float* __restrict__ m, float* __restrict__ v, float c1,
                                  float c2, float lr, float inv_n, float* __restrict__ loss_out) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= MLP_SLOT) return;
  double s = 0.0;
  for (int b = 0; b < nblk; ++b) s += (double)part[(long long)b * MLP_SLOT + p];
  if (p == MLP_PARAMS) {
    if (loss_out) *loss_out = (float)(s * (double)inv_n);
    return;
  }
  const float g = (float)s;
  if (grad_out) grad_out[p] = g;
  if (lr > 0.f) {
    const float beta1 = 0.9f, beta2 = 0.999f, eps = 1e-8f;
    const float mm = beta1 * m[p] + (1.f - beta1) * g;
    const float vv = beta2 * v[p] + (1.f - beta2) * g * g;
    m[p] = mm;
    v[p] = vv;
    theta[p] -= lr * (mm * c1) / (sqrtf(vv * c2) + eps);
  }
}

// y[i] = network(X[i]) for n samples, one warp per sample.
__global__ void mlp_forward_kernel(const float* __restrict__ X, long long n, const float* __restrict__ theta,
                                   float* __restrict__ y) {
  const int lane = threadIdx.x & 31;
  const long long w0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long s = w0; s < n; s += nw) {
    float x[MLP_IN];
#pragma unroll
    for (int k = 0; k < MLP_IN; ++k) x[k] = X[s * MLP_IN + k];
    MlpAct a;
    mlp_forward_warp(theta, x, lane, a);
    if (lane == 0) y[s] = a.y;
  }
}

int mlp_grad_blocks(long long nb) {
  return (int)std::max<long long>(1, std::min<long long>((nb + MLP_WARPS - 1) / MLP_WARPS, 152 * 4));
}

cudaError_t launch_mlp_grad(const float* X, const float* t, long long s0, int nb, const float* theta, float inv_n,
                            float* part, int nblk, cudaStream_t st) {
  mlp_grad_kernel<<<nblk, MLP_WARPS * 32, 0, st>>>(X, t, s0, nb, theta, inv_n, part);
  return cudaGetLastError();
}

cudaError_t launch_mlp_reduce(const float* part, int nblk, float* grad_out, float* theta, float* m, float* v, int step,
                              float lr, float inv_n, float* loss_out, cudaStream_t st) {
  const float c1 = step > 0 ? (float)(1.0 / (1.0 - std::pow(0.9, step))) : 1.f;
  const float c2 = step > 0 ? (float)(1.0 / (1.0 - std::pow(0.999, step))) : 1.f;
  mlp_reduce_kernel<<<(MLP_SLOT + 255) / 256, 256, 0, st>>>(part, nblk, grad_out, theta, m, v, c1, c2, lr, inv_n,
                                                             loss_out);
  return cudaGetLastError();
}

cudaError_t launch_mlp_forward(const float* X, long long n, const float* theta, float* y, cudaStream_t st) {
  const int blocks = (int)std::max<long long>(1, std::min<long long>((n + 7) / 8, 152 * 8));
  mlp_forward_kernel<<<blocks, 256, 0, st>>>(X, n, theta, y);
  return cudaGetLastError();
}

}  // namespace ftg
