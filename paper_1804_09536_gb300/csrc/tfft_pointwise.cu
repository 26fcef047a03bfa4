// Pointwise kernels on a stage buffer for the spectral-weight loss
// L = sum_k |y_k w_k|^2 and its gradient seed z = c w^2 y (c read on the
// device, so that the backward needs no host synchronisation).
//
// The reduction is deterministic: a fixed grid of blocks each sums a fixed
// strided subset in double precision with a fixed tree order, and one block
// then adds the block sums in index order.
#include "tfft_internal.h"

namespace tfft {

namespace {

constexpr int kRedThreads = 256;

__global__ void __launch_bounds__(kRedThreads) k_weighted_energy_part(const float2* __restrict__ y,
                                                                      const float* __restrict__ w, int64_t n,
                                                                      double* __restrict__ part) {
  __shared__ double red[kRedThreads];
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * kRedThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kRedThreads) {
    const float2 v = y[i];
    const double ww = (double)w[i] * (double)w[i];
    acc += ww * ((double)v.x * v.x + (double)v.y * v.y);
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = kRedThreads / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

__global__ void __launch_bounds__(kRedThreads) k_sum_parts(const double* __restrict__ part, int nparts,
                                                           double* __restrict__ out) {
  __shared__ double red[kRedThreads];
  double acc = 0.0;
  for (int i = threadIdx.x; i < nparts; i += kRedThreads) acc += part[i];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = kRedThreads / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}

__global__ void k_weight_scale(const float2* __restrict__ y, const float* __restrict__ w,
                               const double* __restrict__ coef, double scale, int64_t n, float2* __restrict__ z) {
  const float c = (float)(scale * (coef ? *coef : 1.0));
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float2 v = y[i];
    const float f = c * w[i] * w[i];
    z[i] = make_float2(f * v.x, f * v.y);
  }
}

}  // namespace

cudaError_t launch_weighted_energy(const float2* y, const float* w, int64_t n, double* parts, int nparts,
                                   double* out, cudaStream_t s) {
  k_weighted_energy_part<<<nparts, kRedThreads, 0, s>>>(y, w, n, parts);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_sum_parts<<<1, kRedThreads, 0, s>>>(parts, nparts, out);
  return cudaGetLastError();
}

cudaError_t launch_weight_scale(const float2* y, const float* w, const double* coef, double scale, int64_t n,
                                float2* z, cudaStream_t s) {
  int64_t blocks = (n + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  if (blocks < 1) return cudaSuccess;
  k_weight_scale<<<(unsigned)blocks, 256, 0, s>>>(y, w, coef, scale, n, z);
  return cudaGetLastError();
}

}  // namespace tfft
