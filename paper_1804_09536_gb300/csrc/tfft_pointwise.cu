// Pointwise kernels on a stage buffer for the spectral-weight loss
// L = sum_k |y_k w_k|^2 and its gradient seed z = c w^2 y (c read on the
// device, so that the backward needs no host synchronisation).
//
// The reduction is deterministic: a fixed grid of blocks each sums a fixed
// strided subset (per thread in compensated FP32, about 48 bits, then in
// double with a fixed tree order), and one block then adds the block sums in
// index order.
#include "tfft_internal.h"

namespace tfft {

namespace {

constexpr int kRedThreads = 256;

// Error-free transformations in FP32 (Knuth's two-sum, the FMA two-product):
// a value is carried as the unevaluated sum hi + lo of two floats, about 48
// significant bits.  FP64 throughput on this part is a small fraction of
// FP32, so the per-element work stays in FP32 and only each thread's final
// sum is converted to double.  The intrinsics keep the compiler from
// contracting or reordering the steps.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
  p = __fmul_rn(a, b);
  e = __fmaf_rn(a, b, -p);
}

// |v|^2 w^2 as hi + lo (relative error a few units of 2^-48).
__device__ __forceinline__ void weighted_term(float2 v, float w, float& hi, float& lo) {
  float p1, e1, p2, e2, s, es, q, eq;
  two_prod(v.x, v.x, p1, e1);
  two_prod(v.y, v.y, p2, e2);
  two_sum(p1, p2, s, es);
  const float sl = __fadd_rn(__fadd_rn(e1, e2), es);  // |v|^2 = s + sl
  two_prod(w, w, q, eq);                              // w^2 = q + eq exactly
  float et;
  two_prod(s, q, hi, et);
  lo = __fmaf_rn(s, eq, __fmaf_rn(sl, q, et));
}

// With U = true the same sweep also writes u = w^2 y (the gradient seed up to
// its scalar factor), which may alias y.
template <bool U>
__global__ void __launch_bounds__(kRedThreads) k_weighted_energy_part(const float2* y, const float* __restrict__ w,
                                                                      int64_t n, double* __restrict__ part,
                                                                      float2* u) {
  __shared__ double red[kRedThreads];
  float ah = 0.f, al = 0.f;  // running sum, renormalised after every term
  for (int64_t i = (int64_t)blockIdx.x * kRedThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kRedThreads) {
    float th, tl, s, e;
    const float2 v = y[i];
    const float wi = w[i];
    weighted_term(v, wi, th, tl);
    if constexpr (U) {
      const float f = wi * wi;
      u[i] = make_float2(f * v.x, f * v.y);
    }
    two_sum(ah, th, s, e);
    const float l = __fadd_rn(__fadd_rn(al, e), tl);
    ah = __fadd_rn(s, l);  // fast two-sum: |s| >= |l|
    al = __fsub_rn(l, __fsub_rn(ah, s));
  }
  red[threadIdx.x] = (double)ah + (double)al;
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
                                   double* out, float2* u, cudaStream_t s) {
  if (u)
    k_weighted_energy_part<true><<<nparts, kRedThreads, 0, s>>>(y, w, n, parts, u);
  else
    k_weighted_energy_part<false><<<nparts, kRedThreads, 0, s>>>(y, w, n, parts, nullptr);
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
