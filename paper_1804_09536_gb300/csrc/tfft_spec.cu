// Compile-time specialised FFT passes for the axis lengths of the benchmark
// workloads (32, 64, 96, 128, 160, 256, 512).  Same Stockham schedule as the
// runtime-dispatched kernels (tfft_kernels.cu), but with the length, the
// radix sequence, the threads per line and the tile width fixed at compile
// time: every index, span and twiddle stride folds to a constant, the row
// tables hold 32-bit offsets, and the register budget is known to ptxas.
#include <type_traits>

#include "tfft_internal.h"
#include "tfft_tiles.cuh"

namespace tfft {

namespace {

using namespace tiles;

template <int L, int E, int B, int... Rs>
__global__ void __launch_bounds__((L / E) * B, min_blocks(E, (L / E) * B, 512))
    k_contig_spec(const ContigArgs a) {
  extern __shared__ float2 smem[];
  for (int64_t tile = blockIdx.x; tile * B < a.nlines; tile += gridDim.x)
    contig_tile<L, E, B, false, Rs...>(a, tile, smem, opaque_tid_x(), threadIdx.y);
}

template <int L, int E, int W, int... Rs>
__global__ void __launch_bounds__(W * (L / E), min_blocks(E, W * (L / E), 1024))
    k_strided_spec(const StridedArgs a) {
  extern __shared__ float2 smem[];
  const int64_t ntiles = a.nouter * a.ncolblocks;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x)
    strided_tile<L, E, W, false, Rs...>(a, tile, smem, threadIdx.x, opaque_tid_y(), threadIdx.y * W + threadIdx.x);
}

// ------------------------------------------------------------ real lines
//
// Real-to-complex along the innermost axis (footnote to Eq. multifft: the
// Hermitian half k = 0 .. N/2).  A real line of N = 2L values is read as L
// complex values z[n] = x[2n] + i x[2n+1]; Z = FFT_L(z); then with
// w = exp(-2 pi i / N):  X[k] = (Z[k] + conj Z[L-k]) / 2
//                              - (i / 2) w^k (Z[k] - conj Z[L-k]),  k = 0 .. L.
// Complex-to-real inverts it: Z[k] = (X[k] + conj X[L-k])
//                              + i w^-k (X[k] - conj X[L-k]),  k < L,
// z = backward FFT_L(Z), x[2n] = Re z[n], x[2n+1] = Im z[n]; the imaginary
// parts of X[0] and X[L] are ignored (taken as zero).

template <int L, int E, int B, int... Rs>
__global__ void __launch_bounds__((L / E) * B, min_blocks(E, (L / E) * B, 512))
    k_r2c_spec(const RealArgs a) {
  constexpr int T = L / E, NST = sizeof...(Rs);
  constexpr int LP = line_pitch<L, Rs...>();
  constexpr int P = pad_every<Rs...>();
  extern __shared__ float2 smem[];
  const int ly = threadIdx.y;
  float2* sl = smem + ly * LP;
  for (int64_t base = (int64_t)blockIdx.x * B; base < a.nlines; base += (int64_t)gridDim.x * B) {
    const int64_t line = base + ly;
    const bool act = line < a.nlines;
    const float2* src = reinterpret_cast<const float2*>(a.rin) + line * L;
    float2* dst = a.cout + line * (L + 1);
    const int jt = opaque_tid_x();
    float2 v[emax<L, E, Rs...>()];
    static_for<0, NST>([&](auto S) {
      constexpr int s = decltype(S)::value;
      constexpr int R = radix_at<s, Rs...>();
      constexpr int Ns = span_at<s, Rs...>();
      if constexpr (s == 0) {
#pragma unroll
        for (int q = 0; q < nbf<L, E, R>(); ++q)
#pragma unroll
          for (int r = 0; r < R; ++r)
            v[q * R + r] = (act && bf_exists<L, E, R>(jt, q)) ? src[jt + q * T + r * (L / R)] : make_float2(0.f, 0.f);
      } else {
        constexpr int Rp = radix_at<s - 1, Rs...>();
        constexpr int Nsp = Ns / Rp;
        line_sync<T>();
#pragma unroll
        for (int q = 0; q < nbf<L, E, Rp>(); ++q)
          if (bf_exists<L, E, Rp>(jt, q))
#pragma unroll
            for (int r = 0; r < Rp; ++r) sl[padp<P>(stockham_out_index(jt + q * T, Nsp, Rp, r))] = v[q * Rp + r];
        line_sync<T>();
#pragma unroll
        for (int q = 0; q < nbf<L, E, R>(); ++q)
          if (bf_exists<L, E, R>(jt, q))
#pragma unroll
            for (int r = 0; r < R; ++r) v[q * R + r] = sl[padp<P>(jt + q * T + r * (L / R))];
      }
      spec_stage<L, E, R, Ns>(v, jt, a.tw);
    });
    constexpr int RL = radix_at<NST - 1, Rs...>();
    line_sync<T>();
#pragma unroll
    for (int q = 0; q < nbf<L, E, RL>(); ++q)
      if (bf_exists<L, E, RL>(jt, q))
#pragma unroll
        for (int r = 0; r < RL; ++r) sl[padp<P>(jt + q * T + r * (L / RL))] = v[q * RL + r];
    line_sync<T>();
    for (int k = jt; k <= L; k += T) {
      const float2 zk = sl[padp<P>(k == L ? 0 : k)];
      const float2 zm = sl[padp<P>(k == 0 ? 0 : L - k)];
      const float2 e = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));   // (Z[k] + conj Z[L-k]) / 2
      const float2 d = make_float2(0.5f * (zk.x - zm.x), 0.5f * (zk.y + zm.y));   // (Z[k] - conj Z[L-k]) / 2
      const float2 o = cmul(__ldg(&a.tw2[k]), mul_mi(d));                          // -i w^k d
      if (act) dst[k] = cscale(cadd(e, o), a.scale);
    }
  }
}

template <int L, int E, int B, int... Rs>
__global__ void __launch_bounds__((L / E) * B, min_blocks(E, (L / E) * B, 512))
    k_c2r_spec(const RealArgs a) {
  constexpr int T = L / E, NST = sizeof...(Rs);
  constexpr int LP = line_pitch<L, Rs...>() + 1;
  constexpr int P = pad_every<Rs...>();
  extern __shared__ float2 smem[];
  const int ly = threadIdx.y;
  float2* sl = smem + ly * LP;
  for (int64_t base = (int64_t)blockIdx.x * B; base < a.nlines; base += (int64_t)gridDim.x * B) {
    const int64_t line = base + ly;
    const bool act = line < a.nlines;
    const float2* src = a.cin + line * (L + 1);
    float2* dst = reinterpret_cast<float2*>(a.rout) + line * L;
    const int jt = opaque_tid_x();
    // the L + 1 inputs: every load issued before the first shared store, so
    // that they are all in flight together
    constexpr int NK = E + 1;  // ceil((L + 1) / T)
    float2 xin[NK];
#pragma unroll
    for (int i = 0; i < NK; ++i) {
      const int k = jt + i * T;
      xin[i] = (act && k <= L) ? src[k] : make_float2(0.f, 0.f);
    }
    line_sync<T>();  // the previous line group is done with sl
#pragma unroll
    for (int i = 0; i < NK; ++i) {
      const int k = jt + i * T;
      if (k <= L) {
        float2 x = xin[i];
        if (k == 0 || k == L) x.y = 0.f;
        sl[padp<P>(k)] = x;
      }
    }
    line_sync<T>();
    float2 v[emax<L, E, Rs...>()];
    static_for<0, NST>([&](auto S) {
      constexpr int s = decltype(S)::value;
      constexpr int R = radix_at<s, Rs...>();
      constexpr int Ns = span_at<s, Rs...>();
      if constexpr (s == 0) {
#pragma unroll
        for (int q = 0; q < nbf<L, E, R>(); ++q)
#pragma unroll
          for (int r = 0; r < R; ++r) {
            const int k = bf_exists<L, E, R>(jt, q) ? jt + q * T + r * (L / R) : 0;
            const float2 xk = sl[padp<P>(k)];
            const float2 xm = sl[padp<P>(L - k)];
            const float2 e = make_float2(xk.x + xm.x, xk.y - xm.y);      // X[k] + conj X[L-k]
            const float2 d = make_float2(xk.x - xm.x, xk.y + xm.y);      // X[k] - conj X[L-k]
            const float2 w = __ldg(&a.tw2[k]);
            const float2 od = cmul(make_float2(w.x, -w.y), d);           // w^-k d
            const float2 z = make_float2(e.x - od.y, e.y + od.x);         // e + i w^-k d
            v[q * R + r] = make_float2(z.x, -z.y);                        // backward = conj o forward o conj
          }
      } else {
        constexpr int Rp = radix_at<s - 1, Rs...>();
        constexpr int Nsp = Ns / Rp;
        line_sync<T>();
#pragma unroll
        for (int q = 0; q < nbf<L, E, Rp>(); ++q)
          if (bf_exists<L, E, Rp>(jt, q))
#pragma unroll
            for (int r = 0; r < Rp; ++r) sl[padp<P>(stockham_out_index(jt + q * T, Nsp, Rp, r))] = v[q * Rp + r];
        line_sync<T>();
#pragma unroll
        for (int q = 0; q < nbf<L, E, R>(); ++q)
          if (bf_exists<L, E, R>(jt, q))
#pragma unroll
            for (int r = 0; r < R; ++r) v[q * R + r] = sl[padp<P>(jt + q * T + r * (L / R))];
      }
      spec_stage<L, E, R, Ns>(v, jt, a.tw);
    });
    constexpr int RL = radix_at<NST - 1, Rs...>();
#pragma unroll
    for (int q = 0; q < nbf<L, E, RL>(); ++q)
#pragma unroll
      for (int r = 0; r < RL; ++r) {
        const float2 z = v[q * RL + r];
        if (act && bf_exists<L, E, RL>(jt, q)) dst[jt + q * T + r * (L / RL)] = make_float2(z.x * a.scale, -z.y * a.scale);
      }
  }
}

template <class K>
cudaError_t allow_smem(K kernel) {
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
}

constexpr int64_t kMaxGrid = 1 << 20;

template <int L, int E, int B, int... Rs>
cudaError_t run_contig(const ContigArgs& a, cudaStream_t s) {
  static cudaError_t attr = allow_smem(k_contig_spec<L, E, B, Rs...>);
  if (attr != cudaSuccess) return attr;
  const size_t smem = (size_t)B * line_pitch<L, Rs...>() * sizeof(float2);
  int64_t grid = (a.nlines + B - 1) / B;
  if (grid > kMaxGrid) grid = kMaxGrid;
  if (grid < 1) return cudaSuccess;
  k_contig_spec<L, E, B, Rs...><<<(unsigned)grid, dim3(L / E, B), smem, s>>>(a);
  return cudaGetLastError();
}

template <int L, int E, int W, int... Rs>
cudaError_t run_strided(const StridedArgs& a, cudaStream_t s) {
  static cudaError_t attr = allow_smem(k_strided_spec<L, E, W, Rs...>);
  if (attr != cudaSuccess) return attr;
  if (a.W != W) return cudaErrorInvalidValue;
  const size_t smem = (size_t)L * W * sizeof(float2) + 2 * (size_t)L * sizeof(int);
  int64_t grid = a.nouter * a.ncolblocks;
  if (grid > kMaxGrid) grid = kMaxGrid;
  if (grid < 1) return cudaSuccess;
  k_strided_spec<L, E, W, Rs...><<<(unsigned)grid, dim3(W, L / E), smem, s>>>(a);
  return cudaGetLastError();
}

// The table of specialisations: length; contiguous passes: elements per
// thread and lines per CTA; strided passes: elements per thread and tile
// width; radices.  "Elements per thread" is L / (threads per line); for the
// lengths with 2, 3 and 5 all present no radix set divides it, and the
// threads carry ceil(butterflies / threads) butterflies per stage (nbf()).
#define TFFT_SPECS(X)                       \
  X(32, 8, 64, 8, 32, 8, 4)                 \
  X(64, 8, 32, 8, 32, 8, 8)                 \
  X(96, 12, 32, 12, 32, 4, 4, 3, 2)         \
  X(128, 16, 32, 16, 32, 16, 8)             \
  X(160, 20, 32, 20, 32, 5, 4, 4, 2)        \
  X(256, 16, 16, 16, 32, 16, 16)            \
  X(512, 32, 16, 32, 16, 32, 16)            \
  X(60, 15, 64, 15, 64, 4, 5, 3)            \
  X(120, 15, 32, 15, 32, 8, 5, 3)           \
  X(240, 15, 16, 15, 16, 16, 5, 3)          \
  X(480, 30, 16, 30, 16, 16, 5, 3, 2)

struct SpecRow {
  int L, EC, B, ES, W, nst, radix[6];
};

const SpecRow kSpecs[] = {
#define X(L, EC, B, ES, W, ...) \
  {L, EC, B, ES, W, (int)(sizeof((int[]){__VA_ARGS__}) / sizeof(int)), {__VA_ARGS__}},
    TFFT_SPECS(X)
#undef X
};

template <int L, int E, int B, int... Rs>
cudaError_t run_real(const RealArgs& a, cudaStream_t s) {
  const int64_t grid0 = (a.nlines + B - 1) / B;
  const int64_t grid = grid0 > kMaxGrid ? kMaxGrid : grid0;
  if (grid < 1) return cudaSuccess;
  if (a.dir < 0) {
    static cudaError_t attr = allow_smem(k_r2c_spec<L, E, B, Rs...>);
    if (attr != cudaSuccess) return attr;
    const size_t smem = (size_t)B * line_pitch<L, Rs...>() * sizeof(float2);
    k_r2c_spec<L, E, B, Rs...><<<(unsigned)grid, dim3(L / E, B), smem, s>>>(a);
  } else {
    static cudaError_t attr = allow_smem(k_c2r_spec<L, E, B, Rs...>);
    if (attr != cudaSuccess) return attr;
    const size_t smem = (size_t)B * (line_pitch<L, Rs...>() + 1) * sizeof(float2);
    k_c2r_spec<L, E, B, Rs...><<<(unsigned)grid, dim3(L / E, B), smem, s>>>(a);
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_real_spec(const RealArgs& a, cudaStream_t s) {
  switch (a.ap.L) {
#define X(L, EC, B, ES, W, ...) \
  case L:                       \
    return run_real<L, EC, B, __VA_ARGS__>(a, s);
    TFFT_SPECS(X)
#undef X
    default:
      return cudaErrorInvalidValue;
  }
}

bool spec_plan(int L, bool strided, int64_t nelems, AxisPlan& ap, int& width) {
  if (nelems >= (int64_t(1) << 31)) return false;  // 32-bit row offsets
  for (const SpecRow& r : kSpecs) {
    if (r.L != L) continue;
    const int E = strided ? r.ES : r.EC;
    ap.L = L;
    ap.E = E;
    ap.T = L / E;
    ap.nst = r.nst;
    ap.code = 0;
    for (int s = 0; s < r.nst; ++s) {
      ap.radix[s] = r.radix[s];
      ap.code |= (uint64_t)r.radix[s] << (5 * s);
    }
    ap.spec = 1;
    width = strided ? r.W : r.B;
    return true;
  }
  return false;
}

cudaError_t launch_contig_spec(const ContigArgs& a, cudaStream_t s) {
  switch (a.ap.L) {
#define X(L, EC, B, ES, W, ...) \
  case L:                       \
    return run_contig<L, EC, B, __VA_ARGS__>(a, s);
    TFFT_SPECS(X)
#undef X
    default:
      return cudaErrorInvalidValue;
  }
}

cudaError_t launch_strided_spec(const StridedArgs& a, cudaStream_t s) {
  switch (a.ap.L) {
#define X(L, EC, B, ES, W, ...) \
  case L:                       \
    return run_strided<L, ES, W, __VA_ARGS__>(a, s);
    TFFT_SPECS(X)
#undef X
    default:
      return cudaErrorInvalidValue;
  }
}

}  // namespace tfft
