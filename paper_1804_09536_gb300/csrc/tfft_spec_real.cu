// Compile-time specialised real-line passes (r2c / c2r along the innermost
// axis) for the lengths of tfft_spec_table.h (the complex half-length).
#include "tfft_internal.h"
#include "tfft_spec_table.h"
#include "tfft_tiles.cuh"

namespace tfft {

namespace {

using namespace tiles;

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
__global__ void __launch_bounds__((L / E) * B, min_blocks(E, (L / E) * B, 1024))
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
    float2* dst = a.cout + line * a.cpitch;
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
    // outputs k and L - k together: with e, o of k, X[k] = e + o and, as
    // w^(L-k) = -conj(w^k) and the roles of Z[k], Z[L-k] swap,
    // X[L-k] = conj(e - o) -- one pair of shared loads and one twiddle for two
    // outputs (k = 0 gives X[0] and X[L]; k = L/2 is its own partner)
    for (int k = jt; k <= L / 2; k += T) {
      const float2 zk = sl[padp<P>(k)];
      const float2 zm = sl[padp<P>(k == 0 ? 0 : L - k)];
      const float2 e = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));   // (Z[k] + conj Z[L-k]) / 2
      const float2 d = make_float2(0.5f * (zk.x - zm.x), 0.5f * (zk.y + zm.y));   // (Z[k] - conj Z[L-k]) / 2
      const float2 o = cmul(__ldg(&a.tw2[k]), mul_mi(d));                          // -i w^k d
      if (act) {
        dst[k] = cscale(cadd(e, o), a.scale);
        if (2 * k != L) dst[L - k] = cscale(make_float2(e.x - o.x, o.y - e.y), a.scale);
      }
    }
  }
}

template <int L, int E, int B, int... Rs>
__global__ void __launch_bounds__((L / E) * B, min_blocks(E, (L / E) * B, 1024))
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
    const float2* src = a.cin + line * a.cpitch;
    float2* dst = reinterpret_cast<float2*>(a.rout) + line * L;
    const int jt = opaque_tid_x();
    // the L + 1 inputs as the pairs (X[k], X[L-k]), k <= L/2 (k = 0 pairs
    // X[0] with X[L]): every load issued before the first shared store, so
    // that they are all in flight together
    constexpr int NP = (L / 2) / T + 1;
    float2 xa[NP], xb[NP];
#pragma unroll
    for (int i = 0; i < NP; ++i) {
      const int k = jt + i * T;
      const bool ok = act && k <= L / 2;
      xa[i] = ok ? src[k] : make_float2(0.f, 0.f);
      xb[i] = ok ? src[L - k] : make_float2(0.f, 0.f);
    }
    line_sync<T>();  // the previous line group is done with sl
    // Z[k] and Z[L-k] of each pair: with e, q = i w^-k d of k, Z[k] = e + q
    // and (w^-(L-k) = -w^k, the roles of X[k], X[L-k] swap) Z[L-k] =
    // conj(e - q); stored conjugated (backward = conj o forward o conj).
    // The imaginary parts of X[0] and X[L] are ignored; k = L/2 is its own
    // partner.
#pragma unroll
    for (int i = 0; i < NP; ++i) {
      const int k = jt + i * T;
      if (k <= L / 2) {
        float2 xk = xa[i], xm = xb[i];
        if (k == 0) {
          xk.y = 0.f;
          xm.y = 0.f;
        }
        const float2 e = make_float2(xk.x + xm.x, xk.y - xm.y);      // X[k] + conj X[L-k]
        const float2 d = make_float2(xk.x - xm.x, xk.y + xm.y);      // X[k] - conj X[L-k]
        const float2 w = __ldg(&a.tw2[k]);
        const float2 od = cmul(make_float2(w.x, -w.y), d);           // w^-k d
        const float2 qv = make_float2(-od.y, od.x);                  // i w^-k d
        sl[padp<P>(k)] = make_float2(e.x + qv.x, -(e.y + qv.y));     // conj Z[k]
        if (k > 0 && 2 * k != L) sl[padp<P>(L - k)] = make_float2(e.x - qv.x, e.y - qv.y);  // conj Z[L-k]
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
            v[q * R + r] = sl[padp<P>(k)];
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

// the kernel's shared-memory limit raised to 227 KB, once per device
#define TFFT_ALLOW_SMEM(kernel)                          \
  static PerDevice<cudaError_t> attr_cache;              \
  const cudaError_t attr = smem_attr_once(attr_cache, kernel, 227 * 1024)

constexpr int64_t kMaxGrid = 1 << 20;

template <int L, int E, int B, int... Rs>
cudaError_t run_real(const RealArgs& a, cudaStream_t s) {
  const int64_t grid0 = (a.nlines + B - 1) / B;
  const int64_t grid = grid0 > kMaxGrid ? kMaxGrid : grid0;
  if (grid < 1) return cudaSuccess;
  if (a.dir < 0) {
    TFFT_ALLOW_SMEM((k_r2c_spec<L, E, B, Rs...>));
    if (attr != cudaSuccess) return attr;
    const size_t smem = (size_t)B * line_pitch<L, Rs...>() * sizeof(float2);
    k_r2c_spec<L, E, B, Rs...><<<(unsigned)grid, dim3(L / E, B), smem, s>>>(a);
  } else {
    TFFT_ALLOW_SMEM((k_c2r_spec<L, E, B, Rs...>));
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

}  // namespace tfft
