// Host emulation of the kernels' Stockham schedule (test infrastructure).
// Runs the same per-thread work-item mapping, butterflies and twiddle
// indexing as the CUDA kernels, one emulated thread after another between
// the shared-memory exchanges, on host memory.
#include <cmath>
#include <cstdint>
#include <vector>

#include "tfft_common.cuh"

using namespace tfft;

template <int E, int R>
static void stage(float2 (&v)[E], int jt, int T, int Ns, int L, const float2* tw) {
  for (int q = 0; q < E / R; ++q) {
    if (Ns > 1) {
      const int j = jt + q * T;
      const int step = (j % Ns) * (L / (Ns * R));
      for (int r = 1; r < R; ++r) v[q * R + r] = cmul(v[q * R + r], tw[r * step]);
    }
    Dft<R>::run(&v[q * R]);
  }
}

template <int E, class F>
static void with_radix(int R, F&& f) {
  switch (R) {
    case 2: if constexpr (E % 2 == 0) f(std::integral_constant<int, 2>{}); break;
    case 3: if constexpr (E % 3 == 0) f(std::integral_constant<int, 3>{}); break;
    case 4: if constexpr (E % 4 == 0) f(std::integral_constant<int, 4>{}); break;
    case 5: if constexpr (E % 5 == 0) f(std::integral_constant<int, 5>{}); break;
    case 8: if constexpr (E % 8 == 0) f(std::integral_constant<int, 8>{}); break;
    case 16: if constexpr (E % 16 == 0) f(std::integral_constant<int, 16>{}); break;
    case 32: if constexpr (E % 32 == 0) f(std::integral_constant<int, 32>{}); break;
  }
}

template <int E>
static int run(int L, const int* radix, int nst, const float2* in, float2* out, int sign) {
  const int T = L / E;
  std::vector<float2> tw(L), sm(L);
  for (int m = 0; m < L; ++m) {
    const double a = 2.0 * M_PI * m / L;
    tw[m] = make_float2((float)std::cos(a), (float)-std::sin(a));
  }
  std::vector<std::vector<float2>> regs(T, std::vector<float2>(E));
  auto V = [&](int t) -> float2(&)[E] { return *reinterpret_cast<float2(*)[E]>(regs[t].data()); };
  int Ns = 1;
  for (int s = 0; s < nst; ++s) {
    const int R = radix[s];
    if (s == 0) {
      for (int t = 0; t < T; ++t)
        with_radix<E>(R, [&](auto rc) {
          constexpr int RR = decltype(rc)::value;
          for (int q = 0; q < E / RR; ++q)
            for (int r = 0; r < RR; ++r) {
              float2 x = in[t + q * T + r * (L / RR)];
              if (sign > 0) x.y = -x.y;
              V(t)[q * RR + r] = x;
            }
        });
    } else {
      const int Rp = radix[s - 1], Nsp = Ns / Rp;
      for (int t = 0; t < T; ++t)
        with_radix<E>(Rp, [&](auto rc) {
          constexpr int RR = decltype(rc)::value;
          for (int q = 0; q < E / RR; ++q)
            for (int r = 0; r < RR; ++r) sm[stockham_out_index(t + q * T, Nsp, RR, r)] = V(t)[q * RR + r];
        });
      for (int t = 0; t < T; ++t)
        with_radix<E>(R, [&](auto rc) {
          constexpr int RR = decltype(rc)::value;
          for (int q = 0; q < E / RR; ++q)
            for (int r = 0; r < RR; ++r) V(t)[q * RR + r] = sm[t + q * T + r * (L / RR)];
        });
    }
    for (int t = 0; t < T; ++t)
      with_radix<E>(R, [&](auto rc) {
        constexpr int RR = decltype(rc)::value;
        stage<E, RR>(V(t), t, T, Ns, L, tw.data());
      });
    Ns *= R;
  }
  if (Ns != L) return -1;
  for (int t = 0; t < T; ++t)
    with_radix<E>(radix[nst - 1], [&](auto rc) {
      constexpr int RR = decltype(rc)::value;
      for (int q = 0; q < E / RR; ++q)
        for (int r = 0; r < RR; ++r) {
          float2 x = V(t)[q * RR + r];
          if (sign > 0) x.y = -x.y;
          out[t + q * T + r * (L / RR)] = x;
        }
    });
  return 0;
}

extern "C" int emulate_fft(int L, int E, const int* radix, int nst, const float* in, float* out,
                           int sign) {
  const float2* i2 = reinterpret_cast<const float2*>(in);
  float2* o2 = reinterpret_cast<float2*>(out);
  switch (E) {
    case 2: return run<2>(L, radix, nst, i2, o2, sign);
    case 3: return run<3>(L, radix, nst, i2, o2, sign);
    case 4: return run<4>(L, radix, nst, i2, o2, sign);
    case 5: return run<5>(L, radix, nst, i2, o2, sign);
    case 6: return run<6>(L, radix, nst, i2, o2, sign);
    case 8: return run<8>(L, radix, nst, i2, o2, sign);
    case 10: return run<10>(L, radix, nst, i2, o2, sign);
    case 12: return run<12>(L, radix, nst, i2, o2, sign);
    case 15: return run<15>(L, radix, nst, i2, o2, sign);
    case 16: return run<16>(L, radix, nst, i2, o2, sign);
    case 20: return run<20>(L, radix, nst, i2, o2, sign);
    case 24: return run<24>(L, radix, nst, i2, o2, sign);
    case 32: return run<32>(L, radix, nst, i2, o2, sign);
  }
  return -2;
}
