// Host/device shared definitions of the CUDA path: layout addressing on the
// virtual process grid, radix butterflies and the Stockham index schedule.
// Compiled by nvcc for the kernels and by the host compiler for the plan code.
#pragma once

#include <stdint.h>
#include <vector_types.h>
#include <vector_functions.h>

#if defined(__CUDACC__)
#define TFFT_HD __host__ __device__ __forceinline__
#else
#define TFFT_HD inline
#endif

namespace tfft {

constexpr int MAXD = 4;        // array dimensions
constexpr int MAXG = 3;        // grid dimensions
constexpr int MAXSTAGES = 12;  // radix stages of one 1-D FFT
constexpr int MAXLEN = 4096;   // longest transformed axis

// One alignment ("stage") of a d-D global array on the virtual grid.  Axis m
// is cut in Mx[m] parts by one grid direction (Mx[m] = 1 when the stage holds
// it whole) with the balanced block decomposition of Eq. decompose; the part
// index along that direction contributes part * rs[m] to the rank.  A rank's
// local array is C ordered and sits at element offset[rank] of the stage
// buffer.
struct DevLayout {
  int d;
  int64_t N[MAXD];
  int64_t Mx[MAXD];
  int64_t rs[MAXD];
  const int64_t* offset;  // nranks entries (device memory in kernels)
  int64_t pitch;          // > 0: the innermost axis is stored `pitch` apart (a padded internal layout)
};

// Inverse of Eq. decompose: which part (coord) of N split in M holds global
// index g, g's index inside that part, and the part's length.  Extents are
// below 2^31, so 32-bit division suffices.
TFFT_HD void locate(int64_t N64, int64_t M64, int64_t g64, int64_t& coord, int64_t& local,
                    int64_t& n) {
  const uint32_t N = (uint32_t)N64, M = (uint32_t)M64, g = (uint32_t)g64;
  const uint32_t q = N / M, r = N - q * M;
  const uint32_t big = r * (q + 1);
  if (g < big) {
    const uint32_t c = g / (q + 1);
    coord = c;
    local = g - c * (q + 1);
    n = q + 1;
  } else {
    const uint32_t h = g - big;  // q >= 1 here because g < N
    const uint32_t c = h / q;
    coord = r + c;
    local = h - c * q;
    n = q;
  }
}

// ------------------------------------------------------------ complex math

TFFT_HD float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
TFFT_HD float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
// The rounding order is spelled out on the device, so every kernel that
// applies the same twiddle gets the same bits, however the compiler would
// otherwise contract the products into FMAs.
TFFT_HD float2 cmul(float2 a, float2 b) {
#ifdef __CUDA_ARCH__
  return make_float2(__fmaf_rn(a.x, b.x, -__fmul_rn(a.y, b.y)), __fmaf_rn(a.x, b.y, __fmul_rn(a.y, b.x)));
#else
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
#endif
}
TFFT_HD float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
// multiply by -i (the forward quarter turn)
TFFT_HD float2 mul_mi(float2 a) { return make_float2(a.y, -a.x); }

// Forward (sign -1) DFTs of size R on v[0..R-1], in place, natural order out.
template <int R>
struct Dft;

template <>
struct Dft<2> {
  TFFT_HD static void run(float2* v) {
    const float2 a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
  }
};

template <>
struct Dft<3> {
  TFFT_HD static void run(float2* v) {
    const float c = -0.5f, s = 0.86602540378443864676f;  // cos, sin of 2 pi / 3
    const float2 t = cadd(v[1], v[2]), u = csub(v[1], v[2]);
    const float2 a = v[0];
    const float2 m = make_float2(a.x + c * t.x, a.y + c * t.y);
    const float2 su = make_float2(s * u.y, -s * u.x);  // -i s u
    v[0] = cadd(a, t);
    v[1] = cadd(m, su);
    v[2] = csub(m, su);
  }
};

template <>
struct Dft<4> {
  TFFT_HD static void run(float2* v) {
    const float2 t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
    const float2 t2 = cadd(v[1], v[3]), t3 = mul_mi(csub(v[1], v[3]));
    v[0] = cadd(t0, t2);
    v[2] = csub(t0, t2);
    v[1] = cadd(t1, t3);
    v[3] = csub(t1, t3);
  }
};

template <>
struct Dft<5> {
  TFFT_HD static void run(float2* v) {
    const float c1 = 0.30901699437494742410f;   // cos(2 pi / 5)
    const float c2 = -0.80901699437494742410f;  // cos(4 pi / 5)
    const float s1 = 0.95105651629515357212f;   // sin(2 pi / 5)
    const float s2 = 0.58778525229247312917f;   // sin(4 pi / 5)
    const float2 a = v[0];
    const float2 t1 = cadd(v[1], v[4]), u1 = csub(v[1], v[4]);
    const float2 t2 = cadd(v[2], v[3]), u2 = csub(v[2], v[3]);
    const float2 m1 = make_float2(a.x + c1 * t1.x + c2 * t2.x, a.y + c1 * t1.y + c2 * t2.y);
    const float2 m2 = make_float2(a.x + c2 * t1.x + c1 * t2.x, a.y + c2 * t1.y + c1 * t2.y);
    // -i (s1 u1 + s2 u2) and -i (s2 u1 - s1 u2)
    const float2 p1 = mul_mi(make_float2(s1 * u1.x + s2 * u2.x, s1 * u1.y + s2 * u2.y));
    const float2 p2 = mul_mi(make_float2(s2 * u1.x - s1 * u2.x, s2 * u1.y - s1 * u2.y));
    v[0] = make_float2(a.x + t1.x + t2.x, a.y + t1.y + t2.y);
    v[1] = cadd(m1, p1);
    v[4] = csub(m1, p1);
    v[2] = cadd(m2, p2);
    v[3] = csub(m2, p2);
  }
};

template <>
struct Dft<8> {
  TFFT_HD static void run(float2* v) {
    const float h = 0.70710678118654752440f;  // sqrt(1/2)
    float2 e[4] = {v[0], v[2], v[4], v[6]};
    float2 o[4] = {v[1], v[3], v[5], v[7]};
    Dft<4>::run(e);
    Dft<4>::run(o);
    // o[k] *= exp(-2 pi i k / 8)
    o[1] = make_float2(h * (o[1].x + o[1].y), h * (o[1].y - o[1].x));
    o[2] = mul_mi(o[2]);
    o[3] = make_float2(h * (o[3].y - o[3].x), -h * (o[3].x + o[3].y));
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      v[k] = cadd(e[k], o[k]);
      v[k + 4] = csub(e[k], o[k]);
    }
  }
};

template <>
struct Dft<16> {
  TFFT_HD static void run(float2* v) {
    // 16 = 4 x 4: inner DFT4 over n2 for each n1 (n = 4 n2 + n1), twiddle
    // exp(-2 pi i n1 k1 / 16), outer DFT4 over n1; output k = k1 + 4 k2.
    const float c = 0.92387953251128675613f;  // cos(pi / 8)
    const float s = 0.38268343236508977173f;  // sin(pi / 8)
    const float h = 0.70710678118654752440f;
    float2 y[4][4];
#pragma unroll
    for (int n1 = 0; n1 < 4; ++n1) {
      y[n1][0] = v[n1];
      y[n1][1] = v[4 + n1];
      y[n1][2] = v[8 + n1];
      y[n1][3] = v[12 + n1];
      Dft<4>::run(y[n1]);
    }
    // twiddles w16^(n1 k1) for n1, k1 in 1..3
    const float2 w1 = make_float2(c, -s), w2 = make_float2(h, -h), w3 = make_float2(s, -c);
    const float2 w6 = make_float2(-h, -h), w9 = make_float2(-c, s);
    y[1][1] = cmul(y[1][1], w1);
    y[1][2] = cmul(y[1][2], w2);
    y[1][3] = cmul(y[1][3], w3);
    y[2][1] = cmul(y[2][1], w2);
    y[2][2] = mul_mi(y[2][2]);
    y[2][3] = cmul(y[2][3], w6);
    y[3][1] = cmul(y[3][1], w3);
    y[3][2] = cmul(y[3][2], w6);
    y[3][3] = cmul(y[3][3], w9);
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
      float2 z[4] = {y[0][k1], y[1][k1], y[2][k1], y[3][k1]};
      Dft<4>::run(z);
      v[k1] = z[0];
      v[k1 + 4] = z[1];
      v[k1 + 8] = z[2];
      v[k1 + 12] = z[3];
    }
  }
};

// exp(-2 pi i m / 32) for 0 <= m < 32, from cos(pi j / 16), j = 0..8, by
// the symmetries of the circle.
TFFT_HD float2 w32(int m) {
  const float c[9] = {1.0f,
                      0.98078528040323044913f,
                      0.92387953251128675613f,
                      0.83146961230254523708f,
                      0.70710678118654752440f,
                      0.55557023301960222474f,
                      0.38268343236508977173f,
                      0.19509032201612826785f,
                      0.0f};
  // cos and sin of pi m / 16 for m in [0, 32)
  const int q = m & 7, oct = m >> 3;  // m = 8 oct + q
  float cs, sn;
  switch (oct) {
    case 0: cs = c[q]; sn = c[8 - q]; break;
    case 1: cs = -c[8 - q]; sn = c[q]; break;
    case 2: cs = -c[q]; sn = -c[8 - q]; break;
    default: cs = c[8 - q]; sn = -c[q]; break;
  }
  return make_float2(cs, -sn);
}

template <>
struct Dft<32> {
  TFFT_HD static void run(float2* v) {
    // 32 = 4 x 8: inner DFT8 over n2 for each n1 (n = 4 n2 + n1), twiddle
    // exp(-2 pi i n1 k1 / 32), outer DFT4 over n1; output k = k1 + 8 k2.
    float2 y[4][8];
#pragma unroll
    for (int n1 = 0; n1 < 4; ++n1) {
#pragma unroll
      for (int n2 = 0; n2 < 8; ++n2) y[n1][n2] = v[4 * n2 + n1];
      Dft<8>::run(y[n1]);
    }
#pragma unroll
    for (int n1 = 1; n1 < 4; ++n1)
#pragma unroll
      for (int k1 = 1; k1 < 8; ++k1) y[n1][k1] = cmul(y[n1][k1], w32(n1 * k1));
#pragma unroll
    for (int k1 = 0; k1 < 8; ++k1) {
      float2 z[4] = {y[0][k1], y[1][k1], y[2][k1], y[3][k1]};
      Dft<4>::run(z);
#pragma unroll
      for (int k2 = 0; k2 < 4; ++k2) v[k1 + 8 * k2] = z[k2];
    }
  }
};

// ------------------------------------------------------------ Stockham schedule
//
// A length-L FFT with radices R_0, R_1, ... (product L).  Stage s has span
// Ns = R_0 ... R_{s-1}.  Work item j (0 <= j < L / R) of a stage reads
// x[j + r L / R] (r < R), multiplies input r by exp(-2 pi i r k / (Ns R)),
// k = j mod Ns, runs a size-R DFT and writes output r to
// (j / Ns) Ns R + k + r Ns.  After the last stage the result is in natural
// order (self-sorting).  Twiddles are read from one table of the L roots
// exp(-2 pi i m / L), index m = r k L / (Ns R) < L.

TFFT_HD int stockham_out_index(int j, int Ns, int R, int r) {
  const int k = j % Ns;
  return (j / Ns) * Ns * R + k + r * Ns;
}

TFFT_HD int stockham_tw_index(int j, int Ns, int R, int r, int L) {
  const int k = j % Ns;
  return r * k * (L / (Ns * R));
}

// FFT plan of one axis length, shared by host planning and device kernels.
// The radices are also packed 5 bits per stage in `code` so that kernels read
// stage s's radix with a shift instead of an indexed load.
struct AxisPlan {
  int L;           // transform length
  int E;           // elements per thread (every radix divides E)
  int T;           // threads per line = L / E
  int nst;         // number of radix stages
  uint64_t code;   // radix of stage s = (code >> 5 s) & 31
  int spec;        // 1: a compile-time specialised kernel exists for this plan
  int width;       // lines per CTA (contiguous) or tile width W (strided)
  int radix[MAXSTAGES];
  int blue_m;      // > 0: length without a 2/3/5 plan, done by Bluestein with this convolution length
  int blue_spec;   // 1: that convolution length has compile-time specialised kernels (width is theirs)
};

TFFT_HD int stage_radix(uint64_t code, int s) { return (int)((code >> (5 * s)) & 31); }

}  // namespace tfft
