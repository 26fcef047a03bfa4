// CUDA kernels of the transpose-algorithm FFT on a virtual process grid
// (sm_103a).  Every 1-D FFT runs as a self-sorting Stockham schedule (see
// tfft_common.cuh): each thread keeps E elements of a line in registers, the
// radix-R butterflies of a stage run on them, and the line is exchanged
// through shared memory between stages.  Global memory is touched once per
// element per pass: the first stage loads straight from HBM and the last
// stage stores straight to HBM.
#include <type_traits>

#include "tfft_internal.h"

namespace tfft {

namespace {

template <int E, class F>
__device__ __forceinline__ void with_radix(int R, F&& f) {
  switch (R) {
    case 2:
      if constexpr (E % 2 == 0) f(std::integral_constant<int, 2>{});
      break;
    case 3:
      if constexpr (E % 3 == 0) f(std::integral_constant<int, 3>{});
      break;
    case 4:
      if constexpr (E % 4 == 0) f(std::integral_constant<int, 4>{});
      break;
    case 5:
      if constexpr (E % 5 == 0) f(std::integral_constant<int, 5>{});
      break;
    case 8:
      if constexpr (E % 8 == 0) f(std::integral_constant<int, 8>{});
      break;
    case 16:
      if constexpr (E % 16 == 0) f(std::integral_constant<int, 16>{});
      break;
    default:
      break;
  }
}

// Twiddle and butterfly of the E / R work items a thread owns in one stage.
// Work item q of thread jt is j = jt + q T; its inputs sit in v[q R + r].
template <int E, int R>
__device__ __forceinline__ void radix_stage(float2 (&v)[E], int jt, int T, int Ns, int L,
                                            const float2* __restrict__ tw) {
#pragma unroll
  for (int q = 0; q < E / R; ++q) {
    if (Ns > 1) {
      const int j = jt + q * T;
      const int step = (j % Ns) * (L / (Ns * R));
#pragma unroll
      for (int r = 1; r < R; ++r) v[q * R + r] = cmul(v[q * R + r], __ldg(&tw[r * step]));
    }
    Dft<R>::run(&v[q * R]);
  }
}

__device__ __forceinline__ int padpos(int pos) { return pos + (pos >> 4); }

// ------------------------------------------------------------ contiguous lines

template <int E>
__global__ void __launch_bounds__(512, 2) k_fft_contig(const ContigArgs a) {
  const float oscale = contig_scale(a);
  extern __shared__ float2 smem[];
  const int L = a.ap.L, T = a.ap.T, nst = a.ap.nst;
  const int jt = threadIdx.x, ly = threadIdx.y, B = blockDim.y;
  const int Lp = L + (L >> 4);
  float2* sl = smem + ly * Lp;
  const bool inv = a.sign > 0;
  for (int64_t base = (int64_t)blockIdx.x * B; base < a.nlines; base += (int64_t)gridDim.x * B) {
    const int64_t line = base + ly;
    const bool act = line < a.nlines;
    const float2* src = a.in + line * L;
    float2* dst = a.out + line * L;
    if (nst == 0) {  // length-1 axis: the DFT is the identity
      if (act && jt == 0) dst[0] = cscale(src[0], oscale);
      continue;
    }
    float2 v[E];
    int Ns = 1;
    for (int s = 0; s < nst; ++s) {
      const int R = stage_radix(a.ap.code, s);
      if (s == 0) {
        with_radix<E>(R, [&](auto rc) {
          constexpr int RR = decltype(rc)::value;
#pragma unroll
          for (int q = 0; q < E / RR; ++q)
#pragma unroll
            for (int r = 0; r < RR; ++r) {
              const int pos = jt + q * T + r * (L / RR);
              float2 x = act ? src[pos] : make_float2(0.f, 0.f);
              if (inv) x.y = -x.y;
              v[q * RR + r] = x;
            }
        });
      } else {
        const int Rp = stage_radix(a.ap.code, s - 1);
        const int Nsp = Ns / Rp;
        __syncthreads();
        with_radix<E>(Rp, [&](auto rc) {
          constexpr int RR = decltype(rc)::value;
#pragma unroll
          for (int q = 0; q < E / RR; ++q)
#pragma unroll
            for (int r = 0; r < RR; ++r)
              sl[padpos(stockham_out_index(jt + q * T, Nsp, RR, r))] = v[q * RR + r];
        });
        __syncthreads();
        with_radix<E>(R, [&](auto rc) {
          constexpr int RR = decltype(rc)::value;
#pragma unroll
          for (int q = 0; q < E / RR; ++q)
#pragma unroll
            for (int r = 0; r < RR; ++r) v[q * RR + r] = sl[padpos(jt + q * T + r * (L / RR))];
        });
      }
      with_radix<E>(R, [&](auto rc) {
        constexpr int RR = decltype(rc)::value;
        radix_stage<E, RR>(v, jt, T, Ns, L, a.tw);
      });
      Ns *= R;
    }
    with_radix<E>(stage_radix(a.ap.code, nst - 1), [&](auto rc) {
      constexpr int RR = decltype(rc)::value;
#pragma unroll
      for (int q = 0; q < E / RR; ++q)
#pragma unroll
        for (int r = 0; r < RR; ++r) {
          float2 x = cscale(v[q * RR + r], oscale);
          if (inv) x.y = -x.y;
          if (act) dst[jt + q * T + r * (L / RR)] = x;
        }
    });
  }
}

// ------------------------------------------------------------ strided lines

template <int E>
__global__ void __launch_bounds__(512, 1) k_fft_strided(const StridedArgs a) {
  extern __shared__ float2 smem[];
  const int L = a.ap.L, T = a.ap.T, nst = a.ap.nst, W = a.W;
  const int cx = threadIdx.x, jt = threadIdx.y;
  const int tid = jt * W + cx, nthr = W * T;
  int64_t* rin = reinterpret_cast<int64_t*>(smem + (size_t)L * W);
  int64_t* rout = rin + L;
  const bool inv = a.sign > 0;
  const int64_t ntiles = a.nouter * a.ncolblocks;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const StridedTilePos tp(a, tile);
    const int2 blk = tp.blk;
    const TileRows ri(a, a.lin, tp), ro(a, a.lout, tp);
    __syncthreads();  // the previous tile is done with the row tables
    for (int i = tid; i < L; i += nthr) {
      rin[i] = ri.row(a.lin, i);
      rout[i] = ro.row(a.lout, i);
    }
    __syncthreads();
    const bool act = cx < blk.y;
    if (nst == 0) {
      if (act && jt == 0) a.out[rout[0] + cx] = cscale(a.in[rin[0] + cx], a.scale);
      continue;
    }
    float2 v[E];
    int Ns = 1;
    for (int s = 0; s < nst; ++s) {
      const int R = stage_radix(a.ap.code, s);
      if (s == 0) {
        with_radix<E>(R, [&](auto rc) {
          constexpr int RR = decltype(rc)::value;
#pragma unroll
          for (int q = 0; q < E / RR; ++q)
#pragma unroll
            for (int r = 0; r < RR; ++r) {
              const int pos = jt + q * T + r * (L / RR);
              float2 x = act ? a.in[rin[pos] + cx] : make_float2(0.f, 0.f);
              if (inv) x.y = -x.y;
              v[q * RR + r] = x;
            }
        });
      } else {
        const int Rp = stage_radix(a.ap.code, s - 1);
        const int Nsp = Ns / Rp;
        __syncthreads();
        with_radix<E>(Rp, [&](auto rc) {
          constexpr int RR = decltype(rc)::value;
#pragma unroll
          for (int q = 0; q < E / RR; ++q)
#pragma unroll
            for (int r = 0; r < RR; ++r)
              smem[stockham_out_index(jt + q * T, Nsp, RR, r) * W + cx] = v[q * RR + r];
        });
        __syncthreads();
        with_radix<E>(R, [&](auto rc) {
          constexpr int RR = decltype(rc)::value;
#pragma unroll
          for (int q = 0; q < E / RR; ++q)
#pragma unroll
            for (int r = 0; r < RR; ++r)
              v[q * RR + r] = smem[(jt + q * T + r * (L / RR)) * W + cx];
        });
      }
      with_radix<E>(R, [&](auto rc) {
        constexpr int RR = decltype(rc)::value;
        radix_stage<E, RR>(v, jt, T, Ns, L, a.tw);
      });
      Ns *= R;
    }
    with_radix<E>(stage_radix(a.ap.code, nst - 1), [&](auto rc) {
      constexpr int RR = decltype(rc)::value;
#pragma unroll
      for (int q = 0; q < E / RR; ++q)
#pragma unroll
        for (int r = 0; r < RR; ++r) {
          const int pos = jt + q * T + r * (L / RR);
          float2 x = cscale(v[q * RR + r], a.scale);
          if (inv) x.y = -x.y;
          if (act) a.out[rout[pos] + cx] = x;
        }
    });
  }
}

// ------------------------------------------------------------ generic lengths
//
// Lengths whose radices have no common register budget (those with all of
// 2, 3 and 5 as factors, e.g. 60 or 120) keep the whole line in shared memory
// between stages: two buffers, each stage reads one and writes the other,
// every thread looping over the stage's L / R work items.

template <int R>
__device__ __forceinline__ void generic_stage(const float2* __restrict__ src, float2* __restrict__ dst,
                                              int L, int Ns, int T, int jt, int stride, int cx,
                                              const float2* __restrict__ tw) {
  for (int j = jt; j < L / R; j += T) {
    float2 x[R];
#pragma unroll
    for (int r = 0; r < R; ++r) x[r] = src[(j + r * (L / R)) * stride + cx];
    if (Ns > 1) {
      const int step = (j % Ns) * (L / (Ns * R));
#pragma unroll
      for (int r = 1; r < R; ++r) x[r] = cmul(x[r], __ldg(&tw[r * step]));
    }
    Dft<R>::run(x);
#pragma unroll
    for (int r = 0; r < R; ++r) dst[stockham_out_index(j, Ns, R, r) * stride + cx] = x[r];
  }
}

// Runs every stage between the two shared buffers; returns the buffer that
// holds the result.
__device__ __forceinline__ float2* generic_fft(float2* b0, float2* b1, const AxisPlan& ap, int jt,
                                               int stride, int cx, const float2* __restrict__ tw) {
  int Ns = 1;
  float2* src = b0;
  float2* dst = b1;
  for (int s = 0; s < ap.nst; ++s) {
    const int R = stage_radix(ap.code, s);
    switch (R) {
      case 2: generic_stage<2>(src, dst, ap.L, Ns, ap.T, jt, stride, cx, tw); break;
      case 3: generic_stage<3>(src, dst, ap.L, Ns, ap.T, jt, stride, cx, tw); break;
      case 4: generic_stage<4>(src, dst, ap.L, Ns, ap.T, jt, stride, cx, tw); break;
      case 5: generic_stage<5>(src, dst, ap.L, Ns, ap.T, jt, stride, cx, tw); break;
      case 8: generic_stage<8>(src, dst, ap.L, Ns, ap.T, jt, stride, cx, tw); break;
      case 16: generic_stage<16>(src, dst, ap.L, Ns, ap.T, jt, stride, cx, tw); break;
      default: break;
    }
    __syncthreads();
    float2* t = src;
    src = dst;
    dst = t;
    Ns *= R;
  }
  return src;
}

__global__ void __launch_bounds__(512) k_fft_contig_generic(const ContigArgs a) {
  const float oscale = contig_scale(a);
  extern __shared__ float2 smem[];
  const int L = a.ap.L, T = a.ap.T;
  const int jt = threadIdx.x, ly = threadIdx.y, B = blockDim.y;
  float2* b0 = smem + (size_t)ly * L;
  float2* b1 = smem + (size_t)(B + ly) * L;
  const bool inv = a.sign > 0;
  for (int64_t base = (int64_t)blockIdx.x * B; base < a.nlines; base += (int64_t)gridDim.x * B) {
    const int64_t line = base + ly;
    const bool act = line < a.nlines;
    __syncthreads();
    for (int i = jt; i < L; i += T) {
      float2 x = act ? a.in[line * L + i] : make_float2(0.f, 0.f);
      if (inv) x.y = -x.y;
      b0[i] = x;
    }
    __syncthreads();
    const float2* res = generic_fft(b0, b1, a.ap, jt, 1, 0, a.tw);
    for (int i = jt; i < L; i += T) {
      float2 x = cscale(res[i], oscale);
      if (inv) x.y = -x.y;
      if (act) a.out[line * L + i] = x;
    }
  }
}

__global__ void __launch_bounds__(512) k_fft_strided_generic(const StridedArgs a) {
  extern __shared__ float2 smem[];
  const int L = a.ap.L, T = a.ap.T, W = a.W;
  const int cx = threadIdx.x, jt = threadIdx.y;
  const int tid = jt * W + cx, nthr = W * T;
  float2* b0 = smem;
  float2* b1 = smem + (size_t)L * W;
  int64_t* rin = reinterpret_cast<int64_t*>(smem + 2 * (size_t)L * W);
  int64_t* rout = rin + L;
  const bool inv = a.sign > 0;
  const int64_t ntiles = a.nouter * a.ncolblocks;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const StridedTilePos tp(a, tile);
    const int2 blk = tp.blk;
    const TileRows ri(a, a.lin, tp), ro(a, a.lout, tp);
    __syncthreads();
    for (int i = tid; i < L; i += nthr) {
      rin[i] = ri.row(a.lin, i);
      rout[i] = ro.row(a.lout, i);
    }
    __syncthreads();
    for (int idx = tid; idx < L * W; idx += nthr) {
      const int pos = idx / W, c = idx - (idx / W) * W;
      float2 x = (c < blk.y) ? a.in[rin[pos] + c] : make_float2(0.f, 0.f);
      if (inv) x.y = -x.y;
      b0[idx] = x;
    }
    __syncthreads();
    const float2* res = generic_fft(b0, b1, a.ap, jt, W, cx, a.tw);
    for (int idx = tid; idx < L * W; idx += nthr) {
      const int pos = idx / W, c = idx - (idx / W) * W;
      float2 x = cscale(res[idx], a.scale);
      if (inv) x.y = -x.y;
      if (c < blk.y) a.out[rout[pos] + c] = x;
    }
  }
}

// ------------------------------------------------------------ Bluestein
//
// A line of length N with no 2/3/5 factorisation: with c[n] = exp(i pi n^2 / N),
// X[k] = conj(c[k]) * sum_n (x[n] conj(c[n])) c[k - n], a circular
// convolution once a = x conj(c) is zero-padded to M >= 2N - 1 and c is
// wrapped around (b[m] = b[M - m] = c[m]).  The convolution is done as
// FFT_M(a) * (FFT_M(b) / M) followed by an inverse FFT, taken as
// conj o FFT_M o conj.

__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }

// Convolution of the chirped, zero-padded column (stride, cx) held in b0;
// returns the buffer (b0 or b1) holding conj(a (*) b).
__device__ __forceinline__ float2* blue_convolve(float2* b0, float2* b1, const BlueArgs& b, int jt, int T,
                                                 int stride, int cx) {
  float2* r = generic_fft(b0, b1, b.apm, jt, stride, cx, b.twm);
  for (int i = jt; i < b.M; i += T) r[i * stride + cx] = cconj(cmul(r[i * stride + cx], __ldg(&b.bhat[i])));
  __syncthreads();
  return generic_fft(r, r == b0 ? b1 : b0, b.apm, jt, stride, cx, b.twm);
}

__global__ void __launch_bounds__(512) k_blue_contig(const ContigArgs a, const BlueArgs b) {
  const float oscale = contig_scale(a);
  extern __shared__ float2 smem[];
  const int N = b.N, M = b.M, T = b.apm.T;
  const int jt = threadIdx.x, ly = threadIdx.y, B = blockDim.y;
  float2* b0 = smem + (size_t)ly * M;
  float2* b1 = smem + (size_t)(B + ly) * M;
  const bool inv = a.sign > 0;
  for (int64_t base = (int64_t)blockIdx.x * B; base < a.nlines; base += (int64_t)gridDim.x * B) {
    const int64_t line = base + ly;
    const bool act = line < a.nlines;
    __syncthreads();
    for (int i = jt; i < M; i += T) {
      float2 v = make_float2(0.f, 0.f);
      if (act && i < N) {
        v = a.in[line * N + i];
        if (inv) v.y = -v.y;
        v = cmul(v, __ldg(&b.chirp[i]));
      }
      b0[i] = v;
    }
    __syncthreads();
    const float2* r = blue_convolve(b0, b1, b, jt, T, 1, 0);
    for (int k = jt; k < N; k += T) {
      float2 y = cscale(cmul(cconj(r[k]), __ldg(&b.chirp[k])), oscale);
      if (inv) y.y = -y.y;
      if (act) a.out[line * N + k] = y;
    }
  }
}

__global__ void __launch_bounds__(512) k_blue_strided(const StridedArgs a, const BlueArgs b) {
  extern __shared__ float2 smem[];
  const int N = b.N, M = b.M, T = b.apm.T, W = a.W;
  const int cx = threadIdx.x, jt = threadIdx.y;
  const int tid = jt * W + cx, nthr = W * T;
  float2* b0 = smem;
  float2* b1 = smem + (size_t)M * W;
  int64_t* rin = reinterpret_cast<int64_t*>(smem + 2 * (size_t)M * W);
  int64_t* rout = rin + N;
  const bool inv = a.sign > 0;
  const int64_t ntiles = a.nouter * a.ncolblocks;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const StridedTilePos tp(a, tile);
    const int2 blk = tp.blk;
    const TileRows ri(a, a.lin, tp), ro(a, a.lout, tp);
    __syncthreads();
    for (int i = tid; i < N; i += nthr) {
      rin[i] = ri.row(a.lin, i);
      rout[i] = ro.row(a.lout, i);
    }
    __syncthreads();
    for (int idx = tid; idx < M * W; idx += nthr) {
      const int pos = idx / W, c = idx - (idx / W) * W;
      float2 v = make_float2(0.f, 0.f);
      if (pos < N && c < blk.y) {
        v = a.in[rin[pos] + c];
        if (inv) v.y = -v.y;
        v = cmul(v, __ldg(&b.chirp[pos]));
      }
      b0[idx] = v;
    }
    __syncthreads();
    const float2* r = blue_convolve(b0, b1, b, jt, T, W, cx);
    for (int idx = tid; idx < N * W; idx += nthr) {
      const int pos = idx / W, c = idx - (idx / W) * W;
      float2 y = cscale(cmul(cconj(r[idx]), __ldg(&b.chirp[pos])), a.scale);
      if (inv) y.y = -y.y;
      if (c < blk.y) a.out[rout[pos] + c] = y;
    }
  }
}

// ------------------------------------------------------------ box copy

// One CTA per copy task.  The task's rows are spread over the CTA in slots of
// `lpr` lanes (the smallest power of two covering the row, at most 256), and
// every thread keeps U rows' loads in flight before it stores them; no
// division per row or element.  T is float4 (pairs of complex64) when every
// offset, stride and row length of the launch is even, else float2.
template <class T, int U>
__global__ void __launch_bounds__(256) k_boxcopy(const BoxArgs a) {
  constexpr int K = sizeof(T) / sizeof(float2);
  const CopyTask* tp = a.tasks + blockIdx.x;
  const int nrows = tp->nrows;
  const int rowlen = tp->rowlen / K;  // in copy units
  if (nrows <= 0 || rowlen <= 0) return;
  const T* src = reinterpret_cast<const T*>(a.in + tp->src);
  T* dst = reinterpret_cast<T*>(a.out + tp->dst);
  const int64_t ss = tp->ss / K, ds = tp->ds / K;
  const int lpr = rowlen >= 256 ? 256 : (rowlen <= 1 ? 1 : 1 << (32 - __clz(rowlen - 1)));
  const int slots = 256 / lpr;
  const int lane = threadIdx.x % lpr, slot = threadIdx.x / lpr;
  for (int r0 = slot; r0 < nrows; r0 += slots * U) {
    for (int c = lane; c < rowlen; c += lpr) {
      T v[U];
#pragma unroll
      for (int k = 0; k < U; ++k) {
        const int r = r0 + k * slots;
        if (r < nrows) v[k] = src[r * ss + c];
      }
#pragma unroll
      for (int k = 0; k < U; ++k) {
        const int r = r0 + k * slots;
        if (r < nrows) dst[r * ds + c] = v[k];
      }
    }
  }
}

// ------------------------------------------------------------ twiddles

// exp(-2 pi i m / L) for m < L, evaluated in double precision and rounded to
// float (the only double-precision arithmetic of the path besides the
// normalisation factor).
__global__ void k_twiddles(float2* tw, int L) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m < L) {
    double s, c;
    sincospi(2.0 * (double)m / (double)L, &s, &c);
    tw[m] = make_float2((float)c, (float)(-s));
  }
}

// the kernel's shared-memory limit raised to 227 KB, once per device
#define TFFT_ALLOW_SMEM(kernel)                          \
  static PerDevice<cudaError_t> attr_cache;              \
  const cudaError_t attr = smem_attr_once(attr_cache, kernel, 227 * 1024)

constexpr int64_t kMaxGrid = 1 << 20;

template <int E>
cudaError_t launch_contig_E(const ContigArgs& a, cudaStream_t s) {
  TFFT_ALLOW_SMEM(k_fft_contig<E>);
  if (attr != cudaSuccess) return attr;
  const int B = a.lines_per_cta;
  const int L = a.ap.L;
  const size_t smem = (size_t)B * (L + (L >> 4)) * sizeof(float2);
  int64_t grid = (a.nlines + B - 1) / B;
  if (grid > kMaxGrid) grid = kMaxGrid;
  if (grid < 1) return cudaSuccess;
  k_fft_contig<E><<<(unsigned)grid, dim3(a.ap.T, B), smem, s>>>(a);
  return cudaGetLastError();
}

template <int E>
cudaError_t launch_strided_E(const StridedArgs& a, cudaStream_t s) {
  TFFT_ALLOW_SMEM(k_fft_strided<E>);
  if (attr != cudaSuccess) return attr;
  const int L = a.ap.L;
  const size_t smem = (size_t)L * a.W * sizeof(float2) + 2 * (size_t)L * sizeof(int64_t);
  int64_t grid = a.nouter * a.ncolblocks;
  if (grid > kMaxGrid) grid = kMaxGrid;
  if (grid < 1) return cudaSuccess;
  k_fft_strided<E><<<(unsigned)grid, dim3(a.W, a.ap.T), smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace

#define TFFT_FOR_EACH_E(X) \
  X(1) X(2) X(3) X(4) X(5) X(6) X(8) X(10) X(12) X(15) X(16) X(20) X(24)

bool kernel_supports_E(int E) {
  switch (E) {
#define X(e) case e:
    TFFT_FOR_EACH_E(X)
#undef X
    return true;
    default:
      return false;
  }
}

cudaError_t launch_contig(const ContigArgs& a, cudaStream_t s) {
  if (a.ap.spec) return launch_contig_spec(a, s);
  if (a.ap.E == 0) {
    TFFT_ALLOW_SMEM(k_fft_contig_generic);
    if (attr != cudaSuccess) return attr;
    const int B = a.lines_per_cta;
    const size_t smem = 2 * (size_t)B * a.ap.L * sizeof(float2);
    int64_t grid = (a.nlines + B - 1) / B;
    if (grid > kMaxGrid) grid = kMaxGrid;
    if (grid < 1) return cudaSuccess;
    k_fft_contig_generic<<<(unsigned)grid, dim3(a.ap.T, B), smem, s>>>(a);
    return cudaGetLastError();
  }
  switch (a.ap.E) {
#define X(e) \
  case e:    \
    return launch_contig_E<e>(a, s);
    TFFT_FOR_EACH_E(X)
#undef X
    default:
      return cudaErrorInvalidValue;
  }
}

cudaError_t launch_strided(const StridedArgs& a, cudaStream_t s) {
  if (a.ap.spec) return launch_strided_spec(a, s);
  if (a.ap.E == 0) {
    TFFT_ALLOW_SMEM(k_fft_strided_generic);
    if (attr != cudaSuccess) return attr;
    const int L = a.ap.L;
    const size_t smem = 2 * (size_t)L * a.W * sizeof(float2) + 2 * (size_t)L * sizeof(int64_t);
    int64_t grid = a.nouter * a.ncolblocks;
    if (grid > kMaxGrid) grid = kMaxGrid;
    if (grid < 1) return cudaSuccess;
    k_fft_strided_generic<<<(unsigned)grid, dim3(a.W, a.ap.T), smem, s>>>(a);
    return cudaGetLastError();
  }
  switch (a.ap.E) {
#define X(e) \
  case e:    \
    return launch_strided_E<e>(a, s);
    TFFT_FOR_EACH_E(X)
#undef X
    default:
      return cudaErrorInvalidValue;
  }
}

cudaError_t launch_contig_blue(const ContigArgs& a, const BlueArgs& b, cudaStream_t s) {
  if (a.ap.blue_spec) return launch_contig_blue_spec(a, b, s);
  TFFT_ALLOW_SMEM(k_blue_contig);
  if (attr != cudaSuccess) return attr;
  const int B = a.lines_per_cta;
  const size_t smem = 2 * (size_t)B * b.M * sizeof(float2);
  int64_t grid = (a.nlines + B - 1) / B;
  if (grid > kMaxGrid) grid = kMaxGrid;
  if (grid < 1) return cudaSuccess;
  k_blue_contig<<<(unsigned)grid, dim3(b.apm.T, B), smem, s>>>(a, b);
  return cudaGetLastError();
}

cudaError_t launch_strided_blue(const StridedArgs& a, const BlueArgs& b, cudaStream_t s) {
  if (a.ap.blue_spec) return launch_strided_blue_spec(a, b, s);
  TFFT_ALLOW_SMEM(k_blue_strided);
  if (attr != cudaSuccess) return attr;
  const size_t smem = 2 * (size_t)b.M * a.W * sizeof(float2) + 2 * (size_t)b.N * sizeof(int64_t);
  int64_t grid = a.nouter * a.ncolblocks;
  if (grid > kMaxGrid) grid = kMaxGrid;
  if (grid < 1) return cudaSuccess;
  k_blue_strided<<<(unsigned)grid, dim3(a.W, b.apm.T), smem, s>>>(a, b);
  return cudaGetLastError();
}

cudaError_t launch_boxcopy(const BoxArgs& a, cudaStream_t s) {
  if (a.ntasks <= 0) return cudaSuccess;
  if (a.ntasks > 0x7fffffff) return cudaErrorInvalidConfiguration;
  if (a.vec2)
    k_boxcopy<float4, 4><<<(unsigned)a.ntasks, 256, 0, s>>>(a);
  else
    k_boxcopy<float2, 4><<<(unsigned)a.ntasks, 256, 0, s>>>(a);
  return cudaGetLastError();
}

int current_device() {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return -1;
  return dev;
}

int device_sm_count() {
  static PerDevice<int> cache;
  const int dev = current_device();
  return cache.get(dev, [dev] {
    int v = 0;
    if (dev < 0 || cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) v = 0;
    return v > 0 ? v : 1;
  });
}

cudaError_t launch_twiddles(float2* tw, int L, cudaStream_t s) {
  k_twiddles<<<(L + 255) / 256, 256, 0, s>>>(tw, L);
  return cudaGetLastError();
}

}  // namespace tfft
