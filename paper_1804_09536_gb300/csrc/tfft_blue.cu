// Bluestein passes with compile-time specialised convolution lengths.
//
// A line of length N with no 2/3/5 factorisation (the paper only needs some
// serial 1-D FFT per axis; App. A's 42 x 127 x 256 has two such axes) is
// transformed as a circular convolution: with the chirp c[n] = exp(-i pi
// (n^2 mod 2N) / N),  X[k] = c[k] sum_n (x[n] c[n]) conj(c[k - n]),  i.e.
// y = x c zero-padded to M = 2^ceil(log2(2N - 1)), Y = FFT_M(y) bhat with
// bhat = FFT_M(b) / M for the wrapped filter b[m] = b[M - m] = conj(c[m]),
// X = c IFFT_M(Y), the inverse taken as conj o FFT_M o conj.  Here both
// length-M FFTs run as register-resident Stockham stages (the specialised
// radices of that length), the first one straight on the chirped input, the
// pointwise filter on its output registers, one exchange through shared
// memory back to the first stage's order, the second FFT, and the output
// chirp on its registers: one read and one write of every element, as in
// the other passes.  The chirp and filter tables are built on the host in
// double precision and rounded once.
#include "tfft_tiles.cuh"

namespace tfft {

namespace {

using namespace tiles;

__device__ __forceinline__ float2 conjf2(float2 a) { return make_float2(a.x, -a.y); }

// ------------------------------------------------------------ contiguous lines

// B lines per CTA, thread jt of line ly; lines are N long in memory.
template <int M, int E, int B, int... Rs>
__global__ void __launch_bounds__((M / E) * B, min_blocks(E, (M / E) * B, 512))
    k_blue_contig_spec(const ContigArgs a, const BlueArgs b) {
  constexpr int T = M / E, NST = sizeof...(Rs);
  constexpr int R0 = radix_at<0, Rs...>(), RL = radix_at<NST - 1, Rs...>();
  constexpr int LP = line_pitch<M, Rs...>();
  constexpr int P = pad_every<Rs...>();
  extern __shared__ float2 smem[];
  const int N = b.N;
  const int ly = threadIdx.y;
  float2* sl = smem + ly * LP;
  const bool inv = a.sign > 0;
  const float oscale = contig_scale(a);
  for (int64_t base = (int64_t)blockIdx.x * B; base < a.nlines; base += (int64_t)gridDim.x * B) {
    const int64_t line = base + ly;
    const bool act = line < a.nlines;
    const float2* src = a.in + line * N;
    float2* dst = a.out + line * N;
    const int jt = opaque_tid_x();
    float2 v[E];
#pragma unroll
    for (int q = 0; q < E / R0; ++q)
#pragma unroll
      for (int r = 0; r < R0; ++r) {
        const int pos = jt + q * T + r * (M / R0);
        float2 x = make_float2(0.f, 0.f);
        if (act && pos < N) {
          x = src[pos];
          if (inv) x.y = -x.y;
          x = cmul(x, __ldg(&b.chirp[pos]));
        }
        v[q * R0 + r] = x;
      }
    line_stages<M, E, Rs...>(v, sl, jt, b.twm);
    // filter, conjugated for the inverse, then back to the first stage's order
    line_sync<T>();
#pragma unroll
    for (int q = 0; q < E / RL; ++q)
#pragma unroll
      for (int r = 0; r < RL; ++r) {
        const int p = jt + q * T + r * (M / RL);
        sl[padp<P>(p)] = conjf2(cmul(v[q * RL + r], __ldg(&b.bhat[p])));
      }
    line_sync<T>();
#pragma unroll
    for (int q = 0; q < E / R0; ++q)
#pragma unroll
      for (int r = 0; r < R0; ++r) v[q * R0 + r] = sl[padp<P>(jt + q * T + r * (M / R0))];
    line_stages<M, E, Rs...>(v, sl, jt, b.twm);
#pragma unroll
    for (int q = 0; q < E / RL; ++q)
#pragma unroll
      for (int r = 0; r < RL; ++r) {
        const int p = jt + q * T + r * (M / RL);
        if (act && p < N) {
          float2 y = cscale(cmul(conjf2(v[q * RL + r]), __ldg(&b.chirp[p])), oscale);
          if (inv) y.y = -y.y;
          dst[p] = y;
        }
      }
    line_sync<T>();  // the line slot is free for the next group
  }
}

// ------------------------------------------------------------ strided lines

// Tile = the N rows of W columns, held as M x W in shared memory between the
// stages; row tables of the input and output layouts (tile_fold /
// row_offset) and a per-CTA table of every row's part and index.
template <int M, int W>
__host__ __device__ constexpr size_t blue_strided_smem(int N) {
  return (size_t)M * W * sizeof(float2) + 2 * (size_t)N * sizeof(int) + sizeof(TileShared) +
         2 * (size_t)N * sizeof(uint32_t);
}

// Registers sized for 768 resident threads per SM (three 256-thread CTAs at
// M = 256, a few bytes of spill): the pass is bound by instruction issue, and
// the third CTA's warps raise it (512 x 127 x 512: 0.383 -> 0.334 ms per
// pass); a 1024-thread target spills hundreds of bytes.
template <int M, int E, int W, int... Rs>
__global__ void __launch_bounds__(W * (M / E), min_blocks(E, W * (M / E), 768))
    k_blue_strided_spec(const StridedArgs a, const BlueArgs b) {
  constexpr int T = M / E, NST = sizeof...(Rs);
  constexpr int R0 = radix_at<0, Rs...>(), RL = radix_at<NST - 1, Rs...>();
  static_assert(W * T > 32, "the two layouts' folds are computed by threads 0 and 32");
  extern __shared__ float2 smem[];
  const int N = b.N;
  int* rin = reinterpret_cast<int*>(smem + M * W);
  int* rout = rin + N;
  TileShared* ts = reinterpret_cast<TileShared*>(rout + N);
  uint32_t* rp = reinterpret_cast<uint32_t*>(ts + 1);
  const int cx = threadIdx.x;
  const int tid = threadIdx.y * W + cx;
  const bool inv = a.sign > 0;
  const int64_t ntiles = a.nouter * a.ncolblocks;
  // part and index of every row of both layouts, once per CTA
  for (int i = tid; i < 2 * N; i += W * T) {
    const bool out = i >= N;
    const int row = out ? i - N : i;
    const int64_t NN = out ? a.lout.N[a.axis] : a.lin.N[a.axis];
    const int64_t MM = out ? a.lout.Mx[a.axis] : a.lin.Mx[a.axis];
    int64_t c = 0, l = row, n = NN;
    if (MM > 1) locate(NN, MM, row, c, l, n);
    rp[i] = ((uint32_t)c << 16) | (uint32_t)l;
  }
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    __syncthreads();  // the previous tile is done with the tables, the scalars and smem
    if (tid == 0) {
      const StridedTilePos tp(a, tile);
      tile_fold(a, a.lin, tp, ts, 0);
      ts->blk = tp.blk;
    } else if (tid == 32) {
      const StridedTilePos tp(a, tile);
      tile_fold(a, a.lout, tp, ts, 1);
    }
    __syncthreads();
    for (int i = tid; i < 2 * N; i += W * T) {
      const bool out = i >= N;
      const int row = out ? i - N : i;
      const int64_t c = rp[i] >> 16, l = rp[i] & 0xFFFF;
      if (out)
        rout[row] = row_offset(a.lout, a.axis, ts, 1, c, l);
      else
        rin[row] = row_offset(a.lin, a.axis, ts, 0, c, l);
    }
    __syncthreads();
    const int2 blk = ts->blk;
    const bool act = cx < blk.y;
    const int jt = opaque_tid_y();
    float2 v[E];
#pragma unroll
    for (int q = 0; q < E / R0; ++q)
#pragma unroll
      for (int r = 0; r < R0; ++r) {
        const int pos = jt + q * T + r * (M / R0);
        float2 x = make_float2(0.f, 0.f);
        if (act && pos < N) {
          x = a.in[rin[pos] + cx];
          if (inv) x.y = -x.y;
          x = cmul(x, __ldg(&b.chirp[pos]));
        }
        v[q * R0 + r] = x;
      }
    strided_stages<M, E, W, Rs...>(v, smem, cx, jt, b.twm);
    __syncthreads();
#pragma unroll
    for (int q = 0; q < E / RL; ++q)
#pragma unroll
      for (int r = 0; r < RL; ++r) {
        const int p = jt + q * T + r * (M / RL);
        smem[p * W + cx] = conjf2(cmul(v[q * RL + r], __ldg(&b.bhat[p])));
      }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < E / R0; ++q)
#pragma unroll
      for (int r = 0; r < R0; ++r) v[q * R0 + r] = smem[(jt + q * T + r * (M / R0)) * W + cx];
    strided_stages<M, E, W, Rs...>(v, smem, cx, jt, b.twm);
#pragma unroll
    for (int q = 0; q < E / RL; ++q)
#pragma unroll
      for (int r = 0; r < RL; ++r) {
        const int p = jt + q * T + r * (M / RL);
        if (act && p < N) {
          float2 y = cscale(cmul(conjf2(v[q * RL + r]), __ldg(&b.chirp[p])), a.scale);
          if (inv) y.y = -y.y;
          a.out[rout[p] + cx] = y;
        }
      }
  }
}

// Compiled convolution lengths.  Contiguous: M, elements per thread, lines
// per CTA, radices; strided: M, elements per thread, tile width, radices
// (uniform plans; at most 16 values per thread except the 512 tiles, so that
// two FFTs, the chirps and the filter fit the registers without spilling).
#define TFFT_BLUE_CONTIG(X)        \
  X(32, 8, 64, 8, 4)               \
  X(64, 8, 32, 8, 8)               \
  X(128, 16, 32, 16, 8)            \
  X(256, 16, 16, 16, 16)           \
  X(512, 16, 8, 16, 8, 4)          \
  X(1024, 16, 4, 16, 16, 4)        \
  X(2048, 16, 2, 16, 16, 8)        \
  X(4096, 16, 1, 16, 16, 16)
#define TFFT_BLUE_STRIDED(X)       \
  X(32, 8, 32, 8, 4)               \
  X(64, 8, 32, 8, 8)               \
  X(128, 16, 32, 16, 8)            \
  X(256, 16, 16, 16, 16)           \
  X(512, 32, 8, 32, 16)            \
  X(1024, 16, 8, 16, 16, 4)        \
  X(2048, 16, 4, 16, 16, 8)        \
  X(4096, 16, 2, 16, 16, 16)

// the kernel's shared-memory limit raised to 227 KB, once per device
#define TFFT_ALLOW_SMEM(kernel)                          \
  static PerDevice<cudaError_t> attr_cache;              \
  const cudaError_t attr = smem_attr_once(attr_cache, kernel, 227 * 1024)

constexpr int64_t kMaxGrid = 1 << 20;

template <int M, int E, int B, int... Rs>
cudaError_t run_blue_contig(const ContigArgs& a, const BlueArgs& b, cudaStream_t s) {
  TFFT_ALLOW_SMEM((k_blue_contig_spec<M, E, B, Rs...>));
  if (attr != cudaSuccess) return attr;
  if (a.lines_per_cta != B) return cudaErrorInvalidValue;
  const size_t smem = (size_t)B * line_pitch<M, Rs...>() * sizeof(float2);
  int64_t grid = (a.nlines + B - 1) / B;
  if (grid > kMaxGrid) grid = kMaxGrid;
  if (grid < 1) return cudaSuccess;
  k_blue_contig_spec<M, E, B, Rs...><<<(unsigned)grid, dim3(M / E, B), smem, s>>>(a, b);
  return cudaGetLastError();
}

template <int M, int E, int W, int... Rs>
cudaError_t run_blue_strided(const StridedArgs& a, const BlueArgs& b, cudaStream_t s) {
  TFFT_ALLOW_SMEM((k_blue_strided_spec<M, E, W, Rs...>));
  if (attr != cudaSuccess) return attr;
  if (a.W != W || 2 * b.N > M) return cudaErrorInvalidValue;
  const size_t smem = blue_strided_smem<M, W>(b.N);
  // persistent: the per-CTA row table is computed once
  static PerDevice<int64_t> slots_cache;
  const int64_t slots = slots_cache.get(current_device(), [&] {
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_blue_strided_spec<M, E, W, Rs...>, W * (M / E),
                                                  blue_strided_smem<M, W>(M / 2));
    return (int64_t)device_sm_count() * (per_sm > 0 ? per_sm : 1);
  });
  int64_t grid = a.nouter * a.ncolblocks;
  if (grid > slots) grid = slots;
  if (grid < 1) return cudaSuccess;
  k_blue_strided_spec<M, E, W, Rs...><<<(unsigned)grid, dim3(W, M / E), smem, s>>>(a, b);
  return cudaGetLastError();
}

}  // namespace

bool blue_spec_plan(int M, int& lines_per_cta, int& tile_width) {
  bool c = false, t = false;
#define X(MM, E, B, ...) \
  if (M == MM) {         \
    lines_per_cta = B;   \
    c = true;            \
  }
  TFFT_BLUE_CONTIG(X)
#undef X
#define X(MM, E, W, ...) \
  if (M == MM) {         \
    tile_width = W;      \
    t = true;            \
  }
  TFFT_BLUE_STRIDED(X)
#undef X
  return c && t;
}

cudaError_t launch_contig_blue_spec(const ContigArgs& a, const BlueArgs& b, cudaStream_t s) {
#define X(MM, E, B, ...) \
  if (b.M == MM) return run_blue_contig<MM, E, B, __VA_ARGS__>(a, b, s);
  TFFT_BLUE_CONTIG(X)
#undef X
  return cudaErrorInvalidValue;
}

cudaError_t launch_strided_blue_spec(const StridedArgs& a, const BlueArgs& b, cudaStream_t s) {
#define X(MM, E, W, ...) \
  if (b.M == MM) return run_blue_strided<MM, E, W, __VA_ARGS__>(a, b, s);
  TFFT_BLUE_STRIDED(X)
#undef X
  return cudaErrorInvalidValue;
}

}  // namespace tfft
