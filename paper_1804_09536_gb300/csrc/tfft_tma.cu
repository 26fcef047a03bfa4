// TMA-staged FFT passes (sm_103a).
//
// Strided passes with the redistribution fused in: when every virtual rank of
// the input and output stage holds an equal block (the decomposition divides
// every cut axis), a stage buffer is a regular 5-D array
// [rank dim][rank dim][n0][n1][n2] and one tensor map describes it.  A tile
// (all L rows of the FFT axis x W columns of the innermost axis) is then one
// cp.async.bulk.tensor copy each way -- the box spans the local rows and the
// rank coordinate of the subgroup that cuts the FFT axis, so the gather of
// the line from its M owners (Alg. 3's subarray boxes) is done by the copy
// engine -- and the result goes back the same way into the output stage,
// whose box spans the other subgroup (the scatter).  Tiles are
// buffered three deep -- the copy of tile i+1 runs while tile i is
// transformed and the store of tile i-1 drains -- or two deep where the
// smaller footprint lets one more CTA share the SM.
//
// The same kernel also runs in-place passes along the leading axis of layouts
// whose ranks do NOT hold equal blocks (an uneven split of Eq. decompose):
// each rank's local array is then a 2-D array (L rows x the product of the
// other extents), the ranks with equal blocks form at most four groups whose
// offsets are affine in the rank coordinates, and one tensor map per group
// describes them.  A tile is W consecutive elements of that merged inner
// extent (columns of independent lines) over all L rows of one rank; the
// last tile of a rank may be partial -- the copy fills the missing columns
// with zeros and the store skips them.
//
// The equal-block view also serves a column window of the innermost axis
// (TmaGeo::c0): the gathering pass of a real-to-complex pencil plan reads a
// padded internal stage 0 and writes the last stage's ranks of one even
// width, both described from the window's first column on.
//
// Every wait on an mbarrier is bounded: on expiry the CTA records
// TFFT_DEVICE_ETIMEOUT in the plan's status word and leaves.
#include "tfft_tiles.cuh"
#include "tfft_tma.cuh"

namespace tfft {

namespace {

using namespace tiles;
using namespace tma;

// CTAs of `bytes` of shared memory each that fit one SM's 228 KB (1 KB
// reserved per CTA), at most three.
__host__ __device__ constexpr int strided_tma_ctas(size_t bytes) {
  return 228 * 1024 / (bytes + 1024) < 3 ? (int)(228 * 1024 / (bytes + 1024)) : 3;
}

// Tile buffers of the strided TMA kernel (L x (W + 1) each). Three let the
// load of tile i+1 and the store of tile i-1 overlap the transform of tile i;
// two make the load wait for the previous store to finish reading its buffer,
// which pays wherever the smaller footprint adds a CTA per SM: length 384
// (one CTA -> two: 0.202 -> 0.180 ms per 384^3 pass), length 128 with 32
// columns (12.2 -> 11.8 us per 128^3 pass), length 256 with 16 columns (the
// batch of 48 1.881 -> 1.864 ms, the r2c slab's rank-group pass 22.9 -> 22.3
// us; alone, a 256^3 pass 48.3 -> 49.4 us, 2 % slower, which the batch, where
// these kernels share the GPU with others, more than wins back).
__host__ __device__ constexpr int strided_tma_nbuf(int L, int W) {
  return strided_tma_ctas(2 * (size_t)L * (W + 1) * sizeof(float2) + 3 * sizeof(uint64_t)) >
                 strided_tma_ctas(3 * (size_t)L * (W + 1) * sizeof(float2) + 3 * sizeof(uint64_t))
             ? 2
             : 3;
}

__host__ __device__ constexpr size_t strided_tma_smem(int L, int W) {
  return strided_tma_nbuf(L, W) * (size_t)L * (W + 1) * sizeof(float2) + 3 * sizeof(uint64_t);
}

// Tiles of the equal-block view: (outer index, column block), gathered and
// scattered through the 5-D TmaGeo views of the input and output layouts.
struct BlockTiles {
  CUtensorMap tin, tout;
  TmaGeo gin, gout;
  __host__ __device__ __forceinline__ int64_t ntiles(const StridedArgs& a) const { return a.nouter * a.ncolblocks; }
  template <int W>
  __device__ __forceinline__ void load(const StridedArgs& a, int64_t tile, float2* dst, uint64_t* bar) const {
    int64_t o;
    int2 blk;
    tile_place(a, tile, o, blk);
    const int tax = (a.oax0 >= 0) ? a.oax0 : -1;  // the outer axis (d == 3)
    for (int k = 0; k < gin.nops; ++k) {
      int c[5];
      tile_coords(gin, a.axis, k, (int64_t)blk.x - gin.c0, o, tax, c);
      tma_load_5d(dst + (size_t)k * gin.rows_per_op * W, &tin, bar, c);
    }
  }
  template <int W>
  __device__ __forceinline__ void store(const StridedArgs& a, int64_t tile, const float2* src) const {
    int64_t o;
    int2 blk;
    tile_place(a, tile, o, blk);
    const int tax = (a.oax0 >= 0) ? a.oax0 : -1;
    for (int k = 0; k < gout.nops; ++k) {
      int c[5];
      tile_coords(gout, a.axis, k, (int64_t)blk.x - gout.c0, o, tax, c);
      tma_store_5d(&tout, src + (size_t)k * gout.rows_per_op * W, c);
    }
  }
};

// Tiles of the rank-group view (uneven blocks, in-place leading-axis pass):
// group g covers tiles [first[g], first[g + 1]), nblk[g] column blocks per
// rank, its ranks numbered r1 + ext1[g] r0; its tensor maps view it as
// [inner][rows / a][a... ] = [inner][a][L / a][ext1][ext0] (a = rows of the
// inner row box, at most 256).
struct RankGroupTiles {
  CUtensorMap tin[kMaxRankGroups], tout[kMaxRankGroups];
  RankGroupGeo geo;
  __host__ __device__ __forceinline__ int64_t ntiles(const StridedArgs&) const { return geo.first[geo.ngroups]; }
  __device__ __forceinline__ int place(int64_t tile, int (&c)[5]) const {
    int g = 0;
    while (g + 1 < geo.ngroups && tile >= geo.first[g + 1]) ++g;
    const int64_t local = tile - geo.first[g];
    const int64_t rank = local / geo.nblk[g];
    const int blk = (int)(local - rank * geo.nblk[g]);
    c[0] = blk * geo.width;
    c[1] = 0;
    c[2] = 0;
    c[3] = (int)(rank % geo.ext1[g]);
    c[4] = (int)(rank / geo.ext1[g]);
    return g;
  }
  template <int W>
  __device__ __forceinline__ void load(const StridedArgs&, int64_t tile, float2* dst, uint64_t* bar) const {
    int c[5];
    const int g = place(tile, c);
    tma_load_5d(dst, &tin[g], bar, c);
  }
  template <int W>
  __device__ __forceinline__ void store(const StridedArgs&, int64_t tile, const float2* src) const {
    int c[5];
    const int g = place(tile, c);
    tma_store_5d(&tout[g], src, c);
  }
};

template <int L, int E, int W, class Geo, int... Rs>
__global__ void __launch_bounds__(W * (L / E), strided_tma_ctas(strided_tma_smem(L, W)))
    k_strided_tma(const StridedArgs a, const __grid_constant__ Geo geo) {
  constexpr int T = L / E, NST = sizeof...(Rs);
  constexpr int WP = (W % 16 == 0) ? W : W + 1;  // exchange pitch (bank-conflict padding)
  constexpr int BUF = L * (W + 1);
  extern __shared__ __align__(128) float2 smem[];
  // NB tile buffers: tile i is transformed in buffer i % NB while tile i+1 is
  // loaded into the next one; with three, the store of tile i-1 still reads
  // its own meanwhile, with two it has finished before the load is issued
  constexpr int NB = strided_tma_nbuf(L, W);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + NB * BUF);
  const int cx = threadIdx.x;
  const int tid = threadIdx.y * W + cx;
  const bool inv = a.sign > 0;
  const int64_t ntiles = geo.ntiles(a);
  const uint32_t tile_bytes = (uint32_t)(L * W * sizeof(float2));

  if (tid == 0) {
    for (int b = 0; b < NB; ++b) mbar_init(&bars[b], 1);
    fence_mbar_init();
    fence_proxy_async();
  }
  __syncthreads();

  auto issue_load = [&](int64_t tile, float2* dst, uint64_t* bar) {
    mbar_expect_tx(bar, tile_bytes);
    geo.template load<W>(a, tile, dst, bar);
  };

  int64_t tile = blockIdx.x;
  if (tid == 0 && tile < ntiles) issue_load(tile, smem, &bars[0]);
  StageTwiddles<L, E, Rs...> twr;
  twr.load(threadIdx.y, a.tw);
  int it = 0, b = 0;  // b = it % NB
  for (; tile < ntiles; tile += gridDim.x, ++it, b = (b == NB - 1) ? 0 : b + 1) {
    float2* cur = smem + b * BUF;
    const int bn = (b == NB - 1) ? 0 : b + 1;
    const int64_t next = tile + gridDim.x;
    if (tid == 0 && next < ntiles) {
      // the store of tile it+1-NB has finished reading buffer bn
      if constexpr (NB == 3) bulk_wait_read<1>();
      else bulk_wait_read<0>();
      fence_proxy_async();
      issue_load(next, smem + bn * BUF, &bars[bn]);
    }
    bool ok = true;
    if (!mbar_wait(&bars[b], (it / NB) & 1, a.wait_limit)) ok = false;
    if (__syncthreads_or(!ok)) {
      if (tid == 0) {
        atomicOr(a.status, TFFT_DEVICE_ETIMEOUT);
        // give the copies still in flight (this tile's and the next one's) a
        // bounded chance to land before the CTA leaves
        mbar_wait(&bars[b], (it / NB) & 1, kWaitLimit);
        if (next < ntiles) mbar_wait(&bars[bn], ((it + 1) / NB) & 1, kWaitLimit);
      }
      break;
    }
    const int jt = opaque_tid_y();
    float2 v[E];
    static_for<0, NST>([&](auto S) {
      constexpr int s = decltype(S)::value;
      constexpr int R = radix_at<s, Rs...>();
      constexpr int Ns = span_at<s, Rs...>();
      if constexpr (s == 0) {
#pragma unroll
        for (int q = 0; q < E / R; ++q)
#pragma unroll
          for (int r = 0; r < R; ++r) {
            float2 x = cur[(jt + q * T + r * (L / R)) * W + cx];
            if (inv) x.y = -x.y;
            v[q * R + r] = x;
          }
      } else {
        constexpr int Rp = radix_at<s - 1, Rs...>();
        constexpr int Nsp = Ns / Rp;
        __syncthreads();
#pragma unroll
        for (int q = 0; q < E / Rp; ++q)
#pragma unroll
          for (int r = 0; r < Rp; ++r)
            cur[stockham_out_index(jt + q * T, Nsp, Rp, r) * WP + cx] = v[q * Rp + r];
        __syncthreads();
#pragma unroll
        for (int q = 0; q < E / R; ++q)
#pragma unroll
          for (int r = 0; r < R; ++r) v[q * R + r] = cur[(jt + q * T + r * (L / R)) * WP + cx];
      }
      twr.template stage<s>(v);
    });
    constexpr int RL = radix_at<NST - 1, Rs...>();
    __syncthreads();
#pragma unroll
    for (int q = 0; q < E / RL; ++q)
#pragma unroll
      for (int r = 0; r < RL; ++r) {
        float2 x = cscale(v[q * RL + r], a.scale);
        if (inv) x.y = -x.y;
        cur[(jt + q * T + r * (L / RL)) * W + cx] = x;
      }
    fence_proxy_async();
    __syncthreads();
    if (tid == 0) {
      geo.template store<W>(a, tile, cur);
      bulk_commit();
    }
  }
  if (tid == 0) bulk_wait_all();
}

// the kernel's shared-memory limit raised to 227 KB, once per device
#define TFFT_ALLOW_SMEM(kernel)                          \
  static PerDevice<cudaError_t> attr_cache;              \
  const cudaError_t attr = smem_attr_once(attr_cache, kernel, 227 * 1024)

template <class K>
int64_t persistent_grid(K kernel, int threads, size_t smem, int64_t ntiles) {
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem);
  if (per_sm < 1) per_sm = 1;
  const int64_t g = (int64_t)per_sm * device_sm_count();
  return ntiles < g ? ntiles : g;
}

template <int L, int E, int W, class Geo, int... Rs>
cudaError_t run_strided_tma(const StridedArgs& a, const Geo& geo, cudaStream_t s) {
  auto kern = k_strided_tma<L, E, W, Geo, Rs...>;
  TFFT_ALLOW_SMEM(kern);
  if (attr != cudaSuccess) return attr;
  if (a.W != W) return cudaErrorInvalidValue;
  const size_t smem = strided_tma_smem(L, W);
  const int threads = W * (L / E);
  static PerDevice<int64_t> slots_cache;
  const int64_t slots =
      slots_cache.get(current_device(), [&] { return persistent_grid(kern, threads, smem, int64_t(1) << 40); });
  const int64_t ntiles = geo.ntiles(a);
  const int64_t grid = ntiles < slots ? ntiles : slots;
  if (grid < 1) return cudaSuccess;
  kern<<<(unsigned)grid, dim3(W, L / E), smem, s>>>(a, geo);
  return cudaGetLastError();
}

// Strided TMA variants: length, elements per thread, tile width, radices.
// The first row of a length is its default; tma_strided_variant() can pick
// another (autotuning).  256: 16-column tiles at two CTAs per SM beat 32
// columns at one (256^3 on 4 x 8 / 2 x 2 / 2 x 4: 0.048 vs 0.052 ms per pass;
// the 48-transform batch 1.96 vs 2.01 ms); 8 elements per thread (radices
// 8, 8, 4) took 0.057 ms.  512: 8-column tiles at two CTAs per SM took 0.361
// vs 0.336 ms per 512^3 pass (64-byte rows).
#define TFFT_TMA_STRIDED(X)     \
  X(64, 8, 32, 8, 8)            \
  X(96, 12, 32, 4, 4, 3, 2)     \
  X(128, 16, 32, 16, 8)         \
  X(160, 20, 16, 5, 4, 4, 2)    \
  X(384, 24, 16, 8, 8, 3, 2)    \
  X(1024, 32, 8, 32, 32)        \
  X(256, 16, 16, 16, 16)        \
  X(256, 16, 32, 16, 16)        \
  X(512, 32, 16, 32, 16)        \
  X(512, 16, 16, 8, 8, 8)

}  // namespace

bool tma_strided_variant(int L, int want_W, int want_E, int& E, int& W) {
  bool found = false;
#define X(LL, EE, WW, ...)                                             \
  if (LL == L) {                                                        \
    const bool match = WW == want_W && (want_E == 0 || EE == want_E);  \
    if (!found || match) {                                              \
      E = EE;                                                           \
      W = WW;                                                           \
      found = true;                                                     \
      if (match) return true;                                           \
    }                                                                   \
  }
  TFFT_TMA_STRIDED(X)
#undef X
  return found;
}

cudaError_t launch_strided_tma(const StridedArgs& a, int E, const TmaGeo& gi, const TmaGeo& go,
                               const void* tmap_in, const void* tmap_out, cudaStream_t s) {
  BlockTiles geo;
  geo.tin = *static_cast<const CUtensorMap*>(tmap_in);
  geo.tout = *static_cast<const CUtensorMap*>(tmap_out);
  geo.gin = gi;
  geo.gout = go;
#define X(LL, EE, WW, ...)                   \
  if (a.ap.L == LL && E == EE && a.W == WW) \
    return run_strided_tma<LL, EE, WW, BlockTiles, __VA_ARGS__>(a, geo, s);
  TFFT_TMA_STRIDED(X)
#undef X
  return cudaErrorInvalidValue;
}

cudaError_t launch_strided_tma_groups(const StridedArgs& a, int E, const RankGroupGeo& g, const void* const* tmaps_in,
                                      const void* const* tmaps_out, cudaStream_t s) {
  if (g.ngroups < 1 || g.ngroups > kMaxRankGroups || g.width != a.W) return cudaErrorInvalidValue;
  RankGroupTiles geo;
  for (int k = 0; k < g.ngroups; ++k) {
    geo.tin[k] = *static_cast<const CUtensorMap*>(tmaps_in[k]);
    geo.tout[k] = *static_cast<const CUtensorMap*>(tmaps_out[k]);
  }
  geo.geo = g;
#define X(LL, EE, WW, ...)                   \
  if (a.ap.L == LL && E == EE && a.W == WW) \
    return run_strided_tma<LL, EE, WW, RankGroupTiles, __VA_ARGS__>(a, geo, s);
  TFFT_TMA_STRIDED(X)
#undef X
  return cudaErrorInvalidValue;
}

}  // namespace tfft
