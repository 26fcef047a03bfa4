// Batched persistent executor: the passes of many independent transforms
// (each on its own virtual grid) in one kernel launch.
//
// Work items are the tiles of every (transform, pass) segment, ordered pass
// by pass.  Each CTA takes the next item from a global counter, waits until
// every tile of the same transform's previous pass is done (the next pass
// gathers its lines from all of them), runs the tile with the same tile body
// as the standalone passes (loads through L2, because other SMs wrote the
// data during this launch), then publishes its completion.  Items are taken
// in order, so the item a CTA waits for was taken earlier by a running CTA:
// the waits always end.  Each wait is bounded anyway: past the limit the CTA
// records TFFT_DEVICE_ETIMEOUT, raises the launch's abort flag and leaves.
//
// Strided segments whose layouts have equal blocks can run TMA-staged tiles:
// within an item the copy of tile i+1 runs while tile i is transformed (two
// tile buffers), loads and stores are one cp.async.bulk.tensor each, and the
// item is published only after its stores have completed.
#include "tfft_tiles.cuh"
#include "tfft_tma.cuh"

namespace tfft {

namespace {

using namespace tiles;
using namespace tma;

// Tile variants the executor can run, all with 256 threads per CTA:
// id, kind (0 contiguous / 1 strided), length, elements per thread,
// lines per group (contiguous) or tile width (strided), radices.
#define TFFT_BATCH_VARIANTS(X)          \
  X(0, 0, 64, 8, 32, 8, 8)              \
  X(1, 0, 96, 12, 32, 4, 4, 3, 2)       \
  X(2, 0, 128, 16, 32, 16, 8)           \
  X(3, 0, 160, 20, 32, 5, 4, 4, 2)      \
  X(4, 0, 256, 16, 16, 16, 16)          \
  X(5, 0, 256, 8, 8, 8, 8, 4)           \
  X(6, 0, 128, 8, 16, 8, 8, 2)          \
  X(7, 0, 32, 8, 64, 8, 4)              \
  X(8, 1, 64, 8, 32, 8, 8)              \
  X(9, 1, 96, 12, 32, 4, 4, 3, 2)       \
  X(10, 1, 128, 16, 32, 16, 8)          \
  X(11, 1, 160, 20, 32, 5, 4, 4, 2)     \
  X(12, 1, 256, 16, 16, 16, 16)         \
  X(13, 1, 256, 8, 8, 8, 8, 4)          \
  X(14, 1, 128, 8, 16, 8, 8, 2)

// TMA-staged strided variants: id, length, elements per thread, tile width
// (W * L / E = 256 threads), radices.
#define TFFT_BATCH_TMA_VARIANTS(X) \
  X(15, 64, 8, 32, 8, 8)           \
  X(16, 128, 16, 32, 16, 8)        \
  X(17, 256, 16, 16, 16, 16)       \
  X(18, 96, 12, 32, 4, 4, 3, 2)

constexpr int kBatchThreads = 256;

// Bounded mbarrier wait in clock cycles (the executor's limit unit); the
// first poll does not block.
__device__ __forceinline__ bool mbar_wait_cycles(uint64_t* bar, uint32_t parity, long long limit) {
  if (mbar_test_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (clock64() - t0 <= limit)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// The tiles [t0, t1) of one TMA-staged strided segment, double-buffered in
// `smem` (which must be 128-byte aligned: a tensor copy's shared-memory end).
// ph[b] is the phase the next completion of buffer b's barrier will have
// (the same in every thread).  Returns 0, or the device status bit of the
// failure (TFFT_DEVICE_ETIMEOUT: a copy wait expired).
template <int L, int E, int W, int... Rs>
__device__ int tma_item(const BatchSeg& S, int64_t t0, int64_t t1, float2* smem, int tid, uint64_t* bars,
                        uint32_t (&ph)[2], long long limit) {
  constexpr int T = L / E, NST = sizeof...(Rs);
  const StridedArgs& a = S.sa;
  const CUtensorMap* tin = static_cast<const CUtensorMap*>(S.tin);
  const CUtensorMap* tout = static_cast<const CUtensorMap*>(S.tout);
  const int tax = a.oax0;
  const int cx = tid % W, jt = tid / W;
  const bool inv = a.sign > 0;
  auto issue_load = [&](int64_t tile, float2* dst, uint64_t* bar) {
    int64_t o;
    int2 blk;
    tile_place(a, tile, o, blk);
    mbar_expect_tx(bar, (uint32_t)(L * W * sizeof(float2)));
    for (int k = 0; k < S.gin.nops; ++k) {
      int c[5];
      tile_coords(S.gin, a.axis, k, blk.x, o, tax, c);
      tma_load_5d(dst + (size_t)k * S.gin.rows_per_op * W, tin, bar, c);
    }
  };
  if (tid == 0) {
    // the previous pass wrote through the generic proxy (plain tiles); this
    // CTA's earlier tiles used the buffers through it too
    asm volatile("fence.proxy.async.global;" ::: "memory");
    fence_proxy_async();
    issue_load(t0, smem, &bars[0]);
  }
  int err = 0;
  for (int64_t tile = t0; tile < t1; ++tile) {
    const int bi = (int)((tile - t0) & 1);
    float2* cur = smem + (size_t)bi * L * W;
    const bool more = tile + 1 < t1;
    if (tid == 0 && more) {
      bulk_wait_read<0>();  // the previous tile's store has read the other buffer
      fence_proxy_async();
      issue_load(tile + 1, smem + (size_t)(bi ^ 1) * L * W, &bars[bi ^ 1]);
    }
    const bool got = mbar_wait_cycles(&bars[bi], ph[bi], limit);
    ph[bi] ^= 1;
    if (__syncthreads_or(!got)) {
      if (tid == 0) {  // let the copies in flight land before the CTA leaves
        if (!got) mbar_wait(&bars[bi], ph[bi] ^ 1, kWaitLimit);
        if (more) mbar_wait(&bars[bi ^ 1], ph[bi ^ 1], kWaitLimit);
      }
      err = TFFT_DEVICE_ETIMEOUT;
      break;
    }
    float2 v[E];
    static_for<0, NST>([&](auto St) {
      constexpr int s = decltype(St)::value;
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
          for (int r = 0; r < Rp; ++r) cur[stockham_out_index(jt + q * T, Nsp, Rp, r) * W + cx] = v[q * Rp + r];
        __syncthreads();
#pragma unroll
        for (int q = 0; q < E / R; ++q)
#pragma unroll
          for (int r = 0; r < R; ++r) v[q * R + r] = cur[(jt + q * T + r * (L / R)) * W + cx];
      }
      spec_stage<L, E, R, Ns>(v, jt, a.tw);
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
      int64_t o;
      int2 blk;
      tile_place(a, tile, o, blk);
      for (int k = 0; k < S.gout.nops; ++k) {
        int c[5];
        tile_coords(S.gout, a.axis, k, blk.x, o, tax, c);
        tma_store_5d(tout, cur + (size_t)k * S.gout.rows_per_op * W, c);
      }
      bulk_commit();
    }
  }
  if (tid == 0) bulk_wait_all();  // the item's stores are complete before it is published
  return err;
}

template <int KIND, int L, int E, int BW, int... Rs>
__device__ __forceinline__ void run_tile(const BatchSeg& S, int64_t tile, float2* smem, int tid) {
  if constexpr (KIND == 0)
    contig_tile<L, E, BW, true, Rs...>(S.ca, tile, smem, tid % (L / E), tid / (L / E));
  else
    strided_tile<L, E, BW, true, Rs...>(S.sa, tile, smem, tid % BW, tid / BW, tid);
}

// Segments whose first-item table fits shared memory use it for the lookup.
constexpr int kSmemSegs = 1024;

__global__ void __launch_bounds__(kBatchThreads, 3) k_batch(const BatchArgs b) {
  extern __shared__ __align__(128) float2 smem_raw[];
  // the dynamic block follows the static shared variables: the tile buffers
  // start at its first 128-byte boundary (batch_smem() adds the slack)
  float2* smem = reinterpret_cast<float2*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
  // the current item's segment, copied out of global memory: read there, its
  // fields would be reloaded after every global store of a tile (the
  // compiler cannot rule out that the store changed them)
  __shared__ __align__(16) BatchSeg s_S;
  __shared__ long long s_first[kSmemSegs];
  __shared__ long long s_item;
  __shared__ int s_seg;
  __shared__ int s_abort;
  __shared__ __align__(8) uint64_t s_bars[2];  // TMA tile buffers 0 and 1
  const int tid = threadIdx.x;
  const bool seg_in_smem = b.nsegs <= kSmemSegs;
  if (seg_in_smem)
    for (int i = tid; i < b.nsegs; i += kBatchThreads) s_first[i] = b.segs[i].first;
  if (tid == 0) {
    mbar_init(&s_bars[0], 1);
    mbar_init(&s_bars[1], 1);
    fence_mbar_init();
  }
  uint32_t ph[2] = {0, 0};
  // items are taken one ahead: the next one is claimed while the current one runs
  long long next = 0;
  if (tid == 0) next = (long long)atomicAdd(b.head, 1ull);
  int cur_seg = -1;
  __syncthreads();
  for (;;) {
    if (tid == 0) {
      const long long item = next;
      int seg = 0, abort = 0;
      if (item < b.nitems) {
        next = (long long)atomicAdd(b.head, 1ull);
        int lo = 0, hi = b.nsegs - 1;
        while (lo < hi) {  // last segment whose first item <= item
          const int mid = (lo + hi + 1) >> 1;
          const long long f = seg_in_smem ? s_first[mid] : b.segs[mid].first;
          if (f <= item) lo = mid;
          else hi = mid - 1;
        }
        seg = lo;
        const int prev = b.segs[seg].prev;
        if (prev >= 0) {
          const int need = (int)b.segs[prev].nitems;
          const long long t0 = clock64();
          while (*(volatile int*)&b.done[prev] < need) {
            if (*(volatile int*)b.abort) {
              abort = 1;
              break;
            }
            if (clock64() - t0 > b.spin_limit) {
              atomicOr(b.status, TFFT_DEVICE_ETIMEOUT);
              atomicExch(b.abort, 1);
              abort = 1;
              break;
            }
            __nanosleep(64);
          }
          __threadfence();  // the previous pass's stores are visible before its data is read
        }
      }
      s_item = item;
      s_seg = seg;
      s_abort = abort;
    }
    __syncthreads();
    const long long item = s_item;
    const int seg = s_seg;
    if (item >= b.nitems || s_abort) break;
    if (seg != cur_seg) {
      static_assert(sizeof(BatchSeg) % sizeof(int) == 0, "segment copied as words");
      const int* src = reinterpret_cast<const int*>(&b.segs[seg]);
      int* dst = reinterpret_cast<int*>(&s_S);
      for (int i = tid; i < (int)(sizeof(BatchSeg) / sizeof(int)); i += kBatchThreads) dst[i] = src[i];
      cur_seg = seg;
      __syncthreads();
    }
    const BatchSeg& S = s_S;
    // an item is a run of up to `per_item` consecutive tiles of one segment
    const int64_t t0 = (item - S.first) * S.per_item;
    const int64_t t1 = (t0 + S.per_item < S.ntiles) ? t0 + S.per_item : S.ntiles;
    if (S.tma) {
      // the tensor copies need a 128-byte aligned shared-memory end
      int err = (static_cast<uint32_t>(__cvta_generic_to_shared(smem)) & 127) ? TFFT_DEVICE_EALIGN : 0;
      if (!err) switch (S.variant) {
#define X(ID, L, E, W, ...)                                                            \
  case ID:                                                                             \
    err = tma_item<L, E, W, __VA_ARGS__>(S, t0, t1, smem, tid, s_bars, ph, b.spin_limit); \
    break;
          TFFT_BATCH_TMA_VARIANTS(X)
#undef X
          default:
            break;
        }
      if (err) {
        if (tid == 0) {
          atomicOr(b.status, err);
          atomicExch(b.abort, 1);
        }
        break;
      }
      __syncthreads();
    } else
    for (int64_t tile = t0; tile < t1; ++tile) {
      switch (S.variant) {
#define X(ID, KIND, L, E, BW, ...)                              \
  case ID:                                                      \
    run_tile<KIND, L, E, BW, __VA_ARGS__>(S, tile, smem, tid);  \
    break;
        TFFT_BATCH_VARIANTS(X)
#undef X
        default:
          break;
      }
      __syncthreads();  // shared memory is free for the next tile
    }
    __threadfence();
    __syncthreads();  // every thread's stores are issued and fenced; s_item may be reused
    if (tid == 0) atomicAdd(&b.done[seg], 1);
  }
}

constexpr size_t batch_smem() {
  size_t m = 0;
#define X(ID, KIND, L, E, BW, ...)                                                                     \
  {                                                                                                    \
    const size_t v = (KIND == 0) ? (size_t)BW * line_pitch<L, __VA_ARGS__>() * sizeof(float2) \
                                 : strided_tile_smem<L, BW>(false);                                 \
    m = v > m ? v : m;                                                                                 \
  }
  TFFT_BATCH_VARIANTS(X)
#undef X
#define X(ID, L, E, W, ...)                                   \
  {                                                           \
    const size_t v = 2 * (size_t)L * W * sizeof(float2);      \
    m = v > m ? v : m;                                        \
  }
  TFFT_BATCH_TMA_VARIANTS(X)
#undef X
  return m + 128;  // slack to align the tile buffers (see k_batch)
}

}  // namespace

bool batch_variant(int id, int& kind, int& L, int& E, int& BW, AxisPlan& ap) {
  switch (id) {
#define X(ID, KIND, LL, EE, BWW, ...)                                   \
  case ID: {                                                            \
    const int r[] = {__VA_ARGS__};                                      \
    kind = KIND;                                                        \
    L = LL;                                                             \
    E = EE;                                                             \
    BW = BWW;                                                           \
    ap = AxisPlan{};                                                    \
    ap.L = LL;                                                          \
    ap.E = EE;                                                          \
    ap.T = LL / EE;                                                     \
    ap.nst = (int)(sizeof(r) / sizeof(int));                            \
    for (int s = 0; s < ap.nst; ++s) {                                  \
      ap.radix[s] = r[s];                                               \
      ap.code |= (uint64_t)r[s] << (5 * s);                             \
    }                                                                   \
    ap.spec = 1;                                                        \
    ap.width = BWW;                                                     \
    return true;                                                        \
  }
    TFFT_BATCH_VARIANTS(X)
#undef X
#define X(ID, LL, EE, WW, ...)                                          \
  case ID: {                                                            \
    const int r[] = {__VA_ARGS__};                                      \
    kind = 1;                                                           \
    L = LL;                                                             \
    E = EE;                                                             \
    BW = WW;                                                            \
    ap = AxisPlan{};                                                    \
    ap.L = LL;                                                          \
    ap.E = EE;                                                          \
    ap.T = LL / EE;                                                     \
    ap.nst = (int)(sizeof(r) / sizeof(int));                            \
    for (int s = 0; s < ap.nst; ++s) {                                  \
      ap.radix[s] = r[s];                                               \
      ap.code |= (uint64_t)r[s] << (5 * s);                             \
    }                                                                   \
    ap.spec = 1;                                                        \
    ap.width = WW;                                                      \
    return true;                                                        \
  }
    TFFT_BATCH_TMA_VARIANTS(X)
#undef X
    default:
      return false;
  }
}

bool batch_variant_tma(int id) {
  switch (id) {
#define X(ID, ...) case ID:
    TFFT_BATCH_TMA_VARIANTS(X)
#undef X
    return true;
    default:
      return false;
  }
}

int batch_num_variants() {
  int n = 0;
#define X(ID, ...) ++n;
  TFFT_BATCH_VARIANTS(X)
  TFFT_BATCH_TMA_VARIANTS(X)
#undef X
  return n;
}

cudaError_t launch_batch(const BatchArgs& b, int grid, cudaStream_t s) {
  static PerDevice<cudaError_t> attr_cache;
  const cudaError_t attr = smem_attr_once(attr_cache, k_batch, (int)batch_smem());
  if (attr != cudaSuccess) return attr;
  k_batch<<<grid, kBatchThreads, batch_smem(), s>>>(b);
  return cudaGetLastError();
}

int batch_grid() {
  static PerDevice<int> cache;
  return cache.get(current_device(), [] {
    int per = 0;
    cudaFuncSetAttribute(k_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)batch_smem());
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_batch, kBatchThreads, batch_smem());
    if (per < 1) per = 1;
    return device_sm_count() * per;
  });
}

}  // namespace tfft
