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
#include "tfft_tiles.cuh"

namespace tfft {

namespace {

using namespace tiles;

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

constexpr int kBatchThreads = 256;

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
  extern __shared__ float2 smem[];
  // the current item's segment, copied out of global memory: read there, its
  // fields would be reloaded after every global store of a tile (the
  // compiler cannot rule out that the store changed them)
  __shared__ __align__(16) BatchSeg s_S;
  __shared__ long long s_first[kSmemSegs];
  __shared__ long long s_item;
  __shared__ int s_seg;
  __shared__ int s_abort;
  const int tid = threadIdx.x;
  const bool seg_in_smem = b.nsegs <= kSmemSegs;
  if (seg_in_smem)
    for (int i = tid; i < b.nsegs; i += kBatchThreads) s_first[i] = b.segs[i].first;
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
                                 : (size_t)L * BW * sizeof(float2) + 2 * (size_t)L * sizeof(int);     \
    m = v > m ? v : m;                                                                                 \
  }
  TFFT_BATCH_VARIANTS(X)
#undef X
  return m;
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
    default:
      return false;
  }
}

int batch_num_variants() {
  int n = 0;
#define X(ID, ...) ++n;
  TFFT_BATCH_VARIANTS(X)
#undef X
  return n;
}

cudaError_t launch_batch(const BatchArgs& b, int grid, cudaStream_t s) {
  static cudaError_t attr = cudaFuncSetAttribute(k_batch, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)batch_smem());
  if (attr != cudaSuccess) return attr;
  k_batch<<<grid, kBatchThreads, batch_smem(), s>>>(b);
  return cudaGetLastError();
}

int batch_grid() {
  static int g = [] {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaFuncSetAttribute(k_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)batch_smem());
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_batch, kBatchThreads, batch_smem());
    if (per < 1) per = 1;
    return (sms > 0 ? sms : 1) * per;
  }();
  return g;
}

}  // namespace tfft
