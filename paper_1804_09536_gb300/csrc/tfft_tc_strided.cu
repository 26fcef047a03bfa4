// Strided TMA passes of lengths 512 = 32 x 16 and 256 = 16 x 16 whose last,
// radix-16 stage runs on the 5th-generation tensor cores (tcgen05.mma,
// kind::f16, FP32 accumulation in tensor memory): the tensor-core form of the
// fused exchange-and-transform pass of tfft_tma.cu (Eqs. pencil1 / pencil2
// with the redistributions of Eq. gtp1 / gtp2 in the tile copies).
//
// A tile is L rows (the FFT axis) x W columns, gathered by one TMA copy as
// in the FP32 kernel.  Line cx of the tile is the length-L FFT x[n],
// n = n2 + 16 n1 (n2 < 16, n1 < E, L = 16 E): thread (cx, jt = n2) loads
// x[jt + 16 n1] for all n1 and runs the first stage, a size-E DFT over n1,
// in registers; its output k1 times the twiddle exp(-2 pi i jt k1 / L) is
// input jt of the 16-point sub-transform (cx, k1).  The W x E = 512
// sub-transforms of a tile are the rows of A (K = 32 reals: re/im of their
// 16 inputs) and the 16-point DFT is the 32 x 32 real matrix B, so
// D = A B^T holds every sub-transform's 16 outputs X[k1 + E k2]; with A and
// B split in hi + lo 16-bit parts, D = A_hi B_hi + A_lo B_hi + A_hi B_lo
// (FP32 accumulation) keeps about twice the 16-bit mantissa.  FP16 operands
// are range-scaled per line (a power of two from the line's largest
// magnitude, undone on the accumulator).
//
// Software pipeline: in iteration i the CTA runs the first stage of tile i,
// writes its A operands over the tile's own buffer and issues its MMAs into
// one of two tensor-memory accumulators, then reads back the accumulator of
// tile i-1 (whose MMAs ran meanwhile) and stores it straight to global
// memory (the scatter of the redistribution): in an equal-block layout an
// output row's element offset is affine in its rank part and local index,
// so every thread computes its rows' offsets from the tile geometry; the
// TMA copy of tile i+1 is in flight all along.  No
// tile buffer waits for a store, so three buffers give every load a whole
// iteration of lead.  Four MMA groups of M = 128 rows, N = 32, K = 32 (two
// K = 16 steps, three products each) per tile, issued by one thread and
// committed to one of two mbarriers.  Every wait is bounded; tensor memory
// is released before the CTA leaves unless MMAs are still running after the
// clean-up wait.
#include "tfft_tc.cuh"
#include "tfft_tma.cuh"

namespace tfft {

namespace {

using namespace tiles;
using namespace tma;
using namespace tc;

// Dense K-major operand layout (no swizzle): core matrix = 8 rows x 16 B,
// K-adjacent core matrices 128 B apart, 8-row groups 512 B apart.
constexpr uint32_t kLBO = 128, kSBO = 512;
constexpr int kRows = 512;                     // sub-transforms per tile (W x E)
constexpr uint32_t kOpBytes = kRows * 64;      // one 512 x 32 16-bit operand
constexpr uint32_t kBBytes = 32 * 64;          // the 32 x 32 DFT operand
constexpr uint32_t kAccCols = 128;             // one tile: four FP32 groups of 32 columns
constexpr uint32_t kTmemCols = 2 * kAccCols;   // two accumulators

__device__ __forceinline__ uint32_t op_off(int row, int k) {
  return (uint32_t)((row >> 3) * kSBO + (k >> 3) * kLBO + (row & 7) * 16 + (k & 7) * 2);
}

// Twiddle slot with one spare entry every 16: the lanes of a warp read
// indices jt k1 for two consecutive jt, so stride-k1 patterns spread out.
__device__ __forceinline__ int tws(int i) { return i + (i >> 4); }

// Element offsets of a tile's rows in an equal-block output layout (the
// 5-D view of TmaGeo): rank r holds its (n0, n1, n2) block at r x local, and
// global index g of axis m lies in rank part g / n[m] (rank stride rmul[m])
// at local index g % n[m] when that axis is cut.  Row n of the tile (global
// index n of the FFT axis `ax`) is at base + part(n) + col, with base fixed
// by the tile's outer index and column block.
struct OutRows {
  int64_t base, local, sa;  // tile base, elements per rank, local stride of the FFT axis
  int na, rma, cut;         // local extent of the FFT axis, its rank stride, whether it is cut
  __device__ __forceinline__ OutRows(const TmaGeo& G, int ax, int tax, int64_t o, int col0) {
    local = (int64_t)G.n[0] * G.n[1] * G.n[2];
    const int64_t st[3] = {(int64_t)G.n[1] * G.n[2], (int64_t)G.n[2], 1};
    const int64_t gi[3] = {tax == 0 ? o : 0, tax == 1 ? o : 0, (int64_t)col0};
    int64_t rank = 0, idx = 0;
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      if (m == ax) continue;
      int64_t g = gi[m];
      if (G.cut[m]) {
        const int64_t p = g / G.n[m];
        rank += p * G.rmul[m];
        g -= p * G.n[m];
      }
      idx += g * st[m];
    }
    base = rank * local + idx;
    sa = (ax == 0) ? st[0] : (ax == 1) ? st[1] : 1;
    na = G.n[ax];
    rma = G.rmul[ax];
    cut = G.cut[ax];
  }
  __device__ __forceinline__ int64_t row(int n) const {
    if (!cut) return base + (int64_t)n * sa;
    const int p = n / na;
    return base + (int64_t)p * rma * local + (int64_t)(n - p * na) * sa;
  }
};

// Shared memory, in order: three L x W tile buffers (the TMA tile, then the
// A operands over it), B hi / lo, the padded twiddle table, per-column
// maxima and unscale factors (two tiles), six mbarriers (three copy
// barriers, two MMA barriers, spare) and the tensor-memory slot.
template <int L, int W>
struct TcSmem {
  static constexpr size_t tiles = 0;
  static constexpr size_t b = tiles + 3 * (size_t)L * W * sizeof(float2);
  static constexpr size_t tw = b + 2 * kBBytes;
  static constexpr size_t smax = tw + (L + L / 16) * sizeof(float2);
  static constexpr size_t unscale = smax + 2 * W * sizeof(int);
  static constexpr size_t bars = (unscale + 2 * W * sizeof(float) + 7) / 8 * 8;
  static constexpr size_t slot = bars + 6 * sizeof(uint64_t);
  static constexpr size_t total = slot + 2 * sizeof(uint32_t);
};

template <int L, int E, int W, int FMT>
__global__ void __launch_bounds__(W * 16, 1)
    k_strided_tma_tc(const StridedArgs a, const TmaGeo gin, const TmaGeo gout,
                     const __grid_constant__ CUtensorMap tin) {
  static_assert(L == 16 * E && W * E == kRows, "tile = 512 sub-transforms of 16 points");
  static_assert((size_t)L * W * sizeof(float2) >= 2 * kOpBytes, "A fits in a tile buffer");
  using SM = TcSmem<L, W>;
  constexpr int NT = W * 16;  // threads: 16 per line
  constexpr int NW = NT / 32; // warps
  constexpr int BUF = L * W;
  extern __shared__ __align__(128) uint8_t smraw[];
  float2* tiles = reinterpret_cast<float2*>(smraw + SM::tiles);
  uint8_t* b_hi = smraw + SM::b;
  uint8_t* b_lo = b_hi + kBBytes;
  float2* s_tw = reinterpret_cast<float2*>(smraw + SM::tw);
  int* s_max = reinterpret_cast<int*>(smraw + SM::smax);            // [2][W] column maxima (float bits)
  float* s_unscale = reinterpret_cast<float*>(smraw + SM::unscale); // [2][W] factors 2^-s
  uint64_t* bars = reinterpret_cast<uint64_t*>(smraw + SM::bars);   // [0..2] copies, [3..4] MMA
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smraw + SM::slot);

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // a warp holds 16 columns x 2 consecutive jt: its first-stage reads of
  // adjacent rows are contiguous (W = 16), and its A stores spread over 16 banks
  const int cx = (lane & 15) + 16 * (warp % (W / 16));
  const int jt = (lane >> 4) + 2 * (warp / (W / 16));
  const bool inv = a.sign > 0;
  const int64_t ntiles = a.nouter * a.ncolblocks;
  const int tax = (a.oax0 >= 0) ? a.oax0 : -1;
  const uint32_t tile_bytes = (uint32_t)(L * W * sizeof(float2));

  if (tid == 0) {
    for (int k = 0; k < 5; ++k) mbar_init(&bars[k], 1);
    fence_mbar_init();
  }
  build_dft16_operand<FMT>(b_hi, b_lo, kLBO, kSBO, a.tw, L, tid, NT);
  for (int i = tid; i < L; i += NT) s_tw[tws(i)] = __ldg(&a.tw[i]);
  if (tid < 2 * W) s_max[tid] = 0;
  if (warp == 0) {
    tmem_alloc(tmem_slot, kTmemCols);
    tmem_relinquish();
  }
  fence_proxy_async();  // B, written by plain stores, is read by the MMA unit
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  constexpr uint32_t idesc = instr_desc((uint32_t)FMT, 128, 32);

  auto issue_load = [&](int64_t t, float2* dst, uint64_t* bar) {
    int64_t o;
    int2 blk;
    tile_place(a, t, o, blk);
    mbar_expect_tx(bar, tile_bytes);
    for (int k = 0; k < gin.nops; ++k) {
      int c[5];
      tile_coords(gin, a.axis, k, blk.x, o, tax, c);
      tma_load_5d(dst + (size_t)k * gin.rows_per_op * W, &tin, bar, c);
    }
  };
  // accumulator of tile j read back from tensor memory and stored
  auto epilogue = [&](int j, int64_t t) {
    const int k = j & 1;
    int64_t o;
    int2 blk;
    tile_place(a, t, o, blk);
    const OutRows rows(gout, a.axis, tax, o, blk.x);
    const uint32_t acc = tmem + (uint32_t)k * kAccCols;
#pragma unroll
    for (int g = warp >> 2; g < 4; g += NW / 4) {
      float r[32];
      tmem_ld32(acc + ((uint32_t)(32 * (warp & 3)) << 16) + 32 * g, r);
      // lane t of group g is row R = 128 g + 32 (w % 4) + t: sub-transform
      // k1 = R / W of column R % W, whose output k2 is X[k1 + E k2]
      const int R = 128 * g + 32 * (warp & 3) + lane;
      const int k1 = R / W, c = R % W;
      const float fs = (FMT == 0) ? a.scale * s_unscale[k * W + c] : a.scale;
      if (c < blk.y) {
#pragma unroll
        for (int k2 = 0; k2 < 16; ++k2) {
          float2 y = make_float2(r[2 * k2] * fs, r[2 * k2 + 1] * fs);
          if (inv) y.y = -y.y;
          a.out[rows.row(k1 + E * k2) + c] = y;
        }
      }
    }
  };

  const int64_t tile0 = blockIdx.x;
  if (tid == 0 && tile0 < ntiles) issue_load(tile0, tiles, &bars[0]);
  int it = 0, b = 0;   // b = it % 3
  int issued = 0;      // MMA groups committed (tiles 0 .. issued-1)
  int waited = 0;      // MMA commits waited for (tiles 0 .. waited-1)
  bool failed = false;
  for (int64_t tile = tile0; tile < ntiles; tile += gridDim.x, ++it, b = (b == 2) ? 0 : b + 1) {
    float2* cur = tiles + b * BUF;
    const int bn = (b == 2) ? 0 : b + 1;
    const int64_t next = tile + gridDim.x;
    const int k = it & 1;
    // the copy of tile it+1 goes into the buffer of tile it-2, whose A
    // operands were consumed by MMAs waited for in iteration it-1
    if (tid == 0 && next < ntiles) issue_load(next, tiles + bn * BUF, &bars[bn]);
    if (tid == 32 && FMT == 0) {
      for (int c = 0; c < W; ++c) s_max[(k ^ 1) * W + c] = 0;  // tile it+1's maxima
    }
    const bool ok = mbar_wait(&bars[b], (it / 3) & 1, a.wait_limit);
    if (__syncthreads_or(!ok)) {
      if (tid == 0) {
        atomicOr(a.status, TFFT_DEVICE_ETIMEOUT);
        mbar_wait(&bars[b], (it / 3) & 1, kWaitLimit);
        if (next < ntiles) mbar_wait(&bars[bn], ((it + 1) / 3) & 1, kWaitLimit);
      }
      failed = true;
      break;
    }
    // first stage: size-E DFT over n1 of x[jt + 16 n1], then the twiddles
    float2 v[E];
#pragma unroll
    for (int r = 0; r < E; ++r) {
      float2 x = cur[(jt + 16 * r) * W + cx];
      if (inv) x.y = -x.y;
      v[r] = x;
    }
    Dft<E>::run(v);
#pragma unroll
    for (int k1 = 1; k1 < E; ++k1)
      if (jt != 0) v[k1] = cmul(v[k1], s_tw[tws(jt * k1)]);
    if constexpr (FMT == 0) {
      float m = 0.f;
#pragma unroll
      for (int k1 = 0; k1 < E; ++k1) m = fmaxf(m, fmaxf(fabsf(v[k1].x), fabsf(v[k1].y)));
      m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 16));  // the lane of the same column
      if (lane < 16) atomicMax(&s_max[k * W + cx], __float_as_int(m));  // magnitudes: int order = float order
    }
    __syncthreads();  // S1: the tile is read (A may overwrite it), the maxima are complete
    float sc = 1.f;
    if constexpr (FMT == 0) {
      const int sh = fp16_range_shift(__int_as_float(s_max[k * W + cx]));
      sc = exp2_int(sh);
      if (jt == 0) s_unscale[k * W + cx] = exp2_int(-sh);
    }
    uint8_t* a_hi = reinterpret_cast<uint8_t*>(cur);
    uint8_t* a_lo = a_hi + kOpBytes;
#pragma unroll
    for (int k1 = 0; k1 < E; ++k1) {
      uint32_t lo;
      const uint32_t hi = Half16<FMT>::pack_hi_lo(v[k1].x * sc, v[k1].y * sc, lo);
      const uint32_t off = op_off(k1 * W + cx, 2 * jt);
      *reinterpret_cast<uint32_t*>(a_hi + off) = hi;
      *reinterpret_cast<uint32_t*>(a_lo + off) = lo;
    }
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();  // S2: A and the scale factors of tile it are complete
    tc_fence_after();
    if (tid == 0) {
      const uint32_t ah = smem_u32(a_hi), al = smem_u32(a_lo), bh = smem_u32(b_hi), bl = smem_u32(b_lo);
      const uint32_t acc = tmem + (uint32_t)k * kAccCols;
#pragma unroll
      for (int g = 0; g < 4; ++g) {
        const uint32_t d = acc + 32 * g;
        const uint32_t arow = g * (128 / 8) * kSBO;
#pragma unroll
        for (int kk = 0; kk < 2; ++kk) {
          const uint32_t koff = kk * 2 * kLBO;
          umma_f16(d, smem_desc(ah + arow + koff, kLBO, kSBO), smem_desc(bh + koff, kLBO, kSBO), idesc, kk);
          umma_f16(d, smem_desc(al + arow + koff, kLBO, kSBO), smem_desc(bh + koff, kLBO, kSBO), idesc, 1);
          umma_f16(d, smem_desc(ah + arow + koff, kLBO, kSBO), smem_desc(bl + koff, kLBO, kSBO), idesc, 1);
        }
      }
      umma_commit(&bars[3 + k]);
    }
    ++issued;
    // tile it-1: its MMAs ran during this tile's first stage
    if (it > 0) {
      const int j = it - 1;
      const bool mok = mbar_wait(&bars[3 + (j & 1)], (j >> 1) & 1, a.wait_limit);
      if (__syncthreads_or(!mok)) {
        if (tid == 0) {
          atomicOr(a.status, TFFT_DEVICE_ETIMEOUT);
          if (next < ntiles) mbar_wait(&bars[bn], ((it + 1) / 3) & 1, kWaitLimit);
        }
        failed = true;
        break;
      }
      ++waited;
      tc_fence_after();
      epilogue(j, tile - gridDim.x);
      tc_fence_before();
    }
  }
  // the last tile's accumulator
  if (!failed && issued > waited) {
    const int j = issued - 1;
    const bool mok = mbar_wait(&bars[3 + (j & 1)], (j >> 1) & 1, a.wait_limit);
    if (__syncthreads_or(!mok)) {
      if (tid == 0) atomicOr(a.status, TFFT_DEVICE_ETIMEOUT);
    } else {
      ++waited;
      tc_fence_after();
      epilogue(j, tile0 + (int64_t)j * gridDim.x);
    }
  }
  // MMAs committed but never waited for (a wait gave up): wait for their
  // commits, bounded by time rather than by the requested poll limit, before
  // their tensor memory is released
  int drained = 1;
  if (tid == 0) {
    const long long t0 = clock64();
    for (int j = waited; j < issued && drained; ++j) {
      bool done = false;
      while (!done && clock64() - t0 < kCleanupCycles) done = mbar_try(&bars[3 + (j & 1)], (j >> 1) & 1);
      drained = done ? 1 : 0;
    }
    if (!drained) atomicOr(a.status, TFFT_DEVICE_ETMEM);
  }
  tc_fence_before();
  drained = __syncthreads_and(drained);
  tc_fence_after();
  if (warp == 0 && drained) tmem_dealloc(tmem, kTmemCols);
}

template <int L, int E, int W, int FMT>
cudaError_t run_tc_strided(const StridedArgs& a, const TmaGeo& gi, const TmaGeo& go, const CUtensorMap& ti,
                           cudaStream_t s) {
  auto kern = k_strided_tma_tc<L, E, W, FMT>;
  constexpr size_t smem = TcSmem<L, W>::total;
  static_assert(smem <= 227 * 1024, "shared memory of one CTA");
  static PerDevice<cudaError_t> attr_cache;
  const cudaError_t attr = smem_attr_once(attr_cache, kern, (int)smem);
  if (attr != cudaSuccess) return attr;
  if (a.W != W) return cudaErrorInvalidValue;
  // one CTA per SM (shared memory), persistent over the tiles
  const int64_t slots = device_sm_count();
  const int64_t ntiles = a.nouter * a.ncolblocks;
  const int64_t grid = ntiles < slots ? ntiles : slots;
  if (grid < 1) return cudaSuccess;
  kern<<<(unsigned)grid, W * 16, smem, s>>>(a, gi, go, ti);
  return cudaGetLastError();
}

}  // namespace

bool tc_strided_supported(int L, int E, int W, int64_t nelems) {
  (void)nelems;  // offsets are 64-bit
  return (L == 512 && E == 32 && W == 16) || (L == 256 && E == 16 && W == 32);
}

cudaError_t launch_strided_tma_tc(const StridedArgs& a, int E, int precision, const TmaGeo& gi, const TmaGeo& go,
                                  const void* tmap_in, const void* tmap_out, cudaStream_t s) {
  (void)tmap_out;  // the results are stored with plain stores at offsets from the output geometry
  const CUtensorMap& ti = *static_cast<const CUtensorMap*>(tmap_in);
  const bool fp16 = precision == 2;
  if (a.ap.L == 512 && E == 32 && a.W == 16)
    return fp16 ? run_tc_strided<512, 32, 16, 0>(a, gi, go, ti, s) : run_tc_strided<512, 32, 16, 1>(a, gi, go, ti, s);
  if (a.ap.L == 256 && E == 16 && a.W == 32)
    return fp16 ? run_tc_strided<256, 16, 32, 0>(a, gi, go, ti, s) : run_tc_strided<256, 16, 32, 1>(a, gi, go, ti, s);
  return cudaErrorInvalidValue;
}

}  // namespace tfft
