// Strided TMA passes of lengths 512 = 32 x 16 and 256 = 16 x 16 whose last,
// radix-16 stage runs on the 5th-generation tensor cores (tcgen05.mma,
// kind::f16, FP32 accumulation in tensor memory): the tensor-core form of the
// fused exchange-and-transform pass of tfft_tma.cu (Eqs. pencil1 / pencil2
// with the redistributions of Eq. gtp1 / gtp2 in the tile copies).
//
// A tile is L rows (the FFT axis) x W columns, loaded and stored by TMA as in
// the FP32 kernel (three buffers: load i+1 / compute i / store i-1).  Line
// cx of the tile is the length-L FFT x[n], n = n2 + 16 n1 (n2 < 16, n1 < E,
// L = 16 E): thread (cx, jt = n2) loads x[jt + 16 n1] for all n1 and runs
// the first stage, a size-E DFT over n1, in registers; its output k1 times
// the twiddle exp(-2 pi i jt k1 / L) is input jt of the 16-point
// sub-transform (cx, k1).  The W x E sub-transforms of a tile are the rows
// of A (K = 32 reals: re/im of their 16 inputs) and the 16-point DFT is the
// 32 x 32 real matrix B, so D = A B^T holds every sub-transform's 16 outputs
// X[k1 + E k2]; with A and B split in hi + lo 16-bit parts,
// D = A_hi B_hi + A_lo B_hi + A_hi B_lo (FP32 accumulation) keeps about
// twice the 16-bit mantissa.  FP16 operands are range-scaled per line (a
// power of two from the line's largest magnitude, undone on the
// accumulator).
//
// A (two operands of W E rows x 64 B) is written over the tile's own buffer
// once the first stage has read it; the MMA result is read back from tensor
// memory (tcgen05.ld) into the same buffer in natural order, and TMA stores
// it.  W E / 128 MMA groups of M = 128 rows, N = 32, K = 32 (two K = 16
// steps, three products each) per tile; one thread issues them and commits
// to an mbarrier.  Narrow tiles (W E = 256 rows, 96 KB of tile buffers) fit
// two CTAs per SM, which overlap each other's barrier and MMA waits.  Every
// wait is bounded; tensor memory is released before the CTA leaves, unless
// MMAs are still running after the clean-up wait.
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
constexpr uint32_t kBBytes = 32 * 64;  // the 32 x 32 DFT operand

__device__ __forceinline__ uint32_t op_off(int row, int k) {
  return (uint32_t)((row >> 3) * kSBO + (k >> 3) * kLBO + (row & 7) * 16 + (k & 7) * 2);
}

// Twiddle slot with one spare entry every 16: the lanes of a warp read
// indices jt k1 for a few consecutive jt, so stride-k1 patterns spread out.
__device__ __forceinline__ int tws(int i) { return i + (i >> 4); }

// Geometry of one compiled variant: rows of A (sub-transforms per tile), MMA
// groups, tensor-memory columns (a power of two >= 32), shared memory, CTAs
// per SM.
template <int L, int E, int W>
struct TcGeo {
  static_assert(L == 16 * E, "last stage of 16 points");
  static constexpr int NT = W * 16;  // threads: 16 per line
  static constexpr int ROWS = W * E;
  static constexpr int NG = ROWS / 128;
  static_assert(ROWS % 128 == 0 && NG >= 1 && NG <= 4, "whole M = 128 groups");
  static constexpr uint32_t OP = ROWS * 64;  // one 16-bit operand
  static constexpr uint32_t TMEM = NG * 32 < 32 ? 32 : (NG == 3 ? 128 : NG * 32);
  static constexpr size_t BUF = (size_t)L * W;  // complex elements per tile buffer
  static_assert(BUF * sizeof(float2) >= 2 * OP, "A fits in a tile buffer");
  // tile buffers: three (load i+1 / compute i / store i-1 drain) unless two
  // let a third CTA fit on the SM
  static constexpr size_t extra = 2 * kBBytes + (L + L / 16) * sizeof(float2) + 5 * sizeof(uint64_t) +
                                  2 * sizeof(uint32_t) + 2 * W * sizeof(float);
  static constexpr int NB = (2 * BUF * sizeof(float2) + extra <= 74 * 1024) ? 2 : 3;
  static constexpr size_t SMEM = NB * BUF * sizeof(float2) + extra;
  static constexpr int CTAS = SMEM <= 74 * 1024 ? 3 : (SMEM <= 113 * 1024 ? 2 : 1);
  static_assert(CTAS * TMEM <= 512, "tensor memory columns per SM");
};

template <int L, int E, int W, int FMT>
__global__ void __launch_bounds__(W * 16, TcGeo<L, E, W>::CTAS)
    k_strided_tma_tc(const StridedArgs a, const TmaGeo gin, const TmaGeo gout,
                     const __grid_constant__ CUtensorMap tin, const __grid_constant__ CUtensorMap tout) {
  using G = TcGeo<L, E, W>;
  constexpr int NT = G::NT, NW = NT / 32;
  constexpr int BUF = (int)G::BUF;
  extern __shared__ __align__(128) float2 smem[];
  constexpr int NB = G::NB;
  uint8_t* b_hi = reinterpret_cast<uint8_t*>(smem + NB * BUF);
  uint8_t* b_lo = b_hi + kBBytes;
  float2* s_tw = reinterpret_cast<float2*>(b_lo + kBBytes);
  uint64_t* bars = reinterpret_cast<uint64_t*>(s_tw + L + L / 16);  // [0..2] copies, [3] MMA
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 5);
  int* s_max = reinterpret_cast<int*>(tmem_slot + 2);                // W column maxima (float bits)
  float* s_unscale = reinterpret_cast<float*>(s_max + W);            // W factors 2^-s

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // W >= 16: a warp holds 16 columns x 2 consecutive jt (its first-stage
  // reads of adjacent rows are contiguous when W = 16); W = 8: 8 columns x 4
  // consecutive jt, so that its A stores cover the 8 rows x 4 words of a
  // core matrix -- all 32 banks
  constexpr int CW = W >= 16 ? 16 : W;  // columns per warp
  const int cx = (lane % CW) + CW * (warp % (W / CW));
  const int jt = (lane / CW) + (32 / CW) * (warp / (W / CW));
  const bool inv = a.sign > 0;
  const int64_t ntiles = a.nouter * a.ncolblocks;
  const int tax = (a.oax0 >= 0) ? a.oax0 : -1;
  const uint32_t tile_bytes = (uint32_t)(L * W * sizeof(float2));

  if (tid == 0) {
    for (int b = 0; b < 4; ++b) mbar_init(&bars[b], 1);
    fence_mbar_init();
  }
  build_dft16_operand<FMT>(b_hi, b_lo, kLBO, kSBO, a.tw, L, tid, NT);
  for (int i = tid; i < L; i += NT) s_tw[tws(i)] = __ldg(&a.tw[i]);
  if (tid < W) s_max[tid] = 0;
  if (warp == 0) {
    tmem_alloc(tmem_slot, G::TMEM);
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

  int64_t tile = blockIdx.x;
  if (tid == 0 && tile < ntiles) issue_load(tile, smem, &bars[0]);
  int it = 0, b = 0;  // b = it % NB
  uint32_t mma_phase = 0;
  bool mma_pending = false;  // an MMA group may still be running (failure path)
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
    const bool ok = mbar_wait(&bars[b], (it / NB) & 1, a.wait_limit);
    if (__syncthreads_or(!ok)) {
      if (tid == 0) {
        atomicOr(a.status, TFFT_DEVICE_ETIMEOUT);
        mbar_wait(&bars[b], (it / NB) & 1, kWaitLimit);
        if (next < ntiles) mbar_wait(&bars[bn], ((it + 1) / NB) & 1, kWaitLimit);
      }
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
#pragma unroll
      for (int o = CW; o < 32; o <<= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));  // lanes of one column
      if (lane < CW) atomicMax(&s_max[cx], __float_as_int(m));  // magnitudes: int order = float order
    }
    __syncthreads();  // the tile is read (A may overwrite it) and the column maxima are complete
    float sc = 1.f;
    if constexpr (FMT == 0) {
      const int sh = fp16_range_shift(__int_as_float(s_max[cx]));
      sc = exp2_int(sh);
      if (jt == 0) s_unscale[cx] = exp2_int(-sh);
    }
    uint8_t* a_hi = reinterpret_cast<uint8_t*>(cur);
    uint8_t* a_lo = a_hi + G::OP;
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
    __syncthreads();
    tc_fence_after();
    if (tid == 0) {
      const uint32_t ah = smem_u32(a_hi), al = smem_u32(a_lo), bh = smem_u32(b_hi), bl = smem_u32(b_lo);
#pragma unroll
      for (int g = 0; g < G::NG; ++g) {
        const uint32_t d = tmem + 32 * g;
        const uint32_t arow = g * (128 / 8) * kSBO;
#pragma unroll
        for (int kk = 0; kk < 2; ++kk) {
          const uint32_t koff = kk * 2 * kLBO;
          umma_f16(d, smem_desc(ah + arow + koff, kLBO, kSBO), smem_desc(bh + koff, kLBO, kSBO), idesc, kk);
          umma_f16(d, smem_desc(al + arow + koff, kLBO, kSBO), smem_desc(bh + koff, kLBO, kSBO), idesc, 1);
          umma_f16(d, smem_desc(ah + arow + koff, kLBO, kSBO), smem_desc(bl + koff, kLBO, kSBO), idesc, 1);
        }
      }
      umma_commit(&bars[3]);
    }
    if constexpr (FMT == 0) {
      if (tid < W) s_max[tid] = 0;  // every thread read its maximum before the barrier above
    }
    const bool mok = mbar_wait(&bars[3], mma_phase, a.wait_limit);
    mma_phase ^= 1;
    if (__syncthreads_or(!mok)) {
      mma_pending = true;
      if (tid == 0) {
        atomicOr(a.status, TFFT_DEVICE_ETIMEOUT);
        if (next < ntiles) mbar_wait(&bars[bn], ((it + 1) / NB) & 1, kWaitLimit);
      }
      break;
    }
    tc_fence_after();
    // epilogue: warp w reads tensor-memory lanes 32 (w % 4) .. + 31 of its
    // groups; lane t of group g is row R = 128 g + 32 (w % 4) + t, i.e.
    // sub-transform k1 = R / W of column R % W, whose output k2 is X[k1 + E k2]
#pragma unroll
    for (int g = warp >> 2; g < G::NG; g += NW / 4) {
      float r[32];
      tmem_ld32(tmem + ((uint32_t)(32 * (warp & 3)) << 16) + 32 * g, r);
      const int R = 128 * g + 32 * (warp & 3) + lane;
      const int k1 = R / W, c = R % W;
      const float f = (FMT == 0) ? a.scale * s_unscale[c] : a.scale;
#pragma unroll
      for (int k2 = 0; k2 < 16; ++k2) {
        float2 y = make_float2(r[2 * k2] * f, r[2 * k2 + 1] * f);
        if (inv) y.y = -y.y;
        cur[(k1 + E * k2) * W + c] = y;
      }
    }
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (tid == 0) {
      int64_t o;
      int2 blk;
      tile_place(a, tile, o, blk);
      for (int k = 0; k < gout.nops; ++k) {
        int c[5];
        tile_coords(gout, a.axis, k, blk.x, o, tax, c);
        tma_store_5d(&tout, cur + (size_t)k * gout.rows_per_op * W, c);
      }
      bulk_commit();
    }
  }
  if (tid == 0) bulk_wait_all();
  // after a wait gave up, the last MMA group may still be running: wait for
  // its commit (bounded by time, not by the requested poll limit) before its
  // tensor memory is released
  int drained = 1;
  if (mma_pending && tid == 0) {
    drained = 0;
    const long long t0 = clock64();
    while (!drained && clock64() - t0 < kCleanupCycles) drained = mbar_try(&bars[3], mma_phase ^ 1) ? 1 : 0;
    if (!drained) atomicOr(a.status, TFFT_DEVICE_ETMEM);
  }
  tc_fence_before();
  drained = __syncthreads_and(drained);
  tc_fence_after();
  if (warp == 0 && drained) tmem_dealloc(tmem, G::TMEM);
}

template <int L, int E, int W, int FMT>
cudaError_t run_tc_strided(const StridedArgs& a, const TmaGeo& gi, const TmaGeo& go, const CUtensorMap& ti,
                           const CUtensorMap& to, cudaStream_t s) {
  using G = TcGeo<L, E, W>;
  auto kern = k_strided_tma_tc<L, E, W, FMT>;
  static_assert(G::SMEM <= 227 * 1024, "shared memory of one CTA");
  static PerDevice<cudaError_t> attr_cache;
  const cudaError_t attr = smem_attr_once(attr_cache, kern, (int)G::SMEM);
  if (attr != cudaSuccess) return attr;
  if (a.W != W) return cudaErrorInvalidValue;
  // G::CTAS per SM (shared and tensor memory allow it), persistent over the tiles
  const int64_t slots = (int64_t)device_sm_count() * G::CTAS;
  const int64_t ntiles = a.nouter * a.ncolblocks;
  const int64_t grid = ntiles < slots ? ntiles : slots;
  if (grid < 1) return cudaSuccess;
  kern<<<(unsigned)grid, G::NT, G::SMEM, s>>>(a, gi, go, ti, to);
  return cudaGetLastError();
}

// Compiled variants: length, first-stage radix E, tile width W.  The first
// row of a length is its default; TFFT_TC_W="512:16" picks another width.
#define TFFT_TC_STRIDED(X) \
  X(512, 32, 8)            \
  X(512, 32, 16)           \
  X(256, 16, 16)           \
  X(256, 16, 32)

}  // namespace

bool tc_strided_variant(int L, int want_W, int& E, int& W) {
  bool found = false;
#define X(LL, EE, WW)                                      \
  if (LL == L && (!found || WW == want_W)) {               \
    E = EE;                                                \
    W = WW;                                                \
    if (WW == want_W) return true;                         \
    found = true;                                          \
  }
  TFFT_TC_STRIDED(X)
#undef X
  return found;
}

cudaError_t launch_strided_tma_tc(const StridedArgs& a, int E, int precision, const TmaGeo& gi, const TmaGeo& go,
                                  const void* tmap_in, const void* tmap_out, cudaStream_t s) {
  const CUtensorMap& ti = *static_cast<const CUtensorMap*>(tmap_in);
  const CUtensorMap& to = *static_cast<const CUtensorMap*>(tmap_out);
  const bool fp16 = precision == 2;
#define X(LL, EE, WW)                                                              \
  if (a.ap.L == LL && E == EE && a.W == WW)                                        \
    return fp16 ? run_tc_strided<LL, EE, WW, 0>(a, gi, go, ti, to, s)             \
                : run_tc_strided<LL, EE, WW, 1>(a, gi, go, ti, to, s);
  TFFT_TC_STRIDED(X)
#undef X
  return cudaErrorInvalidValue;
}

}  // namespace tfft
