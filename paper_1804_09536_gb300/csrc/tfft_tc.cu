// Contiguous-line pass of length 512 = 32 x 16 whose radix-16 stage runs on
// the 5th-generation tensor cores (tcgen05.mma, kind::f16, FP32 accumulate
// in tensor memory).
//
// After the radix-32 stage (registers) every line holds 32 length-16
// sub-transforms.  Their twiddled inputs form the rows of A (one row per
// sub-transform, K = 32 reals: re/im of the 16 inputs, interleaved) and the
// 16-point DFT is the real 32 x 32 matrix B = [[c, s], [-s, c]] blocks
// (c = cos, s = sin of 2 pi k n / 16); D = A B^T gives each row's 16 outputs,
// re/im interleaved.  A and B are split into hi + lo 16-bit parts (BF16 or
// FP16) and D = A_hi B_hi + A_lo B_hi + A_hi B_lo (FP32 accumulation), which
// keeps roughly twice the 16-bit mantissa.
//
// CTA = 4 warps, 8 lines (16 threads per line, 32 elements each); two MMA
// groups of M = 128 rows (4 lines each), N = 32, K = 32 (two K = 16 steps).
// Operands in shared memory use the no-swizzle K-major core-matrix layout
// (8 rows x 16 bytes per core matrix).  The MMA completion is signalled on an
// mbarrier with a bounded wait; tensor memory is allocated once per CTA and
// released before the CTA exits, on every path.
#include "tfft_tc.cuh"

namespace tfft {

namespace {

using namespace tiles;
using namespace tc;

// Operand layout: K-major, no swizzle, K = 32 16-bit elements per row.  Core
// matrix (row / 8, k / 8) starts at (row / 8) * kSBO + (k / 8) * kLBO; inside
// it row % 8 sits at 16 B and k % 8 at 2 B.  kLBO = 144 and kSBO = 592 (not
// the dense 128 / 512) put the 16 column pairs two lines write at once on
// distinct shared-memory banks.
constexpr uint32_t kLBO = 144, kSBO = 592;
__device__ __forceinline__ uint32_t op_off(int row, int k) {
  return (uint32_t)((row >> 3) * kSBO + (k >> 3) * kLBO + (row & 7) * 16 + (k & 7) * 2);
}

constexpr int kL = 512, kE = 32, kT = 16, kLines = 8, kThreads = kT * kLines;
constexpr int kRows = kLines * 32;                 // 256 sub-transforms per tile
constexpr uint32_t kOpBytes = (kRows / 8) * kSBO;  // one 256 x 32 16-bit operand
constexpr uint32_t kBBytes = (32 / 8) * kSBO;      // the 32 x 32 DFT operand
constexpr uint32_t kTmemCols = 64;                 // two FP32 groups of 32 columns
// The stage-2 twiddles w^(jt r1) of the 512-root table, kept in shared memory
// with one spare slot every 16: a half-warp reads indices jt * r1 (stride r1),
// which would otherwise put up to 16 lanes on one bank for even r1.
constexpr int kTwSlots = 512 + 512 / 16;
__device__ __forceinline__ int tw_slot(int i) { return i + (i >> 4); }
constexpr int kCtasPerSm = 4;                      // 4 x 64 of the 512 tensor-memory columns
static_assert(kCtasPerSm * kTmemCols <= 512, "tensor memory columns per SM");

template <int FMT>
__global__ void __launch_bounds__(kThreads, kCtasPerSm) k_contig_tc512(const ContigArgs a) {
  extern __shared__ __align__(1024) uint8_t sm[];
  uint8_t* a_hi = sm;
  uint8_t* a_lo = sm + kOpBytes;
  uint8_t* b_hi = sm + 2 * kOpBytes;
  uint8_t* b_lo = b_hi + kBBytes;
  float2* s_tw = reinterpret_cast<float2*>(b_lo + kBBytes);  // the twiddles jt * r1 < 512, padded
  uint64_t* bar = reinterpret_cast<uint64_t*>(s_tw + kTwSlots);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bar + 1);
  float* s_unscale = reinterpret_cast<float*>(tmem_slot + 1);  // 2^-s per line (FP16)
  const int tid = threadIdx.x, warp = tid >> 5;
  const int jt = tid % kT, ly = tid / kT;
  const bool inv = a.sign > 0;

  build_dft16_operand<FMT>(b_hi, b_lo, kLBO, kSBO, a.tw, kL, tid, kThreads);
  for (int i = tid; i < kL; i += kThreads) s_tw[tw_slot(i)] = __ldg(&a.tw[i]);
  if (tid == 0) {
    mbar_init1(bar);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    tmem_alloc(tmem_slot, kTmemCols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  constexpr uint32_t idesc = instr_desc((uint32_t)FMT, 128, 32);
  const float oscale = contig_scale(a);
  bool failed = false;
  uint32_t phase = 0;

  // the loads of a tile: thread jt of line ly holds x[jt + 16 r], r < 32
  float2 v[kE];
  auto load_tile = [&](int64_t t) {
    const int64_t line = t * kLines + ly;
    const bool act = line < a.nlines;
    const float2* src = a.in + line * kL;
#pragma unroll
    for (int r = 0; r < kE; ++r) v[r] = act ? src[jt + kT * r] : make_float2(0.f, 0.f);
  };
  if ((int64_t)blockIdx.x * kLines < a.nlines) load_tile(blockIdx.x);

  for (int64_t tile = blockIdx.x; tile * kLines < a.nlines; tile += gridDim.x) {
    // radix-32 stage on the loaded values
#pragma unroll
    for (int r = 0; r < kE; ++r)
      if (inv) v[r].y = -v[r].y;
    Dft<32>::run(v);
    // output r1 of this thread is input jt of sub-transform j = r1; twiddle
    // exp(-2 pi i jt r1 / 512)
#pragma unroll
    for (int r1 = 1; r1 < kE; ++r1)
      if (jt != 0) v[r1] = cmul(v[r1], s_tw[tw_slot(jt * r1)]);
    float sc = 1.f;
    if constexpr (FMT == 0) {
      float m = 0.f;
#pragma unroll
      for (int r1 = 0; r1 < kE; ++r1) m = fmaxf(m, fmaxf(fabsf(v[r1].x), fabsf(v[r1].y)));
#pragma unroll
      for (int o = 8; o >= 1; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));  // the line's 16 lanes
      const int sh = fp16_range_shift(m);
      sc = exp2_int(sh);
      if (jt == 0) s_unscale[ly] = exp2_int(-sh);
    }
    // the A rows (line, r1), columns 2 jt, 2 jt + 1
#pragma unroll
    for (int r1 = 0; r1 < kE; ++r1) {
      uint32_t lo;
      const uint32_t hi = Half16<FMT>::pack_hi_lo(v[r1].x * sc, v[r1].y * sc, lo);
      const uint32_t off = op_off(ly * 32 + r1, 2 * jt);
      *reinterpret_cast<uint32_t*>(a_hi + off) = hi;
      *reinterpret_cast<uint32_t*>(a_lo + off) = lo;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (tid == 0) {
      const uint32_t ah = smem_addr(a_hi), al = smem_addr(a_lo), bh = smem_addr(b_hi), bl = smem_addr(b_lo);
#pragma unroll
      for (int g = 0; g < 2; ++g) {
        const uint32_t d = tmem + 32 * g;
        const uint32_t arow = g * (128 / 8) * kSBO;  // first 8-row group of this M = 128 block
#pragma unroll
        for (int kk = 0; kk < 2; ++kk) {              // K = 16 per instruction
          const uint32_t koff = kk * 2 * kLBO;        // two core matrices along K
          umma_f16(d, smem_desc(ah + arow + koff, kLBO, kSBO), smem_desc(bh + koff, kLBO, kSBO), idesc, kk);
          umma_f16(d, smem_desc(al + arow + koff, kLBO, kSBO), smem_desc(bh + koff, kLBO, kSBO), idesc, 1);
          umma_f16(d, smem_desc(ah + arow + koff, kLBO, kSBO), smem_desc(bl + koff, kLBO, kSBO), idesc, 1);
        }
      }
      umma_commit(bar);
    }
    // the next tile's loads, in flight while the MMAs and this tile's epilogue run
    {
      const int64_t next = tile + gridDim.x;
      if (next * kLines < a.nlines) load_tile(next);
    }
    // bounded wait for the MMAs (first poll non-blocking)
    bool ok = mbar_test(bar, phase);
    for (uint32_t i = 1; i < a.wait_limit && !ok; ++i) ok = mbar_try(bar, phase);
    phase ^= 1;
    if (__syncthreads_or(!ok)) {
      if (tid == 0) atomicOr(a.status, TFFT_DEVICE_ETIMEOUT);
      failed = true;
      break;
    }
    tc_fence_after();
    // warp w reads rows 32 w .. 32 w + 31 of both groups: group g row 32 w + t is
    // sub-transform j = t of line 4 g + w
#pragma unroll
    for (int g = 0; g < 2; ++g) {
      float r[32];
      tmem_ld32(tmem + ((uint32_t)(32 * warp) << 16) + 32 * g, r);
      const int lline = 4 * g + warp;
      const int64_t gl = tile * kLines + lline;
      if (gl < a.nlines) {
        float2* dst = a.out + gl * kL;
        const int j = tid & 31;
        const float f = (FMT == 0) ? oscale * s_unscale[lline] : oscale;
#pragma unroll
        for (int k = 0; k < 16; ++k) {
          float2 y = make_float2(r[2 * k] * f, r[2 * k + 1] * f);
          if (inv) y.y = -y.y;
          dst[j + 32 * k] = y;
        }
      }
    }
    tc_fence_before();
    __syncthreads();  // TMEM and the A operands are free for the next tile
    tc_fence_after();
  }
  // after a wait gave up, the MMAs of that tile may still be running: wait
  // for their commit (bounded by time, not by the requested poll limit,
  // which may have been tiny on purpose) before their memory is released
  int drained = 1;
  if (failed && tid == 0) {
    drained = 0;
    const long long t0 = clock64();
    while (!drained && clock64() - t0 < kCleanupCycles) drained = mbar_try(bar, phase ^ 1) ? 1 : 0;
    if (!drained) atomicOr(a.status, TFFT_DEVICE_ETMEM);
  }
  tc_fence_before();
  drained = __syncthreads_and(drained);
  tc_fence_after();
  if (warp == 0 && drained) tmem_dealloc(tmem, kTmemCols);
}

template <int FMT>
cudaError_t run_tc(const ContigArgs& a, cudaStream_t s) {
  const size_t smem = 2 * kOpBytes + 2 * kBBytes + kTwSlots * sizeof(float2) + 16 + kLines * sizeof(float);
  static PerDevice<cudaError_t> attr_cache;
  const cudaError_t attr = smem_attr_once(attr_cache, k_contig_tc512<FMT>, (int)smem);
  if (attr != cudaSuccess) return attr;
  // kCtasPerSm resident CTAs per SM (the launch bounds' promise); the grid
  // is a persistent tile loop, so extra CTAs would only queue
  const int slots = device_sm_count() * kCtasPerSm;
  const int64_t ntiles = (a.nlines + kLines - 1) / kLines;
  const int64_t grid = ntiles < slots ? ntiles : slots;
  if (grid < 1) return cudaSuccess;
  k_contig_tc512<FMT><<<(unsigned)grid, kThreads, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace

bool tc_supported(int L) { return L == kL; }

cudaError_t launch_contig_tc(const ContigArgs& a, int precision, cudaStream_t s) {
  if (a.ap.L != kL) return cudaErrorInvalidValue;
  return precision == 2 ? run_tc<0>(a, s) : run_tc<1>(a, s);
}

}  // namespace tfft
