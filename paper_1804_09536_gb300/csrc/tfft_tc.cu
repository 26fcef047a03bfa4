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
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "tfft_tiles.cuh"

namespace tfft {

namespace {

using namespace tiles;

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// ---- tcgen05 wrappers
__device__ __forceinline__ void tmem_alloc(uint32_t* dst_smem, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(dst_smem)),
               "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void umma_f16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_addr(bar))
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&r)[32]) {
  uint32_t u[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]), "=r"(u[6]), "=r"(u[7]),
        "=r"(u[8]), "=r"(u[9]), "=r"(u[10]), "=r"(u[11]), "=r"(u[12]), "=r"(u[13]), "=r"(u[14]), "=r"(u[15]),
        "=r"(u[16]), "=r"(u[17]), "=r"(u[18]), "=r"(u[19]), "=r"(u[20]), "=r"(u[21]), "=r"(u[22]), "=r"(u[23]),
        "=r"(u[24]), "=r"(u[25]), "=r"(u[26]), "=r"(u[27]), "=r"(u[28]), "=r"(u[29]), "=r"(u[30]), "=r"(u[31])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) r[i] = __uint_as_float(u[i]);
}

__device__ __forceinline__ void mbar_init1(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Shared-memory matrix descriptor: no swizzle, K-major core matrices of
// 8 rows x 16 bytes; lbo = bytes between K-adjacent core matrices, sbo =
// bytes between 8-row groups; descriptor version 1.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor, kind::f16: FP32 D, A and B both BF16 (fmt 1) or
// both FP16 (fmt 0), both K-major, N and M.
__host__ __device__ constexpr uint32_t instr_desc(uint32_t fmt, uint32_t M, uint32_t N) {
  return (1u << 4) | (fmt << 7) | (fmt << 10) | ((N >> 3) << 17) | ((M >> 4) << 24);
}

// Operand layout: K-major, no swizzle, K = 32 16-bit elements per row.  Core
// matrix (row / 8, k / 8) starts at (row / 8) * kSBO + (k / 8) * kLBO; inside
// it row % 8 sits at 16 B and k % 8 at 2 B.  kLBO = 144 and kSBO = 592 (not
// the dense 128 / 512) put the 16 column pairs two lines write at once on
// distinct shared-memory banks.
constexpr uint32_t kLBO = 144, kSBO = 592;
__device__ __forceinline__ uint32_t op_off(int row, int k) {
  return (uint32_t)((row >> 3) * kSBO + (k >> 3) * kLBO + (row & 7) * 16 + (k & 7) * 2);
}

template <int FMT>
struct Half16;
template <>
struct Half16<1> {  // BF16
  using T = __nv_bfloat16;
  __device__ static uint32_t pack_hi_lo(float re, float im, uint32_t& lo) {
    const __nv_bfloat16 rh = __float2bfloat16_rn(re), ih = __float2bfloat16_rn(im);
    const __nv_bfloat16 rl = __float2bfloat16_rn(re - __bfloat162float(rh));
    const __nv_bfloat16 il = __float2bfloat16_rn(im - __bfloat162float(ih));
    lo = (uint32_t)__bfloat16_as_ushort(rl) | ((uint32_t)__bfloat16_as_ushort(il) << 16);
    return (uint32_t)__bfloat16_as_ushort(rh) | ((uint32_t)__bfloat16_as_ushort(ih) << 16);
  }
  __device__ static void split(float x, uint16_t& hi, uint16_t& lo) {
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    hi = __bfloat16_as_ushort(h);
    lo = __bfloat16_as_ushort(__float2bfloat16_rn(x - __bfloat162float(h)));
  }
};
template <>
struct Half16<0> {  // FP16
  using T = __half;
  __device__ static uint32_t pack_hi_lo(float re, float im, uint32_t& lo) {
    const __half rh = __float2half_rn(re), ih = __float2half_rn(im);
    const __half rl = __float2half_rn(re - __half2float(rh));
    const __half il = __float2half_rn(im - __half2float(ih));
    lo = (uint32_t)__half_as_ushort(rl) | ((uint32_t)__half_as_ushort(il) << 16);
    return (uint32_t)__half_as_ushort(rh) | ((uint32_t)__half_as_ushort(ih) << 16);
  }
  __device__ static void split(float x, uint16_t& hi, uint16_t& lo) {
    const __half h = __float2half_rn(x);
    hi = __half_as_ushort(h);
    lo = __half_as_ushort(__float2half_rn(x - __half2float(h)));
  }
};

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

// Range scaling of the FP16 operands.  A line's sub-transform inputs are
// multiplied by 2^s, s chosen from their largest magnitude m so that m 2^s
// lies in [2^14, 2^15): the hi parts then stay below the FP16 maximum (65504)
// and the lo parts of everything within 2^17 of the maximum stay normal
// (FP16 subnormals would cut their precision).  The power of two is exact in
// FP32, and the accumulator is multiplied by 2^-s in the epilogue.  BF16 has
// FP32's exponent range and needs no scaling.  s is clamped so that 2^s and
// 2^-s are normal floats; a zero (or NaN) line keeps s = 0.
__device__ __forceinline__ int fp16_range_shift(float m) {
  if (!(m > 0.f)) return 0;
  const int e = ((__float_as_int(m) >> 23) & 255) - 126;  // m < 2^e
  const int sh = 15 - e;
  return sh < -126 ? -126 : (sh > 126 ? 126 : sh);
}
__device__ __forceinline__ float exp2_int(int sh) { return __int_as_float((sh + 127) << 23); }

// Second, clean-up wait for MMAs still in flight after a wait gave up: about
// one second of clock cycles.  Tensor memory is released only once they are
// known to be complete; if even this wait expires, the CTA leaves it
// allocated (status TFFT_DEVICE_ETMEM) rather than free memory an MMA may
// still write.
constexpr long long kCleanupCycles = 2000000000LL;

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

  // the 16-point DFT as a real 32 x 32 operand, hi and lo parts (row = output
  // re/im of k, column = input re/im of n), twiddles from the L-root table
  for (int idx = tid; idx < 32 * 32; idx += kThreads) {
    const int o = idx >> 5, k = idx & 31;
    const int ko = o >> 1, ni = k >> 1;
    const float2 w = __ldg(&a.tw[((ko * ni) & 15) * (kL / 16)]);  // exp(-2 pi i k n / 16)
    const float c = w.x, s = -w.y;                                 // cos, sin
    float v;
    if ((o & 1) == 0) v = (k & 1) == 0 ? c : s;   // Y.re = c x.re + s x.im
    else v = (k & 1) == 0 ? -s : c;               // Y.im = -s x.re + c x.im
    uint16_t h, l;
    Half16<FMT>::split(v, h, l);
    *reinterpret_cast<uint16_t*>(b_hi + op_off(o, k)) = h;
    *reinterpret_cast<uint16_t*>(b_lo + op_off(o, k)) = l;
  }
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
