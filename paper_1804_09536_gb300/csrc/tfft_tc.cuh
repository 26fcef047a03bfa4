// tcgen05 (5th-generation tensor core) building blocks shared by the
// tensor-core FFT passes (tfft_tc.cu: contiguous lines, tfft_tc_strided.cu:
// strided TMA tiles): tensor-memory allocation, kind::f16 MMA issue and
// commit, tensor-memory loads, bounded mbarrier polls, shared-memory matrix
// and instruction descriptors, the hi/lo split of FP32 values into two
// 16-bit parts, the FP16 range scaling and the 16-point DFT operand.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "tfft_tiles.cuh"

namespace tfft {
namespace tc {

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

// The 16-point DFT as a real 32 x 32 operand B (row o = output re/im of
// k = o / 2, column kk = input re/im of n = kk / 2), split in hi and lo parts
// and stored K-major at byte offset (o / 8) sbo + (kk / 8) lbo + (o % 8) 16 +
// (kk % 8) 2 of b_hi / b_lo; the cosines and sines come from the L-root
// table tw (exp(-2 pi i m / L), L a multiple of 16).  D = A B^T then maps a
// row of 16 complex inputs (re, im interleaved) to its 16 outputs.
template <int FMT>
__device__ __forceinline__ void build_dft16_operand(uint8_t* b_hi, uint8_t* b_lo, uint32_t lbo, uint32_t sbo,
                                                    const float2* __restrict__ tw, int L, int tid, int nthreads) {
  for (int idx = tid; idx < 32 * 32; idx += nthreads) {
    const int o = idx >> 5, k = idx & 31;
    const int ko = o >> 1, ni = k >> 1;
    const float2 w = __ldg(&tw[((ko * ni) & 15) * (L / 16)]);  // exp(-2 pi i k n / 16)
    const float c = w.x, s = -w.y;                              // cos, sin
    float v;
    if ((o & 1) == 0) v = (k & 1) == 0 ? c : s;  // Y.re = c x.re + s x.im
    else v = (k & 1) == 0 ? -s : c;              // Y.im = -s x.re + c x.im
    uint16_t h, l;
    Half16<FMT>::split(v, h, l);
    const uint32_t off = (uint32_t)((o >> 3) * sbo + (k >> 3) * lbo + (o & 7) * 16 + (k & 7) * 2);
    *reinterpret_cast<uint16_t*>(b_hi + off) = h;
    *reinterpret_cast<uint16_t*>(b_lo + off) = l;
  }
}

}  // namespace tc
}  // namespace tfft
