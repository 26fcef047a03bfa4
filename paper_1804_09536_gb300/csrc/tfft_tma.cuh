// TMA, bulk-copy and mbarrier building blocks (inline PTX, sm_103a) shared by
// the strided TMA passes (tfft_tma.cu) and the batched executor
// (tfft_batch.cu), and the mapping of a strided tile to tensor-map
// coordinates.  Every mbarrier wait is bounded.
#pragma once

#include <cuda.h>

#include "tfft_internal.h"

namespace tfft {
namespace tma {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ bool mbar_test_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait: false after `limit` polls.  The first poll does not block
// (test_wait); the others may suspend the thread for a while (try_wait).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint32_t limit) {
  if (limit == 0) return false;
  if (mbar_test_wait(bar, parity)) return true;
  for (uint32_t i = 1; i < limit; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void tma_load_5d(void* dst, const CUtensorMap* map, uint64_t* bar,
                                            const int (&c)[5]) {
  asm volatile(
      "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4, %5, %6, %7}], [%2];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(c[0]), "r"(c[1]), "r"(c[2]),
      "r"(c[3]), "r"(c[4])
      : "memory");
}

__device__ __forceinline__ void tma_store_5d(const CUtensorMap* map, const void* src, const int (&c)[5]) {
  asm volatile(
      "cp.async.bulk.tensor.5d.global.shared::cta.tile.bulk_group [%0, {%2, %3, %4, %5, %6}], [%1];" ::"l"(
          reinterpret_cast<uint64_t>(map)),
      "r"(smem_u32(src)), "r"(c[0]), "r"(c[1]), "r"(c[2]), "r"(c[3]), "r"(c[4])
      : "memory");
}

__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }

template <int N>
__device__ __forceinline__ void bulk_wait_read() {
  asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(N) : "memory");
}

__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

constexpr uint32_t kWaitLimit = 1u << 22;  // polls of the second, clean-up wait

// Coordinates of op k of a tile in one stage layout (see TmaGeo).
__device__ __forceinline__ void tile_coords(const TmaGeo& G, int axis, int k, int64_t col, int64_t gt,
                                            int tax, int (&c)[5]) {
#pragma unroll
  for (int i = 0; i < 5; ++i) c[i] = 0;
  if (G.split) {  // [rank][outer][axis / split][split][n2]: the whole tile is op 0
    const int64_t pc = G.cut[2] ? col / G.n[2] : 0;
    const int64_t po = G.cut[tax] ? gt / G.n[tax] : 0;
    c[0] = (int)(col - pc * G.n[2]);
    c[3] = (int)(gt - po * G.n[tax]);
    c[4] = (int)(pc * G.rmul[2] + po * G.rmul[tax]);
    return;
  }
#pragma unroll
  for (int m = 0; m < 3; ++m) {
    int64_t g = (m == axis) ? (int64_t)k * G.rows_per_op : (m == 2) ? col : (m == tax) ? gt : 0;
    if (G.cut[m]) {
      if (m == axis) g = 0;  // the box spans every rank of the subgroup
      const int64_t p = g / G.n[m];
      c[2 - m] = (int)(g - p * G.n[m]);
      c[G.rdim[m]] = (int)p;
    } else {
      c[2 - m] = (int)g;
    }
  }
}

// Outer index and column block of a tile.  The default order runs the column
// blocks fastest; `outer_fastest` runs the outer index fastest, so the CTAs
// that run at the same time share one column block across neighbouring
// outer indices (measured faster for the axis-0 pass of a 3-D array).
__device__ __forceinline__ void tile_place(const StridedArgs& a, int64_t tile, int64_t& o, int2& blk) {
  if (a.outer_fastest) {
    const int64_t cb = tile / a.nouter;
    o = tile - cb * a.nouter;
    blk = a.colblocks[cb];
  } else {
    o = tile / a.ncolblocks;
    blk = a.colblocks[tile - o * a.ncolblocks];
  }
}

}  // namespace tma
}  // namespace tfft
