// Compile-time specialised FFT passes (contiguous and strided) for the
// lengths of tfft_spec_table.h.  Same Stockham schedule as the
// runtime-dispatched kernels (tfft_kernels.cu), but with the length, the
// radix sequence, the threads per line and the tile width fixed at compile
// time: every index, span and twiddle stride folds to a constant, the row
// tables hold 32-bit offsets, and the register budget is known to ptxas.
#include <type_traits>

#include "tfft_internal.h"
#include "tfft_spec_table.h"
#include "tfft_tiles.cuh"

namespace tfft {

namespace {

using namespace tiles;

// Registers sized for 1024 resident threads per SM (four 256-thread CTAs for
// the lengths with up to 16 values per thread; the 20- and 32-value plans
// keep two): more lines in flight per SM.  Against a 512-thread target:
// 256^3 pass 49.4 -> 46.7 us, 240^3 48.8 -> 42.2 us, 128^4 0.667 -> 0.603 ms.
template <int L, int E, int B, int... Rs>
__global__ void __launch_bounds__((L / E) * B, min_blocks(E, (L / E) * B, 1024))
    k_contig_spec(const ContigArgs a) {
  extern __shared__ float2 smem[];
  for (int64_t tile = blockIdx.x; tile * B < a.nlines; tile += gridDim.x)
    contig_tile<L, E, B, false, Rs...>(a, tile, smem, opaque_tid_x(), threadIdx.y);
}

// Whether the plain strided kernel keeps the rows' part/index table for the
// CTA's lifetime (2L words): not at 4096, where it would halve the CTAs per SM.
__host__ __device__ constexpr bool strided_cache_rows(int L) { return L <= 2048; }

// Resident threads per SM the plain strided kernel's registers are sized
// for: 1024 (min_blocks halves it for the plans of 20 or more values per
// thread), and 1536 for the 20- and 24-value plans that fit 80 registers
// without spilling (three 256-thread CTAs instead of two): 320^3 pass 0.166
// -> 0.146 ms, 640 x 640 x 64 0.141 -> 0.136 ms.  The contiguous kernel gained
// nothing from the same change (320^3 0.166 -> 0.165 ms, 160^3 slower).
__host__ __device__ constexpr int strided_target(int L, int E) {
  return E >= 20 && E < 32 && L != 384 && L != 480 ? 1536 : 1024;
}

template <int L, int E, int W, int... Rs>
__global__ void __launch_bounds__(W * (L / E), min_blocks(E, W * (L / E), strided_target(L, E)))
    k_strided_spec(const StridedArgs a) {
  extern __shared__ float2 smem[];
  const int64_t ntiles = a.nouter * a.ncolblocks;
  const int tid = threadIdx.y * W + threadIdx.x;
  uint32_t* rp = nullptr;
  if constexpr (strided_cache_rows(L)) {
    rp = strided_rowparts<L, W>(smem);
    strided_rowparts_init<L>(a, rp, tid, W * (L / E));  // published by the first tile's barriers
  }
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x)
    strided_tile<L, E, W, false, Rs...>(a, tile, smem, threadIdx.x, opaque_tid_y(), tid, rp);
}

// the kernel's shared-memory limit raised to 227 KB, once per device
#define TFFT_ALLOW_SMEM(kernel)                          \
  static PerDevice<cudaError_t> attr_cache;              \
  const cudaError_t attr = smem_attr_once(attr_cache, kernel, 227 * 1024)

constexpr int64_t kMaxGrid = 1 << 20;

template <int L, int E, int B, int... Rs>
cudaError_t run_contig(const ContigArgs& a, cudaStream_t s) {
  TFFT_ALLOW_SMEM((k_contig_spec<L, E, B, Rs...>));
  if (attr != cudaSuccess) return attr;
  const size_t smem = (size_t)B * line_pitch<L, Rs...>() * sizeof(float2);
  int64_t grid = (a.nlines + B - 1) / B;
  if (grid > kMaxGrid) grid = kMaxGrid;
  if (grid < 1) return cudaSuccess;
  k_contig_spec<L, E, B, Rs...><<<(unsigned)grid, dim3(L / E, B), smem, s>>>(a);
  return cudaGetLastError();
}

template <int L, int E, int W, int... Rs>
cudaError_t run_strided(const StridedArgs& a, cudaStream_t s) {
  TFFT_ALLOW_SMEM((k_strided_spec<L, E, W, Rs...>));
  if (attr != cudaSuccess) return attr;
  if (a.W != W) return cudaErrorInvalidValue;
  constexpr size_t smem = strided_tile_smem<L, W>(strided_cache_rows(L));
  // persistent: as many CTAs as fit at once, each taking every gridDim-th
  // tile, so that the row part table is computed once per CTA
  static PerDevice<int64_t> slots_cache;
  const int64_t slots = slots_cache.get(current_device(), [] {
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_strided_spec<L, E, W, Rs...>, W * (L / E), smem);
    return (int64_t)device_sm_count() * (per_sm > 0 ? per_sm : 1);
  });
  int64_t grid = a.nouter * a.ncolblocks;
  if (grid > slots) grid = slots;
  if (grid < 1) return cudaSuccess;
  k_strided_spec<L, E, W, Rs...><<<(unsigned)grid, dim3(W, L / E), smem, s>>>(a);
  return cudaGetLastError();
}

struct SpecRow {
  int L, EC, B, ES, W, nst, radix[6];
};

const SpecRow kSpecs[] = {
#define X(L, EC, B, ES, W, ...) \
  {L, EC, B, ES, W, (int)(sizeof((int[]){__VA_ARGS__}) / sizeof(int)), {__VA_ARGS__}},
    TFFT_SPECS(X)
#undef X
};

// Whether TFFT_SPECS_STRIDED replaces the strided kernel of TFFT_SPECS for L
// (the replaced one is then not instantiated).
constexpr bool strided_overridden(int L) {
#define X(LL, ...) \
  if (L == LL) return true;
  TFFT_SPECS_STRIDED(X)
#undef X
  return false;
}

struct StridedSpecRow {
  int L, ES, W, nst, radix[6];
};

const StridedSpecRow kStridedSpecs[] = {
#define X(L, ES, W, ...) {L, ES, W, (int)(sizeof((int[]){__VA_ARGS__}) / sizeof(int)), {__VA_ARGS__}},
    TFFT_SPECS_STRIDED(X)
#undef X
};

}  // namespace

bool spec_plan(int L, bool strided, int64_t nelems, AxisPlan& ap, int& width) {
  if (nelems >= (int64_t(1) << 31)) return false;  // 32-bit row offsets
  if (strided)
    for (const StridedSpecRow& r : kStridedSpecs) {
      if (r.L != L) continue;
      ap.L = L;
      ap.E = r.ES;
      ap.T = L / r.ES;
      ap.nst = r.nst;
      ap.code = 0;
      for (int s = 0; s < r.nst; ++s) {
        ap.radix[s] = r.radix[s];
        ap.code |= (uint64_t)r.radix[s] << (5 * s);
      }
      ap.spec = 1;
      width = r.W;
      return true;
    }
  for (const SpecRow& r : kSpecs) {
    if (r.L != L) continue;
    const int E = strided ? r.ES : r.EC;
    ap.L = L;
    ap.E = E;
    ap.T = L / E;
    ap.nst = r.nst;
    ap.code = 0;
    for (int s = 0; s < r.nst; ++s) {
      ap.radix[s] = r.radix[s];
      ap.code |= (uint64_t)r.radix[s] << (5 * s);
    }
    ap.spec = 1;
    width = strided ? r.W : r.B;
    return true;
  }
  return false;
}

cudaError_t launch_contig_spec(const ContigArgs& a, cudaStream_t s) {
  switch (a.ap.L) {
#define X(L, EC, B, ES, W, ...) \
  case L:                       \
    return run_contig<L, EC, B, __VA_ARGS__>(a, s);
    TFFT_SPECS(X)
#undef X
    default:
      return cudaErrorInvalidValue;
  }
}

cudaError_t launch_strided_spec(const StridedArgs& a, cudaStream_t s) {
#define X(LL, ES, WW, ...) \
  if (a.ap.L == LL) return a.ap.E == ES ? run_strided<LL, ES, WW, __VA_ARGS__>(a, s) : cudaErrorInvalidValue;
  TFFT_SPECS_STRIDED(X)
#undef X
  switch (a.ap.L) {
#define X(L, EC, B, ES, W, ...)                                          \
  case L:                                                                \
    if constexpr (!strided_overridden(L)) return run_strided<L, ES, W, __VA_ARGS__>(a, s); \
    return cudaErrorInvalidValue;
    TFFT_SPECS(X)
#undef X
    default:
      return cudaErrorInvalidValue;
  }
}

}  // namespace tfft
