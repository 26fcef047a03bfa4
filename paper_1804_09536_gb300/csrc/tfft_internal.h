// Internal interface between the host plan code and the CUDA kernels.
#pragma once

#include <cuda_runtime.h>

#include <string>

#include "tfft_common.cuh"
#include "tfft_device_cache.h"

namespace tfft {

// Bits of the plan's device status word (set by kernels, read by
// tfft_plan_device_status()).
constexpr int TFFT_DEVICE_ETIMEOUT = 1;  // a bounded wait on a copy expired
constexpr int TFFT_DEVICE_EALIGN = 2;    // a TMA tile buffer was not 128-byte aligned (copy skipped)
constexpr int TFFT_DEVICE_ETMEM = 4;     // MMAs still running after the clean-up wait: tensor memory not released

// Batched 1-D FFT of contiguous lines (the axis held whole and innermost,
// Eq. pencil0 / slab0): line l of the buffer is elements [l L, (l + 1) L).
struct ContigArgs {
  const float2* in;
  float2* out;
  int64_t nlines;
  AxisPlan ap;
  const float2* tw;  // ap.L roots exp(-2 pi i m / L)
  int lines_per_cta;
  int sign;
  float scale;
  const double* coef;   // optional device factor on the output (NULL: none)
  int* status;       // device status word
  uint32_t wait_limit;  // polls of a bounded copy wait (TMA passes)
};

// Bluestein's algorithm for a line length N without a 2/3/5 factorisation:
// the DFT as a circular convolution of length M (a power of two >= 2N - 1)
// with a chirp, done with two length-M FFTs.
struct BlueArgs {
  int N, M;
  AxisPlan apm;          // length-M FFT plan (shared-memory stages)
  const float2* twm;     // the M roots exp(-2 pi i m / M)
  const float2* chirp;   // N values exp(-i pi (n^2 mod 2N) / N)
  const float2* bhat;    // M values: the FFT of the wrapped chirp filter, times 1 / M
};

#ifdef __CUDACC__
// Output factor of a contiguous pass: the host's scale, times the device
// coefficient when there is one (formed in double, applied in float).
__device__ __forceinline__ float contig_scale(const ContigArgs& a) {
  return a.coef ? (float)((double)a.scale * __ldg(a.coef)) : a.scale;
}
#endif

// Real-to-complex (dir -1) or complex-to-real (dir +1) along the innermost
// axis: lines of N = 2 L reals <-> lines of L + 1 complex (Hermitian half),
// computed with one complex FFT of length L per line.
struct RealArgs {
  const float* rin;     // r2c input (nlines x 2L floats)
  float2* cout;         // r2c output (nlines x cpitch, the first L + 1 of each written)
  const float2* cin;    // c2r input
  float* rout;          // c2r output
  int64_t nlines;
  AxisPlan ap;          // plan of the length-L complex FFT
  const float2* tw;     // L roots exp(-2 pi i m / L)
  const float2* tw2;    // 2L roots exp(-2 pi i m / 2L)
  int64_t cpitch;       // complex elements from one line's start to the next (>= L + 1)
  int dir;
  float scale;
  int* status;
};

// 1-D FFT along axis `axis` < d - 1 with the redistribution fused into the
// loads (input layout lin) and the stores (output layout lout).  A tile is
// one value of the remaining axes ("outer" index) times a block of up to W
// consecutive columns of the innermost axis d - 1 that lies inside one rank
// of both layouts; the kernel gathers each column's full line from whatever
// virtual ranks hold it and scatters the result the same way.
struct StridedArgs {
  const float2* in;
  float2* out;
  DevLayout lin;
  DevLayout lout;
  int d;
  int axis;
  AxisPlan ap;
  const float2* tw;
  const int2* colblocks;  // (first column, width) along axis d - 1
  int64_t ncolblocks;
  int outer_fastest;      // TMA passes: tiles go (column block, outer) instead of (outer, column block)
  int64_t nouter;
  int oax0, oax1;         // the outer axes (or -1), outer index = g[oax0] * on1 + g[oax1]
  int64_t on1;
  int W;                  // block width (blockDim.x)
  int sign;
  float scale;
  int* status;            // device status word
  uint32_t wait_limit;    // polls of a bounded copy wait (TMA passes)
};

#ifdef __CUDACC__
// Outer index (split into the two outer axes' indices) and column block of
// strided tile `tile`.
struct StridedTilePos {
  int64_t go0, go1;
  int2 blk;
  __device__ __forceinline__ StridedTilePos(const StridedArgs& a, int64_t tile) {
    const int64_t o = tile / a.ncolblocks;
    blk = a.colblocks[tile - o * a.ncolblocks];
    go0 = (a.oax1 >= 0) ? o / a.on1 : o;
    go1 = (a.oax1 >= 0) ? o - go0 * a.on1 : 0;
  }
  // from an outer index and a column block already placed (any tile order)
  __device__ __forceinline__ StridedTilePos(const StridedArgs& a, int64_t o, int2 b) : blk(b) {
    go0 = (a.oax1 >= 0) ? o / a.on1 : o;
    go1 = (a.oax1 >= 0) ? o - go0 * a.on1 : 0;
  }
};

// The rows of one strided tile in one layout, with everything that does not
// depend on the row folded once per tile: the fixed axes' rank part and, in
// the C-order index of a rank's local array, the part before the FFT axis
// (head, scaled by that axis' local extent n_a, which depends on the row's
// part when the split is uneven) and after it (tail, with stride prod).
// Row i is then one locate() along the FFT axis: rank = base + c_a rs_a,
// index = (head n_a + l_a) prod + tail; the element offset is the rank's
// offset plus that index.
struct TileRows {
  int64_t base, head, prod, tail;
  int64_t N, M, rs;  // the FFT axis in this layout
  __device__ __forceinline__ TileRows(const StridedArgs& a, const DevLayout& lay, const StridedTilePos& tp) {
    base = 0;
    head = 0;
    prod = 1;
    tail = 0;
    N = lay.N[a.axis];
    M = lay.Mx[a.axis];
    rs = lay.rs[a.axis];
#pragma unroll
    for (int m = 0; m < MAXD; ++m) {
      if (m >= lay.d || m == a.axis) continue;
      const int64_t g = (m == a.d - 1) ? (int64_t)tp.blk.x : (m == a.oax0) ? tp.go0 : (m == a.oax1) ? tp.go1 : 0;
      int64_t local = g, n = lay.N[m];
      if (lay.Mx[m] > 1) {
        int64_t c;
        locate(lay.N[m], lay.Mx[m], g, c, local, n);
        base += c * lay.rs[m];
      }
      if (m == lay.d - 1 && lay.pitch > 0) n = lay.pitch;  // the innermost axis' storage extent
      if (m < a.axis) {
        head = head * n + local;
      } else {
        tail = tail * n + local;
        prod *= n;
      }
    }
  }
  __device__ __forceinline__ int64_t row(const DevLayout& lay, int i) const {
    int64_t c = 0, l = i, n = N;
    if (M > 1) locate(N, M, i, c, l, n);
    return lay.offset[base + c * rs] + (head * n + l) * prod + tail;
  }
};

#endif


// Tile geometry of one stage layout seen as the 5-D array
// [rank dim 4][rank dim 3][n0][n1][n2] (d = 3, equal blocks on every rank):
// for each axis m, whether it is cut, its local extent and the 5-D dimension
// of the rank coordinate that cuts it; a tile's rows along the FFT axis are
// loaded / stored in `nops` boxes of `rows_per_op` rows.
struct TmaGeo {
  int cut[3];
  int n[3];
  int rdim[3];
  int nops;
  int rows_per_op;
  // split view (uncut FFT axis longer than a 256-row box): the 5-D array is
  // [rank][outer axis][axis / split][split][n2] with the rank as one linear
  // index, so that a whole tile is one copy; rmul[m] = rank stride of cut
  // axis m; split = 0 for the plain view
  int split;
  int rmul[3];
  // first column of the view: a tile's column c is at c - c0 of the tensor
  // map (a view over a window of the innermost axis; 0 for a whole stage)
  int c0;
};

// Rank groups of an uneven stage layout seen by the TMA passes along its
// leading, uncut axis (in place): the ranks that hold blocks of one shape,
// whose offsets are affine in their grid coordinates, described by one
// tensor map each (see the TMA pass).  Tiles are numbered group after group:
// group g has first[g + 1] - first[g] = (its ranks) x nblk[g] tiles, a rank
// r = r1 + ext1[g] r0 of the group holding nblk[g] blocks of `width` merged
// inner columns.
constexpr int kMaxRankGroups = 4;
struct RankGroupGeo {
  int ngroups;
  int width;
  int64_t first[kMaxRankGroups + 1];
  int nblk[kMaxRankGroups];
  int ext1[kMaxRankGroups];
};

// Copy of rectangular boxes: each box has up to MAXD extents, a source and a
// destination base offset and per-axis strides (the innermost stride is 1 on
// both sides).  This is the all-to-all of subarray types of Alg. 3 on the
// virtual grid, and the pack / contiguous exchange / unpack of the
// traditional method.
struct BoxDesc {
  int64_t src;
  int64_t dst;
  int64_t ext[MAXD];
  int64_t ss[MAXD];
  int64_t ds[MAXD];
};

// What the copy kernel runs: a box cut into 2-D tasks of nrows rows of
// rowlen contiguous elements, rows ss / ds elements apart, from src / dst
// (element offsets).  The planner merges box dimensions that are contiguous
// on both sides first, so rows are as long as the layouts allow.
struct CopyTask {
  int64_t src, dst;
  int64_t ss, ds;
  int32_t nrows, rowlen;
};

struct BoxArgs {
  const float2* in;
  float2* out;
  const CopyTask* tasks;
  int64_t ntasks;
  int vec2;  // every offset, stride and row length is even: 16-byte copies
};

cudaError_t launch_contig(const ContigArgs& a, cudaStream_t s);
cudaError_t launch_strided(const StridedArgs& a, cudaStream_t s);
cudaError_t launch_boxcopy(const BoxArgs& a, cudaStream_t s);
cudaError_t launch_contig_blue(const ContigArgs& a, const BlueArgs& b, cudaStream_t s);
cudaError_t launch_strided_blue(const StridedArgs& a, const BlueArgs& b, cudaStream_t s);
// Bluestein passes with a compile-time convolution length (tfft_blue.cu):
// whether M has them, and their lines per CTA and strided tile width.
bool blue_spec_plan(int M, int& lines_per_cta, int& tile_width);
cudaError_t launch_contig_blue_spec(const ContigArgs& a, const BlueArgs& b, cudaStream_t s);
cudaError_t launch_strided_blue_spec(const StridedArgs& a, const BlueArgs& b, cudaStream_t s);
cudaError_t launch_twiddles(float2* tw, int L, cudaStream_t s);

// Batched persistent executor (tfft_batch.cu).  One segment = the tiles of
// one pass of one transform; items are numbered consecutively over the
// segments, pass-major.
struct BatchSeg {
  int kind;         // 0 contiguous, 1 strided
  int variant;      // executor tile variant
  int prev;         // segment that must be complete first (-1: none)
  int transform;
  int64_t first;    // first item of the segment
  int64_t ntiles;
  int64_t per_item; // tiles per work item
  int64_t nitems;   // items of the segment = ceil(ntiles / per_item)
  ContigArgs ca;
  StridedArgs sa;
  // strided tiles staged by TMA (variant of the TMA list): the tile geometry
  // of the input and output layouts and their tensor maps (CUtensorMap, in
  // the batch state, 64-byte aligned)
  int tma;
  TmaGeo gin, gout;
  const void* tin;
  const void* tout;
};

struct BatchArgs {
  const BatchSeg* segs;
  int nsegs;
  int64_t nitems;
  unsigned long long* head;  // next item (zeroed before each launch)
  int* done;                 // completed items per segment (zeroed before each launch)
  int* abort;                // raised when a wait expires (zeroed before each launch)
  int* status;               // device status word
  long long spin_limit;      // clock cycles a wait may last
};

bool batch_variant(int id, int& kind, int& L, int& E, int& BW, AxisPlan& ap);
bool batch_variant_tma(int id);  // a TMA-staged strided variant
int batch_num_variants();
int batch_grid();
cudaError_t launch_batch(const BatchArgs& b, int grid, cudaStream_t s);

// Tensor-core contiguous pass (tfft_tc.cu): length 512 = 32 x 16 with the
// radix-16 stage as split hi/lo 16-bit MMAs; precision 1 = BF16 x3, 2 = FP16 x3.
bool tc_supported(int L);
cudaError_t launch_contig_tc(const ContigArgs& a, int precision, cudaStream_t s);

// Tensor-core strided TMA passes (tfft_tc_strided.cu): lengths 512 (E = 32)
// and 256 (E = 16), the last radix-16 stage on tcgen05; tc_strided_variant
// gives the first-stage radix and tile width of the compiled variant of
// length L with width want_W if there is one, else the default.
bool tc_strided_variant(int L, int want_W, int& E, int& W);
cudaError_t launch_strided_tma_tc(const StridedArgs& a, int E, int precision, const TmaGeo& gin, const TmaGeo& gout,
                                  const void* tmap_in, const void* tmap_out, cudaStream_t s);

// Spectral-weight loss pieces (tfft_pointwise.cu).  The reduction uses
// `nparts` doubles of plan-state scratch.
constexpr int kReductionParts = 1024;
cudaError_t launch_weighted_energy(const float2* y, const float* w, int64_t n, double* parts, int nparts,
                                   double* out, float2* u, cudaStream_t s);
cudaError_t launch_weight_scale(const float2* y, const float* w, const double* coef, double scale, int64_t n,
                                float2* z, cudaStream_t s);

// Message returned by tfft_last_error() on the calling thread.
void set_last_error(const std::string& msg);

// The current device id (-1 if the runtime cannot tell) and its SM count
// (cached per device).
int current_device();
int device_sm_count();

// The kernel's maximum dynamic shared memory set once per device (the
// attribute is per device); `cache` is the caller's static for that kernel.
template <class K>
cudaError_t smem_attr_once(PerDevice<cudaError_t>& cache, K kernel, int bytes) {
  return cache.get(current_device(), [&] {
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  });
}

// Limits of the kernels, used by the planner.
bool kernel_supports_E(int E);

// Compile-time specialised passes (tfft_spec.cu): the plan of length L if one
// exists (and the buffers fit 32-bit offsets), and their launchers.
bool spec_plan(int L, bool strided, int64_t nelems, AxisPlan& ap, int& width);
cudaError_t launch_contig_spec(const ContigArgs& a, cudaStream_t s);
cudaError_t launch_strided_spec(const StridedArgs& a, cudaStream_t s);
cudaError_t launch_real_spec(const RealArgs& a, cudaStream_t s);

// TMA-staged passes (tfft_tma.cu).  tmap_* point to host CUtensorMap objects.
// tma_strided_variant: elements per thread and tile width of the strided TMA
// variant of length L with width want_W if compiled, else the default one.
bool tma_strided_variant(int L, int want_W, int want_E, int& E, int& W);
cudaError_t launch_strided_tma(const StridedArgs& a, int E, const TmaGeo& gin, const TmaGeo& gout,
                               const void* tmap_in, const void* tmap_out, cudaStream_t s);
// The same passes over the rank groups of an uneven layout (in place along
// the leading axis): tmaps_in / tmaps_out hold g.ngroups host CUtensorMaps each.
cudaError_t launch_strided_tma_groups(const StridedArgs& a, int E, const RankGroupGeo& g, const void* const* tmaps_in,
                                      const void* const* tmaps_out, cudaStream_t s);

}  // namespace tfft
