// Device-side building blocks of the compile-time specialised passes: the
// Stockham stage, register-held stage twiddles, shared-memory helpers and the
// per-tile bodies of the contiguous and strided passes.  Included by the pass
// kernels (tfft_spec.cu, tfft_tma.cu, tfft_tc.cu) and by the batched executor
// (tfft_batch.cu).
#pragma once

#include <type_traits>

#include "tfft_internal.h"

namespace tfft {
namespace tiles {

template <int S, int... Rs>
__host__ __device__ constexpr int radix_at() {
  constexpr int r[] = {Rs...};
  return r[S];
}

template <int S, int... Rs>
__host__ __device__ constexpr int span_at() {
  constexpr int r[] = {Rs...};
  int p = 1;
  for (int i = 0; i < S; ++i) p *= r[i];
  return p;
}

template <int I, int N, class F>
__device__ __forceinline__ void static_for(F&& f) {
  if constexpr (I < N) {
    f(std::integral_constant<int, I>{});
    static_for<I + 1, N>(f);
  }
}

// A line of length L has T = L / E threads.  A stage of radix R has L / R
// butterflies, nbf = ceil((L / R) / T) per thread: butterfly j = jt + q T,
// q < nbf, exists when j < L / R.  When every radix divides E this is E / R
// butterflies each and no guard (the usual plans); lengths with 2, 3 and 5
// all present (60, 120, 240, 480) have no such E, so their threads carry one
// butterfly fewer in some stages and hold up to emax() values.
template <int L, int E, int R>
__host__ __device__ constexpr int nbf() {
  return (L / R + L / E - 1) / (L / E);
}

template <int L, int E, int R>
__host__ __device__ constexpr bool nbf_exact() {
  return (L / R) % (L / E) == 0;
}

template <int L, int E, int... Rs>
__host__ __device__ constexpr int emax() {
  constexpr int r[] = {Rs...};
  int m = 0;
  for (int i = 0; i < (int)sizeof...(Rs); ++i) {
    const int v = ((L / r[i] + L / E - 1) / (L / E)) * r[i];
    m = v > m ? v : m;
  }
  return m;
}

// Whether butterfly q of thread jt exists in a stage of radix R.
template <int L, int E, int R>
__device__ __forceinline__ bool bf_exists(int jt, int q) {
  if constexpr (nbf_exact<L, E, R>()) return true;
  else return jt + q * (L / E) < L / R;
}

// Twiddle (stage span Ns > 1) and size-R butterflies of a thread's work items.
template <int L, int E, int R, int Ns, int EM>
__device__ __forceinline__ void spec_stage(float2 (&v)[EM], int jt, const float2* __restrict__ tw) {
  constexpr int T = L / E;
#pragma unroll
  for (int q = 0; q < nbf<L, E, R>(); ++q) {
    if (!bf_exists<L, E, R>(jt, q)) continue;
    if constexpr (Ns > 1) {
      const int j = jt + q * T;
      const int step = (j % Ns) * (L / (Ns * R));
#pragma unroll
      for (int r = 1; r < R; ++r) v[q * R + r] = cmul(v[q * R + r], __ldg(&tw[r * step]));
    }
    Dft<R>::run(&v[q * R]);
  }
}

// Twiddles of every stage after the first for one thread, held in registers.
// They depend only on the thread's position in the line, so a persistent
// kernel loads them once instead of once per tile.  Stage s (span Ns, radix
// R) multiplies item r of butterfly q by w_L^{r (j % Ns) L / (Ns R)} with
// j = jt + q T; the values are stored from offset(s) on, (R - 1) per q.
template <int L, int E, int... Rs>
struct StageTwiddles {
  static_assert(((E % Rs == 0) && ...), "every radix divides E (uniform plans)");
  static constexpr int NST = sizeof...(Rs);
  __host__ __device__ static constexpr int offset(int s) {
    constexpr int r[] = {Rs...};
    int c = 0;
    for (int i = 1; i < s; ++i) c += (E / r[i]) * (r[i] - 1);
    return c;
  }
  static constexpr int COUNT = offset(NST);
  float2 w[COUNT > 0 ? COUNT : 1];

  __device__ __forceinline__ void load(int jt, const float2* __restrict__ tw) {
    constexpr int T = L / E;
    static_for<1, NST>([&](auto S) {
      constexpr int s = decltype(S)::value;
      constexpr int R = radix_at<s, Rs...>();
      constexpr int Ns = span_at<s, Rs...>();
      constexpr int off = offset(s);
#pragma unroll
      for (int q = 0; q < E / R; ++q) {
        const int step = ((jt + q * T) % Ns) * (L / (Ns * R));
#pragma unroll
        for (int r = 1; r < R; ++r) w[off + q * (R - 1) + r - 1] = __ldg(&tw[r * step]);
      }
    });
  }

  // Stage s on a thread's items with the held twiddles.
  template <int s>
  __device__ __forceinline__ void stage(float2 (&v)[E]) const {
    constexpr int R = radix_at<s, Rs...>();
    constexpr int off = offset(s);
#pragma unroll
    for (int q = 0; q < E / R; ++q) {
      if constexpr (s > 0) {
#pragma unroll
        for (int r = 1; r < R; ++r) v[q * R + r] = cmul(v[q * R + r], w[off + q * (R - 1) + r - 1]);
      }
      Dft<R>::run(&v[q * R]);
    }
  }
};

// threadIdx re-read inside a loop body, opaque to the compiler: it keeps the
// per-thread shared-memory addresses from being hoisted out of the tile loop
// (and held in registers across it).
__device__ __forceinline__ int opaque_tid_x() {
  int v;
  asm volatile("mov.u32 %0, %%tid.x;" : "=r"(v));
  return v;
}
__device__ __forceinline__ int opaque_tid_y() {
  int v;
  asm volatile("mov.u32 %0, %%tid.y;" : "=r"(v));
  return v;
}

// CTAs per SM the register budget is sized for: `target` resident threads
// (half that for the 20-element plans, whose butterflies need more registers).
__host__ __device__ constexpr int min_blocks(int E, int threads, int target) {
  const int t = (E >= 20 ? target / 2 : target) / threads;
  return t > 1 ? t : (E >= 20 && threads <= 256 ? 2 : 1);
}

// Synchronises the threads of one line: a warp (or part of one) when a line
// has at most 32 threads, the whole CTA otherwise.
template <int T>
__device__ __forceinline__ void line_sync() {
  if constexpr (T <= 32) {
    __syncwarp();
  } else {
    __syncthreads();
  }
}

// Padded position inside a contiguous line: one spare slot every P elements.
// The first stage writes its outputs at stride R0 (its radix); with P = R0
// that stride becomes R0 + 1, odd, so 16 lanes of 8-byte stores hit 16
// distinct bank pairs.  P = 8 for a first radix below 8 or not a power of two.
template <int... Rs>
__host__ __device__ constexpr int pad_every() {
  constexpr int r[] = {Rs...};
  return (r[0] & (r[0] - 1)) == 0 && r[0] >= 8 ? r[0] : 8;
}

template <int P>
__device__ __forceinline__ int padp(int pos) {
  return pos + pos / P;
}

// Padded line pitch of the contiguous-line kernels (elements).
template <int L, int... Rs>
__host__ __device__ constexpr int line_pitch() {
  return L + L / pad_every<Rs...>();
}

// ------------------------------------------------------------ contiguous lines

// Global load, optionally L2-only (.cg): used where the data was written by
// other SMs earlier in the same launch (the batched executor).
template <bool CG>
__device__ __forceinline__ float2 ld(const float2* p) {
  if constexpr (CG) {
    return __ldcg(p);
  } else {
    return *p;
  }
}

// One group of B contiguous lines (group `tile`): thread jt of line ly.
template <int L, int E, int B, bool CG, int... Rs>
__device__ __forceinline__ void contig_tile(const ContigArgs& a, int64_t tile, float2* smem, int jt, int ly) {
  constexpr int T = L / E, NST = sizeof...(Rs);
  constexpr int LP = line_pitch<L, Rs...>();
  constexpr int P = pad_every<Rs...>();
  float2* sl = smem + ly * LP;
  const bool inv = a.sign > 0;
  const int64_t line = tile * B + ly;
  const bool act = line < a.nlines;
  const float2* src = a.in + line * L;
  float2* dst = a.out + line * L;
  float2 v[emax<L, E, Rs...>()];
  static_for<0, NST>([&](auto S) {
    constexpr int s = decltype(S)::value;
    constexpr int R = radix_at<s, Rs...>();
    constexpr int Ns = span_at<s, Rs...>();
    if constexpr (s == 0) {
#pragma unroll
      for (int q = 0; q < nbf<L, E, R>(); ++q)
#pragma unroll
        for (int r = 0; r < R; ++r) {
          float2 x = (act && bf_exists<L, E, R>(jt, q)) ? ld<CG>(src + jt + q * T + r * (L / R))
                                                        : make_float2(0.f, 0.f);
          if (inv) x.y = -x.y;
          v[q * R + r] = x;
        }
    } else {
      constexpr int Rp = radix_at<s - 1, Rs...>();
      constexpr int Nsp = Ns / Rp;
      line_sync<T>();
#pragma unroll
      for (int q = 0; q < nbf<L, E, Rp>(); ++q)
        if (bf_exists<L, E, Rp>(jt, q))
#pragma unroll
          for (int r = 0; r < Rp; ++r) sl[padp<P>(stockham_out_index(jt + q * T, Nsp, Rp, r))] = v[q * Rp + r];
      line_sync<T>();
#pragma unroll
      for (int q = 0; q < nbf<L, E, R>(); ++q)
        if (bf_exists<L, E, R>(jt, q))
#pragma unroll
          for (int r = 0; r < R; ++r) v[q * R + r] = sl[padp<P>(jt + q * T + r * (L / R))];
    }
    spec_stage<L, E, R, Ns>(v, jt, a.tw);
  });
  constexpr int RL = radix_at<NST - 1, Rs...>();
  const float oscale = contig_scale(a);
#pragma unroll
  for (int q = 0; q < nbf<L, E, RL>(); ++q)
#pragma unroll
    for (int r = 0; r < RL; ++r) {
      float2 x = cscale(v[q * RL + r], oscale);
      if (inv) x.y = -x.y;
      if (act && bf_exists<L, E, RL>(jt, q)) dst[jt + q * T + r * (L / RL)] = x;
    }
  line_sync<T>();  // the line's shared slots are free for the next group
}


// ------------------------------------------------------------ strided lines

// Per-tile scalars of a strided tile, computed by one thread per layout and
// shared through shared memory: the TileRows fold of the input (0) and output
// (1) layouts, the split of the FFT axis in each (part length q, and q + 1
// for the first r parts, Eq. decompose) and the column block.
struct TileShared {
  int64_t base[2], head[2], prod[2], tail[2];
  int q[2], r[2];
  int2 blk;
};

// Bytes of shared memory a strided tile of L x W takes: the tile, the two
// row tables, the shared scalars and, when `cached`, the per-CTA part/index
// table of the rows (two layouts).
template <int L, int W>
__host__ __device__ constexpr size_t strided_tile_smem(bool cached) {
  return (size_t)L * W * sizeof(float2) + 2 * (size_t)L * sizeof(int) + sizeof(TileShared) +
         (cached ? 2 * (size_t)L * sizeof(uint32_t) : 0);
}

template <int L, int W>
__device__ __forceinline__ uint32_t* strided_rowparts(float2* smem) {
  return reinterpret_cast<uint32_t*>(reinterpret_cast<char*>(smem) + strided_tile_smem<L, W>(false));
}

// Part c and index l (packed c << 16 | l) of every row i < L along the FFT
// axis, input layout in [0, L), output layout in [L, 2L): they depend on the
// axis split only, so a persistent CTA computes them once.
template <int L>
__device__ __forceinline__ void strided_rowparts_init(const StridedArgs& a, uint32_t* rp, int tid, int nthreads) {
  for (int i = tid; i < 2 * L; i += nthreads) {
    const int row = i < L ? i : i - L;
    const int64_t N = i < L ? a.lin.N[a.axis] : a.lout.N[a.axis];
    const int64_t M = i < L ? a.lin.Mx[a.axis] : a.lout.Mx[a.axis];
    int64_t c = 0, l = row, n = N;
    if (M > 1) locate(N, M, row, c, l, n);
    rp[i] = ((uint32_t)c << 16) | (uint32_t)l;
  }
}

// The fold of one layout for tile position tp, written to ts slot `k`.
__device__ __forceinline__ void tile_fold(const StridedArgs& a, const DevLayout& lay, const StridedTilePos& tp,
                                          TileShared* ts, int k) {
  const TileRows tr(a, lay, tp);
  ts->base[k] = tr.base;
  ts->head[k] = tr.head;
  ts->prod[k] = tr.prod;
  ts->tail[k] = tr.tail;
  const uint32_t N = (uint32_t)tr.N, M = (uint32_t)tr.M;
  ts->q[k] = (int)(N / M);
  ts->r[k] = (int)(N - (N / M) * M);
}

// Element offset of row i of a layout from the shared fold (slot k): the
// part's offset plus the C-order index inside it.
__device__ __forceinline__ int row_offset(const DevLayout& lay, int axis, const TileShared* ts, int k, int64_t c,
                                          int64_t l) {
  const int64_t n = ts->q[k] + (c < ts->r[k] ? 1 : 0);
  return (int)(lay.offset[ts->base[k] + c * lay.rs[axis]] + (ts->head[k] * n + l) * ts->prod[k] + ts->tail[k]);
}

// One strided tile (outer index and column block `tile`): thread jt of
// column cx; tid = thread index in the CTA (W x T threads).  `rp` is the
// per-CTA part/index table of strided_rowparts_init, or null (then each row
// locates its part itself).
template <int L, int E, int W, bool CG, int... Rs>
__device__ __forceinline__ void strided_tile(const StridedArgs& a, int64_t tile, float2* smem, int cx, int jt,
                                             int tid, const uint32_t* rp = nullptr) {
  constexpr int T = L / E, NST = sizeof...(Rs);
  static_assert(W * T > 32, "the two layouts' folds are computed by threads 0 and 32");
  int* rin = reinterpret_cast<int*>(smem + L * W);
  int* rout = rin + L;
  TileShared* ts = reinterpret_cast<TileShared*>(rout + L);
  const bool inv = a.sign > 0;
  __syncthreads();  // the previous tile is done with the row tables and the scalars
  if (tid == 0) {
    const StridedTilePos tp(a, tile);
    tile_fold(a, a.lin, tp, ts, 0);
    ts->blk = tp.blk;
  } else if (tid == 32) {
    const StridedTilePos tp(a, tile);
    tile_fold(a, a.lout, tp, ts, 1);
  }
  __syncthreads();
  for (int i = tid; i < 2 * L; i += W * T) {
    const bool out = i >= L;
    const int row = out ? i - L : i;
    int64_t c = 0, l = row;
    if (rp != nullptr) {
      c = rp[i] >> 16;
      l = rp[i] & 0xFFFF;
    } else {
      int64_t n;
      const int64_t N = out ? a.lout.N[a.axis] : a.lin.N[a.axis];
      const int64_t M = out ? a.lout.Mx[a.axis] : a.lin.Mx[a.axis];
      if (M > 1) locate(N, M, row, c, l, n);
    }
    if (out)
      rout[row] = row_offset(a.lout, a.axis, ts, 1, c, l);
    else
      rin[row] = row_offset(a.lin, a.axis, ts, 0, c, l);
  }
  __syncthreads();
  const int2 blk = ts->blk;
  const bool act = cx < blk.y;
  float2 v[emax<L, E, Rs...>()];
  static_for<0, NST>([&](auto S) {
    constexpr int s = decltype(S)::value;
    constexpr int R = radix_at<s, Rs...>();
    constexpr int Ns = span_at<s, Rs...>();
    if constexpr (s == 0) {
#pragma unroll
      for (int q = 0; q < nbf<L, E, R>(); ++q)
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const int pos = jt + q * T + r * (L / R);
          float2 x = (act && bf_exists<L, E, R>(jt, q)) ? ld<CG>(a.in + rin[pos] + cx) : make_float2(0.f, 0.f);
          if (inv) x.y = -x.y;
          v[q * R + r] = x;
        }
    } else {
      constexpr int Rp = radix_at<s - 1, Rs...>();
      constexpr int Nsp = Ns / Rp;
      __syncthreads();
#pragma unroll
      for (int q = 0; q < nbf<L, E, Rp>(); ++q)
        if (bf_exists<L, E, Rp>(jt, q))
#pragma unroll
          for (int r = 0; r < Rp; ++r)
            smem[stockham_out_index(jt + q * T, Nsp, Rp, r) * W + cx] = v[q * Rp + r];
      __syncthreads();
#pragma unroll
      for (int q = 0; q < nbf<L, E, R>(); ++q)
        if (bf_exists<L, E, R>(jt, q))
#pragma unroll
          for (int r = 0; r < R; ++r) v[q * R + r] = smem[(jt + q * T + r * (L / R)) * W + cx];
    }
    spec_stage<L, E, R, Ns>(v, jt, a.tw);
  });
  constexpr int RL = radix_at<NST - 1, Rs...>();
#pragma unroll
  for (int q = 0; q < nbf<L, E, RL>(); ++q)
#pragma unroll
    for (int r = 0; r < RL; ++r) {
      float2 x = cscale(v[q * RL + r], a.scale);
      if (inv) x.y = -x.y;
      if (act && bf_exists<L, E, RL>(jt, q)) a.out[rout[jt + q * T + r * (L / RL)] + cx] = x;
    }
}



// ------------------------------------------------------------ stages only

// The Stockham stages of a length-L FFT on the values a thread holds for
// column cx of an L x W tile in shared memory (the strided passes' layout:
// position i of the column at smem[i W + cx]): on entry v holds the first
// stage's inputs x[jt + q T + r L / R0], on exit the outputs at positions
// jt + q T + r L / RL (natural order, self-sorting); between stages the
// column goes through smem.  Starts and ends without a barrier: the caller
// orders smem use around it.
template <int L, int E, int W, int... Rs>
__device__ __forceinline__ void strided_stages(float2 (&v)[emax<L, E, Rs...>()], float2* smem, int cx, int jt,
                                               const float2* __restrict__ tw) {
  constexpr int T = L / E, NST = sizeof...(Rs);
  static_for<0, NST>([&](auto S) {
    constexpr int s = decltype(S)::value;
    constexpr int R = radix_at<s, Rs...>();
    constexpr int Ns = span_at<s, Rs...>();
    if constexpr (s > 0) {
      constexpr int Rp = radix_at<s - 1, Rs...>();
      constexpr int Nsp = Ns / Rp;
      __syncthreads();
#pragma unroll
      for (int q = 0; q < nbf<L, E, Rp>(); ++q)
        if (bf_exists<L, E, Rp>(jt, q))
#pragma unroll
          for (int r = 0; r < Rp; ++r) smem[stockham_out_index(jt + q * T, Nsp, Rp, r) * W + cx] = v[q * Rp + r];
      __syncthreads();
#pragma unroll
      for (int q = 0; q < nbf<L, E, R>(); ++q)
        if (bf_exists<L, E, R>(jt, q))
#pragma unroll
          for (int r = 0; r < R; ++r) v[q * R + r] = smem[(jt + q * T + r * (L / R)) * W + cx];
    }
    spec_stage<L, E, R, Ns>(v, jt, tw);
  });
}

// The same for one contiguous line in its padded line slot sl (the
// contiguous passes' layout), synchronising the line's threads.
template <int L, int E, int... Rs>
__device__ __forceinline__ void line_stages(float2 (&v)[emax<L, E, Rs...>()], float2* sl, int jt,
                                            const float2* __restrict__ tw) {
  constexpr int T = L / E, NST = sizeof...(Rs);
  constexpr int P = pad_every<Rs...>();
  static_for<0, NST>([&](auto S) {
    constexpr int s = decltype(S)::value;
    constexpr int R = radix_at<s, Rs...>();
    constexpr int Ns = span_at<s, Rs...>();
    if constexpr (s > 0) {
      constexpr int Rp = radix_at<s - 1, Rs...>();
      constexpr int Nsp = Ns / Rp;
      line_sync<T>();
#pragma unroll
      for (int q = 0; q < nbf<L, E, Rp>(); ++q)
        if (bf_exists<L, E, Rp>(jt, q))
#pragma unroll
          for (int r = 0; r < Rp; ++r) sl[padp<P>(stockham_out_index(jt + q * T, Nsp, Rp, r))] = v[q * Rp + r];
      line_sync<T>();
#pragma unroll
      for (int q = 0; q < nbf<L, E, R>(); ++q)
        if (bf_exists<L, E, R>(jt, q))
#pragma unroll
          for (int r = 0; r < R; ++r) v[q * R + r] = sl[padp<P>(jt + q * T + r * (L / R))];
    }
    spec_stage<L, E, R, Ns>(v, jt, tw);
  });
}

}  // namespace tiles
}  // namespace tfft
