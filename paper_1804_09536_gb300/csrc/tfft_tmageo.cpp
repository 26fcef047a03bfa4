// Tile geometry of the TMA-staged strided passes: the 5-D view of an
// equal-block stage layout and the tensor map that describes it.
#include "tfft_plan.h"

namespace tfft {
namespace host {

// Rows of the inner dimension when an uncut axis of length L > 256 is viewed
// as two tensor dimensions (L = a x b, both at most 256, a as large as
// possible); 0 when there is no such split.
int split_rows(int L) {
  for (int a = 256; a >= 2; --a)
    if (L % a == 0 && L / a <= 256) return a;
  return 0;
}

// The 5-D view of a stage layout used by the TMA passes exists when d == 3,
// every cut axis splits evenly, and each rank's innermost extent is a
// multiple of the tile width (every tile starts on a 16-byte boundary).
bool tma_geo(tfft_plan p, int stage, int axis, int W, TmaGeo& G) {
  if (p->d != 3 || p->g < 1 || p->g > 2) return false;
  const LayoutH& S = p->st[stage];
  if (S.pitch > 0) return false;  // padded rows: window_side describes those
  const int L = (int)p->cshape[axis];
  G.c0 = 0;
  for (int m = 0; m < 3; ++m) {
    G.cut[m] = S.owner[m] >= 0 ? 1 : 0;
    const int64_t M = G.cut[m] ? p->grid[S.owner[m]] : 1;
    if (p->cshape[m] % M) return false;
    G.n[m] = (int)(p->cshape[m] / M);
    G.rdim[m] = G.cut[m] ? 3 + (p->g - 1 - S.owner[m]) : 0;
  }
  if (G.n[2] % W != 0 || (W & 1)) return false;
  G.split = 0;
  for (int m = 0; m < 3; ++m) G.rmul[m] = G.cut[m] ? (int)p->rstride[S.owner[m]] : 0;
  if (G.cut[axis]) {
    if (G.n[axis] > 256 || p->grid[S.owner[axis]] > 256) return false;
    G.nops = 1;
    G.rows_per_op = L;
  } else if (L > 256 && axis != 2 && split_rows(L) > 0) {
    // one copy per tile: measured, 2 / 4 / 8 copies of 256 / 128 / 64 rows
    // made the 512-row pass take 0.39 / 0.50 / 0.74 ms
    G.split = split_rows(L);
    G.nops = 1;
    G.rows_per_op = L;
  } else {
    G.rows_per_op = L < 256 ? L : 256;
    if (L % G.rows_per_op) return false;
    G.nops = L / G.rows_per_op;
  }
  return true;
}

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      f = nullptr;
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
  }();
  return fn;
}

// Tensor map of a whole stage buffer as [D4][D3][n0][n1][n2] complex64
// elements, with the box of one TMA op of a tile along `axis`.
bool encode_stage_map(tfft_plan p, const TmaGeo& G, int axis, int W, const void* base, CUtensorMap* map) {
  auto enc = tensor_map_encoder();
  if (!enc) return false;
  const int64_t local = (int64_t)G.n[0] * G.n[1] * G.n[2];
  const cuuint64_t D3 = p->g >= 1 ? (cuuint64_t)p->grid[p->g - 1] : 1;
  const cuuint64_t D4 = p->g == 2 ? (cuuint64_t)p->grid[0] : 1;
  cuuint64_t dims[5] = {(cuuint64_t)G.n[2], (cuuint64_t)G.n[1], (cuuint64_t)G.n[0], D3, D4};
  cuuint64_t strides[4] = {(cuuint64_t)G.n[2] * 8, (cuuint64_t)G.n[1] * G.n[2] * 8, (cuuint64_t)local * 8,
                           (cuuint64_t)local * 8 * D3};
  cuuint32_t box[5] = {(cuuint32_t)W, 1, 1, 1, 1};
  if (G.split) {  // [rank][outer][axis / a][a][n2] with a = G.split, see TmaGeo
    const int tax = 1 - axis;  // the other non-innermost axis (d == 3)
    const int64_t sa = axis == 0 ? (int64_t)G.n[1] * G.n[2] : G.n[2];
    const int64_t so = tax == 0 ? (int64_t)G.n[1] * G.n[2] : G.n[2];
    dims[1] = (cuuint64_t)G.split;
    dims[2] = (cuuint64_t)(G.n[axis] / G.split);
    dims[3] = (cuuint64_t)G.n[tax];
    dims[4] = (cuuint64_t)p->nranks;
    strides[0] = (cuuint64_t)sa * 8;
    strides[1] = (cuuint64_t)sa * G.split * 8;
    strides[2] = (cuuint64_t)so * 8;
    strides[3] = (cuuint64_t)local * 8;
    box[1] = (cuuint32_t)G.split;
    box[2] = (cuuint32_t)(G.n[axis] / G.split);
  } else if (G.cut[axis]) {
    box[2 - axis] = (cuuint32_t)G.n[axis];                             // local rows
    box[G.rdim[axis]] = (cuuint32_t)(p->cshape[axis] / G.n[axis]);     // every rank of the subgroup
  } else {
    box[2 - axis] = (cuuint32_t)G.rows_per_op;
  }
  cuuint32_t estr[5] = {1, 1, 1, 1, 1};
  // L2 fill granule = the tile's row (W complex): measured on 512^3 with
  // 128-byte rows, 128 B beat 256 B by 4 % on the pass whose rows lie 64 KB apart
  const CUtensorMapL2promotion promo =
      W * 8 >= 256 ? CU_TENSOR_MAP_L2_PROMOTION_L2_256B : CU_TENSOR_MAP_L2_PROMOTION_L2_128B;
  CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_UINT64, 5, const_cast<void*>(base), dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, promo, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// Tile width (and optionally elements per thread) requested for the strided
// TMA pass of length L by the environment, TFFT_TMA_W="512:8:16,256:32"
// (TFFT_TC_W for the tensor-core passes; used when tuning); 0 when not given.
int tuned_width(int L, int* E, const char* var) {
  if (E) *E = 0;
  const char* env = std::getenv(var);
  if (!env) return 0;
  std::string v(env);
  size_t pos = 0;
  while (pos < v.size()) {
    size_t comma = v.find(',', pos);
    std::string item = v.substr(pos, comma == std::string::npos ? std::string::npos : comma - pos);
    size_t colon = item.find(':');
    if (colon != std::string::npos && std::atoi(item.substr(0, colon).c_str()) == L) {
      size_t colon2 = item.find(':', colon + 1);
      if (E && colon2 != std::string::npos) *E = std::atoi(item.substr(colon2 + 1).c_str());
      return std::atoi(item.substr(colon + 1).c_str());
    }
    if (comma == std::string::npos) break;
    pos = comma + 1;
  }
  return 0;
}

// Rank groups of stage `stage` for an in-place TMA pass along axis 0 (held
// whole in that stage) when its ranks do not all hold equal blocks.  Each
// grid direction splits its axis into r parts of q + 1 and M - r parts of q
// (Eq. decompose); the ranks of one size class per direction form a group.
// A group qualifies when its ranks' blocks have one shape, its offsets are
// affine in the rank coordinates, and every offset and the merged inner
// extent are even (16-byte aligned rows for the tensor copies).
bool rank_groups(tfft_plan p, int stage, int L, int W, RankGroupGeo& G, std::vector<RankGroupH>& groups) {
  groups.clear();
  if (p->g < 1 || p->g > 2 || p->d < 2) return false;
  const LayoutH& S = p->st[stage];
  if (S.owner[0] >= 0 || p->cshape[0] != L || (W & 1)) return false;
  const int d = p->d;
  // class ranges [lo, hi) of every grid direction
  std::vector<std::pair<int, int>> cls[2];
  for (int i = 0; i < p->g; ++i) {
    int ax = -1;
    for (int m = 0; m < d; ++m)
      if (S.owner[m] == i) ax = m;
    if (ax < 0) return false;
    const int64_t M = p->grid[i], r = p->cshape[ax] % M;
    if (r > 0) cls[i] = {{0, (int)r}, {(int)r, (int)M}};
    else cls[i] = {{0, (int)M}};
  }
  if (p->g == 1) cls[1] = {{0, 1}};
  const int64_t rs0 = p->rstride[0], rs1 = p->g == 2 ? p->rstride[1] : 0;
  for (const auto& c0 : cls[0])
    for (const auto& c1 : cls[1]) {
      // the group's ranks: direction 0 in [c0), direction 1 in [c1)
      auto rank_of = [&](int p0, int p1) { return (int)(p0 * rs0 + p1 * rs1); };
      RankGroupH H;
      const int r00 = rank_of(c0.first, c1.first);
      int64_t inner = 1;
      for (int m = 1; m < d; ++m) inner *= S.size[(size_t)r00 * d + m];
      if (S.size[(size_t)r00 * d] != L || inner == 0) return false;
      H.inner = inner;
      H.base = S.offset[r00];
      // ranks along direction 1 are the fastest group dimension (for a slab,
      // direction 0 takes that place)
      const int e1 = p->g == 2 ? c1.second - c1.first : c0.second - c0.first;
      const int e0 = p->g == 2 ? c0.second - c0.first : 1;
      H.ext1 = e1;
      H.ext0 = e0;
      auto rank_at = [&](int i1, int i0) {
        return p->g == 2 ? rank_of(c0.first + i0, c1.first + i1) : rank_of(c0.first + i1, 0);
      };
      H.s1 = e1 > 1 ? S.offset[rank_at(1, 0)] - H.base : inner * L;
      H.s0 = e0 > 1 ? S.offset[rank_at(0, 1)] - H.base : inner * L * e1;
      for (int i0 = 0; i0 < e0; ++i0)
        for (int i1 = 0; i1 < e1; ++i1) {
          const int rk = rank_at(i1, i0);
          for (int m = 0; m < d; ++m)
            if (S.size[(size_t)rk * d + m] != S.size[(size_t)r00 * d + m]) return false;
          if (S.offset[rk] != H.base + i1 * H.s1 + i0 * H.s0) return false;
        }
      if ((H.inner | H.base | H.s1 | H.s0) & 1) return false;
      groups.push_back(H);
    }
  if (groups.empty() || (int)groups.size() > kMaxRankGroups) return false;
  G = RankGroupGeo{};
  G.ngroups = (int)groups.size();
  G.width = W;
  G.first[0] = 0;
  for (int k = 0; k < G.ngroups; ++k) {
    const RankGroupH& H = groups[k];
    G.nblk[k] = (int)((H.inner + W - 1) / W);
    G.ext1[k] = H.ext1;
    G.first[k + 1] = G.first[k] + (int64_t)G.nblk[k] * H.ext1 * H.ext0;
  }
  return true;
}

// Tensor map of one rank group as [inner][a][L / a][ext1][ext0] complex64
// elements (a = the rows of one box dimension, at most 256), box
// W x a x L / a x 1 x 1: one tile is one copy each way.
bool encode_group_map(const RankGroupH& H, int L, int W, const void* base, CUtensorMap* map) {
  auto enc = tensor_map_encoder();
  if (!enc) return false;
  const int a = L <= 256 ? L : split_rows(L);
  if (a <= 0) return false;
  const char* b = static_cast<const char*>(base) + H.base * 8;
  cuuint64_t dims[5] = {(cuuint64_t)H.inner, (cuuint64_t)a, (cuuint64_t)(L / a), (cuuint64_t)H.ext1,
                        (cuuint64_t)H.ext0};
  cuuint64_t strides[4] = {(cuuint64_t)H.inner * 8, (cuuint64_t)H.inner * 8 * a, (cuuint64_t)H.s1 * 8,
                           (cuuint64_t)H.s0 * 8};
  cuuint32_t box[5] = {(cuuint32_t)W, (cuuint32_t)a, (cuuint32_t)(L / a), 1, 1};
  cuuint32_t estr[5] = {1, 1, 1, 1, 1};
  const CUtensorMapL2promotion promo =
      W * 8 >= 256 ? CU_TENSOR_MAP_L2_PROMOTION_L2_256B : CU_TENSOR_MAP_L2_PROMOTION_L2_128B;
  CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_UINT64, 5, const_cast<char*>(b), dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, promo, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// One side (a stage layout) of a TMA pass along `axis` over the column window
// [c0, c0 + nc) of the innermost axis (d == 3 on a 2-D grid): the 5-D view
// [x][n1][n0][ranks of direction 1][ranks of direction 0] of the ranks that
// hold the window, with the box of one tile (W columns x every row of the
// line: the local rows of all ranks of the subgroup that cuts `axis`).  When
// the layout cuts the innermost axis, the window must be tiled exactly by
// ranks of one width (a multiple of W) whose offsets are affine in their grid
// coordinates; when it does not, the window lies inside every row (rows
// `pitch` apart in a padded layout).  `shift` is the element offset of the
// layout's origin in its buffer.  Every stride and the base must be 16-byte
// aligned, and the view must stay inside the layout's elements: this is
// checked here, before any map is made.
bool window_side(tfft_plan p, int stage, int axis, int W, int64_t c0, int64_t nc, int64_t shift, TmaGeo& G,
                 TmaMapH& D) {
  if (p->d != 3 || p->g != 2 || axis < 0 || axis > 1 || W < 2 || (W & 1) || nc < W) return false;
  if (stage < 0 || stage >= (int)p->st.size()) return false;
  const LayoutH& S = p->st[stage];
  if (S.owner[axis] < 0) return false;  // the box spans the ranks that cut the FFT axis
  G = TmaGeo{};
  G.split = 0;
  G.nops = 1;
  G.rows_per_op = (int)p->cshape[axis];
  G.c0 = (int)c0;
  int lo[2] = {0, 0}, cnt[2] = {p->grid[0], p->grid[1]};
  for (int m = 0; m < 3; ++m) {
    G.cut[m] = S.owner[m] >= 0 ? 1 : 0;
    G.rdim[m] = G.cut[m] ? 3 + (p->g - 1 - S.owner[m]) : 0;
    if (!G.cut[m]) {
      G.n[m] = (int)(m == 2 ? nc : p->cshape[m]);
      continue;
    }
    const int k = S.owner[m];
    const int M = p->grid[k];
    if (m == 2) {
      // the ranks of direction k whose columns tile the window
      int first = -1;
      for (int c = 0; c < M; ++c) {
        int64_t n = 0, s0 = 0;
        decompose(p->cshape[2], M, c, n, s0);
        if (s0 == c0 && n > 0) first = c;
      }
      if (first < 0) return false;
      int64_t q = 0, s0 = 0;
      decompose(p->cshape[2], M, first, q, s0);
      if (nc % q || q % W) return false;
      const int64_t ranks = nc / q;
      for (int64_t j = 0; j < ranks; ++j) {
        int64_t n = 0, s1 = 0;
        if (first + j >= M) return false;
        decompose(p->cshape[2], M, (int)(first + j), n, s1);
        if (n != q || s1 != c0 + j * q) return false;
      }
      G.n[2] = (int)q;
      lo[k] = first;
      cnt[k] = (int)ranks;
    } else {
      if (p->cshape[m] % M) return false;
      G.n[m] = (int)(p->cshape[m] / M);
    }
  }
  const int ka = S.owner[axis];
  if (G.n[axis] > 256 || p->grid[ka] > 256 || lo[ka] != 0 || cnt[ka] != p->grid[ka]) return false;
  // the window's ranks: equal local blocks, offsets affine in (c0, c1)
  auto rank_at = [&](int i0, int i1) { return (int)((lo[0] + i0) * p->rstride[0] + (lo[1] + i1) * p->rstride[1]); };
  const int r00 = rank_at(0, 0);
  const int64_t rowlen = S.pitch > 0 ? S.pitch : (G.cut[2] ? G.n[2] : p->cshape[2]);
  const int64_t block = (int64_t)G.n[0] * G.n[1] * rowlen;
  const int64_t sd[2] = {cnt[0] > 1 ? S.offset[rank_at(1, 0)] - S.offset[r00] : block,
                         cnt[1] > 1 ? S.offset[rank_at(0, 1)] - S.offset[r00] : block};
  for (int i0 = 0; i0 < cnt[0]; ++i0)
    for (int i1 = 0; i1 < cnt[1]; ++i1) {
      const int r = rank_at(i0, i1);
      for (int m = 0; m < 3; ++m) {
        const int64_t want = (m == 2 && !G.cut[2]) ? p->cshape[2] : G.n[m];
        if (S.size[(size_t)r * 3 + m] != want) return false;
      }
      if (S.offset[r] != S.offset[r00] + i0 * sd[0] + i1 * sd[1]) return false;
    }
  if (!G.cut[2] && c0 + nc > p->cshape[2]) return false;
  D = TmaMapH{};
  D.base = S.offset[r00] + (G.cut[2] ? 0 : c0);
  D.dims[0] = (uint64_t)(G.cut[2] ? G.n[2] : nc);
  D.dims[1] = (uint64_t)G.n[1];
  D.dims[2] = (uint64_t)G.n[0];
  D.dims[3] = (uint64_t)cnt[1];  // direction g - 1 = 1
  D.dims[4] = (uint64_t)cnt[0];  // direction 0
  D.strides[0] = (uint64_t)rowlen * 8;
  D.strides[1] = (uint64_t)(G.n[1] * rowlen) * 8;
  D.strides[2] = (uint64_t)sd[1] * 8;
  D.strides[3] = (uint64_t)sd[0] * 8;
  D.box[0] = (uint32_t)W;
  D.box[2 - axis] = (uint32_t)G.n[axis];
  D.box[G.rdim[axis]] = (uint32_t)p->grid[ka];
  // 16-byte alignment of the base and every stride
  if ((shift + D.base) & 1) return false;
  for (int i = 0; i < 4; ++i)
    if ((D.strides[i] % 16) || D.strides[i] == 0) return false;
  // the farthest element the view can address stays inside the layout's
  // buffer (S.total elements from the buffer's start)
  int64_t last = D.base + (int64_t)D.dims[0] - 1;
  for (int i = 0; i < 4; ++i) last += (int64_t)(D.dims[i + 1] - 1) * (int64_t)(D.strides[i] / 8);
  if (D.base < 0 || shift < 0 || shift + last >= S.total) return false;
  return true;
}

bool encode_window_map(const TmaMapH& D, int W, const void* base, CUtensorMap* map) {
  auto enc = tensor_map_encoder();
  if (!enc || (int)D.box[0] != W) return false;
  const char* b = static_cast<const char*>(base) + D.base * 8;
  cuuint64_t dims[5];
  cuuint64_t strides[4];
  cuuint32_t box[5];
  for (int i = 0; i < 5; ++i) {
    dims[i] = (cuuint64_t)D.dims[i];
    box[i] = (cuuint32_t)D.box[i];
  }
  for (int i = 0; i < 4; ++i) strides[i] = (cuuint64_t)D.strides[i];
  cuuint32_t estr[5] = {1, 1, 1, 1, 1};
  const CUtensorMapL2promotion promo =
      W * 8 >= 256 ? CU_TENSOR_MAP_L2_PROMOTION_L2_256B : CU_TENSOR_MAP_L2_PROMOTION_L2_128B;
  CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_UINT64, 5, const_cast<char*>(b), dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, promo, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// Padding of the internal complex stage-0 buffer of a real-to-complex plan
// (d == 3, 2-D grid, FP32): when the gathering pass along axis 1 cannot run
// TMA-staged on the plain layouts -- the Hermitian half N2 = n/2 + 1 is odd,
// so stage-0 rows are not 16-byte multiples and the last stage's split of
// N2 is uneven -- the stage-0 rows are padded to an even pitch with a lead
// that puts the first column of the TMA-describable rank class on a 16-byte
// boundary.  That class (the ranks of one width, a multiple of the tile
// width) then runs TMA-staged; the other class runs the plain kernel.
bool plan_padding(tfft_plan p) {
  if (p->kind != TFFT_R2C || p->d != 3 || p->g != 2 || !p->use_tma || p->precision != TFFT_FP32) return false;
  const int ax = p->d - 2;
  const int L = (int)p->cshape[ax];
  auto it = p->aplan_s.find(L);
  if (it == p->aplan_s.end() || !it->second.spec) return false;
  int wantE = 0, Et = 0, Wt = 0;
  const int wantW = tuned_width(L, &wantE);
  if (!tma_strided_variant(L, wantW, wantE, Et, Wt)) return false;
  TmaGeo a{}, b{};
  if (tma_geo(p, 0, ax, Wt, a) && tma_geo(p, p->g, ax, Wt, b)) return false;  // no padding needed
  const LayoutH& S = p->st[p->g];
  const int k2 = S.owner[2];
  if (k2 < 0) return false;
  const int64_t N2 = p->cshape[2], M = p->grid[k2], q = N2 / M, r = N2 % M;
  // candidate classes: the r ranks of width q + 1, the M - r ranks of width q
  int64_t c0 = -1, nc = 0;
  if (r > 0 && (q + 1) % Wt == 0 && r * (q + 1) > nc) {
    c0 = 0;
    nc = r * (q + 1);
  }
  if (M - r > 0 && q > 0 && q % Wt == 0 && (M - r) * q > nc) {
    c0 = r * (q + 1);
    nc = (M - r) * q;
  }
  if (c0 < 0) return false;
  // the window's first column on a 128-byte line (16 complex): every tile row
  // of the padded side is then whole lines (measured on 512^3, 4 x 8: with
  // 16-byte alignment only, rows straddled two lines and the window pass ran
  // at 0.85 of HBM); 16-byte alignment when 128 would cost over 1/16 more
  // memory
  int64_t lead = (16 - c0 % 16) % 16;
  int64_t pitch = (lead + N2 + 15) / 16 * 16;
  if (16 * (pitch - N2) > N2) {
    lead = c0 & 1;
    pitch = (lead + N2 + 1) & ~int64_t(1);
  }
  LayoutH P;
  build_layout(p, p->cshape, 0, P, pitch);
  if (P.total >= (int64_t(1) << 31)) return false;  // 32-bit row offsets of the plain kernel
  p->st.push_back(P);
  const int idx = (int)p->st.size() - 1;
  TmaGeo gi{}, go{};
  TmaMapH mi{}, mo{};
  if (!window_side(p, idx, ax, Wt, c0, nc, lead, gi, mi) || !window_side(p, p->g, ax, Wt, c0, nc, 0, go, mo)) {
    p->st.pop_back();
    return false;
  }
  p->st[idx].state_off = image_add(p, p->st[idx].offset.data(), p->st[idx].offset.size() * 8);
  p->pad_stage = idx;
  p->pad_lead = lead;
  p->win_c0 = c0;
  p->win_nc = nc;
  p->win_E = Et;
  p->win_W = Wt;
  return true;
}

// Workspace of the fused path: one stage buffer, or the padded stage-0
// buffer of a real-to-complex plan when that is larger.
size_t fused_work_bytes(tfft_plan p) {
  size_t b = (size_t)p->nelems * sizeof(float2);
  if (p->pad_stage >= 0) b = std::max(b, (size_t)p->st[p->pad_stage].total * sizeof(float2));
  return b;
}

}  // namespace host
}  // namespace tfft
