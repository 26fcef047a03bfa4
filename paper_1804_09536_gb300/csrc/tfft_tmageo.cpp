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
  const int L = (int)p->cshape[axis];
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

}  // namespace host
}  // namespace tfft
