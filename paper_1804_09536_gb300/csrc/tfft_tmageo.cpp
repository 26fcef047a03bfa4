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

}  // namespace host
}  // namespace tfft
