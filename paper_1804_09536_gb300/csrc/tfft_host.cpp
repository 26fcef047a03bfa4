// Host side of the C ABI (include/tfft.h): plan construction on the virtual
// process grid, state image, pass lists and launches.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <map>
#include <new>
#include <stdexcept>
#include <numeric>
#include <string>
#include <tuple>
#include <vector>

#include <cuda.h>
#include <cudaTypedefs.h>

#include "tfft.h"
#include "tfft_internal.h"

using namespace tfft;

namespace {

thread_local std::string g_err;

int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  g_err = std::string(what) + ": " + cudaGetErrorString(e);
  return TFFT_ECUDA;
}

// Eq. decompose / Alg. 1.
void decompose(int64_t N, int64_t M, int64_t p, int64_t& n, int64_t& s) {
  const int64_t q = N / M, r = N % M;
  n = q + (r > p ? 1 : 0);
  s = q * p + std::min(r, p);
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

struct LayoutH {
  int d = 0;
  int64_t N[MAXD] = {0, 0, 0, 0};
  int owner[MAXD] = {-1, -1, -1, -1};
  int nranks = 0;
  std::vector<int64_t> start, size, offset;  // nranks * d, nranks * d, nranks
  int64_t total = 0;
  size_t state_off = 0;  // rank offset table in the state image (bytes)
};

enum StepKind { S_CONTIG, S_STRIDED, S_BOX, S_REAL };
constexpr int kAdjoint = 2;  // key of the adjoint's step list
enum BufId { BUF_IN, BUF_OUT, BUF_W0, BUF_W1 };

struct Step {
  StepKind kind;
  int src = BUF_IN, dst = BUF_OUT;
  bool inplace_ok = true;
  // FFT passes
  int axis = 0, lin = 0, lout = 0, L = 1, W = 16;
  int64_t nlines = 0;
  size_t cb_off = 0;
  int64_t ncb = 0;
  int sign = -1;
  bool scaled = false;
  double scale_value = 1.0;
  const double* coef = nullptr;  // device factor on a contiguous pass's output (one call only)
  // box copies: the copy tasks of the step's box list
  size_t box_off = 0;
  int64_t ntasks = 0;
  int vec2 = 0;
  int64_t box_elems = 0;
  // TMA-staged strided pass: variant, its column blocks and the tile
  // geometry of the input and output layouts
  bool tma = false;
  int tma_E = 0, tma_W = 0;
  size_t tma_cb_off = 0;
  int64_t tma_ncb = 0;
  bool tma_outer_fastest = false;  // tile order of the TMA pass
  TmaGeo gin{}, gout{};
};

struct ExchangeBoxes {  // one adjacent-stage exchange
  std::vector<BoxDesc> direct, pack, xchg, unpack;
  bool pack_identity = false, unpack_identity = false;
};

// A box list as the copy kernel runs it: offset of its task table in the
// plan state, task count, whether 16-byte copies apply, elements copied.
struct BoxList {
  size_t off = 0;
  int64_t ntasks = 0;
  int vec2 = 1;
  int64_t elems = 0;
};

}  // namespace

void tfft::set_last_error(const std::string& msg) { g_err = msg; }

struct tfft_plan_s {
  int d = 0, g = 0, kind = TFFT_C2C, precision = TFFT_FP32, flags = 0;
  int64_t shape[MAXD] = {1, 1, 1, 1};
  int64_t cshape[MAXD] = {1, 1, 1, 1};
  int grid[MAXG] = {1, 1, 1};
  int64_t rstride[MAXG] = {0, 0, 0};
  int nranks = 1;
  int64_t nelems = 0;  // complex elements of every stage buffer
  int64_t nreal = 0;   // real elements of the real stage-0 buffer (R2C)
  LayoutH real0;       // real stage-0 layout (R2C)
  AxisPlan rplan{};    // complex FFT of half the innermost length (R2C)
  bool transformable = true;  // every axis length has an FFT plan
  bool use_tma = true;        // TMA-staged passes where their conditions hold
  size_t red_off = 0;         // reduction scratch in the state (kReductionParts doubles)
  uint32_t wait_limit = 1u << 22;  // polls of a bounded copy wait
  std::vector<LayoutH> st;
  std::map<int, AxisPlan> aplan;   // contiguous-line passes
  std::map<int, AxisPlan> aplan_s; // strided passes
  std::map<int, size_t> tw_off;
  struct BlueH {       // Bluestein lengths: convolution plan and the offsets of their tables
    int M = 0;
    AxisPlan apm{};
    size_t chirp_off = 0, bhat_off = 0;
  };
  std::map<int, BlueH> blue;
  std::map<std::tuple<int, int, int>, std::pair<size_t, int64_t>> colblocks;  // (lin,lout,W)
  std::map<std::pair<int, int>, ExchangeBoxes> xboxes;                       // (from,to)
  std::map<std::pair<int, int>, std::vector<BoxList>> xbox_off;  // direct, pack, xchg, unpack
  std::map<std::pair<int, int>, std::vector<Step>> steps;        // (sign, mode)
  std::vector<uint8_t> image;
  size_t state_bytes = 0;
  char* d_state = nullptr;
  int device = -1;  // device the state was bound on
  std::vector<cudaEvent_t> events;
  // copy streams and events of tfft_execute_host (created on first use)
  struct HostIo {
    int device = -1;
    cudaStream_t cin = nullptr, cout = nullptr;
    cudaEvent_t in_done[2] = {}, comp_done[2] = {}, out_done[2] = {}, start = nullptr, end = nullptr;
  } io;
  ~tfft_plan_s() {
    if (io.device < 0) return;
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(io.device);
    for (cudaEvent_t e : {io.in_done[0], io.in_done[1], io.comp_done[0], io.comp_done[1], io.out_done[0],
                          io.out_done[1], io.start, io.end})
      if (e) cudaEventDestroy(e);
    if (io.cin) cudaStreamDestroy(io.cin);
    if (io.cout) cudaStreamDestroy(io.cout);
    cudaSetDevice(cur);
  }
};

namespace {

size_t image_add(tfft_plan p, const void* data, size_t bytes) {
  const size_t off = align_up(p->image.size(), 256);
  p->image.resize(off + bytes, 0);
  if (data && bytes) std::memcpy(p->image.data() + off, data, bytes);
  return off;
}

void build_layout(tfft_plan p, const int64_t* shape, int stage, LayoutH& L) {
  L.d = p->d;
  for (int m = 0; m < MAXD; ++m) {
    L.N[m] = m < p->d ? shape[m] : 1;
    L.owner[m] = -1;
  }
  for (int i = 0; i < p->g; ++i) {
    const int axis = (i < p->g - stage) ? i : i + 1;
    L.owner[axis] = i;
  }
  L.nranks = p->nranks;
  L.start.assign((size_t)p->nranks * p->d, 0);
  L.size.assign((size_t)p->nranks * p->d, 0);
  L.offset.assign(p->nranks, 0);
  int64_t off = 0;
  for (int r = 0; r < p->nranks; ++r) {
    int64_t coords[MAXG] = {0, 0, 0};
    int64_t rr = r;
    for (int i = p->g - 1; i >= 0; --i) {
      coords[i] = rr % p->grid[i];
      rr /= p->grid[i];
    }
    int64_t cnt = 1;
    for (int m = 0; m < p->d; ++m) {
      int64_t n = L.N[m], s = 0;
      if (L.owner[m] >= 0) decompose(L.N[m], p->grid[L.owner[m]], coords[L.owner[m]], n, s);
      L.start[(size_t)r * p->d + m] = s;
      L.size[(size_t)r * p->d + m] = n;
      cnt *= n;
    }
    L.offset[r] = off;
    off += cnt;
  }
  L.total = off;
}

DevLayout dev_layout(tfft_plan p, const LayoutH& L) {
  DevLayout D;
  D.d = L.d;
  for (int m = 0; m < MAXD; ++m) {
    D.N[m] = L.N[m];
    D.Mx[m] = L.owner[m] >= 0 ? p->grid[L.owner[m]] : 1;
    D.rs[m] = L.owner[m] >= 0 ? p->rstride[L.owner[m]] : 0;
  }
  D.offset = reinterpret_cast<const int64_t*>(p->d_state + L.state_off);
  return D;
}

// 1-D FFT plan: radices from {16, 8, 5, 4, 3, 2} that all divide E, fewest
// stages first, then the largest smallest radix, then E preference.
// `strided`: the line is one column of a W-wide tile of at most 512 threads,
// so plans with at most 32 threads per line (W >= 16 columns) are preferred.
bool make_axis_plan(int L, bool strided, AxisPlan& best) {
  best = AxisPlan{};
  if (L == 1) {
    best = AxisPlan{1, 1, 1, 0, 0, 0, 1, {}};
    return true;
  }
  static const int Es[] = {8, 16, 4, 12, 20, 24, 10, 6, 15, 5, 3, 2};
  static const int Rs[] = {16, 8, 5, 4, 3, 2};
  bool found = false;
  double best_cost = 1e30;
  for (int E : Es) {
    if (L % E != 0 || !kernel_supports_E(E)) continue;
    if (L / E > 1024) continue;
    // enumerate factorizations by depth-first search over non-increasing radices
    std::vector<int> cur, bestv;
    double bc = 1e30;
    std::vector<int> allowed;
    for (int R : Rs)
      if (E % R == 0) allowed.push_back(R);
    std::function<void(int, int)> dfs = [&](int rem, int maxi) {
      if ((int)cur.size() > MAXSTAGES) return;
      if (rem == 1) {
        int mn = *std::min_element(cur.begin(), cur.end());
        double c = cur.size() * 10.0 - mn * 0.1;
        if (c < bc) {
          bc = c;
          bestv = cur;
        }
        return;
      }
      for (int k = maxi; k < (int)allowed.size(); ++k) {
        const int R = allowed[k];
        if (rem % R == 0) {
          cur.push_back(R);
          dfs(rem / R, k);
          cur.pop_back();
        }
      }
    };
    dfs(L, 0);
    if (bestv.empty()) continue;
    double cost = bc + (E == 8 ? 0.0 : E == 16 ? 0.5 : E <= 16 ? 1.0 : 2.0);
    if (strided && L / E > 64) cost += 3.0;
    if (cost < best_cost) {
      best_cost = cost;
      best.L = L;
      best.E = E;
      best.T = L / E;
      best.nst = (int)bestv.size();
      best.code = 0;
      for (int s = 0; s < best.nst; ++s) {
        best.radix[s] = bestv[s];
        best.code |= (uint64_t)bestv[s] << (5 * s);
      }
      found = true;
    }
  }
  if (!found) {
    // no register budget fits every radix: the shared-memory-resident kernel
    // (E = 0) with a greedy factorisation, largest radices first
    std::vector<int> f;
    int rem = L;
    for (int R : Rs)
      while (rem % R == 0 && (int)f.size() < MAXSTAGES) {
        f.push_back(R);
        rem /= R;
      }
    if (rem != 1) return false;
    int items = 1;
    for (int R : f) items = std::max(items, L / R);
    best.L = L;
    best.E = 0;
    best.T = std::min(items, strided ? 32 : 128);
    best.nst = (int)f.size();
    best.code = 0;
    for (int s = 0; s < best.nst; ++s) {
      best.radix[s] = f[s];
      best.code |= (uint64_t)f[s] << (5 * s);
    }
    found = true;
  }
  return found;
}

int strided_width(const AxisPlan& ap) {
  if (ap.spec) return ap.width;
  int W = std::max(1, std::min(32, 512 / ap.T));
  // shared memory: L x W elements (two buffers for the generic kernel; two of
  // the convolution length for Bluestein) + row tables
  const size_t budget = 200 * 1024 - 16 * (size_t)ap.L;
  const size_t per_col = ap.blue_m ? 2 * 8 * (size_t)ap.blue_m : (ap.E == 0 ? 2 : 1) * 8 * (size_t)ap.L;
  while (W > 1 && (size_t)W * per_col > budget) --W;
  return W;
}

// Column blocks along axis d-1 that lie inside one rank of both layouts.
std::pair<size_t, int64_t> get_colblocks(tfft_plan p, int lin, int lout, int W) {
  auto key = std::make_tuple(lin, lout, W);
  auto it = p->colblocks.find(key);
  if (it != p->colblocks.end()) return it->second;
  const int last = p->d - 1;
  const int64_t N = p->cshape[last];
  std::vector<int64_t> cuts = {0, N};
  for (int li : {lin, lout}) {
    const LayoutH& L = p->st[li];
    if (L.owner[last] >= 0) {
      const int M = p->grid[L.owner[last]];
      for (int q = 0; q < M; ++q) {
        int64_t n, s;
        decompose(N, M, q, n, s);
        cuts.push_back(s);
      }
    }
  }
  std::sort(cuts.begin(), cuts.end());
  cuts.erase(std::unique(cuts.begin(), cuts.end()), cuts.end());
  std::vector<int2> blocks;
  for (size_t k = 0; k + 1 < cuts.size(); ++k)
    for (int64_t c = cuts[k]; c < cuts[k + 1]; c += W)
      blocks.push_back(make_int2((int)c, (int)std::min<int64_t>(W, cuts[k + 1] - c)));
  const size_t off = image_add(p, blocks.data(), blocks.size() * sizeof(int2));
  auto v = std::make_pair(off, (int64_t)blocks.size());
  p->colblocks[key] = v;
  return v;
}

// Column blocks of a (lin, lout, W) strided pass as a list (for the batch).
// Sorted cut points of the innermost axis: 0, its length and the first
// column of every rank of `lin` and `lout` that cut it.
std::vector<int64_t> column_cuts(tfft_plan p, int lin, int lout) {
  const int last = p->d - 1;
  const int64_t N = p->cshape[last];
  std::vector<int64_t> cuts = {0, N};
  for (int li : {lin, lout}) {
    const LayoutH& L = p->st[li];
    if (L.owner[last] >= 0) {
      const int M = p->grid[L.owner[last]];
      for (int q = 0; q < M; ++q) {
        int64_t n, s;
        decompose(N, M, q, n, s);
        cuts.push_back(s);
      }
    }
  }
  std::sort(cuts.begin(), cuts.end());
  cuts.erase(std::unique(cuts.begin(), cuts.end()), cuts.end());
  return cuts;
}

std::vector<int2> colblock_list(tfft_plan p, int lin, int lout, int W) {
  const std::vector<int64_t> cuts = column_cuts(p, lin, lout);
  std::vector<int2> blocks;
  for (size_t k = 0; k + 1 < cuts.size(); ++k)
    for (int64_t c = cuts[k]; c < cuts[k + 1]; c += W)
      blocks.push_back(make_int2((int)c, (int)std::min<int64_t>(W, cuts[k + 1] - c)));
  return blocks;
}

BoxDesc make_box(int d, const int64_t* ext, int64_t src, const int64_t* ss, int64_t dst,
                 const int64_t* ds) {
  BoxDesc b;
  b.src = src;
  b.dst = dst;
  const int pad = MAXD - d;
  for (int m = 0; m < MAXD; ++m) {
    if (m < pad) {
      b.ext[m] = 1;
      b.ss[m] = 0;
      b.ds[m] = 0;
    } else {
      b.ext[m] = ext[m - pad];
      b.ss[m] = ss[m - pad];
      b.ds[m] = ds[m - pad];
    }
  }
  return b;
}

void row_major_strides(int d, const int64_t* ext, int64_t* st) {
  int64_t s = 1;
  for (int m = d - 1; m >= 0; --m) {
    st[m] = s;
    s *= ext[m];
  }
}

// A flat copy of n contiguous elements as boxes of (n / 1024, 1024) rows plus a tail.
void add_flat(std::vector<BoxDesc>& out, int64_t src, int64_t dst, int64_t n) {
  const int64_t C = 1024;
  if (n <= 0) return;
  const int64_t rows = n / C, tail = n - rows * C;
  if (rows > 0) {
    const int64_t ext[2] = {rows, C}, st[2] = {C, 1};
    out.push_back(make_box(2, ext, src, st, dst, st));
  }
  if (tail > 0) {
    const int64_t ext[1] = {tail}, st[1] = {1};
    out.push_back(make_box(1, ext, src + rows * C, st, dst + rows * C, st));
  }
}

// Copy tasks of a box list.  Each box first loses its unit dimensions and
// merges every pair of neighbouring dimensions that is contiguous on both
// sides (outer stride = inner stride x inner extent); the innermost run is
// then one row.  A run longer than kRowMax elements becomes rows of kRowChunk
// (plus a tail row); otherwise the next dimension out supplies the rows.
// Rows are grouped into tasks of about kTaskElems elements, and every other
// dimension is enumerated on the host.
constexpr int64_t kRowMax = 4096, kRowChunk = 2048, kTaskElems = 16384;

void box_tasks(const BoxDesc& b, std::vector<CopyTask>& out) {
  struct Dim {
    int64_t e, s, d;
  };
  std::vector<Dim> dims;
  for (int m = 0; m < MAXD; ++m)
    if (b.ext[m] != 1) dims.push_back({b.ext[m], b.ss[m], b.ds[m]});
  for (const Dim& x : dims)
    if (x.e <= 0) return;  // empty box
  if (dims.empty()) dims.push_back({1, 1, 1});
  for (size_t k = dims.size() - 1; k > 0; --k) {  // merge contiguous neighbours, innermost first
    Dim& in = dims[k];
    const Dim& o = dims[k - 1];
    if (o.s == in.s * in.e && o.d == in.d * in.e) {
      in.e *= o.e;
      dims.erase(dims.begin() + (long)(k - 1));
    }
  }
  // innermost run (stride 1 on both sides; a unit-extent innermost axis
  // leaves a strided last dimension, whose elements are then rows of one)
  if (dims.back().s != 1 || dims.back().d != 1) dims.push_back({1, 1, 1});
  const Dim run = dims.back();
  dims.pop_back();
  std::vector<Dim> outer = dims;  // enumerated on the host
  int64_t rows = 1, rs = 0, rd = 0, rowlen = run.e, tail = 0;
  if (run.e > kRowMax) {
    rowlen = kRowChunk;
    rows = run.e / kRowChunk;
    tail = run.e - rows * kRowChunk;
    rs = rd = kRowChunk;
  } else if (!outer.empty()) {
    rows = outer.back().e;
    rs = outer.back().s;
    rd = outer.back().d;
    outer.pop_back();
  }
  const int64_t rows_per_task = std::max<int64_t>(1, kTaskElems / std::max<int64_t>(1, rowlen));
  int64_t count = 1;
  for (const Dim& x : outer) count *= x.e;
  for (int64_t idx = 0; idx < count; ++idx) {
    int64_t so = b.src, dof = b.dst, r = idx;
    for (size_t k = outer.size(); k-- > 0;) {
      const int64_t i = r % outer[k].e;
      r /= outer[k].e;
      so += i * outer[k].s;
      dof += i * outer[k].d;
    }
    for (int64_t r0 = 0; r0 < rows; r0 += rows_per_task) {
      CopyTask t;
      t.src = so + r0 * rs;
      t.dst = dof + r0 * rd;
      t.ss = rs;
      t.ds = rd;
      t.nrows = (int32_t)std::min(rows_per_task, rows - r0);
      t.rowlen = (int32_t)rowlen;
      out.push_back(t);
    }
    if (tail > 0) {
      CopyTask t;
      t.src = so + rows * kRowChunk;
      t.dst = dof + rows * kRowChunk;
      t.ss = t.ds = tail;
      t.nrows = 1;
      t.rowlen = (int32_t)tail;
      out.push_back(t);
    }
  }
}

BoxList add_box_list(tfft_plan p, const std::vector<BoxDesc>& boxes) {
  std::vector<CopyTask> tasks;
  BoxList L;
  for (const BoxDesc& b : boxes) {
    box_tasks(b, tasks);
    L.elems += b.ext[0] * b.ext[1] * b.ext[2] * b.ext[3];
  }
  for (const CopyTask& t : tasks)
    if ((t.src | t.dst | t.ss | t.ds | (int64_t)t.rowlen) & 1) L.vec2 = 0;
  L.ntasks = (int64_t)tasks.size();
  L.off = image_add(p, tasks.data(), tasks.size() * sizeof(CopyTask));
  return L;
}

bool box_contiguous(const BoxDesc& b, const int64_t* st) {
  int64_t rm[MAXD];
  row_major_strides(MAXD, b.ext, rm);
  for (int m = 0; m < MAXD; ++m)
    if (b.ext[m] > 1 && st[m] != rm[m]) return false;
  return true;
}

// Boxes of the exchange between adjacent stages s_from -> s_to (Alg. 2 / Alg. 3).
void build_exchange(tfft_plan p, int s_from, int s_to) {
  const int d = p->d;
  const int i = p->g - std::max(s_from, s_to);
  const LayoutH& A = p->st[s_from];
  const LayoutH& B = p->st[s_to];
  int v = -1, w = -1;
  for (int m = 0; m < d; ++m) {
    if (B.owner[m] == i) v = m;  // A holds v whole, B cuts it
    if (A.owner[m] == i) w = m;  // A cuts w, B holds it whole
  }
  const int M = p->grid[i];
  ExchangeBoxes X;
  X.pack_identity = true;
  X.unpack_identity = true;
  for (int a = 0; a < p->nranks; ++a) {
    const int64_t pa = (a / p->rstride[i]) % M;  // a's coordinate in direction i
    const int64_t* Aext = &A.size[(size_t)a * d];
    int64_t Ast[MAXD];
    row_major_strides(d, Aext, Ast);
    int64_t packed = 0;
    for (int q = 0; q < M; ++q) {
      const int b = (int)(a + (q - pa) * p->rstride[i]);
      const int64_t* Bext = &B.size[(size_t)b * d];
      int64_t Bst[MAXD];
      row_major_strides(d, Bext, Bst);
      int64_t nq, sq, np_, sp;
      decompose(p->cshape[v], M, q, nq, sq);
      decompose(p->cshape[w], M, pa, np_, sp);
      int64_t ext[MAXD];
      int64_t cnt = 1;
      for (int m = 0; m < d; ++m) {
        ext[m] = (m == v) ? nq : Aext[m];
        cnt *= ext[m];
      }
      if (cnt == 0) continue;
      const int64_t src = A.offset[a] + sq * Ast[v];
      const int64_t dst = B.offset[b] + sp * Bst[w];
      X.direct.push_back(make_box(d, ext, src, Ast, dst, Bst));
      // traditional: pack into rank a's send region, chunk q after chunks 0..q-1
      int64_t cst[MAXD];
      row_major_strides(d, ext, cst);
      const int64_t psrc = src, pdst = A.offset[a] + packed;
      BoxDesc pb = make_box(d, ext, psrc, Ast, pdst, cst);
      X.pack.push_back(pb);
      if (!(psrc == pdst && box_contiguous(pb, pb.ss))) X.pack_identity = false;
      packed += cnt;
    }
  }
  // all-to-all of contiguous chunks: rank b receives from p = 0..M-1 in order
  for (int b = 0; b < p->nranks; ++b) {
    const int64_t qb = (b / p->rstride[i]) % M;
    const int64_t* Bext = &B.size[(size_t)b * d];
    int64_t Bst[MAXD];
    row_major_strides(d, Bext, Bst);
    int64_t recv = 0;
    for (int pp = 0; pp < M; ++pp) {
      const int a = (int)(b + (pp - qb) * p->rstride[i]);
      const int64_t* Aext = &A.size[(size_t)a * d];
      // offset of chunk qb inside a's send region
      int64_t before = 0;
      for (int q = 0; q < qb; ++q) {
        int64_t nq, sq;
        decompose(p->cshape[v], M, q, nq, sq);
        int64_t c = 1;
        for (int m = 0; m < d; ++m) c *= (m == v) ? nq : Aext[m];
        before += c;
      }
      int64_t nq, sq, np_, sp;
      decompose(p->cshape[v], M, qb, nq, sq);
      decompose(p->cshape[w], M, pp, np_, sp);
      int64_t ext[MAXD];
      int64_t cnt = 1;
      for (int m = 0; m < d; ++m) {
        ext[m] = (m == v) ? nq : Aext[m];
        cnt *= ext[m];
      }
      if (cnt == 0) continue;
      add_flat(X.xchg, A.offset[a] + before, B.offset[b] + recv, cnt);
      int64_t cst[MAXD];
      row_major_strides(d, ext, cst);
      const int64_t usrc = B.offset[b] + recv, udst = B.offset[b] + sp * Bst[w];
      BoxDesc ub = make_box(d, ext, usrc, cst, udst, Bst);
      X.unpack.push_back(ub);
      if (!(usrc == udst && box_contiguous(ub, ub.ds))) X.unpack_identity = false;
      recv += cnt;
    }
  }
  std::vector<BoxList> offs;
  for (auto* vec : {&X.direct, &X.pack, &X.xchg, &X.unpack}) offs.push_back(add_box_list(p, *vec));
  p->xboxes[{s_from, s_to}] = std::move(X);
  p->xbox_off[{s_from, s_to}] = offs;
}

Step box_step(const BoxList& L) {
  Step s;
  s.kind = S_BOX;
  s.inplace_ok = false;
  s.box_off = L.off;
  s.ntasks = L.ntasks;
  s.vec2 = L.vec2;
  s.box_elems = L.elems;
  return s;
}

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
// (used when tuning); 0 when not given.
int tuned_width(int L, int* E = nullptr) {
  if (E) *E = 0;
  const char* env = std::getenv("TFFT_TMA_W");
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

Step fft_step(tfft_plan p, int axis, int lin, int lout, int sign) {
  Step s;
  s.sign = sign;
  s.axis = axis;
  s.lin = lin;
  s.lout = lout;
  s.L = (int)p->cshape[axis];
  if (axis == p->d - 1) {
    s.kind = S_CONTIG;
    s.inplace_ok = true;
    s.nlines = p->nelems / s.L;
  } else {
    s.kind = S_STRIDED;
    s.inplace_ok = (lin == lout);
    const AxisPlan& ap = p->aplan_s[s.L];
    s.W = strided_width(ap);
    auto cb = get_colblocks(p, lin, lout, s.W);
    s.cb_off = cb.first;
    s.ncb = cb.second;
    int Et = 0, Wt = 0, wantE = 0;
    const int wantW = tuned_width(s.L, &wantE);
    s.tma = p->use_tma && ap.spec && tma_strided_variant(s.L, wantW, wantE, Et, Wt) &&
            tma_geo(p, lin, axis, Wt, s.gin) && tma_geo(p, lout, axis, Wt, s.gout);
    if (s.tma) {
      s.tma_E = Et;
      s.tma_W = Wt;
      auto cbt = get_colblocks(p, lin, lout, Wt);
      s.tma_cb_off = cbt.first;
      s.tma_ncb = cbt.second;
      // measured on 512^3, 4 x 8 grid: the axis-0 pass is faster with the
      // outer index running fastest (16-column tiles: 0.348 vs 0.356 ms), the
      // axis-1 pass with the column blocks running fastest; with 8-column
      // tiles (64-byte rows, 1024 x 1024 x 128) the column-block order wins
      // on axis 0 as well (0.395 vs 0.588 ms)
      s.tma_outer_fastest = axis == 0 && Wt * sizeof(float2) >= 128;
    }
  }
  return s;
}

// The pass along the innermost axis: a complex FFT of contiguous lines, or
// for a real-to-complex plan the r2c (forward) / c2r (backward) pass between
// the real and the complex stage-0 buffers.
Step last_axis_step(tfft_plan p, int sign) {
  if (p->kind != TFFT_R2C) return fft_step(p, p->d - 1, 0, 0, sign);
  Step s;
  s.kind = S_REAL;
  s.sign = sign;
  s.axis = p->d - 1;
  s.inplace_ok = false;
  s.L = p->rplan.L;
  s.nlines = p->nreal / (2 * (int64_t)p->rplan.L);
  return s;
}

void add_exchange_steps(tfft_plan p, std::vector<Step>& out, int from, int to, int mode) {
  const ExchangeBoxes& X = p->xboxes[{from, to}];
  const std::vector<BoxList>& off = p->xbox_off[{from, to}];
  if (mode == TFFT_MODE_UNFUSED) {
    out.push_back(box_step(off[0]));
  } else {
    if (!X.pack_identity) out.push_back(box_step(off[1]));
    out.push_back(box_step(off[2]));
    if (!X.unpack_identity) out.push_back(box_step(off[3]));
  }
}

// Logical step list of one direction and mode (buffers assigned later).
std::vector<Step> build_steps(tfft_plan p, int sign, int mode) {
  const int d = p->d, g = p->g;
  std::vector<Step> v;
  if (mode == TFFT_MODE_FUSED) {
    if (sign == TFFT_FORWARD) {
      v.push_back(last_axis_step(p, sign));
      for (int a = d - 2; a >= 0; --a) v.push_back(fft_step(p, a, a == d - 2 ? 0 : g, g, sign));
    } else {
      for (int a = 0; a <= d - 2; ++a) v.push_back(fft_step(p, a, g, a == d - 2 ? 0 : g, sign));
      v.push_back(last_axis_step(p, sign));
    }
  } else {
    if (sign == TFFT_FORWARD) {
      v.push_back(last_axis_step(p, sign));
      for (int a = d - 2; a >= g; --a) v.push_back(fft_step(p, a, 0, 0, sign));
      for (int s = 1; s <= g; ++s) {
        add_exchange_steps(p, v, s - 1, s, mode);
        v.push_back(fft_step(p, g - s, s, s, sign));
      }
    } else {
      for (int s = g; s >= 1; --s) {
        v.push_back(fft_step(p, g - s, s, s, sign));
        add_exchange_steps(p, v, s, s - 1, mode);
      }
      for (int a = g; a <= d - 2; ++a) v.push_back(fft_step(p, a, 0, 0, sign));
      v.push_back(last_axis_step(p, sign));
    }
  }
  // normalisation on the last FFT pass of the scaled direction
  const bool scale_here = (sign == TFFT_FORWARD) == !(p->flags & TFFT_NORM_BACKWARD);
  if (scale_here) {
    for (int k = (int)v.size() - 1; k >= 0; --k)
      if (v[k].kind != S_BOX) {
        v[k].scaled = true;
        v[k].scale_value = 1.0 / (double)(p->kind == TFFT_R2C ? p->nreal : p->nelems);
        break;
      }
  }
  return v;
}

// Assign buffers: the first step reads the input; in-place passes keep the
// current buffer (the input itself only when it may be overwritten);
// layout-changing steps alternate between the work buffers; the last
// layout-changing step (or the first pass when there is none) writes `out`.
void assign_buffers(std::vector<Step>& v, bool destroy_input) {
  int last_move = -1;
  for (int k = 0; k < (int)v.size(); ++k)
    if (!v[k].inplace_ok) last_move = k;
  int cur = BUF_IN;
  for (int k = 0; k < (int)v.size(); ++k) {
    Step& s = v[k];
    s.src = cur;
    if (s.inplace_ok) {
      if (cur == BUF_IN) {
        if (last_move < k) s.dst = BUF_OUT;
        else s.dst = destroy_input ? BUF_IN : BUF_W0;
      } else {
        s.dst = cur;
      }
    } else {
      if (k == last_move) s.dst = BUF_OUT;
      else s.dst = (cur == BUF_W0) ? BUF_W1 : BUF_W0;
    }
    cur = s.dst;
  }
}

int check_ptr(const void* ptr, const char* name) {
  if (!ptr) return fail(TFFT_EINVAL, std::string(name) + " is NULL");
  if (reinterpret_cast<uintptr_t>(ptr) & 15)
    return fail(TFFT_EALIGN, std::string(name) + " is not 16-byte aligned");
  return TFFT_OK;
}

// The plan is bound, and the calling thread's current device is the one it
// was bound on (its state, twiddles and tensor maps live there).
int check_bound(tfft_plan p) {
  if (!p->d_state) return fail(TFFT_ESTATE, "plan is not bound");
  const int dev = current_device();
  if (dev != p->device)
    return fail(TFFT_EINVAL, "the current device (" + std::to_string(dev) + ") is not the device the plan was bound on (" +
                                 std::to_string(p->device) + ")");
  return TFFT_OK;
}

BlueArgs blue_args(tfft_plan p, int N);

int launch_step(tfft_plan p, const Step& s, void* const* bufs, cudaStream_t st) {
  const float2* in = static_cast<const float2*>(bufs[s.src]);
  float2* out = static_cast<float2*>(bufs[s.dst]);
  cudaError_t e = cudaSuccess;
  if (s.kind == S_CONTIG) {
    ContigArgs a;
    a.in = in;
    a.out = out;
    a.nlines = s.nlines;
    a.ap = p->aplan[s.L];
    a.tw = reinterpret_cast<const float2*>(p->d_state + p->tw_off[s.L]);
    a.lines_per_cta = a.ap.spec ? a.ap.width : std::max(1, 256 / a.ap.T);
    a.sign = s.sign;
    a.scale = s.scaled ? (float)s.scale_value : 1.0f;
    a.coef = s.coef;
    a.status = reinterpret_cast<int*>(p->d_state);
    a.wait_limit = p->wait_limit;
    if (a.ap.blue_m)
      e = launch_contig_blue(a, blue_args(p, s.L), st);
    else if (p->precision != TFFT_FP32 && tc_supported(a.ap.L))
      e = launch_contig_tc(a, p->precision, st);
    else
      e = launch_contig(a, st);
  } else if (s.kind == S_STRIDED) {
    StridedArgs a;
    a.in = in;
    a.out = out;
    a.lin = dev_layout(p, p->st[s.lin]);
    a.lout = dev_layout(p, p->st[s.lout]);
    a.d = p->d;
    a.axis = s.axis;
    a.ap = p->aplan_s[s.L];
    a.tw = reinterpret_cast<const float2*>(p->d_state + p->tw_off[s.L]);
    a.colblocks = reinterpret_cast<const int2*>(p->d_state + s.cb_off);
    a.ncolblocks = s.ncb;
    a.outer_fastest = 0;
    int oax[2] = {-1, -1}, no = 0;
    int64_t nouter = 1;
    for (int m = 0; m < p->d - 1; ++m)
      if (m != s.axis) {
        oax[no++] = m;
        nouter *= p->cshape[m];
      }
    a.nouter = nouter;
    a.oax0 = oax[0];
    a.oax1 = oax[1];
    a.on1 = oax[1] >= 0 ? p->cshape[oax[1]] : 1;
    a.W = s.W;
    a.sign = s.sign;
    a.scale = s.scaled ? (float)s.scale_value : 1.0f;
    a.status = reinterpret_cast<int*>(p->d_state);
    a.wait_limit = p->wait_limit;
    bool done = false;
    if (s.tma) {
      alignas(64) CUtensorMap ti, to;
      if (encode_stage_map(p, s.gin, s.axis, s.tma_W, in, &ti) &&
          encode_stage_map(p, s.gout, s.axis, s.tma_W, out, &to)) {
        StridedArgs at = a;
        at.W = s.tma_W;
        at.colblocks = reinterpret_cast<const int2*>(p->d_state + s.tma_cb_off);
        at.ncolblocks = s.tma_ncb;
        at.outer_fastest = s.tma_outer_fastest ? 1 : 0;
        if (p->precision != TFFT_FP32 && tc_strided_supported(s.L, s.tma_E, s.tma_W, p->nelems))
          e = launch_strided_tma_tc(at, s.tma_E, p->precision, s.gin, s.gout, &ti, &to, st);
        else
          e = launch_strided_tma(at, s.tma_E, s.gin, s.gout, &ti, &to, st);
        done = true;
      }
    }
    if (!done && a.ap.blue_m) {
      e = launch_strided_blue(a, blue_args(p, s.L), st);
      done = true;
    }
    if (!done) e = launch_strided(a, st);
  } else if (s.kind == S_REAL) {
    RealArgs a;
    a.rin = reinterpret_cast<const float*>(bufs[s.src]);
    a.cout = static_cast<float2*>(bufs[s.dst]);
    a.cin = static_cast<const float2*>(bufs[s.src]);
    a.rout = static_cast<float*>(bufs[s.dst]);
    a.nlines = s.nlines;
    a.ap = p->rplan;
    a.tw = reinterpret_cast<const float2*>(p->d_state + p->tw_off[p->rplan.L]);
    a.tw2 = reinterpret_cast<const float2*>(p->d_state + p->tw_off[2 * p->rplan.L]);
    a.dir = s.sign;
    a.scale = s.scaled ? (float)s.scale_value : 1.0f;
    a.status = reinterpret_cast<int*>(p->d_state);
    e = launch_real_spec(a, st);
  } else {
    BoxArgs a;
    a.in = in;
    a.out = out;
    a.tasks = reinterpret_cast<const CopyTask*>(p->d_state + s.box_off);
    a.ntasks = s.ntasks;
    a.vec2 = s.vec2;
    e = launch_boxcopy(a, st);
  }
  if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
  return TFFT_OK;
}

int run_steps(tfft_plan p, const std::vector<Step>& steps, void* const* bufs, cudaStream_t st) {
  const bool timed = !p->events.empty();
  for (size_t k = 0; k < steps.size(); ++k) {
    if (timed) {
      cudaError_t e = cudaEventRecord(p->events[k], st);
      if (e != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
    }
    int rc = launch_step(p, steps[k], bufs, st);
    if (rc != TFFT_OK) return rc;
  }
  if (timed) {
    cudaError_t e = cudaEventRecord(p->events[steps.size()], st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
  }
  return TFFT_OK;
}

bool is_smooth_235(int64_t n) {
  if (n < 1) return false;
  for (int f : {2, 3, 5})
    while (n % f == 0) n /= f;
  return n == 1;
}

// Bluestein plan for a length N without a 2/3/5 factorisation: convolution
// length M = the power of two >= 2N - 1 (at most MAXLEN), and the tables,
// evaluated in double and rounded once: chirp[n] = exp(-i pi (n^2 mod 2N) / N)
// and bhat = FFT_M(b) / M for the wrapped filter b[m] = b[M - m] = conj(chirp[m]).
bool make_bluestein(tfft_plan p, int N) {
  int M = 1;
  while (M < 2 * N - 1) M <<= 1;
  AxisPlan apm{};
  if (M > MAXLEN || !make_axis_plan(M, false, apm)) return false;
  const double pi = 3.14159265358979323846;
  std::vector<float2> chirp(N), bhat(M);
  std::vector<std::complex<double>> b(M, 0.0), w(M);
  for (int n = 0; n < N; ++n) {
    const int64_t r = ((int64_t)n * n) % (2 * (int64_t)N);
    const double ang = pi * (double)r / (double)N;
    chirp[n] = make_float2((float)std::cos(ang), (float)-std::sin(ang));
    b[n] = std::complex<double>(std::cos(ang), std::sin(ang));
    if (n > 0) b[M - n] = b[n];
  }
  for (int m = 0; m < M; ++m) w[m] = std::polar(1.0, -2.0 * pi * (double)m / (double)M);
  std::vector<int> nz;
  for (int m = 0; m < M; ++m)
    if (b[m] != 0.0) nz.push_back(m);
  for (int k = 0; k < M; ++k) {
    std::complex<double> acc = 0.0;
    for (int m : nz) acc += b[m] * w[((int64_t)m * k) % M];
    acc /= (double)M;
    bhat[k] = make_float2((float)acc.real(), (float)acc.imag());
  }
  tfft_plan_s::BlueH h;
  h.M = M;
  h.apm = apm;
  h.chirp_off = image_add(p, chirp.data(), chirp.size() * sizeof(float2));
  h.bhat_off = image_add(p, bhat.data(), bhat.size() * sizeof(float2));
  if (!p->tw_off.count(M)) p->tw_off[M] = image_add(p, nullptr, (size_t)M * sizeof(float2));
  if (!p->tw_off.count(N)) p->tw_off[N] = image_add(p, nullptr, (size_t)N * sizeof(float2));
  AxisPlan ap{};
  ap.L = N;
  ap.E = 0;
  ap.T = apm.T;
  ap.blue_m = M;
  ap.width = std::max(1, std::min(4096 / M, 512 / apm.T));  // lines per CTA (two M-buffers each)
  AxisPlan aps = ap;
  aps.width = strided_width(aps);
  p->aplan[N] = ap;
  p->aplan_s[N] = aps;
  p->blue[N] = h;
  return true;
}

BlueArgs blue_args(tfft_plan p, int N) {
  const tfft_plan_s::BlueH& h = p->blue.at(N);
  BlueArgs b;
  b.N = N;
  b.M = h.M;
  b.apm = h.apm;
  b.twm = reinterpret_cast<const float2*>(p->d_state + p->tw_off.at(h.M));
  b.chirp = reinterpret_cast<const float2*>(p->d_state + h.chirp_off);
  b.bhat = reinterpret_cast<const float2*>(p->d_state + h.bhat_off);
  return b;
}

}  // namespace

// ============================================================== ABI

// Runs an entry point's body so that no C++ exception (host allocation
// failure, a library error) crosses the C ABI: it becomes an error status.
template <class F>
int guarded(const char* name, F&& body) {
  try {
    return body();
  } catch (const std::bad_alloc&) {
    return fail(TFFT_EINVAL, std::string(name) + ": out of host memory");
  } catch (const std::exception& e) {
    return fail(TFFT_EINVAL, std::string(name) + ": " + e.what());
  } catch (...) {
    return fail(TFFT_EINVAL, std::string(name) + ": unexpected error");
  }
}

extern "C" {

const char* tfft_status_string(int status) {
  switch (status) {
    case TFFT_OK: return "TFFT_OK";
    case TFFT_EINVAL: return "TFFT_EINVAL";
    case TFFT_EUNSUPPORTED: return "TFFT_EUNSUPPORTED";
    case TFFT_EALIGN: return "TFFT_EALIGN";
    case TFFT_EWORKSPACE: return "TFFT_EWORKSPACE";
    case TFFT_ECUDA: return "TFFT_ECUDA";
    case TFFT_ESTATE: return "TFFT_ESTATE";
    default: return "TFFT_UNKNOWN";
  }
}

const char* tfft_last_error(void) { return g_err.c_str(); }

int tfft_version(void) { return 100; }

int tfft_decompose(int64_t N, int64_t M, int64_t p, int64_t* n, int64_t* s) {
  if (!n || !s) return fail(TFFT_EINVAL, "decompose: NULL output");
  if (N < 0 || M <= 0 || p < 0 || p >= M) return fail(TFFT_EINVAL, "decompose: need N >= 0, M > 0, 0 <= p < M");
  decompose(N, M, p, *n, *s);
  return TFFT_OK;
}

int tfft_plan_create(tfft_plan* plan, int ndims, const int64_t* shape, int grid_ndims,
                     const int* grid, int kind, int precision, int flags) {
  return guarded("tfft_plan_create", [&]() -> int {
    if (!plan) return fail(TFFT_EINVAL, "plan is NULL");
    *plan = nullptr;
    if (ndims < 1 || ndims > MAXD) return fail(TFFT_EINVAL, "ndims must be 1..4");
    if (!shape) return fail(TFFT_EINVAL, "shape is NULL");
    if (grid_ndims < 0 || grid_ndims > ndims - 1 || grid_ndims > MAXG)
      return fail(TFFT_EINVAL, "grid_ndims must be 0..min(3, ndims - 1) (Sec. 3.6)");
    if (grid_ndims > 0 && !grid) return fail(TFFT_EINVAL, "grid is NULL");
    if (kind != TFFT_C2C && kind != TFFT_R2C) return fail(TFFT_EINVAL, "kind must be TFFT_C2C or TFFT_R2C");
    if (precision != TFFT_FP32 && precision != TFFT_TC_BF16X3 && precision != TFFT_TC_FP16X3)
      return fail(TFFT_EINVAL, "precision must be TFFT_FP32, TFFT_TC_BF16X3 or TFFT_TC_FP16X3");
    if (flags & ~(TFFT_NORM_BACKWARD | TFFT_NO_TMA)) return fail(TFFT_EINVAL, "unknown flag bits");
    auto p = new tfft_plan_s();
    p->d = ndims;
    p->g = grid_ndims;
    p->kind = kind;
    p->precision = precision;
    p->flags = flags;
    int64_t n = 1;
    for (int m = 0; m < ndims; ++m) {
      if (shape[m] < 1 || shape[m] > (int64_t(1) << 31)) {
        delete p;
        return fail(TFFT_EINVAL, "every extent must be in 1 .. 2^31");
      }
      p->shape[m] = p->cshape[m] = shape[m];
      n *= shape[m];
    }
    p->nreal = n;
    if (kind == TFFT_R2C) {
      if (shape[ndims - 1] % 2) {
        delete p;
        return fail(TFFT_EUNSUPPORTED, "real-to-complex needs an even innermost extent");
      }
      p->cshape[ndims - 1] = shape[ndims - 1] / 2 + 1;  // Hermitian half (footnote to Eq. multifft)
      n = n / shape[ndims - 1] * p->cshape[ndims - 1];
    }
    p->nelems = n;
    int64_t nr = 1;
    for (int i = 0; i < grid_ndims; ++i) {
      if (grid[i] < 1 || grid[i] > 65536) {
        delete p;
        return fail(TFFT_EINVAL, "grid extents must be in 1 .. 65536");
      }
      p->grid[i] = grid[i];
      nr *= grid[i];
    }
    if (nr > (1 << 20)) {
      delete p;
      return fail(TFFT_EINVAL, "too many virtual ranks");
    }
    p->nranks = (int)nr;
    for (int i = grid_ndims - 1, s = 1; i >= 0; --i) {
      p->rstride[i] = s;
      s *= grid[i];
    }
    // stage layouts and their rank offset tables
    p->use_tma = !(flags & TFFT_NO_TMA);
    image_add(p, nullptr, 256);  // device status word(s) at offset 0
    p->red_off = image_add(p, nullptr, kReductionParts * sizeof(double));
    p->st.resize(p->g + 1);
    for (int s = 0; s <= p->g; ++s) {
      build_layout(p, p->cshape, s, p->st[s]);
      p->st[s].state_off = image_add(p, p->st[s].offset.data(), p->st[s].offset.size() * 8);
    }
    if (kind == TFFT_R2C) build_layout(p, p->shape, 0, p->real0);
    // per-length FFT plans and twiddle table slots (a plan whose lengths do not
    // factor into 2, 3, 5 up to 4096 still redistributes, but does not transform)
    if (kind == TFFT_R2C) {
      const int Lh = (int)(p->shape[ndims - 1] / 2);
      int width = 0;
      p->rplan = AxisPlan{};
      if (spec_plan(Lh, false, p->nelems, p->rplan, width)) {
        p->rplan.width = width;
        if (!p->tw_off.count(Lh)) p->tw_off[Lh] = image_add(p, nullptr, (size_t)Lh * sizeof(float2));
        if (!p->tw_off.count(2 * Lh)) p->tw_off[2 * Lh] = image_add(p, nullptr, (size_t)2 * Lh * sizeof(float2));
      } else {
        p->transformable = false;  // half length without a compiled real-line kernel
      }
    }
    for (int m = 0; m < ndims; ++m) {
      if (kind == TFFT_R2C && m == ndims - 1) break;  // the innermost axis is the real pass
      const int L = (int)p->cshape[m];
      if (p->aplan.count(L)) continue;
      AxisPlan ap{}, aps{};
      if (!is_smooth_235(L) && L <= MAXLEN / 2) {
        if (!make_bluestein(p, L)) p->transformable = false;
        continue;
      }
      if (L > MAXLEN || !is_smooth_235(L) || !make_axis_plan(L, false, ap) ||
          !make_axis_plan(L, true, aps)) {
        p->transformable = false;
        continue;
      }
      int width = 0;
      if (spec_plan(L, false, p->nelems, ap, width)) ap.width = width;
      if (spec_plan(L, true, p->nelems, aps, width)) aps.width = width;
      p->aplan[L] = ap;
      p->aplan_s[L] = aps;
      if (!p->tw_off.count(L)) p->tw_off[L] = image_add(p, nullptr, (size_t)L * sizeof(float2));
    }
    // exchange boxes between adjacent stages, both directions
    for (int s = 1; s <= p->g; ++s) {
      build_exchange(p, s - 1, s);
      build_exchange(p, s, s - 1);
    }
    if (p->transformable) {
      // pass lists
      for (int sign : {TFFT_FORWARD, TFFT_BACKWARD})
        for (int mode : {TFFT_MODE_FUSED, TFFT_MODE_UNFUSED, TFFT_MODE_PACKED})
          p->steps[{sign, mode}] = build_steps(p, sign, mode);
      // the adjoint of the forward (kAdjoint): the backward steps, with 1/N on
      // the last pass when the forward carries the normalisation
      if (p->kind == TFFT_C2C)
        for (int mode : {TFFT_MODE_FUSED, TFFT_MODE_UNFUSED, TFFT_MODE_PACKED}) {
          std::vector<Step> v = build_steps(p, TFFT_BACKWARD, mode);
          if (!(p->flags & TFFT_NORM_BACKWARD))
            for (int k = (int)v.size() - 1; k >= 0; --k)
              if (v[k].kind != S_BOX) {
                v[k].scaled = true;
                v[k].scale_value = 1.0 / (double)p->nelems;
                break;
              }
          p->steps[{kAdjoint, mode}] = v;
        }
      // column blocks for in-place partial transforms of every stage
      for (int s = 0; s <= p->g; ++s)
        for (auto& kv : p->aplan_s) get_colblocks(p, s, s, strided_width(kv.second));
    }
    p->state_bytes = align_up(p->image.size(), 256);
    p->image.resize(p->state_bytes, 0);
    *plan = p;
    return TFFT_OK;
  });
}

int tfft_plan_destroy(tfft_plan plan) {
  if (!plan) return fail(TFFT_EINVAL, "plan is NULL");
  delete plan;
  return TFFT_OK;
}

int tfft_plan_num_stages(tfft_plan p, int* nstages) {
  if (!p || !nstages) return fail(TFFT_EINVAL, "NULL argument");
  *nstages = p->g + 1;
  return TFFT_OK;
}

int tfft_plan_num_ranks(tfft_plan p, int* nranks) {
  if (!p || !nranks) return fail(TFFT_EINVAL, "NULL argument");
  *nranks = p->nranks;
  return TFFT_OK;
}

int tfft_plan_stage_axis(tfft_plan p, int stage, int* axis) {
  if (!p || !axis) return fail(TFFT_EINVAL, "NULL argument");
  if (stage < 0 || stage > p->g) return fail(TFFT_EINVAL, "stage out of range");
  *axis = p->g - stage;
  return TFFT_OK;
}

int tfft_plan_stage_elems(tfft_plan p, int stage, int real, int64_t* elems) {
  if (!p || !elems) return fail(TFFT_EINVAL, "NULL argument");
  if (stage < 0 || stage > p->g) return fail(TFFT_EINVAL, "stage out of range");
  if (real) {
    if (p->kind != TFFT_R2C) return fail(TFFT_EINVAL, "not a real-to-complex plan");
    if (stage != 0) return fail(TFFT_EINVAL, "the real buffer is the stage-0 alignment");
    *elems = p->real0.total;
    return TFFT_OK;
  }
  *elems = p->st[stage].total;
  return TFFT_OK;
}

int tfft_plan_local_box(tfft_plan p, int stage, int real, int rank, int64_t* start,
                        int64_t* size, int64_t* offset) {
  if (!p || !start || !size || !offset) return fail(TFFT_EINVAL, "NULL argument");
  if (stage < 0 || stage > p->g) return fail(TFFT_EINVAL, "stage out of range");
  if (rank < 0 || rank >= p->nranks) return fail(TFFT_EINVAL, "rank out of range");
  if (real && p->kind != TFFT_R2C) return fail(TFFT_EINVAL, "not a real-to-complex plan");
  if (real && stage != 0) return fail(TFFT_EINVAL, "the real buffer is the stage-0 alignment");
  const LayoutH& L = real ? p->real0 : p->st[stage];
  for (int m = 0; m < p->d; ++m) {
    start[m] = L.start[(size_t)rank * p->d + m];
    size[m] = L.size[(size_t)rank * p->d + m];
  }
  *offset = L.offset[rank];
  return TFFT_OK;
}

int tfft_plan_state_bytes(tfft_plan p, size_t* bytes) {
  if (!p || !bytes) return fail(TFFT_EINVAL, "NULL argument");
  *bytes = p->state_bytes;
  return TFFT_OK;
}

int tfft_plan_bind(tfft_plan p, void* d_state, size_t bytes, void* stream) {
  return guarded("tfft_plan_bind", [&]() -> int {
    if (!p) return fail(TFFT_EINVAL, "plan is NULL");
    int rc = check_ptr(d_state, "d_state");
    if (rc) return rc;
    if (bytes < p->state_bytes) return fail(TFFT_EINVAL, "state buffer too small");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemcpyAsync(d_state, p->image.data(), p->state_bytes, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync (plan state)");
    for (auto& kv : p->tw_off) {
      e = launch_twiddles(reinterpret_cast<float2*>(static_cast<char*>(d_state) + kv.second), kv.first, st);
      if (e != cudaSuccess) return cuda_fail(e, "twiddle generation");
    }
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize (bind)");
    p->d_state = static_cast<char*>(d_state);
    p->device = current_device();
    return TFFT_OK;
  });
}

int tfft_plan_workspace_bytes(tfft_plan p, int mode, int keep_input, size_t* bytes) {
  if (!p || !bytes) return fail(TFFT_EINVAL, "NULL argument");
  const size_t stage = (size_t)p->nelems * sizeof(float2);
  switch (mode) {
    case TFFT_MODE_FUSED: *bytes = (keep_input || p->kind == TFFT_R2C) ? stage : 0; break;
    case TFFT_MODE_UNFUSED:
    case TFFT_MODE_PACKED: *bytes = 2 * stage; break;
    default: return fail(TFFT_EINVAL, "unknown mode");
  }
  return TFFT_OK;
}

int tfft_redistribute(tfft_plan p, int axis_v, int axis_w, const void* in, void* out, void* stream) {
  return guarded("tfft_redistribute", [&]() -> int {
    if (!p) return fail(TFFT_EINVAL, "plan is NULL");
    if (int rcb = check_bound(p)) return rcb;
    const int sf = p->g - axis_v, stt = p->g - axis_w;
    if (sf < 0 || sf > p->g || stt < 0 || stt > p->g || std::abs(sf - stt) != 1)
      return fail(TFFT_EINVAL, "axis_v / axis_w are not the aligned axes of two adjacent stages");
    int rc = check_ptr(in, "in");
    if (rc) return rc;
    rc = check_ptr(out, "out");
    if (rc) return rc;
    const size_t bytes = (size_t)p->nelems * sizeof(float2);
    const char* a = static_cast<const char*>(in);
    const char* b = static_cast<const char*>(out);
    if (a < b + bytes && b < a + bytes) return fail(TFFT_EINVAL, "in and out overlap");
    Step s = box_step(p->xbox_off[{sf, stt}][0]);
    s.src = BUF_IN;
    s.dst = BUF_OUT;
    void* bufs[4] = {const_cast<void*>(in), out, nullptr, nullptr};
    return launch_step(p, s, bufs, static_cast<cudaStream_t>(stream));
  });
}

int tfft_partial(tfft_plan p, int stage, int axis, int sign, void* inout, void* stream) {
  return guarded("tfft_partial", [&]() -> int {
    if (!p) return fail(TFFT_EINVAL, "plan is NULL");
    if (int rcb = check_bound(p)) return rcb;
    if (stage < 0 || stage > p->g) return fail(TFFT_EINVAL, "stage out of range");
    if (axis < 0 || axis >= p->d) return fail(TFFT_EINVAL, "axis out of range");
    if (sign != TFFT_FORWARD && sign != TFFT_BACKWARD) return fail(TFFT_EINVAL, "sign must be -1 or +1");
    if (p->st[stage].owner[axis] >= 0) return fail(TFFT_EINVAL, "axis is distributed in this stage");
    if (!p->aplan.count((int)p->cshape[axis]))
      return fail(TFFT_EUNSUPPORTED, "axis length has no transform plan (2/3/5 lengths up to 4096, others up to 2048)");
    int rc = check_ptr(inout, "inout");
    if (rc) return rc;
    Step s = fft_step(p, axis, stage, stage, sign);
    s.src = BUF_IN;
    s.dst = BUF_IN;
    if (sign == TFFT_FORWARD) {
      s.scaled = true;
      s.scale_value = 1.0 / (double)p->cshape[axis];
    }
    void* bufs[4] = {inout, inout, nullptr, nullptr};
    return launch_step(p, s, bufs, static_cast<cudaStream_t>(stream));
  });
}

int tfft_plan_num_launches(tfft_plan p, int sign, int mode, int* n) {
  if (!p || !n) return fail(TFFT_EINVAL, "NULL argument");
  if (!p->transformable) return fail(TFFT_EUNSUPPORTED, "an axis length has no transform plan (2/3/5 lengths up to 4096, others up to 2048)");
  auto it = p->steps.find({sign, mode});
  if (it == p->steps.end()) return fail(TFFT_EINVAL, "bad sign or mode");
  *n = (int)it->second.size();
  return TFFT_OK;
}

int tfft_plan_launch_info(tfft_plan p, int sign, int mode, int index, char* name, int name_len,
                          int64_t* bytes) {
  return guarded("tfft_plan_launch_info", [&]() -> int {
    if (!p || !bytes || (name_len > 0 && !name)) return fail(TFFT_EINVAL, "NULL argument");
    if (!p->transformable) return fail(TFFT_EUNSUPPORTED, "an axis length has no transform plan (2/3/5 lengths up to 4096, others up to 2048)");
    auto it = p->steps.find({sign, mode});
    if (it == p->steps.end()) return fail(TFFT_EINVAL, "bad sign or mode");
    if (index < 0 || index >= (int)it->second.size()) return fail(TFFT_EINVAL, "launch index out of range");
    const Step& s = it->second[index];
    std::string nm;
    int64_t elems = 0;
    if (s.kind == S_REAL) {
      nm = std::string(sign == TFFT_FORWARD ? "fft_r2c_L" : "fft_c2r_L") + std::to_string(2 * p->rplan.L);
      *bytes = p->nreal * (int64_t)sizeof(float) + p->nelems * (int64_t)sizeof(float2);
      if (name_len > 0) {
        std::strncpy(name, nm.c_str(), (size_t)name_len - 1);
        name[name_len - 1] = 0;
      }
      return TFFT_OK;
    }
    if (s.kind == S_BOX) {
      nm = "box_copy";
      elems = s.box_elems;
    } else {
      const AxisPlan& ap = (s.kind == S_CONTIG) ? p->aplan[s.L] : p->aplan_s[s.L];
      const bool tma = s.kind == S_STRIDED && s.tma;
      const bool tc = p->precision != TFFT_FP32 &&
                      ((s.kind == S_CONTIG && tc_supported(ap.L)) ||
                       (tma && tc_strided_supported(s.L, s.tma_E, s.tma_W, p->nelems)));
      nm = std::string(s.kind == S_CONTIG ? "fft_contig" : "fft_strided") +
           (tma ? "_tma" : "") + (tc ? (p->precision == TFFT_TC_BF16X3 ? "_tc_bf16x3" : "_tc_fp16x3") : "") +
           (ap.blue_m ? "_bluestein_L" + std::to_string(ap.L)
                      : ap.spec ? "_L" + std::to_string(ap.L)
                                : ap.E == 0 ? std::string("_generic") : "_E" + std::to_string(ap.E));
      elems = p->nelems;
    }
    *bytes = 2 * elems * (int64_t)sizeof(float2);  // one read and one write of every element
    if (name_len > 0) {
      std::strncpy(name, nm.c_str(), (size_t)name_len - 1);
      name[name_len - 1] = 0;
    }
    return TFFT_OK;
  });
}

int tfft_plan_copy_tasks(tfft_plan p, int sign, int mode, int index, int64_t* tasks, int64_t max_tasks,
                         int64_t* ntasks) {
  return guarded("tfft_plan_copy_tasks", [&]() -> int {
    if (!p || !ntasks || (max_tasks > 0 && !tasks)) return fail(TFFT_EINVAL, "NULL argument");
    auto it = p->steps.find({sign, mode});
    if (it == p->steps.end()) return fail(TFFT_EINVAL, "bad sign or mode");
    if (index < 0 || index >= (int)it->second.size()) return fail(TFFT_EINVAL, "launch index out of range");
    const Step& s = it->second[index];
    if (s.kind != S_BOX) return fail(TFFT_EINVAL, "launch is not a box copy");
    *ntasks = s.ntasks;
    const CopyTask* t = reinterpret_cast<const CopyTask*>(p->image.data() + s.box_off);
    for (int64_t k = 0; k < std::min<int64_t>(max_tasks, s.ntasks); ++k) {
      int64_t* o = tasks + 6 * k;
      o[0] = t[k].src;
      o[1] = t[k].dst;
      o[2] = t[k].ss;
      o[3] = t[k].ds;
      o[4] = t[k].nrows;
      o[5] = t[k].rowlen;
    }
    return TFFT_OK;
  });
}

int tfft_plan_set_wait_limit(tfft_plan p, uint32_t polls) {
  if (!p) return fail(TFFT_EINVAL, "plan is NULL");
  p->wait_limit = polls > 0 ? polls : (1u << 22);
  return TFFT_OK;
}

int tfft_plan_device_status(tfft_plan p, int* status, int reset, void* stream) {
  if (!p || !status) return fail(TFFT_EINVAL, "NULL argument");
  if (int rcb = check_bound(p)) return rcb;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int v = 0;
  cudaError_t e = cudaMemcpyAsync(&v, p->d_state, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess && reset) {
    const int zero = 0;
    e = cudaMemcpyAsync(p->d_state, &zero, sizeof(int), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  }
  if (e != cudaSuccess) return cuda_fail(e, "reading the device status word");
  *status = v;
  return TFFT_OK;
}

int tfft_plan_set_launch_events(tfft_plan p, void* const* events, int count) {
  if (!p) return fail(TFFT_EINVAL, "plan is NULL");
  if (count < 0 || (count > 0 && !events)) return fail(TFFT_EINVAL, "bad events");
  p->events.clear();
  for (int k = 0; k < count; ++k) {
    if (!events[k]) return fail(TFFT_EINVAL, "NULL event");
    p->events.push_back(static_cast<cudaEvent_t>(events[k]));
  }
  return TFFT_OK;
}

static int execute_impl(tfft_plan p, int key, int sign, int mode, const void* in, void* out, void* work,
                        size_t work_bytes, void* stream, const double* coef = nullptr, double factor = 1.0);

int tfft_execute(tfft_plan p, int sign, int mode, const void* in, void* out, void* work,
                 size_t work_bytes, void* stream) {
  return guarded("tfft_execute", [&]() -> int {
    return execute_impl(p, sign, sign, mode, in, out, work, work_bytes, stream);
  });
}

int tfft_adjoint(tfft_plan p, int mode, const void* in, void* out, void* work, size_t work_bytes,
                 const double* d_coef, void* stream) {
  return guarded("tfft_adjoint", [&]() -> int {
    if (p && p->kind != TFFT_C2C) return fail(TFFT_EUNSUPPORTED, "the adjoint is built for complex-to-complex plans");
    if (d_coef && (reinterpret_cast<uintptr_t>(d_coef) & 7)) return fail(TFFT_EINVAL, "d_coef is misaligned");
    return execute_impl(p, kAdjoint, TFFT_BACKWARD, mode, in, out, work, work_bytes, stream, d_coef);
  });
}

int tfft_weighted_energy_grad(tfft_plan p, int mode, const void* u, void* out, void* work, size_t work_bytes,
                              const double* d_g, void* stream) {
  return guarded("tfft_weighted_energy_grad", [&]() -> int {
    if (p && p->kind != TFFT_C2C) return fail(TFFT_EUNSUPPORTED, "the adjoint is built for complex-to-complex plans");
    if (d_g && (reinterpret_cast<uintptr_t>(d_g) & 7)) return fail(TFFT_EINVAL, "d_g is misaligned");
    // d/dRe x + i d/dIm x of g sum |F(x) w|^2 = 2 g F^H (w^2 F x): the factor 2
    // joins the adjoint's own scale on its last pass, g is read there on the device
    return execute_impl(p, kAdjoint, TFFT_BACKWARD, mode, u, out, work, work_bytes, stream, d_g, 2.0);
  });
}

// ---------------------------------------------------------------- host buffers

namespace {

constexpr int kHostSetBufs = 4;  // per buffer set: input, intermediate, output, workspace

size_t host_buf_bytes(tfft_plan p) { return align_up((size_t)p->nelems * sizeof(float2), 256); }

int ensure_host_io(tfft_plan p) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  auto& io = p->io;
  if (io.device >= 0) {
    if (io.device != dev) return fail(TFFT_EINVAL, "tfft_execute_host: called on another device than before");
    return TFFT_OK;
  }
  io.device = dev;
  e = cudaStreamCreateWithFlags(&io.cin, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&io.cout, cudaStreamNonBlocking);
  for (cudaEvent_t* ev : {&io.in_done[0], &io.in_done[1], &io.comp_done[0], &io.comp_done[1], &io.out_done[0],
                          &io.out_done[1], &io.start, &io.end})
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
  if (e != cudaSuccess) return cuda_fail(e, "tfft_execute_host: stream / event creation");
  return TFFT_OK;
}

int check_pinned(const void* ptr, const char* name) {
  if (!ptr) return fail(TFFT_EINVAL, std::string(name) + " has a NULL entry");
  cudaPointerAttributes a;
  cudaError_t e = cudaPointerGetAttributes(&a, ptr);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(TFFT_EINVAL, std::string(name) + ": not a CUDA-registered pointer");
  }
  if (a.type != cudaMemoryTypeHost)
    return fail(TFFT_EINVAL, std::string(name) + " must be page-locked host memory (cudaHostAlloc / pinned)");
  return TFFT_OK;
}

}  // namespace

int tfft_host_space_bytes(tfft_plan p, size_t* bytes) {
  if (!p || !bytes) return fail(TFFT_EINVAL, "NULL argument");
  *bytes = 2 * kHostSetBufs * host_buf_bytes(p);
  return TFFT_OK;
}

int tfft_execute_host(tfft_plan p, int nsigns, const int* signs, int count, const void* const* h_in,
                      void* const* h_out, void* d_space, size_t space_bytes, void* stream) {
  return guarded("tfft_execute_host", [&]() -> int {
    if (!p) return fail(TFFT_EINVAL, "plan is NULL");
    if (int rcb = check_bound(p)) return rcb;
    if (nsigns < 1 || !signs) return fail(TFFT_EINVAL, "need at least one transform direction");
    for (int j = 0; j < nsigns; ++j) {
      if (signs[j] != TFFT_FORWARD && signs[j] != TFFT_BACKWARD) return fail(TFFT_EINVAL, "sign must be -1 or +1");
      if (j > 0 && signs[j] == signs[j - 1])
        return fail(TFFT_EINVAL, "directions must alternate (a forward leaves stage g, a backward stage 0)");
    }
    if (count < 0 || (count > 0 && (!h_in || !h_out))) return fail(TFFT_EINVAL, "bad host buffer lists");
    int rc = check_ptr(d_space, "d_space");
    if (rc) return rc;
    const size_t B = host_buf_bytes(p);
    if (space_bytes < 2 * kHostSetBufs * B) return fail(TFFT_EWORKSPACE, "d_space smaller than tfft_host_space_bytes");
    for (int k = 0; k < count; ++k) {
      if ((rc = check_pinned(h_in[k], "h_in")) || (rc = check_pinned(h_out[k], "h_out"))) return rc;
    }
    if (count == 0) return TFFT_OK;
    if ((rc = ensure_host_io(p))) return rc;
    auto& io = p->io;
    const bool r2c = p->kind == TFFT_R2C;
    const size_t cbytes = (size_t)p->nelems * sizeof(float2), rbytes = (size_t)p->nreal * sizeof(float);
    const size_t in_bytes = (r2c && signs[0] == TFFT_FORWARD) ? rbytes : cbytes;
    const size_t out_bytes = (r2c && signs[nsigns - 1] == TFFT_BACKWARD) ? rbytes : cbytes;
    cudaStream_t cs = static_cast<cudaStream_t>(stream);
    auto ok = [](cudaError_t e) { return e == cudaSuccess; };
    cudaError_t e = cudaEventRecord(io.start, cs);  // after the caller's earlier work
    if (ok(e)) e = cudaStreamWaitEvent(io.cin, io.start, 0);
    if (ok(e)) e = cudaStreamWaitEvent(io.cout, io.start, 0);
    // array k uses buffer set k % 2: its copy-in overlaps the transform of array
    // k - 1 and the copy-out of array k - 2
    for (int k = 0; k < count && ok(e); ++k) {
      const int s = k & 1;
      char* base = static_cast<char*>(d_space) + (size_t)s * kHostSetBufs * B;
      char* bin = base;
      char* bmid = base + B;
      char* bout = base + 2 * B;
      char* bwork = base + 3 * B;
      if (k >= 2) e = cudaStreamWaitEvent(io.cin, io.comp_done[s], 0);  // array k-2 is done with bin
      if (ok(e)) e = cudaMemcpyAsync(bin, h_in[k], in_bytes, cudaMemcpyHostToDevice, io.cin);
      if (ok(e)) e = cudaEventRecord(io.in_done[s], io.cin);
      if (ok(e)) e = cudaStreamWaitEvent(cs, io.in_done[s], 0);
      if (ok(e) && k >= 2) e = cudaStreamWaitEvent(cs, io.out_done[s], 0);  // bout copied out
      if (!ok(e)) break;
      char* src = bin;
      for (int j = 0; j < nsigns; ++j) {
        char* dst = (j == nsigns - 1) ? bout : ((j % 2 == 0) ? bmid : bin);
        rc = execute_impl(p, signs[j], signs[j], TFFT_MODE_FUSED, src, dst, bwork, B, stream);
        if (rc) return rc;
        src = dst;
      }
      e = cudaEventRecord(io.comp_done[s], cs);
      if (ok(e)) e = cudaStreamWaitEvent(io.cout, io.comp_done[s], 0);
      if (ok(e)) e = cudaMemcpyAsync(h_out[k], bout, out_bytes, cudaMemcpyDeviceToHost, io.cout);
      if (ok(e)) e = cudaEventRecord(io.out_done[s], io.cout);
    }
    if (ok(e)) e = cudaEventRecord(io.end, io.cout);
    if (ok(e)) e = cudaStreamWaitEvent(cs, io.end, 0);  // the caller's stream sees the copied results
    if (!ok(e)) return cuda_fail(e, "tfft_execute_host");
    return TFFT_OK;
  });
}

int tfft_weighted_energy(tfft_plan p, int stage, const void* y, const float* w, double* d_loss, void* u,
                         void* stream) {
  return guarded("tfft_weighted_energy", [&]() -> int {
    if (!p) return fail(TFFT_EINVAL, "plan is NULL");
    if (int rcb = check_bound(p)) return rcb;
    if (stage < 0 || stage > p->g) return fail(TFFT_EINVAL, "stage out of range");
    int rc = check_ptr(y, "y");
    if (rc) return rc;
    if (!w || (reinterpret_cast<uintptr_t>(w) & 15)) return fail(TFFT_EALIGN, "w is NULL or not 16-byte aligned");
    if (!d_loss || (reinterpret_cast<uintptr_t>(d_loss) & 7)) return fail(TFFT_EINVAL, "d_loss is NULL or misaligned");
    if (u && (rc = check_ptr(u, "u"))) return rc;
    cudaError_t e = launch_weighted_energy(static_cast<const float2*>(y), w, p->st[stage].total,
                                           reinterpret_cast<double*>(p->d_state + p->red_off), kReductionParts,
                                           d_loss, static_cast<float2*>(u), static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
    return TFFT_OK;
  });
}

int tfft_weight_scale(tfft_plan p, int stage, const void* y, const float* w, const double* d_coef, double scale,
                      void* z, void* stream) {
  return guarded("tfft_weight_scale", [&]() -> int {
    if (!p) return fail(TFFT_EINVAL, "plan is NULL");
    if (int rcb = check_bound(p)) return rcb;
    if (stage < 0 || stage > p->g) return fail(TFFT_EINVAL, "stage out of range");
    int rc = check_ptr(y, "y");
    if (rc) return rc;
    rc = check_ptr(z, "z");
    if (rc) return rc;
    if (!w || (reinterpret_cast<uintptr_t>(w) & 15)) return fail(TFFT_EALIGN, "w is NULL or not 16-byte aligned");
    cudaError_t e = launch_weight_scale(static_cast<const float2*>(y), w, d_coef, scale, p->st[stage].total,
                                        static_cast<float2*>(z), static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
    return TFFT_OK;
  });
}

static int execute_impl(tfft_plan p, int key, int sign, int mode, const void* in, void* out, void* work,
                        size_t work_bytes, void* stream, const double* coef, double factor) {
  if (!p) return fail(TFFT_EINVAL, "plan is NULL");
  if (int rcb = check_bound(p)) return rcb;
  if (sign != TFFT_FORWARD && sign != TFFT_BACKWARD) return fail(TFFT_EINVAL, "sign must be -1 or +1");
  if (mode < TFFT_MODE_FUSED || mode > TFFT_MODE_PACKED) return fail(TFFT_EINVAL, "unknown mode");
  if (!p->transformable) return fail(TFFT_EUNSUPPORTED, "an axis length has no transform plan (2/3/5 lengths up to 4096, others up to 2048)");
  int rc = check_ptr(in, "in");
  if (rc) return rc;
  rc = check_ptr(out, "out");
  if (rc) return rc;
  const size_t stage = (size_t)p->nelems * sizeof(float2);
  const bool r2c = p->kind == TFFT_R2C;
  const size_t real_bytes = (size_t)p->nreal * sizeof(float);
  const size_t in_bytes = (r2c && sign == TFFT_FORWARD) ? real_bytes : stage;
  const size_t out_bytes = (r2c && sign == TFFT_BACKWARD) ? real_bytes : stage;
  {
    const char* a = static_cast<const char*>(in);
    const char* b = static_cast<const char*>(out);
    if (a < b + out_bytes && b < a + in_bytes) return fail(TFFT_EINVAL, "in and out overlap");
  }
  std::vector<Step> steps = p->steps[{key, mode}];
  if (coef || factor != 1.0) {  // device coefficient and host factor go on the last transform pass
    int k = (int)steps.size() - 1;
    while (k >= 0 && steps[k].kind == S_BOX) --k;
    if (k < 0 || steps[k].kind != S_CONTIG)
      return fail(TFFT_EUNSUPPORTED, "a device coefficient needs a contiguous last pass");
    steps[k].coef = coef;
    steps[k].scale_value = (steps[k].scaled ? steps[k].scale_value : 1.0) * factor;
    steps[k].scaled = true;
  }
  void* w0 = nullptr;
  void* w1 = nullptr;
  bool destroy = false;
  if (mode == TFFT_MODE_FUSED) {
    if (work) {
      rc = check_ptr(work, "work");
      if (rc) return rc;
      if (work_bytes < stage) return fail(TFFT_EWORKSPACE, "fused workspace must hold one stage buffer");
      w0 = work;
    } else if (r2c) {
      return fail(TFFT_EWORKSPACE, "real-to-complex plans need a workspace of one complex stage buffer");
    } else {
      destroy = true;
    }
    // a complex-to-real backward uses its input as scratch
    if (r2c && sign == TFFT_BACKWARD) destroy = true;
  } else {
    if (!work || work_bytes < 2 * stage)
      return fail(TFFT_EWORKSPACE, "this mode needs a workspace of two stage buffers");
    rc = check_ptr(work, "work");
    if (rc) return rc;
    w0 = work;
    w1 = static_cast<char*>(work) + stage;
  }
  if (work) {
    const char* a = static_cast<const char*>(work);
    const size_t wb = (mode == TFFT_MODE_FUSED) ? stage : 2 * stage;
    const void* ptrs[2] = {in, out};
    const size_t sizes[2] = {in_bytes, out_bytes};
    for (int k = 0; k < 2; ++k) {
      const char* b = static_cast<const char*>(ptrs[k]);
      if (a < b + sizes[k] && b < a + wb) return fail(TFFT_EINVAL, "work overlaps in or out");
    }
  }
  assign_buffers(steps, destroy);
  if (!p->events.empty() && p->events.size() < steps.size() + 1)
    return fail(TFFT_EINVAL, "fewer launch events than launches + 1");
  void* bufs[4] = {const_cast<void*>(in), out, w0, w1};
  return run_steps(p, steps, bufs, static_cast<cudaStream_t>(stream));
}

}  // extern "C"

// ============================================================== batch

namespace {

struct BatchSegH {
  int t, pass, kind, L, prev;
  int64_t ntiles;
  size_t cb_cap;  // column-block slots reserved (strided)
};

// Issue order of the (transform, pass) segments: pass-major (every
// transform's first pass, then every second pass, ...).  Items are taken in
// this order, so a pass's producer was queued a whole round of passes
// earlier and its waits are rare.  Orders that queue a transform's next pass
// sooner, for L2 reuse, measured slower on the 48-transform workload: the
// waits cost more than the reuse saves.
std::vector<std::pair<int, int>> batch_order(const std::vector<std::vector<Step>>& steps) {
  size_t maxpass = 0;
  for (const auto& v : steps) maxpass = std::max(maxpass, v.size());
  std::vector<std::pair<int, int>> order;
  for (size_t pass = 0; pass < maxpass; ++pass)
    for (size_t t = 0; t < steps.size(); ++t)
      if (pass < steps[t].size()) order.emplace_back((int)t, (int)pass);
  return order;
}

}  // namespace

struct tfft_batch_s {
  int sign = TFFT_FORWARD;
  std::vector<tfft_plan> plans;
  std::vector<std::vector<Step>> steps;       // per transform, fused, buffers assigned at bind
  std::vector<BatchSegH> segs;                // in issue order (batch_order)
  std::map<std::pair<int, int>, int> choice;  // (kind, L) -> executor variant
  std::vector<void*> ins, outs, works;
  char* d_state = nullptr;
  size_t state_bytes = 0, ctr_off = 0, seg_off = 0, cb_off = 0, map_off = 0;  // map_off: 2 tensor maps per segment
  int64_t nitems = 0;
  long long spin_limit = 4000000000LL;  // clock cycles (~2 s at 2 GHz)
};

namespace {

// Executor variants for passes of (kind, L); the first is the default
// before autotuning: TMA-staged strided variants lead (measured faster on
// the 48-transform batch, and a segment that cannot use them falls back to
// the first plain variant by itself).
std::vector<int> batch_candidates(int kind, int L) {
  std::vector<int> tma, plain;
  for (int id = 0; id < batch_num_variants(); ++id) {
    int k, l, e, bw;
    AxisPlan ap{};
    if (batch_variant(id, k, l, e, bw, ap) && k == kind && l == L)
      (batch_variant_tma(id) ? tma : plain).push_back(id);
  }
  tma.insert(tma.end(), plain.begin(), plain.end());
  return tma;
}


// Items, segment table and column blocks for the current variant choices,
// written into the bound state buffer.
int batch_upload(tfft_batch b, cudaStream_t st) {
  const int nseg = (int)b->segs.size();
  std::vector<uint8_t> img(b->state_bytes, 0);
  std::vector<BatchSeg> dsegs(nseg);
  size_t cb = b->cb_off;
  int64_t first = 0;
  for (int i = 0; i < nseg; ++i) {
    BatchSegH& h = b->segs[i];
    tfft_plan p = b->plans[h.t];
    const Step& s = b->steps[h.t][h.pass];
    int v = b->choice[{h.kind, h.L}];
    int k, l, e, bw;
    AxisPlan ap{};
    batch_variant(v, k, l, e, bw, ap);
    void* bufs[4] = {b->ins[h.t], b->outs[h.t], b->works[h.t], nullptr};
    // a TMA variant needs equal blocks and aligned columns in both layouts;
    // other segments of the same length take the first plain variant
    TmaGeo gin{}, gout{};
    bool tma = false;
    if (batch_variant_tma(v)) {
      tma = p->use_tma && tma_geo(p, s.lin, s.axis, bw, gin) && tma_geo(p, s.lout, s.axis, bw, gout);
      if (tma) {
        alignas(64) CUtensorMap maps[2];
        tma = encode_stage_map(p, gin, s.axis, bw, bufs[s.src], &maps[0]) &&
              encode_stage_map(p, gout, s.axis, bw, bufs[s.dst], &maps[1]);
        if (tma) std::memcpy(img.data() + b->map_off + (size_t)i * sizeof(maps), maps, sizeof(maps));
      }
      if (!tma) {
        for (int c : batch_candidates(h.kind, h.L))
          if (!batch_variant_tma(c)) {
            v = c;
            break;
          }
        batch_variant(v, k, l, e, bw, ap);
      }
    }
    BatchSeg& D = dsegs[i];
    std::memset(&D, 0, sizeof(D));
    D.kind = h.kind;
    D.variant = v;
    D.prev = h.prev;
    D.transform = h.t;
    D.first = first;
    const float scale = s.scaled ? (float)s.scale_value : 1.0f;
    int* status = reinterpret_cast<int*>(b->d_state);
    if (s.kind == S_CONTIG) {
      ContigArgs& a = D.ca;
      a.in = static_cast<const float2*>(bufs[s.src]);
      a.out = static_cast<float2*>(bufs[s.dst]);
      a.nlines = s.nlines;
      a.ap = ap;
      a.tw = reinterpret_cast<const float2*>(p->d_state + p->tw_off[s.L]);
      a.lines_per_cta = bw;
      a.sign = s.sign;
      a.scale = scale;
      a.status = status;
      D.ntiles = (s.nlines + bw - 1) / bw;
    } else {
      StridedArgs& a = D.sa;
      a.in = static_cast<const float2*>(bufs[s.src]);
      a.out = static_cast<float2*>(bufs[s.dst]);
      a.lin = dev_layout(p, p->st[s.lin]);
      a.lout = dev_layout(p, p->st[s.lout]);
      a.d = p->d;
      a.axis = s.axis;
      a.ap = ap;
      a.tw = reinterpret_cast<const float2*>(p->d_state + p->tw_off[s.L]);
      std::vector<int2> blocks = colblock_list(p, s.lin, s.lout, bw);
      if (blocks.size() > h.cb_cap) return fail(TFFT_EINVAL, "batch: column-block capacity exceeded");
      std::memcpy(img.data() + cb, blocks.data(), blocks.size() * sizeof(int2));
      a.colblocks = reinterpret_cast<const int2*>(b->d_state + cb);
      a.ncolblocks = (int64_t)blocks.size();
      a.outer_fastest = 0;
      cb += align_up(h.cb_cap * sizeof(int2), 256);
      int oax[2] = {-1, -1}, no = 0;
      int64_t nouter = 1;
      for (int m = 0; m < p->d - 1; ++m)
        if (m != s.axis) {
          oax[no++] = m;
          nouter *= p->cshape[m];
        }
      a.nouter = nouter;
      a.oax0 = oax[0];
      a.oax1 = oax[1];
      a.on1 = oax[1] >= 0 ? p->cshape[oax[1]] : 1;
      a.W = bw;
      a.sign = s.sign;
      a.scale = scale;
      a.status = status;
      D.ntiles = nouter * a.ncolblocks;
      if (tma) {
        D.tma = 1;
        D.gin = gin;
        D.gout = gout;
        D.tin = b->d_state + b->map_off + (size_t)i * 2 * sizeof(CUtensorMap);
        D.tout = b->d_state + b->map_off + ((size_t)i * 2 + 1) * sizeof(CUtensorMap);
      }
    }
    // items of about 32K elements: small tiles are grouped so that the queue,
    // the lookup and the completion fence are paid once per ~512 KB moved
    // (measured on the 48-transform batch: 8K / 16K / 32K / 64K / 128K
    // elements per item gave 2.77 / 2.56 / 2.49 / 2.53 / 2.60 ms)
    const int64_t tile_elems = (int64_t)bw * s.L;
    D.per_item = std::max<int64_t>(1, std::min<int64_t>(16, 32768 / std::max<int64_t>(1, tile_elems)));
    D.nitems = (D.ntiles + D.per_item - 1) / D.per_item;
    h.ntiles = D.ntiles;
    first += D.nitems;
  }
  b->nitems = first;
  std::memcpy(img.data() + b->seg_off, dsegs.data(), dsegs.size() * sizeof(BatchSeg));
  cudaError_t e = cudaMemcpyAsync(b->d_state, img.data(), img.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "batch state upload");
  return TFFT_OK;
}

int batch_launch(tfft_batch b, cudaStream_t st) {
  const size_t ctr_bytes = align_up(16 + b->segs.size() * sizeof(int), 256);
  cudaError_t e = cudaMemsetAsync(b->d_state + b->ctr_off, 0, ctr_bytes, st);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync (batch counters)");
  BatchArgs a;
  a.segs = reinterpret_cast<const BatchSeg*>(b->d_state + b->seg_off);
  a.nsegs = (int)b->segs.size();
  a.nitems = b->nitems;
  a.head = reinterpret_cast<unsigned long long*>(b->d_state + b->ctr_off);
  a.abort = reinterpret_cast<int*>(b->d_state + b->ctr_off + 8);
  a.done = reinterpret_cast<int*>(b->d_state + b->ctr_off + 16);
  a.status = reinterpret_cast<int*>(b->d_state);
  a.spin_limit = b->spin_limit;
  int grid = batch_grid();
  if (grid > b->nitems) grid = (int)std::max<int64_t>(1, b->nitems);
  e = launch_batch(a, grid, st);
  if (e != cudaSuccess) return cuda_fail(e, "batch launch");
  return TFFT_OK;
}

}  // namespace

extern "C" {

int tfft_batch_create(tfft_batch* out, int count, const tfft_plan* plans, int sign) {
  return guarded("tfft_batch_create", [&]() -> int {
    if (!out) return fail(TFFT_EINVAL, "batch is NULL");
    *out = nullptr;
    if (count < 1 || !plans) return fail(TFFT_EINVAL, "need at least one plan");
    if (sign != TFFT_FORWARD && sign != TFFT_BACKWARD) return fail(TFFT_EINVAL, "sign must be -1 or +1");
    auto b = new tfft_batch_s();
    b->sign = sign;
    for (int t = 0; t < count; ++t) {
      tfft_plan p = plans[t];
      if (!p || !p->transformable || p->kind != TFFT_C2C || p->nelems >= (int64_t(1) << 31)) {
        delete b;
        return fail(TFFT_EUNSUPPORTED, "batch plans must be complex-to-complex, transformable, < 2^31 elements");
      }
      b->plans.push_back(p);
      b->steps.push_back(p->steps[{sign, TFFT_MODE_FUSED}]);
      for (const Step& s : b->steps.back()) {
        const int kind = s.kind == S_CONTIG ? 0 : 1;
        if ((s.kind != S_CONTIG && s.kind != S_STRIDED) || batch_candidates(kind, s.L).empty()) {
          delete b;
          return fail(TFFT_EUNSUPPORTED, "batch: no executor tile for a pass of length " + std::to_string(s.L));
        }
        if (!b->choice.count({kind, s.L})) b->choice[{kind, s.L}] = batch_candidates(kind, s.L)[0];
      }
    }
    // segments in issue order (see batch_order); column-block capacity for the
    // narrowest candidate
    std::vector<std::vector<int>> idx(count);
    size_t cb_total = 0;
    for (const auto& tp : batch_order(b->steps)) {
      const int t = tp.first, pass = tp.second;
      const Step& s = b->steps[t][pass];
      BatchSegH h;
      h.t = t;
      h.pass = pass;
      h.kind = s.kind == S_CONTIG ? 0 : 1;
      h.L = s.L;
      h.prev = pass > 0 ? idx[t][pass - 1] : -1;
      h.ntiles = 0;
      h.cb_cap = 0;
      if (h.kind == 1)
        for (int v : batch_candidates(1, s.L)) {
          int k, l, e, bw;
          AxisPlan ap{};
          batch_variant(v, k, l, e, bw, ap);
          h.cb_cap = std::max(h.cb_cap, colblock_list(b->plans[t], s.lin, s.lout, bw).size());
        }
      cb_total += align_up(h.cb_cap * sizeof(int2), 256);
      idx[t].push_back((int)b->segs.size());
      b->segs.push_back(h);
    }
    b->ctr_off = 256;
    b->seg_off = b->ctr_off + align_up(16 + b->segs.size() * sizeof(int), 256);
    b->cb_off = b->seg_off + align_up(b->segs.size() * sizeof(BatchSeg), 256);
    b->map_off = b->cb_off + align_up(cb_total, 256);
    b->state_bytes = b->map_off + b->segs.size() * 2 * sizeof(CUtensorMap);
    b->ins.assign(count, nullptr);
    b->outs.assign(count, nullptr);
    b->works.assign(count, nullptr);
    *out = b;
    return TFFT_OK;
  });
}

int tfft_batch_segment(tfft_batch b, int index, int* transform, int* pass) {
  if (!b || !transform || !pass) return fail(TFFT_EINVAL, "NULL argument");
  if (index < 0 || index >= (int)b->segs.size()) return fail(TFFT_EINVAL, "segment index out of range");
  *transform = b->segs[index].t;
  *pass = b->segs[index].pass;
  return TFFT_OK;
}

int tfft_batch_destroy(tfft_batch b) {
  if (!b) return fail(TFFT_EINVAL, "batch is NULL");
  delete b;
  return TFFT_OK;
}

int tfft_batch_state_bytes(tfft_batch b, size_t* bytes) {
  if (!b || !bytes) return fail(TFFT_EINVAL, "NULL argument");
  *bytes = b->state_bytes;
  return TFFT_OK;
}

int tfft_batch_bind(tfft_batch b, void* d_state, size_t bytes, const void* const* ins, void* const* outs,
                    void* const* works, void* stream) {
  return guarded("tfft_batch_bind", [&]() -> int {
    if (!b || !ins || !outs) return fail(TFFT_EINVAL, "NULL argument");
    int rc = check_ptr(d_state, "d_state");
    if (rc) return rc;
    if (reinterpret_cast<uintptr_t>(d_state) & 255)
      return fail(TFFT_EALIGN, "batch state must be 256-byte aligned (it holds tensor maps)");
    if (bytes < b->state_bytes) return fail(TFFT_EINVAL, "batch state buffer too small");
    const int n = (int)b->plans.size();
    for (int t = 0; t < n; ++t) {
      tfft_plan p = b->plans[t];
      if (!p->d_state) return fail(TFFT_ESTATE, "every plan of the batch must be bound first");
      if ((rc = check_ptr(ins[t], "in"))) return rc;
      if ((rc = check_ptr(outs[t], "out"))) return rc;
      b->ins[t] = const_cast<void*>(ins[t]);
      b->outs[t] = outs[t];
      b->works[t] = works ? works[t] : nullptr;
      if (b->works[t] && (rc = check_ptr(b->works[t], "work"))) return rc;
      b->steps[t] = p->steps[{b->sign, TFFT_MODE_FUSED}];
      assign_buffers(b->steps[t], b->works[t] == nullptr);
    }
    b->d_state = static_cast<char*>(d_state);
    return batch_upload(b, static_cast<cudaStream_t>(stream));
  });
}

int tfft_batch_execute(tfft_batch b, void* stream) {
  return guarded("tfft_batch_execute", [&]() -> int {
    if (!b) return fail(TFFT_EINVAL, "batch is NULL");
    if (!b->d_state) return fail(TFFT_ESTATE, "batch is not bound");
    return batch_launch(b, static_cast<cudaStream_t>(stream));
  });
}

int tfft_batch_num_items(tfft_batch b, int64_t* items, int* segments) {
  if (!b || !items || !segments) return fail(TFFT_EINVAL, "NULL argument");
  *items = b->nitems;
  *segments = (int)b->segs.size();
  return TFFT_OK;
}

int tfft_batch_variant(tfft_batch b, int kind, int L, int* variant) {
  if (!b || !variant) return fail(TFFT_EINVAL, "NULL argument");
  auto it = b->choice.find({kind, L});
  if (it == b->choice.end()) return fail(TFFT_EINVAL, "no pass of that kind and length in the batch");
  *variant = it->second;
  return TFFT_OK;
}

int tfft_batch_autotune(tfft_batch b, int reps, void* stream) {
  return guarded("tfft_batch_autotune", [&]() -> int {
    if (!b) return fail(TFFT_EINVAL, "batch is NULL");
    if (!b->d_state) return fail(TFFT_ESTATE, "batch is not bound");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (reps < 1) reps = 3;
    // cached choices: lines "kind L variant" in $TFFT_AUTOTUNE_CACHE
    const char* cache = std::getenv("TFFT_AUTOTUNE_CACHE");
    std::map<std::pair<int, int>, int> cached;
    if (cache) {
      if (FILE* f = std::fopen(cache, "r")) {
        int k, l, v;
        while (std::fscanf(f, "%d %d %d", &k, &l, &v) == 3) cached[{k, l}] = v;
        std::fclose(f);
      }
    }
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
      return fail(TFFT_ECUDA, "cudaEventCreate");
    int rc = TFFT_OK;
    for (auto& kv : b->choice) {
      const std::vector<int> cands = batch_candidates(kv.first.first, kv.first.second);
      auto hit = cached.find(kv.first);
      if (hit != cached.end() && std::find(cands.begin(), cands.end(), hit->second) != cands.end()) {
        kv.second = hit->second;
        continue;
      }
      if (cands.size() < 2) continue;
      float best = 1e30f;
      int best_v = kv.second;
      for (int v : cands) {
        kv.second = v;
        if ((rc = batch_upload(b, st))) break;
        if ((rc = batch_launch(b, st))) break;  // warm-up
        cudaEventRecord(e0, st);
        for (int r = 0; r < reps && !rc; ++r) rc = batch_launch(b, st);
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) {
          best = ms;
          best_v = v;
        }
      }
      kv.second = best_v;
      if (rc) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    if (cache) {
      if (FILE* f = std::fopen(cache, "w")) {
        for (auto& kv : b->choice) std::fprintf(f, "%d %d %d\n", kv.first.first, kv.first.second, kv.second);
        std::fclose(f);
      }
    }
    return batch_upload(b, st);
  });
}

int tfft_batch_set_variant(tfft_batch b, int kind, int L, int variant, void* stream) {
  return guarded("tfft_batch_set_variant", [&]() -> int {
    if (!b) return fail(TFFT_EINVAL, "batch is NULL");
    if (!b->d_state) return fail(TFFT_ESTATE, "batch is not bound");
    auto it = b->choice.find({kind, L});
    if (it == b->choice.end()) return fail(TFFT_EINVAL, "the batch has no pass of that kind and length");
    const std::vector<int> cands = batch_candidates(kind, L);
    if (std::find(cands.begin(), cands.end(), variant) == cands.end())
      return fail(TFFT_EINVAL, "not a compiled variant for that kind and length");
    it->second = variant;
    return batch_upload(b, static_cast<cudaStream_t>(stream));
  });
}

int tfft_batch_set_wait_limit(tfft_batch b, long long cycles) {
  if (!b) return fail(TFFT_EINVAL, "batch is NULL");
  b->spin_limit = cycles > 0 ? cycles : 4000000000LL;
  return TFFT_OK;
}

int tfft_batch_device_status(tfft_batch b, int* status, int reset, void* stream) {
  if (!b || !status) return fail(TFFT_EINVAL, "NULL argument");
  if (!b->d_state) return fail(TFFT_ESTATE, "batch is not bound");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int v = 0;
  cudaError_t e = cudaMemcpyAsync(&v, b->d_state, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess && reset) {
    const int zero = 0;
    e = cudaMemcpyAsync(b->d_state, &zero, sizeof(int), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  }
  if (e != cudaSuccess) return cuda_fail(e, "reading the batch status word");
  *status = v;
  return TFFT_OK;
}

}  // extern "C"
