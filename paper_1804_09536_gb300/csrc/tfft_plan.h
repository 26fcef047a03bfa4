// Host-side plan objects of the C ABI (include/tfft.h), shared by its
// translation units: tfft_plan.cpp (plan creation, layouts, per-length FFT
// plans, Bluestein tables, queries, binding), tfft_exchange.cpp (subarray
// boxes of the exchange and their copy tasks, Alg. 2 / Alg. 3),
// tfft_tmageo.cpp (tile geometry and tensor maps of the TMA passes),
// tfft_exec.cpp (pass lists, launches, execute / adjoint / partial / loss
// calls), tfft_hostio.cpp (transforms of page-locked host arrays) and
// tfft_batch_host.cpp (the batched executor).
#pragma once

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <map>
#include <mutex>
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

namespace tfft {
namespace host {

// Error status with a message for tfft_last_error() (per thread).
int fail(int code, const std::string& msg);
int cuda_fail(cudaError_t e, const char* what);

// Eq. decompose / Alg. 1.
void decompose(int64_t N, int64_t M, int64_t p, int64_t& n, int64_t& s);

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

struct LayoutH {
  int d = 0;
  int64_t N[MAXD] = {0, 0, 0, 0};
  int owner[MAXD] = {-1, -1, -1, -1};
  int nranks = 0;
  std::vector<int64_t> start, size, offset;  // nranks * d, nranks * d, nranks
  int64_t total = 0;
  size_t state_off = 0;  // rank offset table in the state image (bytes)
  // > 0: every rank's innermost axis is stored `pitch` elements apart (a
  // padded internal copy of a stage; the public stage buffers have none)
  int64_t pitch = 0;
};

enum StepKind { S_CONTIG, S_STRIDED, S_BOX, S_REAL };
constexpr int kAdjoint = 2;  // key of the adjoint's step list
enum BufId { BUF_IN, BUF_OUT, BUF_W0, BUF_W1 };

// One rank group of an uneven stage layout (see RankGroupGeo): the element
// offset of its first rank, the merged extent of the axes after axis 0, the
// offsets between consecutive ranks along its two rank dimensions and their
// extents.
struct RankGroupH {
  int64_t base = 0, inner = 0, s1 = 0, s0 = 0;
  int ext1 = 1, ext0 = 1;
};

// A tensor map described on the host: base element offset inside its buffer,
// extents and byte strides of the 5-D view, and the box of one copy.
struct TmaMapH {
  int64_t base = 0;
  uint64_t dims[5] = {1, 1, 1, 1, 1};
  uint64_t strides[4] = {0, 0, 0, 0};
  uint32_t box[5] = {1, 1, 1, 1, 1};
};

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
  // tensor-core TMA pass (TFFT_TC_* plans): its variant, column blocks and geometry
  bool tc = false;
  int tc_E = 0, tc_W = 0;
  size_t tc_cb_off = 0;
  int64_t tc_ncb = 0;
  bool tc_outer_fastest = false;
  TmaGeo tc_gin{}, tc_gout{};
  // TMA pass over the rank groups of an uneven layout (in place along axis 0)
  bool tma_groups = false;
  RankGroupGeo rg{};
  std::vector<RankGroupH> rgh;
  // TMA pass over one column window [win_c0, win_c0 + win_nc) of the
  // innermost axis (the columns whose ranks are TMA-describable on both
  // sides); the other columns run as the next step, which is marked `cont`
  bool tma_win = false;
  int64_t win_c0 = 0, win_nc = 0;
  TmaMapH win_min{}, win_mout{};
  // this step runs on the previous step's buffers (the rest of its columns)
  bool cont = false;
  int64_t ncols = -1;  // columns of the innermost axis the step covers (-1: all)
  // element shifts of the input / output pointers (a padded internal buffer
  // starts its rows `pad_lead` elements in) and the complex row pitch of a
  // real pass (0: L + 1)
  int64_t in_shift = 0, out_shift = 0;
  int64_t cpitch = 0;
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

}  // namespace host
}  // namespace tfft

using namespace tfft;
using namespace tfft::host;

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
  // real-to-complex plans whose gathering pass along axis d - 2 runs
  // TMA-staged over a column window: the complex stage-0 buffer of the fused
  // path (internal) is stored with rows `pitch` elements apart, starting
  // `pad_lead` elements in, as layout st[pad_stage]; -1 when not padded
  int pad_stage = -1;
  int64_t pad_lead = 0;
  int64_t win_c0 = 0, win_nc = 0;  // the TMA column window of that pass
  int win_E = 0, win_W = 0;        // its TMA variant
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
  // Graphs of repeated executes: a call that repeats an earlier one (same
  // direction, mode, buffers, device coefficient, factor and wait limit)
  // replays the launches captured the second time they were requested (at
  // most kGraphCache per plan, least recently used dropped).
  struct GraphKey {
    int key = 0, mode = 0;
    const void* in = nullptr;
    const void* out = nullptr;
    const void* w0 = nullptr;
    const void* w1 = nullptr;
    const double* coef = nullptr;
    double factor = 1.0;
    uint32_t wait_limit = 0;
    bool operator<(const GraphKey& o) const {
      return std::tie(key, mode, in, out, w0, w1, coef, factor, wait_limit) <
             std::tie(o.key, o.mode, o.in, o.out, o.w0, o.w1, o.coef, o.factor, o.wait_limit);
    }
  };
  struct GraphEntry {
    int calls = 0;
    uint64_t last = 0;
    cudaGraphExec_t exec = nullptr;
  };
  std::map<GraphKey, GraphEntry> graphs;
  std::mutex graph_mutex;  // calls on one plan from several threads share the cache
  uint64_t graph_clock = 0;
  int graph_device = -1;
  cudaStream_t capture_stream = nullptr;  // private stream the launches are captured on
  void release_graphs() {
    if (graph_device < 0) return;
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(graph_device);
    for (auto& kv : graphs)
      if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    if (capture_stream) cudaStreamDestroy(capture_stream);
    cudaSetDevice(cur);
    graphs.clear();
    capture_stream = nullptr;
    graph_device = -1;
  }
  // copy streams and events of tfft_execute_host (created on first use)
  struct HostIo {
    int device = -1;
    cudaStream_t cin = nullptr, cout = nullptr;
    cudaEvent_t in_done[2] = {}, comp_done[2] = {}, out_done[2] = {}, start = nullptr, end = nullptr;
  } io;
  ~tfft_plan_s() {
    release_graphs();
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

namespace tfft {
namespace host {

// ---- plan state image, layouts, per-length plans (tfft_plan.cpp)
size_t image_add(tfft_plan p, const void* data, size_t bytes);
void build_layout(tfft_plan p, const int64_t* shape, int stage, LayoutH& L, int64_t pitch = 0);
DevLayout dev_layout(tfft_plan p, const LayoutH& L);
bool make_axis_plan(int L, bool strided, AxisPlan& best);
int strided_width(const AxisPlan& ap);
bool is_smooth_235(int64_t n);
bool make_bluestein(tfft_plan p, int N);
BlueArgs blue_args(tfft_plan p, int N);
int check_ptr(const void* ptr, const char* name);
int check_bound(tfft_plan p);

// ---- column blocks and exchange boxes (tfft_exchange.cpp)
std::pair<size_t, int64_t> get_colblocks(tfft_plan p, int lin, int lout, int W);
std::vector<int64_t> column_cuts(tfft_plan p, int lin, int lout);
std::vector<int2> colblock_list(tfft_plan p, int lin, int lout, int W);
BoxDesc make_box(int d, const int64_t* ext, int64_t src, const int64_t* ss, int64_t dst, const int64_t* ds);
void row_major_strides(int d, const int64_t* ext, int64_t* st);
void build_exchange(tfft_plan p, int s_from, int s_to);
Step box_step(const BoxList& L);

// ---- TMA tile geometry (tfft_tmageo.cpp)
int split_rows(int L);
bool tma_geo(tfft_plan p, int stage, int axis, int W, TmaGeo& G);
bool encode_stage_map(tfft_plan p, const TmaGeo& G, int axis, int W, const void* base, CUtensorMap* map);
int tuned_width(int L, int* E = nullptr, const char* var = "TFFT_TMA_W");
bool rank_groups(tfft_plan p, int stage, int L, int W, RankGroupGeo& G, std::vector<RankGroupH>& groups);
bool encode_group_map(const RankGroupH& H, int L, int W, const void* base, CUtensorMap* map);
bool window_side(tfft_plan p, int stage, int axis, int W, int64_t c0, int64_t nc, int64_t shift, TmaGeo& G,
                 TmaMapH& D);
bool encode_window_map(const TmaMapH& D, int W, const void* base, CUtensorMap* map);
bool plan_padding(tfft_plan p);
size_t fused_work_bytes(tfft_plan p);

// ---- pass lists and launches (tfft_exec.cpp)
Step fft_step(tfft_plan p, int axis, int lin, int lout, int sign);
Step last_axis_step(tfft_plan p, int sign);
std::vector<Step> build_steps(tfft_plan p, int sign, int mode);
void assign_buffers(std::vector<Step>& v, bool destroy_input);
int launch_step(tfft_plan p, const Step& s, void* const* bufs, cudaStream_t st);
int run_steps(tfft_plan p, const std::vector<Step>& steps, void* const* bufs, cudaStream_t st);
int run_steps_cached(tfft_plan p, const tfft_plan_s::GraphKey& k, const std::vector<Step>& steps, void* const* bufs,
                     cudaStream_t st);
int execute_impl(tfft_plan p, int key, int sign, int mode, const void* in, void* out, void* work,
                 size_t work_bytes, void* stream, const double* coef = nullptr, double factor = 1.0,
                 bool allow_graph = true);

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

}  // namespace host
}  // namespace tfft
