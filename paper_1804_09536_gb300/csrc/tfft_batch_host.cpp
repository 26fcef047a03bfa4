// Host side of the batched persistent executor: segment order, tile variant
// choice, the state image of the work queue, the autotuner and its ABI.
#include "tfft_plan.h"

// ============================================================== batch

namespace {

constexpr int kMaxBatchStreams = 16;

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
  // stream executor: transforms per forked stream, and the streams and events
  // of the fork / join (created on the device of the first execute)
  int executor = TFFT_BATCH_PERSISTENT;
  int nstreams = 4;
  std::vector<std::vector<int>> lanes;
  struct Fork {
    int device = -1;
    std::vector<cudaStream_t> s;
    std::vector<cudaEvent_t> done;
    cudaEvent_t start = nullptr;
  } fork;
  void release_fork() {
    if (fork.device < 0) return;
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(fork.device);
    for (cudaStream_t x : fork.s) cudaStreamDestroy(x);
    for (cudaEvent_t x : fork.done) cudaEventDestroy(x);
    if (fork.start) cudaEventDestroy(fork.start);
    cudaSetDevice(cur);
    fork = Fork{};
  }
  ~tfft_batch_s() { release_fork(); }
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

// Stream executor: transforms, longest first, each to the stream with the
// fewest elements so far.
void batch_lanes(tfft_batch b) {
  const int n = (int)b->plans.size();
  const int K = std::max(1, std::min(b->nstreams, n));
  std::vector<int> order(n);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(),
                   [&](int x, int y) { return b->plans[x]->nelems > b->plans[y]->nelems; });
  std::vector<int64_t> load(K, 0);
  b->lanes.assign(K, {});
  for (int t : order) {
    const int j = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    b->lanes[j].push_back(t);
    load[j] += b->plans[t]->nelems;
  }
}

int ensure_fork(tfft_batch b) {
  const int dev = current_device();
  const size_t K = b->lanes.size();
  if (b->fork.device == dev && b->fork.s.size() >= K) return TFFT_OK;
  b->release_fork();
  b->fork.device = dev;
  cudaError_t e = cudaEventCreateWithFlags(&b->fork.start, cudaEventDisableTiming);
  for (size_t j = 0; j < K && e == cudaSuccess; ++j) {
    cudaStream_t x = nullptr;
    cudaEvent_t ev = nullptr;
    e = cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking);
    if (e == cudaSuccess) b->fork.s.push_back(x);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e == cudaSuccess) b->fork.done.push_back(ev);
  }
  if (e != cudaSuccess) {
    b->release_fork();
    return cuda_fail(e, "creating the batch's fork streams");
  }
  return TFFT_OK;
}

// Every transform's fused passes as its plan's own kernels, the transforms of
// lane j in order on forked stream j; the caller's stream waits for all.
int batch_launch_streams(tfft_batch b, cudaStream_t st) {
  const int dev = current_device();
  for (tfft_plan p : b->plans)
    if (p->device != dev) return fail(TFFT_EINVAL, "a plan of the batch is bound on another device than the current one");
  if (b->lanes.empty()) batch_lanes(b);
  int rc = ensure_fork(b);
  if (rc) return rc;
  cudaError_t e = cudaEventRecord(b->fork.start, st);
  if (e != cudaSuccess) return cuda_fail(e, "batch fork");
  // every forked stream is joined back even when a launch fails, so that a
  // stream capture in progress stays well formed (its end reports the error)
  cudaError_t ej = cudaSuccess;
  for (size_t j = 0; j < b->lanes.size(); ++j) {
    cudaStream_t x = b->fork.s[j];
    cudaError_t ef = cudaStreamWaitEvent(x, b->fork.start, 0);
    if (ef != cudaSuccess) {
      if (ej == cudaSuccess) ej = ef;
      continue;
    }
    for (int t : b->lanes[j]) {
      if (rc) break;
      void* bufs[4] = {b->ins[t], b->outs[t], b->works[t], nullptr};
      for (const Step& s : b->steps[t])
        if ((rc = launch_step(b->plans[t], s, bufs, x))) break;
    }
    cudaError_t e2 = cudaEventRecord(b->fork.done[j], x);
    if (e2 == cudaSuccess) e2 = cudaStreamWaitEvent(st, b->fork.done[j], 0);
    if (e2 != cudaSuccess && ej == cudaSuccess) ej = e2;
  }
  if (rc) return rc;
  if (ej != cudaSuccess) return cuda_fail(ej, "batch fork / join");
  return TFFT_OK;
}

int batch_launch_persistent(tfft_batch b, cudaStream_t st) {
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

int batch_launch(tfft_batch b, cudaStream_t st) {
  return b->executor == TFFT_BATCH_STREAMS ? batch_launch_streams(b, st) : batch_launch_persistent(b, st);
}

// Mean ms of `reps` launches of the current executor (after one warm-up).
int time_batch(tfft_batch b, int reps, cudaStream_t st, cudaEvent_t e0, cudaEvent_t e1, float& ms) {
  int rc = batch_launch(b, st);
  if (rc) return rc;
  cudaEventRecord(e0, st);
  for (int r = 0; r < reps && !rc; ++r) rc = batch_launch(b, st);
  cudaEventRecord(e1, st);
  cudaError_t e = cudaEventSynchronize(e1);
  if (e != cudaSuccess) return cuda_fail(e, "timing the batch");
  cudaEventElapsedTime(&ms, e0, e1);
  ms /= (float)reps;
  return rc;
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
    const int exec0 = b->executor;
    b->executor = TFFT_BATCH_PERSISTENT;  // tile variants: the persistent kernel's
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
    // executor: the persistent kernel with the chosen tiles, or the stream
    // executor with 1, 2, 3, 4, 6 or 8 streams, whichever runs the batch fastest
    auto ex = cached.find({-1, -1});
    if (!rc && ex != cached.end()) {
      b->executor = ex->second >= 1 ? TFFT_BATCH_STREAMS : TFFT_BATCH_PERSISTENT;
      if (ex->second >= 1) b->nstreams = std::min(ex->second, kMaxBatchStreams);
      batch_lanes(b);
    } else if (!rc) {
      float best = 1e30f, ms = 0;
      int best_k = 0;
      if (!(rc = batch_upload(b, st)) && !(rc = time_batch(b, reps, st, e0, e1, ms))) best = ms;
      b->executor = TFFT_BATCH_STREAMS;
      for (int k : {1, 2, 3, 4, 6, 8}) {
        if (rc || k > (int)b->plans.size()) break;
        b->nstreams = k;
        batch_lanes(b);
        if ((rc = time_batch(b, reps, st, e0, e1, ms))) break;
        if (ms < best) {
          best = ms;
          best_k = k;
        }
      }
      b->executor = best_k ? TFFT_BATCH_STREAMS : TFFT_BATCH_PERSISTENT;
      if (best_k) b->nstreams = best_k;
      batch_lanes(b);
    }
    if (rc) b->executor = exec0;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    if (cache) {
      if (FILE* f = std::fopen(cache, "w")) {
        for (auto& kv : b->choice) std::fprintf(f, "%d %d %d\n", kv.first.first, kv.first.second, kv.second);
        std::fprintf(f, "-1 -1 %d\n", b->executor == TFFT_BATCH_STREAMS ? b->nstreams : 0);
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

int tfft_batch_set_executor(tfft_batch b, int executor, int nstreams) {
  return guarded("tfft_batch_set_executor", [&]() -> int {
    if (!b) return fail(TFFT_EINVAL, "batch is NULL");
    if (executor != TFFT_BATCH_PERSISTENT && executor != TFFT_BATCH_STREAMS)
      return fail(TFFT_EINVAL, "unknown batch executor");
    if (executor == TFFT_BATCH_STREAMS && (nstreams < 1 || nstreams > kMaxBatchStreams))
      return fail(TFFT_EINVAL, "nstreams must be in 1 .. 16");
    b->executor = executor;
    if (executor == TFFT_BATCH_STREAMS) {
      b->nstreams = nstreams;
      batch_lanes(b);
    }
    return TFFT_OK;
  });
}

int tfft_batch_executor(tfft_batch b, int* executor, int* nstreams) {
  if (!b || !executor || !nstreams) return fail(TFFT_EINVAL, "NULL argument");
  *executor = b->executor;
  *nstreams = b->executor == TFFT_BATCH_STREAMS ? (int)b->lanes.size() : 0;
  return TFFT_OK;
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
  // the persistent kernel reports in the batch state, the stream executor's
  // kernels in their plans' states: the status is the OR of all of them
  std::vector<char*> words = {b->d_state};
  for (tfft_plan p : b->plans)
    if (p->d_state && std::find(words.begin(), words.end(), p->d_state) == words.end()) words.push_back(p->d_state);
  std::vector<int> vals(words.size(), 0);
  cudaError_t e = cudaSuccess;
  for (size_t i = 0; i < words.size() && e == cudaSuccess; ++i)
    e = cudaMemcpyAsync(&vals[i], words[i], sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess && reset) {
    const int zero = 0;
    for (size_t i = 0; i < words.size() && e == cudaSuccess; ++i)
      e = cudaMemcpyAsync(words[i], &zero, sizeof(int), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  }
  if (e != cudaSuccess) return cuda_fail(e, "reading the batch status words");
  int v = 0;
  for (int x : vals) v |= x;
  *status = v;
  return TFFT_OK;
}

}  // extern "C"
