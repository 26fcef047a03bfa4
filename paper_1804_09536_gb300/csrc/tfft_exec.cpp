// Pass lists and launches: the fused step list (redistributions folded into
// the strided passes' loads and stores), the unfused and packed comparison
// lists, buffer assignment, kernel launches, and the execute, adjoint,
// partial-transform and loss entry points.
#include "tfft_plan.h"

namespace tfft {
namespace host {

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
    // uneven blocks: an in-place pass along axis 0 can still run TMA-staged
    // tiles over the layout's rank groups
    if (!s.tma && p->use_tma && ap.spec && lin == lout && axis == 0 &&
        tma_strided_variant(s.L, wantW, wantE, Et, Wt) && rank_groups(p, lin, s.L, Wt, s.rg, s.rgh)) {
      s.tma_groups = true;
      s.tma_E = Et;
      s.tma_W = Wt;
    }
    // tensor-core plans: the tensor-core TMA variant of this length, with its
    // own tile width (and so its own geometry and column blocks)
    int Ec = 0, Wc = 0;
    s.tc = p->precision != TFFT_FP32 && p->use_tma && ap.spec &&
           tc_strided_variant(s.L, tuned_width(s.L, nullptr, "TFFT_TC_W"), Ec, Wc) &&
           tma_geo(p, lin, axis, Wc, s.tc_gin) && tma_geo(p, lout, axis, Wc, s.tc_gout);
    if (s.tc) {
      s.tc_E = Ec;
      s.tc_W = Wc;
      auto cbc = get_colblocks(p, lin, lout, Wc);
      s.tc_cb_off = cbc.first;
      s.tc_ncb = cbc.second;
      s.tc_outer_fastest = axis == 0 && Wc * sizeof(float2) >= 128;
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

// The gathering pass along axis d - 2 of a padded real-to-complex plan
// (plan_padding): one TMA-staged step over the column window, then the plain
// kernel over the remaining columns on the same buffers (marked `cont`).
// `lin` / `lout` name the padded stage-0 layout on its side.
void add_window_pass(tfft_plan p, std::vector<Step>& v, int axis, int lin, int lout, int sign) {
  Step s = fft_step(p, axis, lin, lout, sign);
  s.tma = s.tc = s.tma_groups = false;
  s.in_shift = lin == p->pad_stage ? p->pad_lead : 0;
  s.out_shift = lout == p->pad_stage ? p->pad_lead : 0;
  const int64_t c0 = p->win_c0, c1 = p->win_c0 + p->win_nc;
  auto upload = [&](const std::vector<int2>& b) {
    return std::make_pair(image_add(p, b.data(), b.size() * sizeof(int2)), (int64_t)b.size());
  };
  Step w = s;
  w.tma_win = true;
  w.tma_E = p->win_E;
  w.tma_W = p->win_W;
  w.win_c0 = c0;
  w.win_nc = p->win_nc;
  w.ncols = p->win_nc;
  w.tma_outer_fastest = axis == 0 && w.tma_W * sizeof(float2) >= 128;
  if (!window_side(p, lin, axis, w.tma_W, c0, p->win_nc, s.in_shift, w.gin, w.win_min) ||
      !window_side(p, lout, axis, w.tma_W, c0, p->win_nc, s.out_shift, w.gout, w.win_mout))
    throw std::logic_error("column window geometry changed after planning");
  std::vector<int2> inside, outside;
  for (const int2& b : colblock_list(p, lin, lout, w.tma_W))
    if (b.x >= c0 && b.x + b.y <= c1) inside.push_back(b);
  for (const int2& b : colblock_list(p, lin, lout, s.W))
    if (b.x + b.y <= c0 || b.x >= c1) outside.push_back(b);
  auto cbw = upload(inside);
  w.tma_cb_off = cbw.first;
  w.tma_ncb = cbw.second;
  v.push_back(w);
  if (!outside.empty()) {
    Step r = s;
    r.cont = true;
    r.ncols = p->cshape[p->d - 1] - p->win_nc;
    auto cbr = upload(outside);
    r.cb_off = cbr.first;
    r.ncb = cbr.second;
    v.push_back(r);
  }
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
    // a padded plan keeps its complex stage-0 buffer (internal to the fused
    // path) in the padded layout
    const int pad = p->pad_stage;
    if (sign == TFFT_FORWARD) {
      v.push_back(last_axis_step(p, sign));
      if (pad >= 0) {
        v.back().cpitch = p->st[pad].pitch;
        v.back().out_shift = p->pad_lead;
      }
      for (int a = d - 2; a >= 0; --a) {
        if (pad >= 0 && a == d - 2) add_window_pass(p, v, a, pad, g, sign);
        else v.push_back(fft_step(p, a, a == d - 2 ? 0 : g, g, sign));
      }
    } else {
      for (int a = 0; a <= d - 2; ++a) {
        if (pad >= 0 && a == d - 2) add_window_pass(p, v, a, g, pad, sign);
        else v.push_back(fft_step(p, a, g, a == d - 2 ? 0 : g, sign));
      }
      v.push_back(last_axis_step(p, sign));
      if (pad >= 0) {
        v.back().cpitch = p->st[pad].pitch;
        v.back().in_shift = p->pad_lead;
      }
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
        // a pass split into steps over column ranges scales in each of them
        for (int j = k; j >= 0; --j) {
          v[j].scaled = true;
          v[j].scale_value = 1.0 / (double)(p->kind == TFFT_R2C ? p->nreal : p->nelems);
          if (!v[j].cont) break;
        }
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
    if (!v[k].inplace_ok && !v[k].cont) last_move = k;
  int cur = BUF_IN;
  for (int k = 0; k < (int)v.size(); ++k) {
    Step& s = v[k];
    if (s.cont && k > 0) {  // the rest of the previous step's columns
      s.src = v[k - 1].src;
      s.dst = v[k - 1].dst;
      continue;
    }
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

int launch_step(tfft_plan p, const Step& s, void* const* bufs, cudaStream_t st) {
  const float2* in = static_cast<const float2*>(bufs[s.src]) + s.in_shift;
  float2* out = static_cast<float2*>(bufs[s.dst]) + s.out_shift;
  cudaError_t e = cudaSuccess;
  if (s.kind == S_CONTIG) {
    ContigArgs a;
    a.in = in;
    a.out = out;
    a.nlines = s.nlines;
    a.ap = p->aplan[s.L];
    a.tw = reinterpret_cast<const float2*>(p->d_state + p->tw_off[s.L]);
    a.lines_per_cta = (a.ap.spec || a.ap.blue_spec) ? a.ap.width : std::max(1, 256 / a.ap.T);
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
    if (s.tma_win) {
      alignas(64) CUtensorMap ti, to;
      if (!encode_window_map(s.win_min, s.tma_W, in, &ti) || !encode_window_map(s.win_mout, s.tma_W, out, &to))
        return fail(TFFT_ECUDA, "tensor map of a column window could not be encoded");
      StridedArgs at = a;
      at.W = s.tma_W;
      at.colblocks = reinterpret_cast<const int2*>(p->d_state + s.tma_cb_off);
      at.ncolblocks = s.tma_ncb;
      at.outer_fastest = s.tma_outer_fastest ? 1 : 0;
      e = launch_strided_tma(at, s.tma_E, s.gin, s.gout, &ti, &to, st);
      done = true;
    }
    if (!done && s.tc) {
      alignas(64) CUtensorMap ti, to;
      if (encode_stage_map(p, s.tc_gin, s.axis, s.tc_W, in, &ti) &&
          encode_stage_map(p, s.tc_gout, s.axis, s.tc_W, out, &to)) {
        StridedArgs at = a;
        at.W = s.tc_W;
        at.colblocks = reinterpret_cast<const int2*>(p->d_state + s.tc_cb_off);
        at.ncolblocks = s.tc_ncb;
        at.outer_fastest = s.tc_outer_fastest ? 1 : 0;
        e = launch_strided_tma_tc(at, s.tc_E, p->precision, s.tc_gin, s.tc_gout, &ti, &to, st);
        done = true;
      }
    }
    if (!done && s.tma) {
      alignas(64) CUtensorMap ti, to;
      if (encode_stage_map(p, s.gin, s.axis, s.tma_W, in, &ti) &&
          encode_stage_map(p, s.gout, s.axis, s.tma_W, out, &to)) {
        StridedArgs at = a;
        at.W = s.tma_W;
        at.colblocks = reinterpret_cast<const int2*>(p->d_state + s.tma_cb_off);
        at.ncolblocks = s.tma_ncb;
        at.outer_fastest = s.tma_outer_fastest ? 1 : 0;
        e = launch_strided_tma(at, s.tma_E, s.gin, s.gout, &ti, &to, st);
        done = true;
      }
    }
    if (!done && s.tma_groups) {
      alignas(64) CUtensorMap ti[kMaxRankGroups], to[kMaxRankGroups];
      const void* pin[kMaxRankGroups];
      const void* pout[kMaxRankGroups];
      bool ok = true;
      for (int k = 0; k < s.rg.ngroups && ok; ++k) {
        ok = encode_group_map(s.rgh[k], s.L, s.tma_W, in, &ti[k]) && encode_group_map(s.rgh[k], s.L, s.tma_W, out, &to[k]);
        pin[k] = &ti[k];
        pout[k] = &to[k];
      }
      if (ok) {
        StridedArgs at = a;
        at.W = s.tma_W;
        e = launch_strided_tma_groups(at, s.tma_E, s.rg, pin, pout, st);
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
    a.cout = out;
    a.cin = in;
    a.rout = static_cast<float*>(bufs[s.dst]);
    a.cpitch = s.cpitch > 0 ? s.cpitch : (int64_t)p->rplan.L + 1;
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

int execute_impl(tfft_plan p, int key, int sign, int mode, const void* in, void* out, void* work,
                        size_t work_bytes, void* stream, const double* coef, double factor, bool allow_graph) {
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
      if (work_bytes < fused_work_bytes(p))
        return fail(TFFT_EWORKSPACE, "fused workspace smaller than tfft_plan_workspace_bytes reports");
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
    const size_t wb = (mode == TFFT_MODE_FUSED) ? fused_work_bytes(p) : 2 * stage;
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
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (!allow_graph || !p->events.empty() || (p->flags & TFFT_NO_GRAPH)) return run_steps(p, steps, bufs, st);
  return run_steps_cached(p, tfft_plan_s::GraphKey{key, mode, in, out, w0, w1, coef, factor, p->wait_limit}, steps,
                          bufs, st);
}

// run_steps through the plan's graph cache (see tfft_execute): the first call
// of a key launches directly, the second captures the launches on the plan's
// capture stream and instantiates them, that call and later ones launch the
// graph on `st`.  A stream already being captured by the caller, or a failed
// capture, launches directly.
int run_steps_cached(tfft_plan p, const tfft_plan_s::GraphKey& k, const std::vector<Step>& steps, void* const* bufs,
                     cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
    cudaGetLastError();
    return run_steps(p, steps, bufs, st);
  }
  if (cs != cudaStreamCaptureStatusNone) return run_steps(p, steps, bufs, st);
  std::lock_guard<std::mutex> lock(p->graph_mutex);
  const int dev = current_device();
  if (p->graph_device >= 0 && p->graph_device != dev) p->release_graphs();
  auto& e = p->graphs[k];
  e.last = ++p->graph_clock;
  if (!e.exec && ++e.calls >= 2) {
    if (!p->capture_stream) {
      cudaError_t ce = cudaStreamCreateWithFlags(&p->capture_stream, cudaStreamNonBlocking);
      if (ce != cudaSuccess) {
        p->capture_stream = nullptr;
        return cuda_fail(ce, "creating the plan's capture stream");
      }
      p->graph_device = dev;
    }
    // at most kGraphCache instantiated graphs: drop the least recently used
    constexpr size_t kGraphCache = 8;
    size_t live = 0;
    for (auto& kv : p->graphs) live += kv.second.exec != nullptr;
    while (live >= kGraphCache) {
      auto victim = p->graphs.end();
      for (auto it = p->graphs.begin(); it != p->graphs.end(); ++it)
        if (it->second.exec && (victim == p->graphs.end() || it->second.last < victim->second.last)) victim = it;
      if (victim == p->graphs.end()) break;
      cudaGraphExecDestroy(victim->second.exec);
      victim->second.exec = nullptr;
      victim->second.calls = 0;
      --live;
    }
    cudaGraph_t g = nullptr;
    cudaError_t ce = cudaStreamBeginCapture(p->capture_stream, cudaStreamCaptureModeRelaxed);
    int rc = TFFT_OK;
    if (ce == cudaSuccess) {
      rc = run_steps(p, steps, bufs, p->capture_stream);
      ce = cudaStreamEndCapture(p->capture_stream, &g);
    }
    if (rc == TFFT_OK && ce == cudaSuccess && g) ce = cudaGraphInstantiate(&e.exec, g, 0);
    if (g) cudaGraphDestroy(g);
    if (rc != TFFT_OK || ce != cudaSuccess || !e.exec) {
      // the launches could not be captured: run them directly, now and later
      cudaGetLastError();
      e.exec = nullptr;
      e.calls = -(1 << 30);
      return run_steps(p, steps, bufs, st);
    }
  }
  if (!e.exec) return run_steps(p, steps, bufs, st);
  cudaError_t ce = cudaGraphLaunch(e.exec, st);
  if (ce != cudaSuccess) return cuda_fail(ce, "cudaGraphLaunch");
  return TFFT_OK;
}

}  // namespace host
}  // namespace tfft

extern "C" {

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
      const bool tma = s.kind == S_STRIDED && (s.tma || s.tc || s.tma_groups || s.tma_win);
      const bool tc = p->precision != TFFT_FP32 && ((s.kind == S_CONTIG && tc_supported(ap.L)) || s.tc);
      nm = std::string(s.kind == S_CONTIG ? "fft_contig" : "fft_strided") +
           (tma ? "_tma" : "") + (s.kind == S_STRIDED && s.tma_groups && !s.tc ? "_groups" : "") +
           (s.kind == S_STRIDED && s.tma_win ? "_window" : "") +
           (tc ? (p->precision == TFFT_TC_BF16X3 ? "_tc_bf16x3" : "_tc_fp16x3") : "") +
           (ap.blue_m ? "_bluestein_L" + std::to_string(ap.L)
                      : ap.spec ? "_L" + std::to_string(ap.L)
                                : ap.E == 0 ? std::string("_generic") : "_E" + std::to_string(ap.E));
      elems = p->nelems;
      if (s.ncols >= 0) elems = p->nelems / p->cshape[p->d - 1] * s.ncols;  // a column range of the pass
    }
    *bytes = 2 * elems * (int64_t)sizeof(float2);  // one read and one write of every element
    if (name_len > 0) {
      std::strncpy(name, nm.c_str(), (size_t)name_len - 1);
      name[name_len - 1] = 0;
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

}  // extern "C"
