// Plan creation and queries of the C ABI (include/tfft.h): the balanced
// decomposition (Eq. decompose / Alg. 1), the stage layouts of the virtual
// grid (Secs. 3.3-3.6), the per-length FFT plans and Bluestein tables, the
// plan state image and its binding to caller-allocated device memory.
#include "tfft_plan.h"

namespace tfft {
namespace host {

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


size_t image_add(tfft_plan p, const void* data, size_t bytes) {
  const size_t off = align_up(p->image.size(), 256);
  p->image.resize(off + bytes, 0);
  if (data && bytes) std::memcpy(p->image.data() + off, data, bytes);
  return off;
}

void build_layout(tfft_plan p, const int64_t* shape, int stage, LayoutH& L, int64_t pitch) {
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
      cnt *= (m == p->d - 1 && pitch > 0) ? pitch : n;
    }
    L.offset[r] = off;
    off += cnt;
  }
  L.total = off;
  L.pitch = pitch;
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
  D.pitch = L.pitch;
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
  if (ap.spec || ap.blue_spec) return ap.width;
  int W = std::max(1, std::min(32, 512 / ap.T));
  // shared memory: L x W elements (two buffers for the generic kernel; two of
  // the convolution length for Bluestein) + row tables
  const size_t budget = 200 * 1024 - 16 * (size_t)ap.L;
  const size_t per_col = ap.blue_m ? 2 * 8 * (size_t)ap.blue_m : (ap.E == 0 ? 2 : 1) * 8 * (size_t)ap.L;
  while (W > 1 && (size_t)W * per_col > budget) --W;
  return W;
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
  // compile-time specialised kernels for this convolution length (their own
  // lines per CTA and tile width; 32-bit row offsets)
  int spec_lines = 0, spec_w = 0;
  if (p->nelems < (int64_t(1) << 31) && blue_spec_plan(M, spec_lines, spec_w)) {
    ap.blue_spec = aps.blue_spec = 1;
    ap.width = spec_lines;
    aps.width = spec_w;
  }
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

}  // namespace host
}  // namespace tfft

void tfft::set_last_error(const std::string& msg) { tfft::host::g_err = msg; }

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
    if (flags & ~(TFFT_NORM_BACKWARD | TFFT_NO_TMA | TFFT_NO_GRAPH)) return fail(TFFT_EINVAL, "unknown flag bits");
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
      // padded stage-0 layout of a real-to-complex plan's fused path
      plan_padding(p);
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
    {
      std::lock_guard<std::mutex> lock(p->graph_mutex);
      p->release_graphs();  // captured launches point into the previous state
    }
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
    case TFFT_MODE_FUSED: *bytes = (keep_input || p->kind == TFFT_R2C) ? fused_work_bytes(p) : 0; break;
    case TFFT_MODE_UNFUSED:
    case TFFT_MODE_PACKED: *bytes = 2 * stage; break;
    default: return fail(TFFT_EINVAL, "unknown mode");
  }
  return TFFT_OK;
}

}  // extern "C"
