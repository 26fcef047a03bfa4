// Column blocks of the strided passes and the exchange between adjacent
// stages (Alg. 2 / Alg. 3): the subarray boxes of every (sender, receiver)
// pair, the pack / all-to-all / unpack boxes of the traditional method
// (Sec. 3.3.1), their copy tasks, tfft_redistribute and
// tfft_plan_copy_tasks.
#include "tfft_plan.h"

namespace tfft {
namespace host {

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

}  // namespace host
}  // namespace tfft

extern "C" {

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

}  // extern "C"
