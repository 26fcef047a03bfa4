// tfft_execute_host: transforms of arrays in page-locked host memory, the
// copies in and out overlapped with the transforms on two library streams.
#include "tfft_plan.h"

namespace {

constexpr int kHostSetBufs = 4;  // per buffer set: input, intermediate, output, workspace

size_t host_buf_bytes(tfft_plan p) { return align_up(fused_work_bytes(p), 256); }

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

extern "C" {

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
        // launched directly: instantiating a graph here could synchronise the
        // device in the middle of the copy pipeline, and the copies bound it
        rc = execute_impl(p, signs[j], signs[j], TFFT_MODE_FUSED, src, dst, bwork, B, stream, nullptr, 1.0,
                          false);
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

}  // extern "C"
