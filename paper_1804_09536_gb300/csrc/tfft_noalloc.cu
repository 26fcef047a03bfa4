// tfft_execute_noalloc(): the fused transform with its scratch buffer taken
// from a fixed device array compiled into this library instead of a
// caller-allocated workspace.
//
// Who needs it: callers that may not allocate device memory themselves --
// for example a plugin that runs inside a host framework which owns all
// device memory through its own allocator and forbids (or has no memory left
// for) a stray cudaMalloc, or code with a fixed, audited memory budget.  Such
// a caller can still keep its input intact, which tfft_execute() only does
// when it is given a workspace.  The one exception is the complex-to-real
// backward of a real-to-complex plan: it overwrites its input with either
// entry point.
//
// The scratch is one stage buffer: the fused path writes the input's
// partially transformed copy there before it redistributes it into `out`.
#include <string>

#include "tfft.h"
#include "tfft_internal.h"

namespace {

// One stage buffer of at most TFFT_NOALLOC_SCRATCH_BYTES (16 MiB, 2^21
// complex64 elements, e.g. 128^3).  Every GPU that loads this library holds
// this array until the process exits.
constexpr size_t kNoallocScratchBytes = TFFT_NOALLOC_SCRATCH_BYTES;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

// Device address of the array on the current device.  In host code the
// array's name is only a host-side stand-in, so the address is looked up with
// cudaGetSymbolAddress, with the device current, on every call: the lookup is
// cheap once the module is loaded, and a cached address would go stale after
// a device reset.
int scratch_for_current_device(void** ptr) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess || !p) return TFFT_ECUDA;
  *ptr = p;
  return TFFT_OK;
}

}  // namespace

extern "C" int tfft_execute_noalloc(tfft_plan plan, int sign, const void* in, void* out, void* stream) {
  if (!plan) {
    tfft::set_last_error("tfft_execute_noalloc: plan is NULL");
    return TFFT_EINVAL;
  }
  size_t need = 0;
  int rc = tfft_plan_workspace_bytes(plan, TFFT_MODE_FUSED, 1, &need);
  if (rc != TFFT_OK) return rc;
  if (need > kNoallocScratchBytes) {
    tfft::set_last_error("tfft_execute_noalloc: the plan needs " + std::to_string(need) +
                         " bytes of scratch; the fixed device array holds " +
                         std::to_string(kNoallocScratchBytes));
    return TFFT_EWORKSPACE;
  }
  void* scratch = nullptr;
  rc = scratch_for_current_device(&scratch);
  if (rc != TFFT_OK) {
    tfft::set_last_error("tfft_execute_noalloc: cudaGetSymbolAddress of the scratch array failed");
    return rc;
  }
  // tfft_execute() rejects (TFFT_EINVAL) a current device other than the one
  // the plan was bound on, so the scratch is always the plan's device's array
  return tfft_execute(plan, sign, TFFT_MODE_FUSED, in, out, scratch, kNoallocScratchBytes, stream);
}
