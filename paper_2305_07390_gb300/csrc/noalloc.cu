// noalloc.cu -- ebisu_run_static: a run whose scratch memory is a fixed,
// library-owned device array, for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc or hand the library a workspace: hosts
// that own every byte of device memory through their own pool and forbid
// outside allocations, code with a memory budget fixed at start-up, and
// latency-critical loops where an allocation (which may synchronise the
// device) is not acceptable.  ebisu_run normally needs a caller-provided
// workspace (a control block plus one grid-sized ping-pong buffer).  Here that
// workspace is the array below, of kStaticScratchBytes bytes, reserved on each
// device that loads this part of the library and held until the process
// exits.  Nothing in this file allocates; the run itself is ebisu_run, given
// the array's device address as its workspace.
#include "plan.h"

namespace {

// 64 MiB: one control block plus the ping-pong buffer of grids up to about
// 8.3 M FP64 cells (e.g. 2048 x 2048), 16.7 M FP32 cells or 33 M BF16 cells.
constexpr size_t kStaticScratchBytes = 64ull << 20;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

// The array's device address in the current device's current context.  In
// host code `g_static_scratch` names a host-side stand-in, not device memory,
// so it must never be passed to a kernel directly.  The lookup is a host-side
// query that allocates nothing; it is repeated on every call (with the
// caller's device current) rather than cached, so that a device that was
// reset, or a context other than the primary one, always yields the address
// of its own copy of the array.  The first lookup in a context loads this
// part of the library there, which is what reserves the array.
int scratch_address(void** out)
{
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return fail_cuda(e);
    if (!p) return EBISU_ERR_CUDA;
    *out = p;
    return EBISU_OK;
}

}  // namespace

extern "C" int ebisu_run_static(ebisu_plan_t plan, const void* in, void* out, int64_t steps, void* stream, int wait)
{
    if (!plan || !in || !out) return EBISU_ERR_INVALID_ARG;
    size_t need = 0;
    int rc = ebisu_plan_workspace_bytes(plan, &need);
    if (rc != EBISU_OK) return rc;
    if (need > kStaticScratchBytes) return EBISU_ERR_UNSUPPORTED;  // grid too large for the fixed array
    void* ws = nullptr;
    rc = scratch_address(&ws);
    if (rc != EBISU_OK) return rc;
    rc = ebisu_run(plan, in, out, steps, ws, stream);
    if (rc != EBISU_OK || !wait) return rc;
    return ebisu_sync(ws, stream);
}

extern "C" int ebisu_sync_static(void* stream)
{
    void* ws = nullptr;
    const int rc = scratch_address(&ws);
    if (rc != EBISU_OK) return rc;
    return ebisu_sync(ws, stream);
}
