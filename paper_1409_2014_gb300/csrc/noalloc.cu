// noalloc.cu -- a solve entry point that allocates no device memory.
//
// Who needs it: callers that cannot call cudaMalloc (or any allocating
// library routine) at the point where they solve -- for example code that
// runs while an application-wide allocator forbids new device allocations,
// or a host loop that must not allocate after start-up.  dsnu_solve needs a
// caller-provided workspace of dsnu_workspace_bytes(plan) bytes; this variant
// instead uses one scratch array that is compiled into the library.
//
// The scratch array below is a __device__ variable of fixed size: every GPU
// on which the library is loaded holds it until the process exits.  In host
// code its name is only a host-side stand-in, so its device address is
// fetched with cudaGetSymbolAddress, once per device, with that device
// current, and that address is what the kernels receive.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "internal.h"

namespace {

constexpr size_t kStaticScratchBytes = size_t(32) << 20;  // 32 MiB per device

__device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mutex;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of g_static_scratch on the current device (set-up on the
// first call per device).
dsnu_status static_scratch_address(void** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    dsnu::set_last_error(std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    return DSNU_ECUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) {
    dsnu::set_last_error("device index out of range for the static scratch table");
    return DSNU_EUNSUPPORTED;
  }
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || !p) {
      dsnu::set_last_error(std::string("cudaGetSymbolAddress(static scratch): ") +
                           cudaGetErrorString(e));
      return DSNU_ECUDA;
    }
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return DSNU_OK;
}

}  // namespace

extern "C" {

size_t dsnu_noalloc_scratch_bytes(void) { return kStaticScratchBytes; }

dsnu_status dsnu_solve_noalloc(dsnu_plan plan, const double* rho, double* phi, void* stream) {
  if (!plan) {
    dsnu::set_last_error("NULL plan");
    return DSNU_EINVAL;
  }
  if (!rho || !phi) {
    dsnu::set_last_error("NULL input or output");
    return DSNU_EINVAL;
  }
  if ((reinterpret_cast<uintptr_t>(rho) | reinterpret_cast<uintptr_t>(phi)) & 15) {
    dsnu::set_last_error("input and output must be 16-byte aligned");
    return DSNU_EINVAL;
  }
  const size_t need = plan->ws_layout.total;
  if (need > kStaticScratchBytes) {
    dsnu::set_last_error("dsnu_solve_noalloc: this plan needs " + std::to_string(need) +
                         " bytes of scratch but the library's static scratch holds " +
                         std::to_string(kStaticScratchBytes) +
                         " bytes (32 MiB); use dsnu_solve with a caller workspace");
    return DSNU_EINVAL;
  }
  const size_t nbytes = size_t(plan->geom.nx) * plan->geom.ny * sizeof(double);
  const char* a = reinterpret_cast<const char*>(rho);
  const char* b = reinterpret_cast<const char*>(phi);
  if (a < b + nbytes && b < a + nbytes) {
    dsnu::set_last_error("input and output overlap");
    return DSNU_EINVAL;
  }
  void* scratch = nullptr;
  const dsnu_status s = static_scratch_address(&scratch);
  if (s != DSNU_OK) return s;
  // Every buffer of the workspace is written before it is read within one
  // solve, so nothing in the scratch needs clearing between calls.
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (plan->geom.precision == DSNU_MIXED)
    return dsnu::run_pipeline_f32(plan->geom, plan->tab, plan->ws_layout,
                                  dsnu::single_member(rho, phi, scratch), st, 0, nullptr);
  return dsnu::run_pipeline_f64(plan->geom, plan->tab, plan->ws_layout, dsnu::single_member(rho, phi, scratch),
                                st, 0, nullptr);
}

}  // extern "C"
