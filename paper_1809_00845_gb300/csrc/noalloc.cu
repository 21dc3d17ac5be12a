// bem_apply_static_scratch: the operator apply of bem_apply with its scratch
// (weighted densities and per-CTA partial sums) in one library-wide static
// device buffer instead of the plan's own scratch.
//
// Who needs it: code that must not touch the CUDA allocator at the point
// where it applies the operator.  Typical cases are a process whose device
// memory is fully reserved up front by another framework's pooling allocator
// (a raw cudaMalloc there can fail or fragment the pool), latency-critical
// loops that must not take the allocator's locks or synchronise, and hosts
// whose plug-in rules forbid device allocation after start-up.  This entry
// point calls no cudaMalloc, cudaFree or allocating library routine.
//
// The buffer below is linked into the library: every GPU on which the library
// is loaded and this entry point is used holds kStaticScratchBytes of device
// memory until the process exits.  Its device address is looked up with
// cudaGetSymbolAddress once per device, on the first call made while that
// device is current (make that first call before any stream capture).  All
// calls share the buffer and it keeps the previous call's contents; every
// byte an apply reads is written earlier in the same apply, so nothing has to
// be cleared, but two calls that overlap on the GPU (different streams without
// ordering, or concurrent host threads) race on it.
#include <mutex>
#include <string>

#include "bem_internal.h"

namespace bemfft {
namespace {

constexpr size_t kStaticScratchBytes = size_t(16) << 20;  // 16 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};

}  // namespace
}  // namespace bemfft

using namespace bemfft;

extern "C" bem_status bem_apply_static_scratch(bem_plan_t p, bem_layer layer, const void* in_dev, void* out_dev,
                                               void* stream) {
  if (!p || !in_dev || !out_dev) {
    set_error("bem_apply_static_scratch: null pointer argument");
    return BEM_ERR_ARG;
  }
  if (ranges_overlap(in_dev, out_dev, (size_t)p->nb * p->ncomp * prec_bytes(p))) {
    set_error("bem_apply_static_scratch: input and output must not overlap");
    return BEM_ERR_ARG;
  }
  if (p->pf) {
    set_error("bem_apply_static_scratch: accuracy-mode plans apply through bem_apply");
    return BEM_ERR_UNSUPPORTED;
  }
  if (p->dim != 2) {
    set_error("bem_apply_static_scratch: 3D plans need more scratch than the static buffer holds; use bem_apply");
    return BEM_ERR_UNSUPPORTED;
  }
  const Operator* op = nullptr;
  if (layer == BEM_SINGLE) op = &p->op_single;
  else if (layer == BEM_DOUBLE) op = &p->op_double;
  else if (layer == BEM_SYSTEM) {
    if (!p->have_bc) {
      set_error("bem_apply_static_scratch: BEM_SYSTEM needs bem_set_bc first");
      return BEM_ERR_ARG;
    }
    op = &p->op_system;
  } else {
    set_error("bem_apply_static_scratch: unknown layer");
    return BEM_ERR_ARG;
  }
  int dev = -1;
  BEM_CUDA_TRY(cudaGetDevice(&dev));
  if (dev != p->device || dev < 0 || dev >= kMaxDevices) {
    set_error("bem_apply_static_scratch: the plan's device must be current");
    return BEM_ERR_ARG;
  }
  bem_status rc;
  if ((rc = check_buffer_device(p, in_dev, "bem_apply_static_scratch")) != BEM_OK) return rc;
  if ((rc = check_buffer_device(p, out_dev, "bem_apply_static_scratch")) != BEM_OK) return rc;
  // bytes needed: the densities of every field, then the per-CTA partial sums
  const size_t need = apply_scratch_bytes(p, *op);
  if (need > kStaticScratchBytes) {
    set_error("bem_apply_static_scratch: this plan needs " + std::to_string(need) +
              " bytes of scratch, more than the static buffer's " + std::to_string(kStaticScratchBytes) +
              " bytes; use bem_apply");
    return BEM_ERR_UNSUPPORTED;
  }
  unsigned char* base = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_addr[dev]) {
      void* ptr = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&ptr, g_static_scratch);
      if (e != cudaSuccess || !ptr) {
        set_error(std::string("bem_apply_static_scratch: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        return BEM_ERR_CUDA;
      }
      g_scratch_addr[dev] = ptr;
    }
    base = static_cast<unsigned char*>(g_scratch_addr[dev]);
  }
  ScratchPtrs sp{};
  carve_scratch(p, *op, base, &sp);
  return launch_apply_2d_with(p, *op, in_dev, out_dev, sp, false, static_cast<cudaStream_t>(stream));
}
