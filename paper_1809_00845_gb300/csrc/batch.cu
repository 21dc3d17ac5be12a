// Batched apply: many plans (geometries of uneven grid sizes) applied as one
// CUDA graph.  The graph is captured once: the plans are distributed
// round-robin over a few forked capture streams, so the applies of small
// geometries run side by side, and the whole batch is then replayed with a
// single graph launch per batched apply (no per-kernel launch overhead).
// Inputs and outputs live in two packed device buffers owned by the batch
// (segment of plan i at offset[i], nb_i * ncomp_i values of the common
// precision).
#include <vector>

#include "bem_internal.h"

struct bem_batch_s {
  std::vector<bem_plan_t> plans;
  std::vector<size_t> offset;  // element offsets into the packed buffers
  size_t total = 0;
  int prec = 0;
  void* d_in = nullptr;
  void* d_out = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<cudaStream_t> side;
  std::vector<cudaEvent_t> events;
  int launches = 0;
};

using namespace bemfft;

extern "C" {

bem_status bem_batch_destroy(bem_batch_t b) {
  if (!b) return BEM_OK;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  for (auto s : b->side) cudaStreamDestroy(s);
  for (auto e : b->events) cudaEventDestroy(e);
  cudaFree(b->d_in);
  cudaFree(b->d_out);
  delete b;
  return BEM_OK;
}

bem_status bem_batch_create(bem_batch_t* out, const bem_plan_t* plans, int count, bem_layer layer, int streams,
                            void* stream) {
  if (!out || !plans || count < 1 || streams < 1 || streams > 16) {
    set_error("bem_batch_create: need plans, count >= 1 and 1 <= streams <= 16");
    return BEM_ERR_ARG;
  }
  *out = nullptr;
  for (int i = 0; i < count; ++i) {
    if (!plans[i]) {
      set_error("bem_batch_create: null plan");
      return BEM_ERR_ARG;
    }
    if (plans[i]->prec != plans[0]->prec) {
      set_error("bem_batch_create: all plans must share one precision");
      return BEM_ERR_ARG;
    }
    if (layer == BEM_SYSTEM && !plans[i]->have_bc) {
      set_error("bem_batch_create: BEM_SYSTEM needs bem_set_bc on every plan");
      return BEM_ERR_ARG;
    }
    plans[i]->timing = false;
  }
  auto* b = new bem_batch_s();
  b->prec = plans[0]->prec;
  for (int i = 0; i < count; ++i) {
    b->plans.push_back(plans[i]);
    b->offset.push_back(b->total);
    b->total += (size_t)plans[i]->nb * plans[i]->ncomp;
  }
  const size_t tb = prec_bytes(plans[0]);
  auto fail = [&](bem_status rc) {
    bem_batch_destroy(b);
    return rc;
  };
  if (cudaMalloc(&b->d_in, b->total * tb) != cudaSuccess || cudaMalloc(&b->d_out, b->total * tb) != cudaSuccess) {
    set_error("bem_batch_create: out of device memory");
    return fail(BEM_ERR_OOM);
  }
  cudaMemset(b->d_in, 0, b->total * tb);
  cudaMemset(b->d_out, 0, b->total * tb);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaStream_t cap = nullptr;
  if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) {
    set_error("bem_batch_create: stream creation failed");
    return fail(BEM_ERR_CUDA);
  }
  b->side.push_back(cap);
  for (int s = 1; s < streams; ++s) {
    cudaStream_t x;
    if (cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking) != cudaSuccess) {
      set_error("bem_batch_create: stream creation failed");
      return fail(BEM_ERR_CUDA);
    }
    b->side.push_back(x);
  }
  for (int s = 0; s < 2 * streams; ++s) {
    cudaEvent_t e;
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
      set_error("bem_batch_create: event creation failed");
      return fail(BEM_ERR_CUDA);
    }
    b->events.push_back(e);
  }
  // capture: fork the side streams off the capture stream, apply, join
  if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    set_error("bem_batch_create: stream capture failed to begin");
    return fail(BEM_ERR_CUDA);
  }
  bem_status rc = BEM_OK;
  cudaEventRecord(b->events[0], cap);
  for (int s = 1; s < streams; ++s) cudaStreamWaitEvent(b->side[s], b->events[0], 0);
  for (int i = 0; i < count && rc == BEM_OK; ++i) {
    cudaStream_t s = b->side[i % streams];
    const unsigned char* in = static_cast<const unsigned char*>(b->d_in) + b->offset[i] * tb;
    unsigned char* o = static_cast<unsigned char*>(b->d_out) + b->offset[i] * tb;
    rc = apply_operator(plans[i], layer, in, o, s);
    b->launches += bem_launches_per_apply(plans[i], layer);
  }
  for (int s = 1; s < streams; ++s) {
    cudaEventRecord(b->events[streams + s], b->side[s]);
    cudaStreamWaitEvent(cap, b->events[streams + s], 0);
  }
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(cap, &g);
  if (rc != BEM_OK) {
    if (g) cudaGraphDestroy(g);
    return fail(rc);
  }
  if (e != cudaSuccess || !g) {
    set_error(std::string("bem_batch_create: capture failed: ") + cudaGetErrorString(e));
    return fail(BEM_ERR_CUDA);
  }
  b->graph = g;
  if (cudaGraphInstantiate(&b->exec, g, 0) != cudaSuccess) {
    set_error("bem_batch_create: graph instantiation failed");
    return fail(BEM_ERR_CUDA);
  }
  (void)st;
  *out = b;
  return BEM_OK;
}

bem_status bem_batch_buffers(bem_batch_t b, void** in_dev, void** out_dev, size_t* total) {
  if (!b) {
    set_error("bem_batch_buffers: null batch");
    return BEM_ERR_ARG;
  }
  if (in_dev) *in_dev = b->d_in;
  if (out_dev) *out_dev = b->d_out;
  if (total) *total = b->total;
  return BEM_OK;
}

bem_status bem_batch_offset(bem_batch_t b, int i, size_t* offset) {
  if (!b || !offset || i < 0 || i >= (int)b->plans.size()) {
    set_error("bem_batch_offset: bad argument");
    return BEM_ERR_ARG;
  }
  *offset = b->offset[i];
  return BEM_OK;
}

bem_status bem_batch_apply(bem_batch_t b, void* stream) {
  if (!b || !b->exec) {
    set_error("bem_batch_apply: null batch");
    return BEM_ERR_ARG;
  }
  BEM_CUDA_TRY(cudaGraphLaunch(b->exec, static_cast<cudaStream_t>(stream)));
  return BEM_OK;
}

int bem_batch_launches(bem_batch_t b) { return b ? b->launches : -1; }

}  // extern "C"
