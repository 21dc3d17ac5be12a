// Batched apply: many plans (geometries of uneven grid sizes) applied as one
// CUDA graph.  The graph is captured once: the plans are distributed
// round-robin over a few forked capture streams, so the applies of small
// geometries run side by side, and the whole batch is then replayed with a
// single graph launch per batched apply (no per-kernel launch overhead).
// Inputs and outputs live in two packed device buffers owned by the batch
// (segment of plan i at offset[i], nb_i * ncomp_i values of the common
// precision).  When bem_set_bc has rebuilt a plan's system operator since the
// capture, the next apply captures the graph again.
#include <algorithm>
#include <vector>

#include "bem_internal.h"

using namespace bemfft;

namespace bemfft {

bem_status batch_issue_applies(bem_batch_s* b, const void* in, void* out, cudaStream_t cap) {
  const int S = b->nstreams;
  const size_t tb = prec_bytes(b->plans[0]);
  bem_status rc = BEM_OK;
  BEM_CUDA_TRY(cudaEventRecord(b->events[0], cap));
  for (int s = 1; s < S; ++s) BEM_CUDA_TRY(cudaStreamWaitEvent(b->side[s], b->events[0], 0));
  // grouped launches first (one stream each), then the remaining plans round-robin
  int k = 0;
  for (size_t gi = 0; gi < b->groups.size() && rc == BEM_OK; ++gi, ++k) {
    cudaStream_t s = k % S == 0 ? cap : b->side[k % S];
    rc = group_issue(b->groups[gi], b->plans, b->layer, in, out, b->offset, s);
  }
  for (size_t si = 0; si < b->solo.size() && rc == BEM_OK; ++si, ++k) {
    const int i = b->solo[si];
    cudaStream_t s = k % S == 0 ? cap : b->side[k % S];
    const unsigned char* pin = static_cast<const unsigned char*>(in) + b->offset[i] * tb;
    unsigned char* pout = static_cast<unsigned char*>(out) + b->offset[i] * tb;
    rc = apply_operator(b->plans[i], b->layer, pin, pout, s);
  }
  for (int s = 1; s < S; ++s) {
    BEM_CUDA_TRY(cudaEventRecord(b->events[S + s], b->side[s]));
    BEM_CUDA_TRY(cudaStreamWaitEvent(cap, b->events[S + s], 0));
  }
  return rc;
}

// Plans that share a grid (FP32 four-step, same thread count) and a field
// count are applied by one grouped persistent launch; the kernel parameters of
// a group are built here, before any capture, from the plans' current
// operators.
static bem_status batch_build_groups(bem_batch_s* b) {
  for (auto& g : b->groups) group_free(g);
  b->groups.clear();
  b->solo.clear();
  std::vector<int> keys;  // distinct (thread count, field count) of the eligible plans
  std::vector<std::vector<int>> members;
  for (size_t i = 0; i < b->plans.size(); ++i) {
    const bem_plan_s* p = b->plans[i];
    if (!b->grouped || !group_eligible(p) || (b->layer == BEM_SYSTEM && !p->have_bc)) {
      b->solo.push_back((int)i);
      continue;
    }
    const Operator& op =
        b->layer == BEM_SINGLE ? p->op_single : (b->layer == BEM_DOUBLE ? p->op_double : p->op_system);
    const int key = p->threads * 8 + op.nf;
    size_t k = 0;
    while (k < keys.size() && keys[k] != key) ++k;
    if (k == keys.size()) {
      keys.push_back(key);
      members.emplace_back();
    }
    members[k].push_back((int)i);
  }
  for (size_t k = 0; k < members.size(); ++k) {
    if (members[k].size() < 2) {
      b->solo.push_back(members[k][0]);
      continue;
    }
    BatchGroup g;
    g.members = members[k];
    bem_status rc = group_build(g, b->plans, b->layer);
    if (rc != BEM_OK) {
      group_free(g);
      return rc;
    }
    b->groups.push_back(g);
  }
  std::sort(b->solo.begin(), b->solo.end());
  return BEM_OK;
}

bem_status batch_capture(bem_batch_s* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
  b->launches = 0;
  bem_status grc = batch_build_groups(b);
  if (grc != BEM_OK) return grc;
  cudaStream_t cap = b->side[0];
  if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    set_error("bem_batch: stream capture failed to begin");
    return BEM_ERR_CUDA;
  }
  bem_status rc = batch_issue_applies(b, b->d_in, b->d_out, cap);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(cap, &g);
  if (rc != BEM_OK) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (e != cudaSuccess || !g) {
    set_error(std::string("bem_batch: capture failed: ") + cudaGetErrorString(e));
    return BEM_ERR_CUDA;
  }
  b->graph = g;
  if (cudaGraphInstantiate(&b->exec, g, 0) != cudaSuccess) {
    set_error("bem_batch: graph instantiation failed");
    return BEM_ERR_CUDA;
  }
  b->versions.clear();
  for (auto* p : b->plans) b->versions.push_back(p->op_version);
  for (const auto& g : b->groups) b->launches += 2 * (int)g.members.size() + 1;  // preps, one column launch, reductions
  for (int i : b->solo) b->launches += bem_launches_per_apply(b->plans[i], b->layer);
  return BEM_OK;
}

bem_status batch_refresh(bem_batch_s* b) {
  if (b->layer != BEM_SYSTEM) return BEM_OK;
  for (size_t i = 0; i < b->plans.size(); ++i)
    if (b->plans[i]->op_version != b->versions[i]) return batch_capture(b);
  return BEM_OK;
}

}  // namespace bemfft

extern "C" {

bem_status bem_batch_destroy(bem_batch_t b) {
  if (!b) return BEM_OK;
  batch_solve_free(b);
  if (b->companions) bem_batch_destroy(b->companions);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  for (auto& g : b->groups) group_free(g);
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
  if (layer != BEM_SINGLE && layer != BEM_DOUBLE && layer != BEM_SYSTEM) {
    set_error("bem_batch_create: unknown layer");
    return BEM_ERR_ARG;
  }
  *out = nullptr;
  for (int i = 0; i < count; ++i) {
    if (!plans[i]) {
      set_error("bem_batch_create: null plan");
      return BEM_ERR_ARG;
    }
    for (int k = 0; k < i; ++k)
      if (plans[k] == plans[i]) {
        set_error("bem_batch_create: a plan appears twice (its scratch would be shared by two applies)");
        return BEM_ERR_ARG;
      }
    if (bem_status dc = check_device(plans[i], "bem_batch_create"); dc != BEM_OK) return dc;
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
  b->layer = layer;
  b->nstreams = streams;
  for (int i = 0; i < count; ++i) {
    b->plans.push_back(plans[i]);
    b->offset.push_back(b->total);
    b->total += (size_t)plans[i]->nb * plans[i]->ncomp;
  }
  b->offset.push_back(b->total);
  const size_t tb = prec_bytes(plans[0]);
  auto fail = [&](bem_status rc) {
    bem_batch_destroy(b);
    return rc;
  };
  if (cudaMalloc(&b->d_in, b->total * tb) != cudaSuccess || cudaMalloc(&b->d_out, b->total * tb) != cudaSuccess) {
    set_error("bem_batch_create: out of device memory");
    return fail(BEM_ERR_OOM);
  }
  if (cudaMemset(b->d_in, 0, b->total * tb) != cudaSuccess || cudaMemset(b->d_out, 0, b->total * tb) != cudaSuccess) {
    set_error("bem_batch_create: clearing the batch buffers failed");
    return fail(BEM_ERR_CUDA);
  }
  for (int s = 0; s < streams; ++s) {
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
  bem_status rc = batch_capture(b);
  if (rc != BEM_OK) return fail(rc);
  (void)stream;
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
  bem_status rc = check_device(b->plans[0], "bem_batch_apply");
  if (rc != BEM_OK) return rc;
  if ((rc = batch_refresh(b)) != BEM_OK) return rc;
  BEM_CUDA_TRY(cudaGraphLaunch(b->exec, static_cast<cudaStream_t>(stream)));
  return BEM_OK;
}

int bem_batch_launches(bem_batch_t b) { return b ? b->launches : -1; }

bem_status bem_batch_set_grouping(bem_batch_t b, int enable) {
  if (!b) {
    set_error("bem_batch_set_grouping: null batch");
    return BEM_ERR_ARG;
  }
  b->grouped = enable != 0;
  batch_solve_free(b);  // its step graph holds the old launches
  return batch_capture(b);
}

}  // extern "C"
