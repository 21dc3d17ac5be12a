// Measured choices the shape of a problem does not fix by itself:
//   - the launch shapes of the apply that are runtime choices: the cells per
//     load batch of the 2D fused cell walks (2 or 4; both kernels are built)
//     and the lines per CTA of the 3D z pass;
//   - the number of forked capture streams of a batch graph (how many of the
//     geometries' applies run side by side);
//   - the block size of the block-Jacobi preconditioner (fewer GMRES
//     iterations against a costlier block inversion and apply).
// Each candidate is timed on the device with the caller's own data; the
// winner is kept in a process-wide table keyed by the problem's shape, so
// later plans or batches of the same shape take it without timing again.
#include <chrono>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "bem_internal.h"

namespace bemfft {

static std::mutex g_tune_mu;
static std::map<std::string, int> g_tune;

static bool tune_lookup(const std::string& key, int* v) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_tune.find(key);
  if (it == g_tune.end()) return false;
  *v = it->second;
  return true;
}

static void tune_store(const std::string& key, int v) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune[key] = v;
}

static std::string plan_shape(const bem_plan_s* p) {
  return std::to_string(p->dim) + "/" + std::to_string(p->kernel) + "/" + std::to_string(p->n) + "/" +
         std::to_string(p->nb) + "/" + std::to_string(p->prec) + "/" + std::to_string(p->tc);
}

// (re)create S side streams and 2S events and capture the batch graph again
static bem_status batch_set_streams(bem_batch_s* b, int S) {
  if (S == b->nstreams && b->exec) return BEM_OK;
  for (auto s : b->side) cudaStreamDestroy(s);
  for (auto e : b->events) cudaEventDestroy(e);
  b->side.clear();
  b->events.clear();
  for (int s = 0; s < S; ++s) {
    cudaStream_t x;
    BEM_CUDA_TRY(cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking));
    b->side.push_back(x);
  }
  for (int s = 0; s < 2 * S; ++s) {
    cudaEvent_t e;
    BEM_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    b->events.push_back(e);
  }
  b->nstreams = S;
  batch_solve_free(b);  // its step graph was captured with the old streams
  return batch_capture(b);
}

// the plan whose kernels take the shape: the inner node plan of an
// accuracy-mode plan, else the plan itself
static bem_plan_s* shape_owner(bem_plan_s* p) { return p->pf ? p->pf->inner : p; }

// candidate values of the plan's runtime launch shape (empty: none)
static std::vector<int> shape_candidates(const bem_plan_s* q) {
  if (q->dim == 2 && q->v2 && q->prec == BEM_F32) return {2, 4};  // FP32 and tensor-core fused walks
  if (q->dim == 3) return {1, 2, 4, 8, 16};
  return {};
}

static void set_shape(bem_plan_s* p, int v) {
  bem_plan_s* q = shape_owner(p);
  if (q->dim == 2) q->cell_batch = v;
  else q->zpass_lines = v;
  // captured graphs hold the old launches
  ++q->op_version;
  ++p->op_version;
  ++p->pc_version;
}

}  // namespace bemfft

using namespace bemfft;

extern "C" {

bem_status bem_tune_shapes(bem_plan_t p, int reps, void* stream, int* chosen, double* best_ms_out) {
  if (!p || reps < 1) {
    set_error("bem_tune_shapes: need a plan and reps >= 1");
    return BEM_ERR_ARG;
  }
  if (bem_status dc = check_device(p, "bem_tune_shapes"); dc != BEM_OK) return dc;
  const std::vector<int> cand = shape_candidates(shape_owner(p));
  if (chosen) *chosen = 0;
  if (best_ms_out) *best_ms_out = 0.0;
  if (cand.empty()) return BEM_OK;
  const bem_layer layer = p->have_bc ? BEM_SYSTEM : BEM_SINGLE;
  const std::string key = "shape:" + plan_shape(p) + ":" + std::to_string(p->pf != nullptr) + ":" +
                          std::to_string((int)layer);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int best = 0;
  float best_ms = 0.0f;
  if (!tune_lookup(key, &best)) {
    // device vectors and events for the timing, released on every path
    struct Timing {
      void* in = nullptr;
      void* out = nullptr;
      cudaEvent_t e0 = nullptr, e1 = nullptr;
      ~Timing() {
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        cudaFree(in);
        cudaFree(out);
      }
    } tm;
    const size_t bytes = (size_t)p->nb * p->ncomp * prec_bytes(p);
    BEM_CUDA_TRY(cudaMalloc(&tm.in, bytes));
    BEM_CUDA_TRY(cudaMalloc(&tm.out, bytes));
    BEM_CUDA_TRY(cudaMemsetAsync(tm.in, 0, bytes, st));
    BEM_CUDA_TRY(cudaEventCreate(&tm.e0));
    BEM_CUDA_TRY(cudaEventCreate(&tm.e1));
    for (int v : cand) {
      set_shape(p, v);
      bem_status rc = apply_operator(p, layer, tm.in, tm.out, st);  // warm-up
      if (rc != BEM_OK) return rc;
      BEM_CUDA_TRY(cudaEventRecord(tm.e0, st));
      for (int i = 0; i < reps; ++i)
        if ((rc = apply_operator(p, layer, tm.in, tm.out, st)) != BEM_OK) return rc;
      BEM_CUDA_TRY(cudaEventRecord(tm.e1, st));
      BEM_CUDA_TRY(cudaEventSynchronize(tm.e1));
      float ms = 0.0f;
      BEM_CUDA_TRY(cudaEventElapsedTime(&ms, tm.e0, tm.e1));
      ms /= (float)reps;
      if (best == 0 || ms < best_ms) {
        best = v;
        best_ms = ms;
      }
    }
    tune_store(key, best);
  }
  set_shape(p, best);
  if (chosen) *chosen = best;
  if (best_ms_out) *best_ms_out = best_ms;
  return BEM_OK;
}

bem_status bem_tune_batch(bem_batch_t b, int reps, int* streams_out) {
  if (!b || reps < 1) {
    set_error("bem_tune_batch: need a batch and reps >= 1");
    return BEM_ERR_ARG;
  }
  if (bem_status dc = check_device(b->plans[0], "bem_tune_batch"); dc != BEM_OK) return dc;
  std::string key = "batch";
  for (auto* p : b->plans) key += ":" + plan_shape(p);
  key += ":" + std::to_string((int)b->layer);
  int best = 0;
  bem_status rc;
  if (!tune_lookup(key, &best)) {
    // timing stream and events, released on every path
    struct Timing {
      cudaStream_t ts = nullptr;
      cudaEvent_t e0 = nullptr, e1 = nullptr;
      ~Timing() {
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        if (ts) cudaStreamDestroy(ts);
      }
    } tm;
    BEM_CUDA_TRY(cudaStreamCreateWithFlags(&tm.ts, cudaStreamNonBlocking));
    BEM_CUDA_TRY(cudaEventCreate(&tm.e0));
    BEM_CUDA_TRY(cudaEventCreate(&tm.e1));
    float best_ms = 0.0f;
    for (int S : {1, 2, 4, 8}) {
      if ((rc = batch_set_streams(b, S)) != BEM_OK) return rc;
      for (int i = 0; i < 2; ++i) BEM_CUDA_TRY(cudaGraphLaunch(b->exec, tm.ts));
      BEM_CUDA_TRY(cudaEventRecord(tm.e0, tm.ts));
      for (int i = 0; i < reps; ++i) BEM_CUDA_TRY(cudaGraphLaunch(b->exec, tm.ts));
      BEM_CUDA_TRY(cudaEventRecord(tm.e1, tm.ts));
      BEM_CUDA_TRY(cudaEventSynchronize(tm.e1));
      float ms = 0.0f;
      BEM_CUDA_TRY(cudaEventElapsedTime(&ms, tm.e0, tm.e1));
      if (best == 0 || ms < best_ms) {
        best = S;
        best_ms = ms;
      }
    }
    tune_store(key, best);
  }
  if ((rc = batch_set_streams(b, best)) != BEM_OK) return rc;
  if (streams_out) *streams_out = best;
  return BEM_OK;
}

bem_status bem_tune_preconditioner(bem_plan_t p, const uint8_t* bc, const double* data, double c, double tol,
                                   int max_iter, int restart, int* block_out) {
  if (!p || !bc || !data || !(tol > 0.0)) {
    set_error("bem_tune_preconditioner: null argument or tol <= 0");
    return BEM_ERR_ARG;
  }
  const std::string key = "pc:" + plan_shape(p) + ":" + std::to_string(p->companion != nullptr) + ":" +
                          std::to_string((int)std::floor(std::log10(tol)));
  int best = 0;
  bem_status rc;
  if (!tune_lookup(key, &best)) {
    const int64_t M = p->nb * p->ncomp;
    std::vector<double> u(M), q(M);
    std::vector<int> cand;
    for (int bs : {32, 64, 128, 256})
      if (bs * p->ncomp <= (p->dim == 2 ? 256 : 192)) cand.push_back(bs);  // device-built or small host blocks
    double best_s = 0.0;
    for (int bs : cand) {
      if ((rc = bem_set_preconditioner(p, 1, bs)) != BEM_OK) return rc;
      bem_solve_info info{};
      const auto t0 = std::chrono::steady_clock::now();  // includes building the preconditioner
      rc = bem_solve(p, bc, data, c, tol, max_iter, restart, nullptr, u.data(), q.data(), &info, nullptr);
      const double s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
      if (rc != BEM_OK && rc != BEM_ERR_NOT_CONVERGED) return rc;
      if (rc == BEM_OK && (best == 0 || s < best_s)) {
        best = bs;
        best_s = s;
      }
    }
    if (best == 0) {
      set_error("bem_tune_preconditioner: no candidate block size converged");
      return BEM_ERR_NOT_CONVERGED;
    }
    tune_store(key, best);
  }
  if ((rc = bem_set_preconditioner(p, 1, best)) != BEM_OK) return rc;
  if (block_out) *block_out = best;
  return BEM_OK;
}

}  // extern "C"
