// Batched form: independent structures, each with its own plan, run as the
// branches of one CUDA graph.
//
// At creation every instance gets its plan and its own branch stream; the
// forward and adjoint sequences of all instances are captured once into two
// graphs (a root event fans out to the branch streams and every branch joins
// back), so one cudaGraphLaunch replays the whole batch: no per-instance host
// work, and the GPU overlaps the instances' kernels.  Each branch is exactly
// the single-instance call (ib_forward, ib_backward), so every instance's
// results are bitwise those of the individual entry points.
#include <cstring>
#include <vector>

#include "ib_device.cuh"

struct ib_batch {
  int n;
  int precision;
  std::vector<ib_instance> inst;
  std::vector<ib_plan*> plans;
  std::vector<cudaStream_t> branch;
  std::vector<cudaEvent_t> done;
  double* gparams;            // device [n][IB_MAX_MATERIALS][kParamRow]
  cudaEvent_t root;
  cudaStream_t cap;
  cudaGraphExec_t fwd, adj;
  bool has_adj;
};

namespace ibfe {
namespace {

void destroy(ib_batch* b) {
  if (!b) return;
  if (b->fwd) cudaGraphExecDestroy(b->fwd);
  if (b->adj) cudaGraphExecDestroy(b->adj);
  for (ib_plan* p : b->plans)
    if (p) ib_plan_destroy(p);
  for (cudaStream_t s : b->branch)
    if (s) cudaStreamDestroy(s);
  for (cudaEvent_t e : b->done)
    if (e) cudaEventDestroy(e);
  if (b->gparams) cudaFree(b->gparams);
  if (b->root) cudaEventDestroy(b->root);
  if (b->cap) cudaStreamDestroy(b->cap);
  delete b;
}

ib_status run_forward(ib_batch* b, int i, cudaStream_t s) {
  const ib_instance& in = b->inst[i];
  return ib_forward(b->plans[i], in.mats, in.n_mats, &in.x, in.u, in.G, in.f, in.U, s);
}

ib_status run_adjoint(ib_batch* b, int i, cudaStream_t s) {
  const ib_instance& in = b->inst[i];
  return ib_backward(b->plans[i], in.mats, in.n_mats, &in.x, in.u, in.G, in.gG, in.gf, in.gU,
                     in.gx, in.gu, b->gparams + (size_t)i * kParamRow * IB_MAX_MATERIALS, s);
}

// Capture fn(b, i, branch_i) for every instance as branches of one graph.
ib_status capture(ib_batch* b, ib_status (*fn)(ib_batch*, int, cudaStream_t),
                  cudaGraphExec_t* out) {
  if (cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
    return IB_ERR_CUDA;
  ib_status st = cudaEventRecord(b->root, b->cap) == cudaSuccess ? IB_OK : IB_ERR_CUDA;
  for (int i = 0; i < b->n && st == IB_OK; ++i) {
    if (cudaStreamWaitEvent(b->branch[i], b->root, 0) != cudaSuccess) st = IB_ERR_CUDA;
    if (st == IB_OK) st = fn(b, i, b->branch[i]);
    if (st == IB_OK && (cudaEventRecord(b->done[i], b->branch[i]) != cudaSuccess ||
                        cudaStreamWaitEvent(b->cap, b->done[i], 0) != cudaSuccess))
      st = IB_ERR_CUDA;
  }
  cudaGraph_t g = nullptr;
  const cudaError_t ec = cudaStreamEndCapture(b->cap, &g);
  if (st == IB_OK && ec != cudaSuccess) st = IB_ERR_CUDA;
  if (st == IB_OK && cudaGraphInstantiate(out, g, 0) != cudaSuccess) st = IB_ERR_CUDA;
  if (g) cudaGraphDestroy(g);
  cudaGetLastError();
  return st;
}

}  // namespace
}  // namespace ibfe

using namespace ibfe;

extern "C" {

ib_status ib_batch_create(int32_t n, const ib_instance* inst, int32_t precision, void* stream,
                          ib_batch** out) {
  if (!out) return IB_ERR_INVALID_ARG;
  *out = nullptr;
  if (n <= 0 || !inst) return IB_ERR_INVALID_ARG;
  bool has_adj = true;
  for (int i = 0; i < n; ++i) {
    const ib_instance& in = inst[i];
    if (!in.u || !in.G || !in.f || !in.U) return IB_ERR_INVALID_ARG;
    const bool a = in.gU && in.gf && in.gu && in.gx;
    if (!a) has_adj = false;
  }
  ib_batch* b = new ib_batch();
  b->n = n;
  b->precision = precision;
  b->inst.assign(inst, inst + n);
  b->plans.assign(n, nullptr);
  b->branch.assign(n, nullptr);
  b->done.assign(n, nullptr);
  b->gparams = nullptr;
  b->root = nullptr;
  b->cap = nullptr;
  b->fwd = b->adj = nullptr;
  b->has_adj = has_adj;
  const size_t gbytes = sizeof(double) * kParamRow * IB_MAX_MATERIALS * (size_t)n;
  ib_status st = cudaMalloc((void**)&b->gparams, gbytes) == cudaSuccess &&
                         cudaMemset(b->gparams, 0, gbytes) == cudaSuccess
                     ? IB_OK
                     : IB_ERR_CUDA;
  for (int i = 0; i < n && st == IB_OK; ++i) {
    st = ib_plan_create(&inst[i].mesh, &inst[i].grid, IB_QUAD_GAUSS2, precision, stream,
                        &b->plans[i]);
    if (st == IB_OK)
      st = ib_plan_autotune(b->plans[i], inst[i].mats, inst[i].n_mats, &inst[i].x, inst[i].u,
                            stream, nullptr);
    if (st == IB_OK && (cudaStreamCreateWithFlags(&b->branch[i], cudaStreamNonBlocking) != cudaSuccess ||
                        cudaEventCreateWithFlags(&b->done[i], cudaEventDisableTiming) != cudaSuccess))
      st = IB_ERR_CUDA;
  }
  if (st == IB_OK && (cudaEventCreateWithFlags(&b->root, cudaEventDisableTiming) != cudaSuccess ||
                      cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess))
    st = IB_ERR_CUDA;
  if (st == IB_OK) st = capture(b, run_forward, &b->fwd);
  if (st == IB_OK && has_adj) st = capture(b, run_adjoint, &b->adj);
  if (st != IB_OK) {
    destroy(b);
    return st;
  }
  *out = b;
  return IB_OK;
}

ib_status ib_batch_forward(ib_batch* b, void* stream) {
  if (!b || !b->fwd) return IB_ERR_INVALID_ARG;
  return cudaGraphLaunch(b->fwd, reinterpret_cast<cudaStream_t>(stream)) == cudaSuccess
             ? IB_OK
             : IB_ERR_CUDA;
}

ib_status ib_batch_adjoint(ib_batch* b, void* stream) {
  if (!b || !b->adj) return IB_ERR_INVALID_ARG;
  return cudaGraphLaunch(b->adj, reinterpret_cast<cudaStream_t>(stream)) == cudaSuccess
             ? IB_OK
             : IB_ERR_CUDA;
}

ib_status ib_batch_gparams(ib_batch* b, double* gparams, void* stream) {
  if (!b || !gparams) return IB_ERR_INVALID_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (cudaMemcpyAsync(gparams, b->gparams, sizeof(double) * kParamRow * IB_MAX_MATERIALS * (size_t)b->n,
                      cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return IB_ERR_CUDA;
  return cudaStreamSynchronize(s) == cudaSuccess ? IB_OK : IB_ERR_CUDA;
}

ib_status ib_batch_destroy(ib_batch* b) {
  if (!b) return IB_ERR_INVALID_ARG;
  destroy(b);
  return IB_OK;
}

}  // extern "C"
