// Force-kernel launches of packed plans (the batched form): FP32 split
// positions, hexahedra, each element's h and material row read through its
// instance; the law sets and outputs the forward and the backward use.  The
// grid sizing is fe_run's.
#include "fe_kernel.cuh"

namespace ibfe {

template <bool kAdj, bool kParams, int kLaws>
ib_status fe_run_packed(ib_plan* p, const MatTable& mt, const void* xa, const float* off,
                        const void* v, void* out, cudaStream_t s) {
  FeArgs<float> A = make_args<float>(p, xa, off, v, out);
  const int threads = 128, per_cta = threads / 8;
  const int per_sm = kAdj ? fe8_min_blocks<float, kAdj>() : p->fe_ctas;
  const int blocks = std::min((p->E + per_cta - 1) / per_cta, p->sm_count * per_sm);
  if (cudaMemsetAsync(A.next, 0, sizeof(int), s) != cudaSuccess) return IB_ERR_CUDA;
  k_fe8<float, df, false, kAdj, kParams, kLaws, true><<<blocks, threads, 0, s>>>(A, mt);
  return cudaGetLastError() == cudaSuccess ? IB_OK : IB_ERR_CUDA;
}

#define IBFE_FE_RUN_PACKED(A, P, L)                                                          \
  template ib_status fe_run_packed<A, P, L>(ib_plan*, const MatTable&, const void*,          \
                                            const float*, const void*, void*, cudaStream_t)
IBFE_FE_RUN_PACKED(false, false, kLawBase);
IBFE_FE_RUN_PACKED(false, false, kLawBaseAct);
IBFE_FE_RUN_PACKED(false, false, kLawAll);
IBFE_FE_RUN_PACKED(true, false, kLawBase);
IBFE_FE_RUN_PACKED(true, false, kLawBaseAct);
IBFE_FE_RUN_PACKED(true, false, kLawAll);
IBFE_FE_RUN_PACKED(true, true, kLawBaseAct);
IBFE_FE_RUN_PACKED(true, true, kLawAll);
#undef IBFE_FE_RUN_PACKED

}  // namespace ibfe
