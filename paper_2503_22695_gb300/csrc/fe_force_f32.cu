// Instantiations of the force kernel for split-precision plans (FP32
// arithmetic with the FP64 scalar set): per output, the law sets the host may
// pick (see fe_force.cu).
#include "fe_kernel.cuh"

namespace ibfe {

#define IBFE_FE_RUN(R, S, E, A, P, L)                                                        \
  template ib_status fe_run<R, S, E, A, P, L, IB_ELEM_HEX8>(                                 \
      ib_plan*, const MatTable&, const void*, const float*, const void*, void*, cudaStream_t)

IBFE_FE_RUN(float, df, false, false, false, kLawBase);
IBFE_FE_RUN(float, df, false, false, false, kLawBaseAct);
IBFE_FE_RUN(float, df, false, false, false, kLawAll);
IBFE_FE_RUN(float, df, true, false, false, kLawAll);

}  // namespace ibfe
