// Instantiations of the force kernel and its adjoint for IB_FP32_SPLIT_F32STAB
// plans (every scalar in FP32) and IB_FP64 plans: the full law set, plus the
// base set for the FP32-scalar forward.
#include "fe_kernel.cuh"

namespace ibfe {

#define IBFE_FE_RUN(R, S, E, A, P, L)                                                        \
  template ib_status fe_run<R, S, E, A, P, L, IB_ELEM_HEX8>(                                 \
      ib_plan*, const MatTable&, const void*, const float*, const void*, void*, cudaStream_t)

IBFE_FE_RUN(float, float, false, false, false, kLawBase);
IBFE_FE_RUN(float, float, false, false, false, kLawAll);
IBFE_FE_RUN(float, float, true, false, false, kLawAll);
IBFE_FE_RUN(float, float, false, true, false, kLawAll);
IBFE_FE_RUN(float, float, false, true, true, kLawAll);
IBFE_FE_RUN(double, double, false, false, false, kLawAll);
IBFE_FE_RUN(double, double, true, false, false, kLawAll);
IBFE_FE_RUN(double, double, false, true, false, kLawAll);
IBFE_FE_RUN(double, double, false, true, true, kLawAll);

}  // namespace ibfe
