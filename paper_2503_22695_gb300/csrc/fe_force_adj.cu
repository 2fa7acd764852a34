// Instantiations of the force adjoint for split-precision plans: per output,
// the law sets the host may pick (see fe_force.cu).
#include "fe_kernel.cuh"

namespace ibfe {

#define IBFE_FE_RUN(R, S, E, A, P, L)                                                        \
  template ib_status fe_run<R, S, E, A, P, L, IB_ELEM_HEX8>(                                 \
      ib_plan*, const MatTable&, const void*, const float*, const void*, void*, cudaStream_t)

IBFE_FE_RUN(float, df, false, true, false, kLawBase);
IBFE_FE_RUN(float, df, false, true, false, kLawBaseAct);
IBFE_FE_RUN(float, df, false, true, false, kLawAll);
IBFE_FE_RUN(float, df, false, true, true, kLawBaseAct);
IBFE_FE_RUN(float, df, false, true, true, kLawAll);

}  // namespace ibfe
