// Instantiations of the force kernel and its adjoints for quadratic (P2) tetrahedra
// (every precision, every output, the full law set).
#include "fe_kernel.cuh"

namespace ibfe {

#define IBFE_FE_RUN(R, S, E, A, P)                                                           \
  template ib_status fe_run<R, S, E, A, P, kLawAll, IB_ELEM_TET10>(                           \
      ib_plan*, const MatTable&, const void*, const float*, const void*, void*, cudaStream_t)

IBFE_FE_RUN(float, df, false, false, false);
IBFE_FE_RUN(float, df, true, false, false);
IBFE_FE_RUN(float, df, false, true, false);
IBFE_FE_RUN(float, df, false, true, true);
IBFE_FE_RUN(float, float, false, false, false);
IBFE_FE_RUN(float, float, true, false, false);
IBFE_FE_RUN(float, float, false, true, false);
IBFE_FE_RUN(float, float, false, true, true);
IBFE_FE_RUN(double, double, false, false, false);
IBFE_FE_RUN(double, double, true, false, false);
IBFE_FE_RUN(double, double, false, true, false);
IBFE_FE_RUN(double, double, false, true, true);

}  // namespace ibfe
