// Instantiations of the force kernel and its adjoint for
// IB_FP32_SPLIT_DFVOL plans on linear and quadratic tetrahedra: every law,
// J - 1 from double-float kinematics (fe_kernel.cuh, exact_jm1).
#include "fe_kernel.cuh"

namespace ibfe {

#define IBFE_FE_RUN(E, A, P, T)                                                           \
  template ib_status fe_run<float, df, E, A, P, kLawAll | kLawVolX, T>(                   \
      ib_plan*, const MatTable&, const void*, const float*, const void*, void*, cudaStream_t)

IBFE_FE_RUN(false, false, false, IB_ELEM_TET4);
IBFE_FE_RUN(true, false, false, IB_ELEM_TET4);
IBFE_FE_RUN(false, true, false, IB_ELEM_TET4);
IBFE_FE_RUN(false, true, true, IB_ELEM_TET4);
IBFE_FE_RUN(false, false, false, IB_ELEM_TET10);
IBFE_FE_RUN(true, false, false, IB_ELEM_TET10);
IBFE_FE_RUN(false, true, false, IB_ELEM_TET10);
IBFE_FE_RUN(false, true, true, IB_ELEM_TET10);

}  // namespace ibfe
