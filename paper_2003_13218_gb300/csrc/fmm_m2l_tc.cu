// fmm_m2l_tc.cu -- tensor-core (tcgen05) M2L for the mixed-precision path.
#include "fmm_internal.cuh"

namespace fmm {

bool tc_available(const Plan &, int) { return false; }
fmm_status tc_prepare(Plan &) { return FMM_OK; }
fmm_status launch_m2l_tc(Plan &, int) { return FMM_ERR_UNSUPPORTED; }
void tc_free(Plan &) {}

}  // namespace fmm
