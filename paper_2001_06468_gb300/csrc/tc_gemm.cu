// tc_gemm.cu -- the rank-64 update M -= C R of the Gauss-Jordan inverse on the
// tensor cores.  Placeholder until the tcgen05 kernel lands: reports that no
// tensor-core kernel is available, so the factor entry point rejects the
// TF32 and BF16 precisions instead of silently using another path.
#include "nrs_internal.cuh"

namespace nrs {

bool tc_available() { return false; }

bool launch_tc_gj_update(Ctx &, float *, int64_t, int64_t, const float *, const float *, int)
{
    return false;
}

}  // namespace nrs
