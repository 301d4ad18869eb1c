// tc_gemm.cu -- placeholder until the tcgen05 contraction lands.
#include "tc_gemm.h"

namespace mcinv {

TcGemmPlan *tc_gemm_plan_create(const uint16_t *, size_t, const uint16_t *, size_t, long long, float *,
                                long long, long long, std::string *why)
{
    if (why) *why = "not available in this build";
    return nullptr;
}
cudaError_t tc_gemm_run(TcGemmPlan *, long long, cudaStream_t) { return cudaErrorNotSupported; }
void tc_gemm_plan_destroy(TcGemmPlan *) {}

}  // namespace mcinv
