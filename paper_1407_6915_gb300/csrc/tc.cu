// Tensor-core radix-16 path (split hi+lo FP16/BF16 operands, FP32 accumulate).
#include "plan.h"

namespace fftseg {

struct TcPlan {};

int tc_plan_create(fftseg_plan p)
{
    (void)p;
    return set_error(FFTSEG_E_UNSUPPORTED, "tensor-core precision is not built yet");
}
void tc_plan_destroy(fftseg_plan p) { delete p->tc; p->tc = nullptr; }
int tc_exec(fftseg_plan, const void *, void *, int64_t, cudaStream_t)
{
    return set_error(FFTSEG_E_UNSUPPORTED, "tensor-core precision is not built yet");
}
int64_t tc_launches_per_exec(fftseg_plan) { return 0; }

}  // namespace fftseg
