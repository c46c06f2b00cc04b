// i32 kernels: exact integer and bitwise combiners.
#include "launch.cuh"

namespace pr {
void register_i32() {
    reg_family<IntOp<LdI32, uint64_t, 0>>(PR_I32, PR_SUM, PR_PREC_PLAIN, AUX_NONE, true, true);
    reg_family<IntOp<LdI32, uint32_t, 1>>(PR_I32, PR_PROD, PR_PREC_PLAIN, AUX_NONE, true, true);
    reg_family<IntOp<LdI32, uint32_t, 4>>(PR_I32, PR_AND, PR_PREC_PLAIN, AUX_NONE, true, true);
    reg_family<IntOp<LdI32, uint32_t, 5>>(PR_I32, PR_OR, PR_PREC_PLAIN, AUX_NONE, true, true);
    reg_family<IntOp<LdI32, uint32_t, 6>>(PR_I32, PR_XOR, PR_PREC_PLAIN, AUX_NONE, true, true);
    reg_family<MaxMin<KeyI32, true>>(PR_I32, PR_MAX, PR_PREC_PLAIN, AUX_NONE, true, true);
    reg_family<MaxMin<KeyI32, false>>(PR_I32, PR_MIN, PR_PREC_PLAIN, AUX_NONE, true, true);
    reg_family<ArgExt<KeyI32, true>>(PR_I32, PR_MAX, PR_PREC_PLAIN, AUX_ARG, true, true);
    reg_family<ArgExt<KeyI32, false>>(PR_I32, PR_MIN, PR_PREC_PLAIN, AUX_ARG, true, true);
}
}  // namespace pr
