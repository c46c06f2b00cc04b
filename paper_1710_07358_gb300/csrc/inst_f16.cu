// f16 kernels: sums and products accumulate in fp32, max/min return f16.
#include "launch.cuh"

namespace pr {
void register_f16() {
    using K = KeyF32<LdF16, 2>;
    reg_family<SumF<LdF16, float>>(PR_F16, PR_SUM, PR_PREC_PLAIN, AUX_NONE, true, true);
    reg_family<SumF<LdF16, double>>(PR_F16, PR_SUM, PR_PREC_FP64_COMBINE, AUX_NONE, true, true);
    reg_family<SumComp<LdF16>>(PR_F16, PR_SUM, PR_PREC_COMPENSATED, AUX_NONE, true, true);
    reg_family<ProdF<LdF16>>(PR_F16, PR_PROD, PR_PREC_PLAIN, AUX_NONE, true, true);
    reg_family<MaxMinF<LdF16, 2, true>>(PR_F16, PR_MAX, PR_PREC_PLAIN, AUX_NONE, true, true);
    reg_family<MaxMinF<LdF16, 2, false>>(PR_F16, PR_MIN, PR_PREC_PLAIN, AUX_NONE, true, true);
    reg_family<ArgExtF<LdF16, 2, true>>(PR_F16, PR_MAX, PR_PREC_PLAIN, AUX_ARG, true, true);
    reg_family<ArgExtF<LdF16, 2, false>>(PR_F16, PR_MIN, PR_PREC_PLAIN, AUX_ARG, true, true);
}
}  // namespace pr
