// bf16 kernels: sums and products accumulate in fp32, max/min return bf16.
#include "launch.cuh"

namespace pr {
void register_bf16() {
    using K = KeyF32<LdBF16, 1>;
    reg_family<SumF<LdBF16, float>>(PR_BF16, PR_SUM, PR_PREC_PLAIN, AUX_NONE, true, true);
    reg_family<SumF<LdBF16, double>>(PR_BF16, PR_SUM, PR_PREC_FP64_COMBINE, AUX_NONE, true, true);
    reg_family<SumComp<LdBF16>>(PR_BF16, PR_SUM, PR_PREC_COMPENSATED, AUX_NONE, true, true);
    reg_family<ProdF<LdBF16>>(PR_BF16, PR_PROD, PR_PREC_PLAIN, AUX_NONE, true, true);
    reg_family<MaxMinF<LdBF16, 1, true>>(PR_BF16, PR_MAX, PR_PREC_PLAIN, AUX_NONE, true, true);
    reg_family<MaxMinF<LdBF16, 1, false>>(PR_BF16, PR_MIN, PR_PREC_PLAIN, AUX_NONE, true, true);
    reg_family<ArgExtF<LdBF16, 1, true>>(PR_BF16, PR_MAX, PR_PREC_PLAIN, AUX_ARG, true, true);
    reg_family<ArgExtF<LdBF16, 1, false>>(PR_BF16, PR_MIN, PR_PREC_PLAIN, AUX_ARG, true, true);
}
}  // namespace pr
