// fp32 segmented kernels (also the row reductions behind autograd).
#include "launch.cuh"

namespace pr {
void register_f32_seg() {
    using K = KeyF32<LdF32, 0>;
    reg_family<SumF<LdF32, float>>(PR_F32, PR_SUM, PR_PREC_PLAIN, AUX_NONE, false, true);
    reg_family<SumF<LdF32, double>>(PR_F32, PR_SUM, PR_PREC_FP64_COMBINE, AUX_NONE, false, true);
    reg_family<SumComp<LdF32>>(PR_F32, PR_SUM, PR_PREC_COMPENSATED, AUX_NONE, false, true);
    reg_family<ProdF<LdF32>>(PR_F32, PR_PROD, PR_PREC_PLAIN, AUX_NONE, false, true);
    reg_family<MaxMinF<LdF32, 0, true>>(PR_F32, PR_MAX, PR_PREC_PLAIN, AUX_NONE, false, true);
    reg_family<MaxMinF<LdF32, 0, false>>(PR_F32, PR_MIN, PR_PREC_PLAIN, AUX_NONE, false, true);
    reg_family<ArgExtF<LdF32, 0, true>>(PR_F32, PR_MAX, PR_PREC_PLAIN, AUX_ARG, true, true);
    reg_family<ArgExtF<LdF32, 0, false>>(PR_F32, PR_MIN, PR_PREC_PLAIN, AUX_ARG, true, true);
    reg_family<ProdAux<ProdF<LdF32>>>(PR_F32, PR_PROD, PR_PREC_PLAIN, AUX_PROD, false, true);
}
}  // namespace pr
