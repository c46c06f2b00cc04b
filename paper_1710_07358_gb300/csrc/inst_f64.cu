// fp64 kernels.  The product splits each vector between the fp64 and the
// integer pipes (ProdMix; with the gradient's aux records, the integer pipes
// alone: ProdAux<ProdExt>); the sum uses fp64 adds; max/min compare integer
// keys.
#include "launch.cuh"
#include "prod64.cuh"

namespace pr {
void register_f64() {
    reg_family<SumF64>(PR_F64, PR_SUM, PR_PREC_PLAIN, AUX_NONE, true, true);
    reg_family<ProdMix>(PR_F64, PR_PROD, PR_PREC_PLAIN, AUX_NONE, true, true);
    reg_family<MaxMin<KeyF64, true>>(PR_F64, PR_MAX, PR_PREC_PLAIN, AUX_NONE, true, true);
    reg_family<MaxMin<KeyF64, false>>(PR_F64, PR_MIN, PR_PREC_PLAIN, AUX_NONE, true, true);
    reg_family<ArgExt<KeyF64, true>>(PR_F64, PR_MAX, PR_PREC_PLAIN, AUX_ARG, true, true);
    reg_family<ArgExt<KeyF64, false>>(PR_F64, PR_MIN, PR_PREC_PLAIN, AUX_ARG, true, true);
    reg_family<ProdAux<ProdExt>>(PR_F64, PR_PROD, PR_PREC_PLAIN, AUX_PROD, false, true);
}
}  // namespace pr
