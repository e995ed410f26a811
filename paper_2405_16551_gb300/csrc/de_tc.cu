// de_tc.cu -- split-precision (BF16x3 / TF32x3) tensor-core path.
#include "de_kernels.h"

namespace de {

de_status tc_plan_build(TcPlan& p, std::vector<RunDesc>& runs, const de_config* cfgs, int prec, cudaStream_t s,
                        std::string& err) {
  (void)p; (void)runs; (void)cfgs; (void)prec; (void)s;
  err = "split precision is not available in this build";
  return DE_ERR_UNSUPPORTED;
}
void tc_plan_free(TcPlan& p) { (void)p; }
void tc_generation_launch(const TcPlan& p, const RunDesc* runs, cudaStream_t s) { (void)p; (void)runs; (void)s; }
de_status tc_eval_launch(const TcPlan& p, const RunDesc* runs, int run, const RunDesc& R, const double* x, int64_t ld,
                         int n, double* f, cudaStream_t s, std::string& err) {
  (void)p; (void)runs; (void)run; (void)R; (void)x; (void)ld; (void)n; (void)f; (void)s;
  err = "split precision is not available in this build";
  return DE_ERR_UNSUPPORTED;
}

}  // namespace de
