// batch.cu -- multi-molecule SCF (placeholder until the batched path lands).
#include "hf_internal.h"

extern "C" int hf_scf_solve_batch(hf_basis* const* bases, int count, const hf_scf_opts* opts, hf_scf_result* results,
                                  int* status) {
  (void)bases; (void)count; (void)opts; (void)results; (void)status;
  return hf_fail(HF_ERR_INVALID, "hf_scf_solve_batch: not available in this build");
}
