/* A plain C99 user of include/hf.h (compiled and run by tests/test_abi.py):
 * default options, error strings, and the shape of a J/K call.  Without a
 * GPU, hf_ctx_create returns HF_ERR_CUDA and the program stops there. */
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "hf.h"

int main(void) {
  hf_jk_opts jk;
  hf_scf_opts scf;
  hf_jk_opts_default(&jk);
  hf_scf_opts_default(&scf);
  printf("tau %g max_iter %d\n", jk.schwarz_tau, scf.max_iter);
  printf("%s\n", hf_strerror(HF_ERR_ODD_ELECTRONS));

  hf_ctx* ctx = NULL;
  int rc = hf_ctx_create(&ctx, 0, 0, NULL);
  if (rc != HF_OK) {
    printf("ctx %d\n", rc);
    return 0;
  }
  /* H2, one s shell of one primitive per atom (bohr) */
  hf_atom atoms[2] = {{1, {0.0, 0.0, 0.0}}, {1, {1.4, 0.0, 0.0}}};
  hf_shell shells[2] = {{0, 0, 1, 0}, {1, 0, 1, 1}};
  double exps[2] = {0.8, 0.8}, coefs[2] = {1.0, 1.0};
  hf_basis* b = NULL;
  rc = hf_basis_create(ctx, atoms, 2, shells, 2, exps, coefs, 2, &b);
  if (rc == HF_OK) {
    hf_scf_result r;
    memset(&r, 0, sizeof r); /* no optional outputs (D, C, eps, F, F1 stay NULL) */
    hf_scf_opts o = scf;
    rc = hf_scf_solve(b, &o, &r);
    printf("E %.10f rc %d\n", r.energy, rc);
    hf_basis_destroy(b);
  }
  hf_ctx_destroy(ctx);
  return rc == HF_OK ? 0 : 1;
}
