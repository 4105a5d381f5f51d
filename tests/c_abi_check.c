/* The C ABI used from plain C (no C++, no Python): create a handle, query its environment size,
 * check the state and argument errors and the error strings, destroy.  None of these calls
 * touches a GPU.  Prints "ok <env numel>" on success. */
#include <stdio.h>
#include <string.h>

#include "../include/ctm.h"

int main(void) {
  double h[16];
  for (int i = 0; i < 16; ++i) h[i] = (i % 5 == 0) ? 1.0 : 0.0; /* identity 4x4 */
  ctm_term term = {0, 0, CTM_BOND_H, 1.0, h};
  ctm_desc desc;
  memset(&desc, 0, sizeof desc);
  desc.Lx = 1; desc.Ly = 1; desc.d = 2; desc.D = 2; desc.chi = 4;
  desc.precision = CTM_TF32X3; desc.n_terms = 1; desc.terms = &term;
  desc.svd_cutoff_rel = 0.0; desc.svd_adjoint_eps = -1.0; desc.max_iter = 0;
  ctm_handle* hd = NULL;
  if (ctm_create(&desc, &hd) != CTM_OK || !hd) { printf("create failed\n"); return 1; }
  int64_t n = ctm_env_numel(hd);
  if (n <= 0) { printf("bad numel\n"); return 1; }
  if (ctm_step(hd, 1, NULL, NULL) != CTM_ERR_STATE) { printf("step before init accepted\n"); return 1; }
  if (ctm_init(hd, NULL, NULL, NULL) != CTM_ERR_INVALID_ARG) { printf("null A accepted\n"); return 1; }
  if (strcmp(ctm_error_string(CTM_OK), "ok") != 0) { printf("bad string\n"); return 1; }
  desc.chi = 0;
  ctm_handle* bad = NULL;
  if (ctm_create(&desc, &bad) != CTM_ERR_INVALID_ARG) { printf("chi=0 accepted\n"); return 1; }
  if (ctm_destroy(hd) != CTM_OK) { printf("destroy failed\n"); return 1; }
  printf("ok %lld\n", (long long)n);
  return 0;
}
