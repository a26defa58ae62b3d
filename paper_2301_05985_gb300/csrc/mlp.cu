// mlp.cu -- learned Newton start (placeholder until the network kernels are built).
#include "ctx.h"

int pnp_learned_start(pnp_ctx* c, pnp_solve_stats* st) {
  (void)c;
  (void)st;
  PNP_FAIL(PNP_ERR_STATE, "learned start: no trained network in this context");
}

void pnp_mlp_release(pnp_ctx* c) { (void)c; }
