// Cluster path (placeholder until the shared-memory kernel lands): FP32 plain
// iterations over all particles.
#include "ibm_internal.h"

ibm_status cluster_forcing_step(ibm_ctx *ctx, void *const *u_ptrs, double tau, void *const *f_out) {
    ibm_status s = ensure_field_ptrs(ctx, u_ptrs, f_out);
    if (s != IBM_OK) return s;
    return plain_iterations_f32(ctx, nullptr, ctx->n_p, tau, f_out != nullptr, ctx->cfg.n_forcing);
}

void cluster_free(ibm_ctx *) {}
