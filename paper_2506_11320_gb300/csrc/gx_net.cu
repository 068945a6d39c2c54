// gx_net.cu -- learned GMRES preconditioner (placeholder until the BF16
// network kernels land; every entry reports GX_ENOTIMPL).
#include "gx_internal.cuh"

struct Net {
    int dummy;
};

int gx_net_apply(gx_ctx *c, const double *, double *, cudaStream_t) {
    c->err = "learned preconditioner not available in this build";
    return GX_ENOTIMPL;
}
int gx_net_collect(gx_ctx *, cudaStream_t) { return GX_OK; }
void gx_net_free(gx_ctx *c) {
    delete c->net;
    c->net = nullptr;
}

extern "C" {
int64_t gx_precond_param_count(void) { return 20259; }
int gx_precond_set_weights(gx_ctx *c, const float *, int64_t, int) {
    if (!c) return GX_EINVAL;
    c->err = "learned preconditioner not available in this build";
    return GX_ENOTIMPL;
}
int gx_precond_get_weights(gx_ctx *c, float *, int64_t, int) {
    if (!c) return GX_EINVAL;
    return GX_ENOTIMPL;
}
int gx_precond_collect(gx_ctx *c, int) { return c ? GX_ENOTIMPL : GX_EINVAL; }
int gx_precond_pairs(gx_ctx *c) { return c ? 0 : -1; }
int gx_precond_train(gx_ctx *c, int, int, int, int, float, uint64_t, float *, void *) {
    return c ? GX_ENOTIMPL : GX_EINVAL;
}
int gx_precond_forward(gx_ctx *c, int, int, const float *, float *, void *) { return c ? GX_ENOTIMPL : GX_EINVAL; }
int gx_precond_loss_grad(gx_ctx *c, int, int, const float *, const float *, float *, float *, void *) {
    return c ? GX_ENOTIMPL : GX_EINVAL;
}
}
