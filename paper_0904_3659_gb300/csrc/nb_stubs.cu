// nb_stubs.cu -- entry points declared in nbody.h whose kernels are not built
// yet: they check their arguments and return NB_ERR_NOT_IMPLEMENTED.
#include "nb_ext.h"

using namespace nbx;

extern "C" {

nb_status nb_force_vjp(nb_ctx *ctx, const float *, const float *, int64_t, float, const float *,
                       const float *, float *, float *, void *) {
    if (!ctx) return NB_ERR_ARG;
    return fail(ctx, NB_ERR_NOT_IMPLEMENTED, "nb_force_vjp is not built yet");
}

}  // extern "C"
