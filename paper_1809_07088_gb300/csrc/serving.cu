// Continuous-batching request loop.
#include "api_internal.h"

void serving_shutdown(ds_ctx *) {}
extern "C" ds_status ds_submit(ds_model *m, const ds_qgrid *, const ds_opts *, void *, uint64_t *) {
    return ds_fail(m ? m->ctx : nullptr, DS_ERR_UNSUPPORTED, "serving not built yet");
}
extern "C" ds_status ds_poll(ds_ctx *ctx, uint64_t, ds_result_info *) { return ds_fail(ctx, DS_ERR_UNSUPPORTED, "serving not built yet"); }
extern "C" ds_status ds_wait(ds_ctx *ctx, uint64_t, double, ds_result_info *) { return ds_fail(ctx, DS_ERR_UNSUPPORTED, "serving not built yet"); }
