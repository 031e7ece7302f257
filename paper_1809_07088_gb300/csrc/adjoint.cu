// Adjoint of the FFT method.
#include "api_internal.h"

extern "C" ds_status ds_backward(ds_model *m, const ds_qgrid *, const ds_opts *, const void *, void *, int, void *) {
    return ds_fail(m ? m->ctx : nullptr, DS_ERR_UNSUPPORTED, "adjoint not built yet");
}
