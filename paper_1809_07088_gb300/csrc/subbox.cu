// Exact sub-box averaging (Section V A) for occupancy and spin disorder.
#include "api_internal.h"

template <typename T>
ds_status subbox_run(ds_model *M, const ds_qgrid *, const ds_opts *, T *, cudaStream_t, Scratch &, ds_result_info *) {
    return ds_fail(M->ctx, DS_ERR_UNSUPPORTED, "sub-box averaging not built yet");
}
template ds_status subbox_run<float>(ds_model *, const ds_qgrid *, const ds_opts *, float *, cudaStream_t, Scratch &,
                                     ds_result_info *);
template ds_status subbox_run<double>(ds_model *, const ds_qgrid *, const ds_opts *, double *, cudaStream_t,
                                      Scratch &, ds_result_info *);
