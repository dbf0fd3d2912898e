// pw_batch.cu -- batched ensembles and the tile autotuner (being written).
#include "pw_internal.h"

extern "C" pw_status pw_batch_create(pw_mesh *const *, int, void *, pw_batch **out) {
    if (out) *out = nullptr;
    return pw_fail(PW_ERR_DTYPE, "batches are not built yet");
}
extern "C" void pw_batch_destroy(pw_batch *) {}
extern "C" pw_status pw_batch_set_fields(pw_batch *, void *const *, void *const *, void *const *,
                                         void *const *, void *const *, void *const *, void *) {
    return pw_fail(PW_ERR_DTYPE, "batches are not built yet");
}
extern "C" pw_status pw_advect_batched(pw_batch *, int, void *) {
    return pw_fail(PW_ERR_DTYPE, "batches are not built yet");
}
extern "C" pw_status pw_batch_halo(pw_batch *, void *) {
    return pw_fail(PW_ERR_DTYPE, "batches are not built yet");
}
extern "C" pw_status pw_autotune(pw_mesh *, const void *, const void *, const void *, void *, void *,
                                 void *, const char *, void *, float *) {
    return pw_fail(PW_ERR_DTYPE, "autotune is not built yet");
}
extern "C" pw_status pw_batch_autotune(pw_batch *, const char *, void *, float *) {
    return pw_fail(PW_ERR_DTYPE, "autotune is not built yet");
}
