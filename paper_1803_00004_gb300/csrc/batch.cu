// bf_filter_batch: placeholder sequence of per-image launches (replaced by the
// persistent work-list kernel).
#include <cuda_runtime.h>

#include "bf_internal.h"

extern "C" bf_status bf_filter_batch(const bf_plan *const *plans, const bf_image *images, int n, void *stream) {
    (void)plans;
    (void)images;
    (void)n;
    (void)stream;
    return bfi::fail(BF_ERR_UNSUPPORTED, "bf_filter_batch not built yet");
}
