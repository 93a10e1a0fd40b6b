// Serving loop placeholder.
#include "bf_internal.h"

extern "C" {
bf_status bf_serve_create(const bf_serve_config *, bf_server **out) {
    if (out) *out = nullptr;
    return bfi::fail(BF_ERR_UNSUPPORTED, "server not built yet");
}
bf_status bf_serve_submit(bf_server *, const bf_request *, uint64_t *) { return BF_ERR_UNSUPPORTED; }
bf_status bf_serve_poll(bf_server *, uint64_t, int, bf_result *) { return BF_ERR_UNSUPPORTED; }
bf_status bf_serve_cancel(bf_server *, uint64_t) { return BF_ERR_UNSUPPORTED; }
void bf_serve_destroy(bf_server *) {}
}
