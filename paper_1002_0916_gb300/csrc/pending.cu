// pending.cu -- entry points whose kernels are not in this build yet.
#include "api_internal.h"
#include "common.cuh"

void cgh_ctx::release_all() {
    for (Buffer *b : {&ws, &ws2, &io, &part, &meta}) {
        if (b->ptr) cudaFree(b->ptr);
        b->ptr = nullptr;
        b->bytes = 0;
    }
}

extern "C" {

cgh_status cgh_batch(cgh_handle h, const cgh_problem *, int, int, void *) {
    if (!h) return CGH_ERR_INVALID_ARG;
    return h->fail(CGH_ERR_UNSUPPORTED, "batch not built yet");
}

}  // extern "C"
