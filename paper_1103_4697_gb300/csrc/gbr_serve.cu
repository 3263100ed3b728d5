// Serving (continuous batching) for libgbres.
#include "gbr_core.h"

void gbr_serve_shutdown(gbr_ctx *c) {
    if (!c || !c->serve) return;
}
