// serve.h -- continuous-batching request loop (hlc_serve_*).
#pragma once

#include <stddef.h>
#include <stdint.h>

#include "../../include/hlc.h"

namespace hlc {
struct Serve;
// The serve state of a context and its device (defined with the context).
Serve*& serve_of(hlc_ctx* c);
int device_of(hlc_ctx* c);
// Allow or forbid the persistent (cooperative, grid-barrier) solve kernel.
void set_persistent(hlc_ctx* c, bool on);
// Estimated device bytes of one evaluation of n points.
size_t serve_footprint(int64_t n, const hlc_params& p);
}  // namespace hlc
