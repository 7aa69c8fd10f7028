// serve.cu -- continuous-batching request loop (hlc_serve_*).
#include "../../include/hlc.h"
#include "serve.h"

extern "C" {
int hlc_serve_start(hlc_ctx*, size_t, int) { return HLC_ERR_UNSUPPORTED; }
int hlc_serve_submit(hlc_ctx*, const double*, const double*, int64_t, const hlc_theta*, const hlc_params*,
                     uint64_t*) {
  return HLC_ERR_UNSUPPORTED;
}
int hlc_serve_poll(hlc_ctx*, uint64_t, hlc_result*) { return HLC_ERR_UNSUPPORTED; }
int hlc_serve_stop(hlc_ctx*) { return HLC_OK; }
}
