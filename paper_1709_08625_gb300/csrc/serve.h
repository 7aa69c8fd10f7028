// serve.h -- continuous-batching request loop (hlc_serve_*).
#pragma once

namespace hlc {
struct Serve;
}
