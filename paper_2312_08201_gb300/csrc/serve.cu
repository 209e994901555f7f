// Serving loop (continuous batching) -- placeholder until implemented.
#include "lyap_internal.h"

extern "C" int lyap_serve_create(lyap_ctx*, const lyap_opts*, lyap_server** out) {
  if (out) *out = nullptr;
  return LYAP_EINVAL;
}
extern "C" int lyap_serve_register_seed(lyap_server*, lyap_seed*, int*) { return LYAP_EINVAL; }
extern "C" int lyap_serve_submit(lyap_server*, int, int, const double*, int, uint64_t*) { return LYAP_EINVAL; }
extern "C" int lyap_serve_run(lyap_server*, int, int*) { return LYAP_EINVAL; }
extern "C" int lyap_serve_poll(lyap_server*, uint64_t, double*, double*, lyap_result_info*, double*) {
  return LYAP_EINVAL;
}
extern "C" int lyap_serve_cancel(lyap_server*, uint64_t) { return LYAP_EINVAL; }
extern "C" void lyap_serve_destroy(lyap_server*) {}
