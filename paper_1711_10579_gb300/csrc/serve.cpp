// Serving runtime: queued solves admitted onto the GPU (placeholder until the
// continuous-batching runtime lands).
#include "api_internal.h"

namespace pf {

struct Server {};

void serve_shutdown(pf_ctx) {}
void serve_forget_case(pf_ctx, pf_case) {}

}  // namespace pf

extern "C" {

int pf_submit(pf_ctx, pf_case, const double*, const double*, const double*, const pf_opts*,
              pf_ticket*) {
  return pf::set_error(PF_ERR_UNSUPPORTED, "serving is not built yet");
}

int pf_poll(pf_ctx, pf_ticket, double*, double*, pf_info*) {
  return pf::set_error(PF_ERR_UNSUPPORTED, "serving is not built yet");
}

int pf_drain(pf_ctx, int) { return pf::set_error(PF_ERR_UNSUPPORTED, "serving is not built yet"); }

}  // extern "C"
