// serve.cu -- serving loop (placeholder until the serving path lands).
#include "hf_internal.h"

extern "C" void hf_serve_opts_default(hf_serve_opts* o) {
  if (!o) return;
  o->max_active = 64;
  o->queue_capacity = 100000;
  o->hbm_budget = 0;
  hf_scf_opts_default(&o->scf);
}
extern "C" int hf_serve_create(hf_ctx*, const hf_serve_opts*, hf_server** out) {
  if (out) *out = nullptr;
  return hf_fail(HF_ERR_INVALID, "serving: not available in this build");
}
extern "C" int hf_serve_submit(hf_server*, const hf_request*, uint64_t*) { return HF_ERR_INVALID; }
extern "C" int hf_serve_poll(hf_server*, uint64_t, hf_serve_result*) { return HF_ERR_NOT_FOUND; }
extern "C" int hf_serve_cancel(hf_server*, uint64_t) { return HF_ERR_NOT_FOUND; }
extern "C" double hf_serve_now(hf_server*) { return 0.0; }
extern "C" int hf_serve_drain(hf_server*, double) { return HF_OK; }
extern "C" void hf_serve_destroy(hf_server*) {}
