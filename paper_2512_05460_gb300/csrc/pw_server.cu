// Continuous-batching server (persistent kernel over a device work queue).
#include "pw_internal.h"

extern "C" {

pw_status pw_server_create(pw_graph*, const pw_params*, size_t, pw_server** out) {
  if (out) *out = nullptr;
  return pw::set_error(PW_ERR_ARG, "server not available in this build");
}
pw_status pw_server_submit(pw_server*, int64_t, int64_t, double, int32_t, const uint64_t*, uint64_t*) {
  return pw::set_error(PW_ERR_ARG, "server not available in this build");
}
pw_status pw_server_poll(pw_server*, uint64_t, double*) {
  return pw::set_error(PW_ERR_ARG, "server not available in this build");
}
pw_status pw_server_drain(pw_server*, int64_t) { return pw::set_error(PW_ERR_ARG, "server not available in this build"); }
pw_status pw_server_destroy(pw_server*) { return PW_OK; }

}  // extern "C"
