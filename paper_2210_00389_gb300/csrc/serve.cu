// Serving loop (tc_serve_*): not yet available in this build.
#include "internal.cuh"

using namespace tc;

struct tc_server {};

extern "C" {
int tc_serve_create(const tc_serve_config*, tc_server**) {
  return fail(TC_ERR_INVALID_ARG, "tc_serve_create: serving is not built yet");
}
int tc_serve_register(tc_server*, const tc_csr_view*, uint64_t*) {
  return fail(TC_ERR_INVALID_ARG, "serving is not built yet");
}
int tc_serve_submit(tc_server*, const tc_csr_view*, uint64_t, int, uint64_t*) {
  return fail(TC_ERR_INVALID_ARG, "serving is not built yet");
}
int tc_serve_poll(tc_server*, uint64_t, int*, uint64_t*, int*) {
  return fail(TC_ERR_INVALID_ARG, "serving is not built yet");
}
int tc_serve_destroy(tc_server*) { return TC_OK; }
}
