// Serving loop (continuous batching); filled in below the matching engine.
#include "gs_host.h"

using namespace gs;

extern "C" gs_status gs_serve_create(gs_graph *, const gs_serve_opts *, gs_server **out) {
  if (out) *out = nullptr;
  return fail(GS_ERR_UNSUPPORTED, "serving not built yet");
}
extern "C" gs_status gs_serve_submit(gs_server *, const gs_query *, const gs_match_opts *, uint64_t *) {
  return fail(GS_ERR_UNSUPPORTED, "serving not built yet");
}
extern "C" gs_status gs_serve_poll(gs_server *, uint64_t, gs_result *, double *) {
  return fail(GS_ERR_UNSUPPORTED, "serving not built yet");
}
extern "C" gs_status gs_serve_destroy(gs_server *) { return GS_OK; }
