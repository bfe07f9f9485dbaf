// Serving loop (continuous batching) -- entry points; the scheduler lands in
// a later change.
#include "wf_internal.h"

using namespace wfk;

struct wf_server_s {};

extern "C" {
wf_status wf_server_create(size_t, int, wf_server_t *out) {
  if (out) *out = nullptr;
  set_error("wf_server_create: serving is not available in this build");
  return WF_EINVAL;
}
wf_status wf_submit(wf_server_t, int, int, const double *, const double *, const uint8_t *, const double *, double,
                    uint64_t *) {
  set_error("wf_submit: serving is not available in this build");
  return WF_EINVAL;
}
wf_status wf_poll(wf_server_t, uint64_t, int *done, double *, wf_stats *) {
  if (done) *done = 0;
  set_error("wf_poll: serving is not available in this build");
  return WF_EINVAL;
}
wf_status wf_server_drain(wf_server_t, int) {
  set_error("wf_server_drain: serving is not available in this build");
  return WF_EINVAL;
}
wf_status wf_server_stats(wf_server_t, double *, double *, int64_t *) {
  set_error("wf_server_stats: serving is not available in this build");
  return WF_EINVAL;
}
wf_status wf_server_destroy(wf_server_t) { return WF_OK; }
}
