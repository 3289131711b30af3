// Serving loop (continuous batching of RED solves). Placeholder until the scheduler lands.
#include "red.h"

extern "C" {
red_status red_server_create(size_t, int, red_server *out) {
  if (out) *out = nullptr;
  return RED_EUNSUPPORTED;
}
red_status red_submit(red_server, const red_config *, const float *, float *, int, double, uint64_t *) {
  return RED_EUNSUPPORTED;
}
red_status red_poll(red_server, uint64_t, red_stats *) { return RED_EUNSUPPORTED; }
red_status red_wait(red_server, uint64_t, int, red_stats *) { return RED_EUNSUPPORTED; }
red_status red_server_destroy(red_server) { return RED_OK; }
}
