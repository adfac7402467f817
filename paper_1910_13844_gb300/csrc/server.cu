// Serving entry points (continuous batching); see include/ls.h.
#include "engine.h"

using namespace lsgpu;

extern "C" {

int ls_server_create(const ls_server_options* opt, ls_server** out) {
  (void)opt;
  if (out) *out = nullptr;
  set_last_error("server not available in this build");
  return LS_EINVAL;
}
int ls_submit(ls_server* srv, const ls_request* req, uint64_t* ticket) {
  (void)srv; (void)req; (void)ticket;
  set_last_error("server not available in this build");
  return LS_EINVAL;
}
int ls_poll(ls_server* srv, uint64_t ticket, ls_result* res) {
  (void)srv; (void)ticket; (void)res;
  return LS_ENOTFOUND;
}
void ls_server_destroy(ls_server* srv) { (void)srv; }

}  // extern "C"
