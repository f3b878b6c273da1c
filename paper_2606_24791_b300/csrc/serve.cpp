// Placeholder entry points for the batched and served solves; replaced as those paths land.
#include "internal.h"

extern "C" {

int lamg_server_create(const lamg_server_opts *, const lamg_options *, lamg_server **out) {
    if (out) *out = nullptr;
    return LAMG_ERR_INVALID;
}
int lamg_serve(lamg_server *, const lamg_graph *, const double *, int64_t *) { return LAMG_ERR_INVALID; }
int lamg_serve_poll(lamg_server *, int64_t, lamg_ticket_info *, double *) { return LAMG_ERR_INVALID; }
int lamg_server_drain(lamg_server *, double) { return LAMG_ERR_INVALID; }
void lamg_server_destroy(lamg_server *) {}

}  // extern "C"
