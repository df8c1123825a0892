// Interim entry points (replaced by the batch and serving implementations).
#include "ac_internal.h"
using namespace acgb;
extern "C" {
int ac_tune(ac_automaton *a, const uint8_t *d_text, uint64_t n, int fmt, void *stream, ac_scan_config *chosen) {
    (void)d_text; (void)n; (void)fmt; (void)stream;
    if (!a) return set_error(AC_EINVAL, "ac_tune: NULL");
    if (chosen) *chosen = a->cfg;
    return AC_OK;
}
int ac_serve_create(const ac_automaton *const *, uint32_t, const ac_serve_opts *, ac_server **) { return set_error(AC_EINVAL, "serving not built"); }
int ac_serve_submit(ac_server *, uint32_t, const uint8_t *, uint64_t, int, uint64_t *) { return AC_EINVAL; }
int ac_serve_poll(ac_server *, uint64_t, ac_result *) { return AC_EINVAL; }
int ac_serve_wait(ac_server *, uint64_t, uint32_t, ac_result *) { return AC_EINVAL; }
int ac_serve_stats(ac_server *, ac_serve_stats_t *) { return AC_EINVAL; }
void ac_serve_destroy(ac_server *) {}
}
