// Continuous-batching server (fftsrv_*).
#include "plan.h"

using namespace fftseg;

extern "C" {
int fftsrv_create(fftsrv *out, const fftsrv_config *) { if (out) *out = nullptr; return set_error(FFTSEG_E_UNSUPPORTED, "server not built yet"); }
int fftsrv_submit(fftsrv, const fftsrv_job *, uint64_t *) { return set_error(FFTSEG_E_UNSUPPORTED, "server not built yet"); }
int fftsrv_poll(fftsrv, uint64_t, int64_t, int *) { return set_error(FFTSEG_E_UNSUPPORTED, "server not built yet"); }
int fftsrv_stats(fftsrv, int64_t[5]) { return set_error(FFTSEG_E_UNSUPPORTED, "server not built yet"); }
int fftsrv_destroy(fftsrv) { return set_error(FFTSEG_E_UNSUPPORTED, "server not built yet"); }
}
