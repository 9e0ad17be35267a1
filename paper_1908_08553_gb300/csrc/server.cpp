// Request server (tn_submit / tn_poll / tn_wait).
#include "runtime.h"

namespace tn {
void server_stop(tn_ctx*) {}
}  // namespace tn

extern "C" {
tn_status tn_submit(tn_ctx*, const tn_job*, uint64_t*) {
    tn::set_error("serving is not built yet");
    return TN_ERR_INVALID;
}
tn_status tn_poll(tn_ctx*, uint64_t, tn_result*) { return TN_ERR_INVALID; }
tn_status tn_wait(tn_ctx*, uint64_t, double, tn_result*) { return TN_ERR_INVALID; }
}
