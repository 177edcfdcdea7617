// Continuous-batching request server (placeholder until the scheduler lands).
#include "../../include/bcgpu.h"

extern "C" {
int bc_request_submit(bc_graph_t, const uint32_t*, uint32_t, double, double*, bc_request_t*) { return BC_ERR_INVALID; }
int bc_request_poll(bc_request_t, int*) { return BC_ERR_INVALID; }
int bc_request_wait(bc_request_t, int) { return BC_ERR_INVALID; }
int bc_request_cancel(bc_request_t) { return BC_ERR_INVALID; }
int bc_serving_stats_get(bc_serving_stats*) { return BC_ERR_INVALID; }
int bc_serving_reset(void) { return BC_ERR_INVALID; }
}
