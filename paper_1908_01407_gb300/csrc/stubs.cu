// Entry points of gbx.h that this build does not provide yet.
#include "common.cuh"
using namespace gbx;
#define STUB(name, ...) gb_info name(__VA_ARGS__) { return fail(GB_NOT_IMPLEMENTED, #name " is not implemented"); }
extern "C" {
STUB(gb_bfs_multi, gb_context *ctx, const gb_matrix *A, const uint32_t *srcs, uint32_t k, int32_t *levels, gb_mem mem, const gb_desc *desc, gb_bfs_stats *stats)
STUB(gb_server_create, gb_server **s, gb_context *ctx, const gb_server_cfg *cfg)
STUB(gb_server_add_graph, gb_server *s, const gb_matrix *A, uint32_t *graph_id)
STUB(gb_server_submit, gb_server *s, const gb_request *req, uint64_t *ticket)
STUB(gb_server_wait, gb_server *s, uint64_t ticket, uint32_t timeout_ms, gb_result *res)
STUB(gb_server_fetch, gb_server *s, uint64_t ticket, void *out, gb_mem mem)
STUB(gb_server_stats_get, gb_server *s, gb_server_stats *st)
STUB(gb_server_destroy, gb_server **s)
}
