// Entry points of the solver and serving layers that this build does not provide yet.
#include "mpk_internal.cuh"

extern "C" mpk_status mpk_server_opts_default(mpk_server_opts *o) { (void)o; return MPK_ERR_UNIMPLEMENTED; }
extern "C" mpk_status mpk_server_create(const mpk_server_opts *o, mpk_server_t *out) { (void)o; (void)out; return MPK_ERR_UNIMPLEMENTED; }
extern "C" mpk_status mpk_server_submit(mpk_server_t srv, int64_t n, int64_t nnz, const int32_t *row_ptr,
                                        const int32_t *col, const double *val, const double *b,
                                        double *x_out, int64_t *id) {
    (void)srv; (void)n; (void)nnz; (void)row_ptr; (void)col; (void)val; (void)b; (void)x_out; (void)id;
    return MPK_ERR_UNIMPLEMENTED;
}
extern "C" mpk_status mpk_server_poll(mpk_server_t srv, mpk_server_result *out, int32_t m, int32_t *n_out) {
    (void)srv; (void)out; (void)m; (void)n_out; return MPK_ERR_UNIMPLEMENTED;
}
extern "C" mpk_status mpk_server_pending(mpk_server_t srv, int64_t *n) { (void)srv; (void)n; return MPK_ERR_UNIMPLEMENTED; }
extern "C" mpk_status mpk_server_destroy(mpk_server_t srv) { (void)srv; return MPK_ERR_UNIMPLEMENTED; }
