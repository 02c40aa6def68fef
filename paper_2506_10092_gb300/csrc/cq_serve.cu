// cq_serve.cu -- batched launches and the serving loop (entry points).
#include "cq_internal.h"

using namespace cq;

extern "C" int cq_batch_run(uint32_t n, cq_table* const* tables, const cq_plan* plans, const cq_exec_options* opts,
                            void* cuda_stream, cq_result** results) {
  (void)n; (void)tables; (void)plans; (void)opts; (void)cuda_stream; (void)results;
  return set_error(CQ_ERR_UNSUPPORTED, "batched launches are not built yet");
}

extern "C" int cq_server_create(cq_ctx* ctx, const cq_server_options* opts, cq_server** out) {
  (void)ctx; (void)opts; (void)out;
  return set_error(CQ_ERR_UNSUPPORTED, "the serving loop is not built yet");
}
extern "C" int cq_server_submit(cq_server* srv, cq_table* table, const cq_plan* plan, uint64_t* ticket) {
  (void)srv; (void)table; (void)plan; (void)ticket;
  return set_error(CQ_ERR_UNSUPPORTED, "the serving loop is not built yet");
}
extern "C" int cq_server_wait(cq_server* srv, uint64_t ticket, uint64_t timeout_us, cq_result** res, double* latency_us) {
  (void)srv; (void)ticket; (void)timeout_us; (void)res; (void)latency_us;
  return set_error(CQ_ERR_UNSUPPORTED, "the serving loop is not built yet");
}
extern "C" int cq_server_stats(cq_server* srv, uint64_t* launches, uint64_t* completed) {
  (void)srv; (void)launches; (void)completed;
  return set_error(CQ_ERR_UNSUPPORTED, "the serving loop is not built yet");
}
extern "C" int cq_server_destroy(cq_server* srv) {
  (void)srv;
  return CQ_OK;
}
