// cq_serve.cu -- batched launches (host side), the batch autotuner and the
// serving loop.
//
// A batch is planned query by query with the one-query planner, constrained
// to the persistent kernel's shape; the descriptors, work items and aux
// tables are packed into one control block that a cached CUDA graph uploads
// and runs (init -> persistent kernel -> finalize).  Result buffers of all
// queries of a batch share one pool allocation.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "cq_internal.h"

namespace cq {

// ------------------------------------------------------------------ launch graphs
// One instantiated launch graph and its control block.  The graph's first
// node uploads the pinned staging copy of the control block.  An event
// recorded on the launching stream after each replay tells the host when
// the staging copy may be rewritten (an event recorded inside the graph
// cannot be queried from the host).
struct BatchGraph {
  int device = 0;
  size_t cap = 0;                 // control-block bytes
  unsigned grid = 0;              // persistent CTAs
  int minb = 1;                   // CTAs per SM
  uint8_t* host = nullptr;        // pinned staging
  uint8_t* dev = nullptr;         // control block (device)
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaGraphNode_t upload = nullptr;
  cudaEvent_t done = nullptr;      // recorded after the last replay
  bool filling = false;           // a host thread is writing the staging copy
  ~BatchGraph() {
    cudaSetDevice(device);
    if (done) cudaEventSynchronize(done);
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (done) cudaEventDestroy(done);
    if (dev) cudaFree(dev);
    if (host) cudaFreeHost(host);
  }
};

// Device block and events shared by the results of one batch.
struct BatchShared {
  int device = 0;
  cudaStream_t stream = nullptr;
  void* block = nullptr;
  cudaEvent_t ev_start = nullptr, ev_done = nullptr;
  ~BatchShared() {
    cudaSetDevice(device);
    if (block) cudaFreeAsync(block, stream);
    if (ev_start) cudaEventDestroy(ev_start);
    if (ev_done) cudaEventDestroy(ev_done);
  }
};

static size_t al16(size_t x) { return (x + 15) / 16 * 16; }
static size_t al256(size_t x) { return (x + 255) / 256 * 256; }

// Dynamic shared memory of the batch kernel: the per-block opt-in limit less
// the kernel's static shared memory (its descriptor copy).
static int ensure_batch_kernel(cq_ctx* ctx) {
  if (ctx->batch_smem) return CQ_OK;
  for (int minb = 1; minb <= 2; ++minb) {
    size_t st = 0;
    cudaError_t e = batch_kernel_static_smem(minb, &st);
    if (e != cudaSuccess) return set_error(CQ_ERR_CUDA, "batch kernel attributes: %s", cudaGetErrorString(e));
    const size_t limit = minb == 2 ? ctx->smem_two : ctx->smem_optin;
    const size_t dyn = (limit - st) / 128 * 128;
    e = batch_kernel_set_smem(minb, dyn);
    if (e != cudaSuccess) return set_error(CQ_ERR_CUDA, "batch kernel shared memory: %s", cudaGetErrorString(e));
    if (minb == 2) ctx->batch_smem_two = dyn;
    else ctx->batch_smem = dyn;
  }
  return CQ_OK;
}

static int capture_graph(cq_ctx* ctx, BatchGraph* g) {
  cudaStream_t cs = nullptr;
  CQ_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) e = cudaMemcpyAsync(g->dev, g->host, g->cap, cudaMemcpyHostToDevice, cs);
  if (e == cudaSuccess)
    e = launch_batch(reinterpret_cast<BatchCtl*>(g->dev), cs, g->grid, g->minb,
                     g->minb == 2 ? ctx->batch_smem_two : ctx->batch_smem, (unsigned)ctx->num_sms * 2);
  cudaGraph_t graph = nullptr;
  const cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
  if (e == cudaSuccess) e = e2;
  cudaStreamDestroy(cs);
  if (e != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return set_error(CQ_ERR_CUDA, "batch graph capture failed: %s", cudaGetErrorString(e));
  }
  g->graph = graph;
  size_t n_nodes = 0;
  CQ_CUDA(cudaGraphGetNodes(graph, nullptr, &n_nodes));
  std::vector<cudaGraphNode_t> nodes(n_nodes);
  CQ_CUDA(cudaGraphGetNodes(graph, nodes.data(), &n_nodes));
  for (cudaGraphNode_t n : nodes) {
    cudaGraphNodeType t;
    CQ_CUDA(cudaGraphNodeGetType(n, &t));
    if (t == cudaGraphNodeTypeMemcpy) g->upload = n;
  }
  if (!g->upload) return set_error(CQ_ERR_CUDA, "batch graph has no upload node");
  CQ_CUDA(cudaGraphInstantiate(&g->exec, graph, 0));
  return CQ_OK;
}

// A launch graph whose control block holds `bytes`, marked as being filled.
static int acquire_graph(cq_ctx* ctx, size_t bytes, int minb, BatchGraph** out) {
  const unsigned grid = (unsigned)ctx->num_sms * (unsigned)minb;
  std::unique_lock<std::mutex> lk(ctx->batch_mu);
  for (int pass = 0; pass < 2; ++pass) {
    for (auto& g : ctx->graphs) {
      if (g->filling || g->cap < bytes || g->grid != grid) continue;
      // pass 0 takes an idle graph; pass 1 waits for a busy one
      const cudaError_t q = cudaEventQuery(g->done);
      if (q != cudaSuccess && q != cudaErrorNotReady)
        return set_error(CQ_ERR_CUDA, "batch graph state: %s", cudaGetErrorString(q));
      if (q == cudaErrorNotReady) (void)cudaGetLastError();   // not an error: clear it
      if (q == cudaErrorNotReady && pass == 0) continue;
      g->filling = true;
      BatchGraph* r = g;
      lk.unlock();
      if (q == cudaErrorNotReady) cudaEventSynchronize(r->done);
      *out = r;
      return CQ_OK;
    }
    if (pass == 0 && ctx->graphs.size() < 16) break;   // room for another graph
  }
  std::unique_ptr<BatchGraph> g(new BatchGraph);
  g->device = ctx->device;
  g->cap = 256 * 1024;
  while (g->cap < bytes) g->cap *= 2;
  g->grid = grid;
  g->minb = minb;
  CQ_CUDA(cudaMalloc(&g->dev, g->cap));
  CQ_CUDA(cudaMallocHost(&g->host, g->cap));
  CQ_CUDA(cudaEventCreateWithFlags(&g->done, cudaEventDisableTiming));
  int rc = capture_graph(ctx, g.get());
  if (rc != CQ_OK) return rc;
  g->filling = true;
  *out = g.get();
  ctx->graphs.push_back(g.release());
  return CQ_OK;
}

static void release_graph(cq_ctx* ctx, BatchGraph* g) {
  std::lock_guard<std::mutex> lk(ctx->batch_mu);
  g->filling = false;
}

// ------------------------------------------------------------------ batch kinds
// Whether every column the plan references is RLE or index-encoded (the
// planner then runs the query in segment mode).
static bool plan_is_segment(const cq_table* t, const cq_plan* p) {
  auto ok = [&](uint32_t c) {
    return c < t->cols.size() && (t->cols[c]->enc == ENC_RLE || t->cols[c]->enc == ENC_INDEX);
  };
  for (uint32_t i = 0; i < p->n_preds && p->preds; ++i)
    if (!ok(p->preds[i].col)) return false;
  for (uint32_t i = 0; i < p->n_group_by && p->group_by; ++i)
    if (!ok(p->group_by[i])) return false;
  for (uint32_t i = 0; i < p->n_aggs && p->aggs; ++i) {
    if (p->aggs[i].op != CQ_COUNT && !ok(p->aggs[i].col)) return false;
    if (p->aggs[i].op != CQ_COUNT && p->aggs[i].expr != CQ_EXPR_NONE && !ok(p->aggs[i].col2)) return false;
  }
  return true;
}

static uint32_t ceil_log2(uint64_t x) {
  uint32_t r = 0;
  while ((1ull << r) < x && r < 63) ++r;
  return r;
}

// Autotuner key: log2 of the query count and of the total rows, and the
// share of segment-mode queries in eighths.
static uint64_t batch_key(uint32_t n, cq_table* const* tables, const cq_plan* plans) {
  uint64_t rows = 0;
  uint32_t seg = 0;
  for (uint32_t i = 0; i < n; ++i) {
    rows += tables[i] ? tables[i]->n_rows : 0;
    if (tables[i] && plan_is_segment(tables[i], &plans[i])) ++seg;
  }
  return ((uint64_t)ceil_log2(n) << 16) | ((uint64_t)ceil_log2(rows + 1) << 8) | (uint64_t)(seg * 8 / n);
}

// ------------------------------------------------------------------ one batch
// Device bytes a planned query holds while it runs: its result block plus
// its share of the control block (admission control of the serving loop).
static uint64_t query_footprint(const Planned& P) {
  return al256(query_block_layout(P, false).total) + sizeof(QueryDesc) + 4 * P.aux.size() + 64;
}

// Plan every query of a batch within `smem_limit` bytes of shared memory.
static int plan_batch(uint32_t n, cq_table* const* tables, const cq_plan* plans, uint32_t tile_rows,
                      size_t smem_limit, std::vector<Planned>* P) {
  P->resize(n);
  for (uint32_t i = 0; i < n; ++i) {
    const int rc = plan_batch_query(tables[i], &plans[i], tile_rows, smem_limit, &(*P)[i]);
    if (rc != CQ_OK) {
      const std::string msg = cq_last_error();
      return set_error(rc, "batch query %u: %s", i, msg.c_str());
    }
  }
  return CQ_OK;
}

// Launch n planned queries as one batch on stream s (see cq_batch_run).
static int launch_planned_batch(cq_ctx* ctx, uint32_t n, cq_table* const* tables, std::vector<Planned>& P,
                                uint32_t items_per_cta, int minb, cudaStream_t s, cq_result** results) {
  // ---- work items: C tiles at most, about items_per_cta per CTA, larger first
  const unsigned grid = (unsigned)ctx->num_sms * (unsigned)minb;
  uint64_t total_tiles = 0;
  for (const Planned& p : P) total_tiles += p.q.n_tiles;
  const uint64_t target = (uint64_t)grid * (items_per_cta ? items_per_cta : 4u);
  uint64_t chunk = (total_tiles + target - 1) / (target ? target : 1);
  if (chunk < 1) chunk = 1;
  if (chunk > 0xFFFFFFFFull) chunk = 0xFFFFFFFFull;
  std::vector<BatchItem> items;
  for (uint32_t i = 0; i < n; ++i)
    for (uint64_t t = 0; t < P[i].q.n_tiles; t += chunk) {
      BatchItem it;
      it.query = i;
      it.n_tiles = (uint32_t)std::min<uint64_t>(chunk, P[i].q.n_tiles - t);
      it.t_begin = t;
      items.push_back(it);
    }
  std::stable_sort(items.begin(), items.end(),
                   [](const BatchItem& a, const BatchItem& b) { return a.n_tiles > b.n_tiles; });
  // ---- control block layout: header, descriptors, items, block prefixes, aux tables
  const size_t off_desc = al256(sizeof(BatchCtl));
  const size_t off_items = al16(off_desc + (size_t)n * sizeof(QueryDesc));
  const size_t off_init = al16(off_items + items.size() * sizeof(BatchItem));
  const size_t off_fin = al16(off_init + 4 * ((size_t)n + 1));
  size_t off_aux = al16(off_fin + 4 * ((size_t)n + 1));
  std::vector<size_t> aux_at(n);
  size_t bytes = off_aux;
  for (uint32_t i = 0; i < n; ++i) {
    aux_at[i] = bytes;
    bytes = al16(bytes + 4 * P[i].aux.size());
  }
  // ---- result buffers: one pool allocation, one block per query
  std::vector<QueryBlock> L(n);
  std::vector<size_t> blk_at(n);
  size_t blk_bytes = 0;
  for (uint32_t i = 0; i < n; ++i) {
    L[i] = query_block_layout(P[i], false);
    blk_at[i] = blk_bytes;
    blk_bytes += al256(L[i].total);
  }
  std::shared_ptr<BatchShared> sh(new BatchShared);
  sh->device = ctx->device;
  sh->stream = s;
  cudaError_t e = pool_alloc(&sh->block, blk_bytes, ctx->pool, s);
  if (e != cudaSuccess) {
    sh->block = nullptr;
    return set_error(CQ_ERR_OOM, "device pool allocation of %llu bytes failed: %s", (unsigned long long)blk_bytes,
                     cudaGetErrorString(e));
  }
  CQ_CUDA(cudaEventCreate(&sh->ev_start));
  CQ_CUDA(cudaEventCreate(&sh->ev_done));
  // ---- fill the staging copy of a launch graph's control block
  BatchGraph* g = nullptr;
  int rc = acquire_graph(ctx, bytes, minb, &g);
  if (rc != CQ_OK) return rc;
  uint8_t* h = g->host;
  uint8_t* d = g->dev;
  uint8_t* blk = reinterpret_cast<uint8_t*>(sh->block);
  BatchCtl ctl;
  memset(&ctl, 0, sizeof(ctl));
  ctl.n_queries = n;
  ctl.n_items = (uint32_t)items.size();
  ctl.descs = reinterpret_cast<const QueryDesc*>(d + off_desc);
  ctl.items = reinterpret_cast<const BatchItem*>(d + off_items);
  ctl.init_first = reinterpret_cast<const uint32_t*>(d + off_init);
  ctl.fin_first = reinterpret_cast<const uint32_t*>(d + off_fin);
  uint32_t* init_first = reinterpret_cast<uint32_t*>(h + off_init);
  uint32_t* fin_first = reinterpret_cast<uint32_t*>(h + off_fin);
  uint32_t ib = 0, fb = 0;
  for (uint32_t i = 0; i < n; ++i) {
    bind_query_block(P[i], blk + blk_at[i], L[i], reinterpret_cast<const uint32_t*>(d + aux_at[i]));
    memcpy(h + off_desc + (size_t)i * sizeof(QueryDesc), &P[i].q, sizeof(QueryDesc));
    if (!P[i].aux.empty()) memcpy(h + aux_at[i], P[i].aux.data(), 4 * P[i].aux.size());
    init_first[i] = ib;
    fin_first[i] = fb;
    const uint64_t G = P[i].q.n_groups ? P[i].q.n_groups : 1;
    ib += (uint32_t)((G + kInitGroups - 1) / kInitGroups);
    fb += (uint32_t)((G + 1023) / 1024);
  }
  init_first[n] = ib;
  fin_first[n] = fb;
  ctl.n_init_blocks = ib;
  ctl.n_fin_blocks = fb;
  memcpy(h, &ctl, sizeof(ctl));
  if (!items.empty()) memcpy(h + off_items, items.data(), items.size() * sizeof(BatchItem));
  // ---- replay: upload only the bytes in use
  clear_stale_error("a batch launch");
  e = cudaGraphExecMemcpyNodeSetParams1D(g->exec, g->upload, g->dev, g->host, bytes, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaEventRecord(sh->ev_start, s);
  if (e == cudaSuccess) e = cudaGraphLaunch(g->exec, s);
  if (e == cudaSuccess) e = cudaEventRecord(g->done, s);
  if (e == cudaSuccess) e = cudaEventRecord(sh->ev_done, s);
  release_graph(ctx, g);
  if (e != cudaSuccess) return set_error(CQ_ERR_CUDA, "batch launch failed: %s", cudaGetErrorString(e));
  // ---- results
  for (uint32_t i = 0; i < n; ++i) {
    cq_result* r = new_result(ctx, s, false);
    r->ev_start = r->ev_k0 = sh->ev_start;
    r->ev_done = r->ev_k1 = sh->ev_done;
    attach_outputs(r, P[i]);
    for (int kc : P[i].out_key_col) r->key_cols.push_back(kc >= 0 ? tables[i]->cols[kc] : nullptr);
    for (cq_column* c : tables[i]->cols) c->refs++;
    r->held_cols = tables[i]->cols;
    r->batch_keepalive = sh;
    results[i] = r;
  }
  return CQ_OK;
}

static int run_batch(uint32_t n, cq_table* const* tables, const cq_plan* plans, uint32_t tile_rows,
                     uint32_t items_per_cta, cudaStream_t s, cq_result** results) {
  // two CTAs per SM when every query fits half an SM's shared memory at its
  // preferred tile, else one
  cq_ctx* ctx = tables[0]->ctx;
  std::vector<Planned> P;
  int minb = 2;
  int rc = plan_batch(n, tables, plans, tile_rows, ctx->batch_smem_two, &P);
  if (rc == CQ_OK) {
    for (const Planned& p : P) {
      const uint32_t want = tile_rows ? tile_rows : 8192u;
      if (p.q.tile_rows < want) minb = 1;
    }
  }
  if (rc != CQ_OK || minb == 1) {
    minb = 1;
    clear_error();
    rc = plan_batch(n, tables, plans, tile_rows, ctx->batch_smem, &P);
    if (rc != CQ_OK) return rc;
  }
  return launch_planned_batch(ctx, n, tables, P, items_per_cta, minb, s, results);
}

static int check_batch(uint32_t n, cq_table* const* tables, const cq_plan* plans, cq_result** results,
                       cq_ctx** ctx_out) {
  if (n == 0) return set_error(CQ_ERR_INVALID_ARG, "empty batch");
  if (!tables || !plans) return set_error(CQ_ERR_INVALID_ARG, "NULL tables or plans");
  for (uint32_t i = 0; i < n; ++i) {
    if (!tables[i]) return set_error(CQ_ERR_INVALID_ARG, "batch query %u: NULL table", i);
    if (tables[i]->ctx != tables[0]->ctx) return set_error(CQ_ERR_INVALID_ARG, "batch query %u: another context", i);
  }
  if (results)
    for (uint32_t i = 0; i < n; ++i) results[i] = nullptr;
  cq_ctx* ctx = tables[0]->ctx;
  CQ_CUDA(cudaSetDevice(ctx->device));
  {
    std::lock_guard<std::mutex> lk(ctx->batch_mu);
    const int rc = ensure_batch_kernel(ctx);
    if (rc != CQ_OK) return rc;
  }
  *ctx_out = ctx;
  return CQ_OK;
}

static bool tuned_shape(cq_ctx* ctx, uint64_t key, uint32_t* tile, uint32_t* ipc) {
  std::lock_guard<std::mutex> lk(ctx->batch_mu);
  for (const TunedShape& t : ctx->tuned)
    if (t.key == key) {
      *tile = t.tile_rows;
      *ipc = t.items_per_cta;
      return true;
    }
  return false;
}

}  // namespace cq

using namespace cq;

cq_ctx::~cq_ctx() {
  for (BatchGraph* g : graphs) delete g;
}

extern "C" int cq_batch_run(uint32_t n, cq_table* const* tables, const cq_plan* plans, const cq_exec_options* opts,
                            void* cuda_stream, cq_result** results) {
  clear_error();
  if (!results) return set_error(CQ_ERR_INVALID_ARG, "results is NULL");
  cq_ctx* ctx = nullptr;
  int rc = check_batch(n, tables, plans, results, &ctx);
  if (rc != CQ_OK) return rc;
  if (opts && opts->mode != CQ_EXEC_FUSED) return set_error(CQ_ERR_UNSUPPORTED, "batches run the fused path only");
  uint32_t tile = opts ? opts->tile_rows : 0, ipc = opts ? opts->items_per_cta : 0;
  if (tile == 0 && ipc == 0) tuned_shape(ctx, batch_key(n, tables, plans), &tile, &ipc);
  if (tile && (tile < 1024 || tile > 8192 || (tile & (tile - 1))))
    return set_error(CQ_ERR_INVALID_ARG, "tile_rows must be 1024, 2048, 4096 or 8192");
  cudaStream_t s = cuda_stream ? reinterpret_cast<cudaStream_t>(cuda_stream) : ctx->stream;
  rc = run_batch(n, tables, plans, tile, ipc, s, results);
  if (rc != CQ_OK)
    for (uint32_t i = 0; i < n; ++i)
      if (results[i]) {
        cq_result_destroy(results[i]);
        results[i] = nullptr;
      }
  return rc;
}

extern "C" int cq_batch_tune(uint32_t n, cq_table* const* tables, const cq_plan* plans, void* cuda_stream,
                             cq_exec_options* best, double* best_us) {
  clear_error();
  cq_ctx* ctx = nullptr;
  int rc = check_batch(n, tables, plans, nullptr, &ctx);
  if (rc != CQ_OK) return rc;
  cudaStream_t s = cuda_stream ? reinterpret_cast<cudaStream_t>(cuda_stream) : ctx->stream;
  static const uint32_t kTiles[] = {4096, 8192};
  static const uint32_t kIpc[] = {1, 2, 4, 8};
  std::vector<cq_result*> res(n, nullptr);
  double best_t = 1e300;
  uint32_t best_tile = 0, best_ipc = 4;
  std::string first_failure;
  for (uint32_t tile : kTiles)
    for (uint32_t ipc : kIpc) {
      double t_min = 1e300;
      bool ok = true;
      for (int rep = 0; rep < 3 && ok; ++rep) {   // warm-up, then best of two
        rc = run_batch(n, tables, plans, tile, ipc, s, res.data());
        if (rc != CQ_OK) {
          ok = false;   // e.g. a tile that leaves no room in shared memory
          if (first_failure.empty()) first_failure = cq_last_error();
          break;
        }
        double us = 0;
        rc = cq_result_wait(res[0], UINT64_MAX);
        if (rc == CQ_OK) rc = cq_result_device_time_us(res[0], &us);
        for (cq_result*& r : res) {
          cq_result_destroy(r);
          r = nullptr;
        }
        if (rc != CQ_OK) return rc;
        if (rep > 0) t_min = std::min(t_min, us);
      }
      if (ok && t_min < best_t) {
        best_t = t_min;
        best_tile = tile;
        best_ipc = ipc;
      }
    }
  clear_error();
  if (best_t >= 1e300)
    return set_error(CQ_ERR_UNSUPPORTED, "no candidate shape runs this batch (first failure: %s)",
                     first_failure.c_str());
  {
    const uint64_t key = batch_key(n, tables, plans);
    std::lock_guard<std::mutex> lk(ctx->batch_mu);
    bool found = false;
    for (TunedShape& t : ctx->tuned)
      if (t.key == key) {
        t.tile_rows = best_tile;
        t.items_per_cta = best_ipc;
        found = true;
      }
    if (!found) ctx->tuned.push_back({key, best_tile, best_ipc});
  }
  if (best) {
    memset(best, 0, sizeof(*best));
    best->mode = CQ_EXEC_FUSED;
    best->tile_rows = best_tile;
    best->items_per_cta = best_ipc;
  }
  if (best_us) *best_us = best_t;
  return CQ_OK;
}

// ---------------------------------------------------------------- serving loop
namespace cq {

// A plan with every array and literal it points to copied.
struct PlanCopy {
  std::vector<cq_predicate> preds;
  std::vector<std::vector<int64_t>> ints;
  std::vector<std::vector<std::string>> strs;
  std::vector<std::vector<const char*>> str_ptrs;
  std::vector<std::vector<uint32_t>> str_lens;
  std::vector<uint32_t> group_by;
  std::vector<cq_aggregate> aggs;
  std::vector<cq_filter_node> filter;
  cq_plan plan;

  explicit PlanCopy(const cq_plan& p) {
    preds.assign(p.preds, p.preds + (p.preds ? p.n_preds : 0));
    ints.resize(preds.size());
    strs.resize(preds.size());
    str_ptrs.resize(preds.size());
    str_lens.resize(preds.size());
    for (size_t i = 0; i < preds.size(); ++i) {
      cq_predicate& d = preds[i];
      if (d.in_ints && d.n_in) ints[i].assign(d.in_ints, d.in_ints + d.n_in);
      if (d.strs && d.n_strs) {
        for (uint32_t k = 0; k < d.n_strs; ++k) {
          const size_t len = d.str_lens ? d.str_lens[k] : (d.strs[k] ? strlen(d.strs[k]) : 0);
          strs[i].emplace_back(d.strs[k] ? std::string(d.strs[k], len) : std::string());
        }
      }
      for (const std::string& x : strs[i]) {
        str_ptrs[i].push_back(x.data());
        str_lens[i].push_back((uint32_t)x.size());
      }
      d.in_ints = ints[i].empty() ? nullptr : ints[i].data();
      d.strs = str_ptrs[i].empty() ? nullptr : str_ptrs[i].data();
      d.str_lens = str_lens[i].empty() ? nullptr : str_lens[i].data();
    }
    group_by.assign(p.group_by, p.group_by + (p.group_by ? p.n_group_by : 0));
    aggs.assign(p.aggs, p.aggs + (p.aggs ? p.n_aggs : 0));
    plan.preds = preds.empty() ? nullptr : preds.data();
    plan.n_preds = (uint32_t)preds.size();
    plan.group_by = group_by.empty() ? nullptr : group_by.data();
    plan.n_group_by = (uint32_t)group_by.size();
    plan.aggs = aggs.empty() ? nullptr : aggs.data();
    plan.n_aggs = (uint32_t)aggs.size();
    filter.assign(p.filter, p.filter + (p.filter ? p.n_filter : 0));
    plan.filter = filter.empty() ? nullptr : filter.data();
    plan.n_filter = p.n_filter;
  }
};

using Clock = std::chrono::steady_clock;

struct Request {
  uint64_t ticket = 0;
  cq_table* table = nullptr;
  bool large = false;      // large lane: launched alone, one large launch in flight at a time
  Planned planned;
  uint64_t footprint = 0;
  Clock::time_point submitted;
  // completion
  bool done = false;
  int status = CQ_OK;
  std::string error;
  cq_result* result = nullptr;
  double latency_us = 0;
};

struct InFlight {
  std::vector<std::shared_ptr<Request>> reqs;
  cudaEvent_t done = nullptr;
  uint64_t footprint = 0;
  int stream = 0;
};

}  // namespace cq

struct cq_server {
  cq_ctx* ctx = nullptr;
  cq_server_options opt;
  uint64_t large_rows = 0;   // tables above this many rows go to the large lane
  std::vector<cudaStream_t> streams;
  std::vector<int> stream_busy;             // launches in flight per stream
  std::vector<cudaEvent_t> free_events;
  std::mutex mu;
  std::condition_variable cv_submit, cv_done;
  std::deque<std::shared_ptr<cq::Request>> pending;        // small lane
  std::deque<std::shared_ptr<cq::Request>> pending_large;  // large lane
  std::unordered_map<uint64_t, std::shared_ptr<cq::Request>> by_ticket;
  std::vector<cq::InFlight> inflight;
  uint64_t next_ticket = 1;
  uint64_t used_bytes = 0;
  uint64_t launches = 0, completed = 0;
  bool stop = false;
  std::thread loop;
};

namespace cq {

// Take admitted requests for the next launch: oldest first, while the batch
// has room and their footprints fit the budget beside what is in flight.
static std::vector<std::shared_ptr<Request>> take_batch(cq_server* srv, std::deque<std::shared_ptr<Request>>& from,
                                                         uint32_t max_n) {
  std::vector<std::shared_ptr<Request>> b;
  uint64_t used = srv->used_bytes;
  while (!from.empty() && b.size() < max_n) {
    const std::shared_ptr<Request>& r = from.front();
    if (used + r->footprint > srv->opt.memory_budget_bytes && !(b.empty() && srv->inflight.empty())) break;
    used += r->footprint;
    b.push_back(r);
    from.pop_front();
  }
  srv->used_bytes = used;
  return b;
}

static void finish(cq_server* srv, Request& r, int status, const std::string& err) {
  r.done = true;
  r.status = status;
  r.error = err;
  r.latency_us = std::chrono::duration<double, std::micro>(Clock::now() - r.submitted).count();
  srv->completed++;
}

// State of a launch in flight: cudaSuccess (done), cudaErrorNotReady, or
// the error the launch met.  With CQ_FAULT_INJECT=event:N the N-th poll of
// the process reports a launch failure without asking CUDA (tests of the
// error path).
static cudaError_t poll_launch(cudaEvent_t ev) {
  static const long long fail_at = fault_inject_at("event");
  static std::atomic<long long> polls{0};
  if (fail_at > 0 && ++polls == fail_at) return cudaErrorLaunchFailure;
  const cudaError_t e = cudaEventQuery(ev);
  if (e == cudaErrorNotReady) (void)cudaGetLastError();   // not ready is not an error
  return e;
}

// The serving loop: launch batches while streams and memory allow, poll the
// launches in flight, hand finished results to their waiters.
static void serve(cq_server* srv) {
  cudaSetDevice(srv->ctx->device);
  const auto max_wait = std::chrono::microseconds(srv->opt.max_wait_us);
  std::unique_lock<std::mutex> lk(srv->mu);
  while (true) {
    // ---- completions
    bool any_done = false;
    for (size_t i = 0; i < srv->inflight.size();) {
      InFlight& f = srv->inflight[i];
      const cudaError_t st = poll_launch(f.done);
      if (st == cudaErrorNotReady) {
        ++i;
        continue;
      }
      if (st != cudaSuccess) {
        // the launch failed: its requests end with the error and their
        // results are released once the stream has drained
        const std::string msg = std::string("the launch of this query's batch failed: ") + cudaGetErrorString(st);
        (void)cudaGetLastError();
        cudaStreamSynchronize(srv->streams[f.stream]);
        (void)cudaGetLastError();
        for (auto& r : f.reqs) {
          if (r->result) {
            r->result->stream = srv->ctx->stream;
            if (r->result->batch_keepalive)
              static_cast<BatchShared*>(r->result->batch_keepalive.get())->stream = srv->ctx->stream;
            cq_result_destroy(r->result);
            r->result = nullptr;
          }
          finish(srv, *r, CQ_ERR_CUDA, msg);
        }
        srv->used_bytes -= f.footprint;
        srv->stream_busy[f.stream]--;
        cudaEventDestroy(f.done);
        srv->inflight[i] = std::move(srv->inflight.back());
        srv->inflight.pop_back();
        any_done = true;
        continue;
      }
      for (auto& r : f.reqs) {
        // the result is complete: later frees may go to the context's stream,
        // so results outlive the server's own streams
        if (r->result) {
          r->result->stream = srv->ctx->stream;
          if (r->result->batch_keepalive)
            static_cast<BatchShared*>(r->result->batch_keepalive.get())->stream = srv->ctx->stream;
        }
        finish(srv, *r, CQ_OK, std::string());
      }
      srv->used_bytes -= f.footprint;
      srv->stream_busy[f.stream]--;
      srv->free_events.push_back(f.done);
      srv->inflight[i] = std::move(srv->inflight.back());
      srv->inflight.pop_back();
      any_done = true;
    }
    if (any_done) srv->cv_done.notify_all();
    if (srv->stop && srv->pending.empty() && srv->pending_large.empty() && srv->inflight.empty()) break;
    // ---- launches.  With two lanes, every launch goes to stream 0, at most
    // two queued: a fused kernel fills every SM (one persistent CTA per SM,
    // most of its shared memory), so launches on several streams would only
    // wait for one another.  Waiting small queries go first, as one batch, when
    // nothing runs, the batch is full or the oldest has waited max_wait_us;
    // otherwise the oldest large query runs alone.  With one lane
    // (n_streams == 1) every query is batched, but for those a batch cannot
    // take, which run alone when nothing else waits.
    int sidx = -1;
    std::vector<std::shared_ptr<Request>> b;
    const bool two_lanes = srv->opt.n_streams >= 2;
    if (two_lanes) {
      const size_t in_flight = srv->inflight.size();
      if (in_flight < 2) {
        const bool small_ready =
            !srv->pending.empty() && (in_flight == 0 || srv->pending.size() >= srv->opt.max_batch || srv->stop ||
                                      Clock::now() - srv->pending.front()->submitted >= max_wait);
        if (small_ready) b = take_batch(srv, srv->pending, srv->opt.max_batch);
        else if (srv->pending.empty() && !srv->pending_large.empty()) b = take_batch(srv, srv->pending_large, 1);
        if (!b.empty()) sidx = 0;
      }
    } else if (srv->stream_busy[0] == 0) {
      if (!srv->pending.empty() && (srv->inflight.empty() || srv->pending.size() >= srv->opt.max_batch ||
                                    srv->stop || Clock::now() - srv->pending.front()->submitted >= max_wait))
        b = take_batch(srv, srv->pending, srv->opt.max_batch);
      else if (srv->pending.empty() && !srv->pending_large.empty())
        b = take_batch(srv, srv->pending_large, 1);
      if (!b.empty()) sidx = 0;
    }
    if (!b.empty()) {
      {
        uint64_t fp = 0;
        for (auto& r : b) fp += r->footprint;
        lk.unlock();
        std::vector<cq_table*> tables;
        std::vector<Planned> P;
        for (auto& r : b) {
          tables.push_back(r->table);
          P.push_back(r->planned);
        }
        std::vector<cq_result*> res(b.size(), nullptr);
        // a batch of one runs the one-query kernels (no per-item table
        // resets and flushes, no control-block upload)
        const int rc = b.size() == 1 ? launch_solo(tables[0], P[0], srv->streams[sidx], &res[0])
                                     : launch_planned_batch(srv->ctx, (uint32_t)b.size(), tables.data(), P, 0, 1,
                                                            srv->streams[sidx], res.data());
        const std::string err = rc == CQ_OK ? std::string() : std::string(cq_last_error());
        cudaEvent_t ev = nullptr;
        lk.lock();
        int rc2 = rc;
        std::string err2 = err;
        if (rc == CQ_OK) {
          cudaError_t ee = cudaSuccess;
          if (!srv->free_events.empty()) {
            ev = srv->free_events.back();
            srv->free_events.pop_back();
          } else {
            ee = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
          }
          if (ee == cudaSuccess) ee = cudaEventRecord(ev, srv->streams[sidx]);
          if (ee != cudaSuccess) {
            // without a completion event the launch cannot be tracked: wait
            // for it here and fail its requests
            rc2 = CQ_ERR_CUDA;
            err2 = std::string("completion event of a launch: ") + cudaGetErrorString(ee);
            (void)cudaGetLastError();
            if (ev) cudaEventDestroy(ev);
            cudaStreamSynchronize(srv->streams[sidx]);
            (void)cudaGetLastError();
            for (cq_result* x : res)
              if (x) {
                x->stream = srv->ctx->stream;
                if (x->batch_keepalive) static_cast<BatchShared*>(x->batch_keepalive.get())->stream = srv->ctx->stream;
                cq_result_destroy(x);
              }
          }
        }
        if (rc2 == CQ_OK) {
          for (size_t k = 0; k < b.size(); ++k) b[k]->result = res[k];
          InFlight f;
          f.reqs = std::move(b);
          f.done = ev;
          f.footprint = fp;
          f.stream = sidx;
          srv->stream_busy[sidx]++;
          srv->inflight.push_back(std::move(f));
          srv->launches++;
        } else {
          for (auto& r : b) finish(srv, *r, rc2, err2);
          srv->used_bytes -= fp;
          srv->cv_done.notify_all();
        }
        continue;
      }
    }
    // ---- wait: for a submission, or briefly while launches are in flight
    if (srv->inflight.empty() && srv->pending.empty() && srv->pending_large.empty()) {
      srv->cv_submit.wait(lk);
    } else {
      srv->cv_submit.wait_for(lk, std::chrono::microseconds(20));
    }
  }
}

}  // namespace cq

extern "C" int cq_server_create(cq_ctx* ctx, const cq_server_options* opts, cq_server** out) {
  clear_error();
  if (!ctx || !out) return set_error(CQ_ERR_INVALID_ARG, "NULL context or out");
  *out = nullptr;
  std::unique_ptr<cq_server> srv(new cq_server);
  srv->ctx = ctx;
  memset(&srv->opt, 0, sizeof(srv->opt));
  if (opts) srv->opt = *opts;
  if (!srv->opt.memory_budget_bytes) srv->opt.memory_budget_bytes = 1ull << 30;
  if (!srv->opt.max_batch) srv->opt.max_batch = 256;
  if (!srv->opt.n_streams) srv->opt.n_streams = 2;
  if (!srv->opt.max_wait_us) srv->opt.max_wait_us = 50;
  srv->large_rows = srv->opt.large_rows_log2 ? (1ull << (srv->opt.large_rows_log2 < 63 ? srv->opt.large_rows_log2 : 63))
                                             : (1ull << 22);
  if (srv->opt.n_streams > 16) return set_error(CQ_ERR_INVALID_ARG, "at most 16 streams");
  CQ_CUDA(cudaSetDevice(ctx->device));
  {
    std::lock_guard<std::mutex> lk(ctx->batch_mu);
    const int rc = ensure_batch_kernel(ctx);
    if (rc != CQ_OK) return rc;
  }
  // every launch goes to one stream (n_streams >= 2 selects the two lanes)
  {
    cudaStream_t st = nullptr;
    CQ_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    srv->streams.push_back(st);
    srv->stream_busy.push_back(0);
  }
  ctx->refs++;   // the server keeps its context alive
  cq_server* s = srv.release();
  s->loop = std::thread(serve, s);
  *out = s;
  return CQ_OK;
}

extern "C" int cq_server_submit(cq_server* srv, cq_table* table, const cq_plan* plan, uint64_t* ticket) {
  clear_error();
  if (!srv || !table || !plan || !ticket) return set_error(CQ_ERR_INVALID_ARG, "NULL argument");
  if (table->ctx != srv->ctx) return set_error(CQ_ERR_INVALID_ARG, "table of another context");
  std::shared_ptr<Request> r(new Request);
  r->submitted = Clock::now();
  // large-lane queries always run alone: planned (and their kernel compiled)
  // like cq_query_run's; small ones for a shared batch
  r->large = srv->opt.n_streams >= 2 && table->n_rows > srv->large_rows;
  {
    PlanCopy pc(*plan);   // literals resolved at planning; the copy lives until then
    int rc = r->large ? plan_solo_query(table, &pc.plan, &r->planned)
                      : plan_batch_query(table, &pc.plan, 0, srv->ctx->batch_smem, &r->planned);
    if (rc == CQ_ERR_UNSUPPORTED && !r->large) {
      // what a batch cannot take (a key domain in the global hash table, a
      // table above 2^31 rows) runs alone, in the large lane
      clear_error();
      rc = plan_solo_query(table, &pc.plan, &r->planned);
      r->large = rc == CQ_OK;
    }
    if (rc != CQ_OK) return rc;
  }
  {
    // the kernel specialised to the query's shape is compiled here, on the
    // submitting thread, not in the serving loop (a lone query runs it)
    const int rc = prepare_row_kernel(srv->ctx, r->planned);
    if (rc != CQ_OK) return rc;
  }
  r->footprint = query_footprint(r->planned);
  std::lock_guard<std::mutex> lk(srv->mu);
  if (srv->stop) return set_error(CQ_ERR_INVALID_ARG, "server is shutting down");
  if (r->footprint > srv->opt.memory_budget_bytes)
    return set_error(CQ_ERR_BUSY, "query needs %llu device bytes, the budget is %llu",
                     (unsigned long long)r->footprint, (unsigned long long)srv->opt.memory_budget_bytes);
  r->ticket = srv->next_ticket++;
  // a private binding of the table's columns: the caller may destroy its
  // table handle before the query has run
  r->table = new cq_table(*table);
  for (cq_column* c : table->cols) c->refs++;
  srv->by_ticket[r->ticket] = r;
  if (r->large) srv->pending_large.push_back(r);
  else srv->pending.push_back(r);
  *ticket = r->ticket;
  srv->cv_submit.notify_one();
  return CQ_OK;
}

extern "C" int cq_server_wait(cq_server* srv, uint64_t ticket, uint64_t timeout_us, cq_result** res,
                              double* latency_us) {
  clear_error();
  if (!srv || !res) return set_error(CQ_ERR_INVALID_ARG, "NULL argument");
  *res = nullptr;
  std::unique_lock<std::mutex> lk(srv->mu);
  auto it = srv->by_ticket.find(ticket);
  if (it == srv->by_ticket.end()) return set_error(CQ_ERR_INVALID_ARG, "unknown ticket %llu", (unsigned long long)ticket);
  std::shared_ptr<Request> r = it->second;
  auto ready = [&] { return r->done; };
  if (timeout_us == UINT64_MAX) srv->cv_done.wait(lk, ready);
  else if (!srv->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), ready))
    return set_error(CQ_ERR_NOT_READY, "query %llu still running", (unsigned long long)ticket);
  srv->by_ticket.erase(it);
  lk.unlock();
  cq_table_destroy(r->table);
  r->table = nullptr;
  if (latency_us) *latency_us = r->latency_us;
  if (r->status != CQ_OK) return set_error(r->status, "%s", r->error.c_str());
  *res = r->result;
  r->result = nullptr;
  return CQ_OK;
}

extern "C" int cq_server_stats(cq_server* srv, uint64_t* launches, uint64_t* completed) {
  if (!srv) return set_error(CQ_ERR_INVALID_ARG, "NULL server");
  std::lock_guard<std::mutex> lk(srv->mu);
  if (launches) *launches = srv->launches;
  if (completed) *completed = srv->completed;
  return CQ_OK;
}

extern "C" int cq_server_destroy(cq_server* srv) {
  clear_error();
  if (!srv) return CQ_OK;
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    srv->stop = true;
  }
  srv->cv_submit.notify_all();
  if (srv->loop.joinable()) srv->loop.join();
  cudaSetDevice(srv->ctx->device);
  for (auto& kv : srv->by_ticket) {   // results nobody collected
    if (kv.second->result) cq_result_destroy(kv.second->result);
    cq_table_destroy(kv.second->table);
  }
  for (cudaEvent_t e : srv->free_events) cudaEventDestroy(e);
  for (cudaStream_t st : srv->streams) {
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
  }
  cq_ctx* ctx = srv->ctx;
  delete srv;
  ctx_release(ctx);
  return CQ_OK;
}
