// CUDA graphs of the solvers' outer-iteration phases (graph.cuh).
#include <algorithm>

#include "graph.cuh"

namespace blws {

namespace {

constexpr size_t kMaxGraphs = 12;  // phases cached per context (two phases, two E buffers, spares)
constexpr size_t kMaxSeen = 16;

void destroy_entry(GraphEntry& e) {
  if (e.exec) cudaGraphExecDestroy(e.exec);
  for (TimedPair& t : e.ev) {
    cudaEventDestroy(t.e0);
    cudaEventDestroy(t.e1);
  }
  e.exec = nullptr;
  e.ev.clear();
}

void drop_capture_events(Ctx* ctx) {
  for (TimedPair& t : ctx->cap_ev) {
    if (t.e0) cudaEventDestroy(t.e0);
    if (t.e1) cudaEventDestroy(t.e1);
  }
  ctx->cap_ev.clear();
}

}  // namespace

void graph_key_ctx(const Ctx* ctx, GraphKey& key) {
  key.u(ctx->gen).u(ctx->timing).u(ctx->oz_tail).u((uint64_t)ctx->cfg.precision);
  key.u((uint64_t)ctx->eig_route).u((uint64_t)ctx->tri_route).u((uint64_t)ctx->sms);
}

GraphEntry* graph_find(Ctx* ctx, const GraphKey& key) {
  for (GraphEntry& e : ctx->graphs)
    if (e.key == key.v) return &e;
  return nullptr;
}

bool graph_seen(Ctx* ctx, const GraphKey& key) {
  for (const auto& k : ctx->seen)
    if (k == key.v) return true;
  if (ctx->seen.size() >= kMaxSeen) ctx->seen.erase(ctx->seen.begin());
  ctx->seen.push_back(key.v);
  return false;
}

blws_status graph_replay(Ctx* ctx, cudaStream_t s, GraphEntry* e) {
  BLWS_TRY_CUDA(ctx, cudaEventRecord(ctx->gfork, s));
  BLWS_TRY_CUDA(ctx, cudaStreamWaitEvent(ctx->gstream, ctx->gfork, 0));
  BLWS_TRY_CUDA(ctx, cudaGraphLaunch(e->exec, ctx->gstream));
  BLWS_TRY_CUDA(ctx, cudaEventRecord(ctx->gjoin, ctx->gstream));
  BLWS_TRY_CUDA(ctx, cudaStreamWaitEvent(s, ctx->gjoin, 0));
  ctx->launches += e->nlaunch;
  e->last_use = ++ctx->graph_clock;
  ++ctx->graph_replays;
  if (ctx->timing)
    for (const TimedPair& t : e->ev) ctx->pending_ev.push_back(t);
  return BLWS_OK;
}

blws_status graph_capture_begin(Ctx* ctx, cudaStream_t s) {
  if (!ctx->gstream) {
    BLWS_TRY_CUDA(ctx, cudaStreamCreateWithFlags(&ctx->gstream, cudaStreamNonBlocking));
    BLWS_TRY_CUDA(ctx, cudaEventCreateWithFlags(&ctx->gfork, cudaEventDisableTiming));
    BLWS_TRY_CUDA(ctx, cudaEventCreateWithFlags(&ctx->gjoin, cudaEventDisableTiming));
  }
  // the graph stream is ordered after s before the capture starts, so the
  // replays that follow on it are too
  BLWS_TRY_CUDA(ctx, cudaEventRecord(ctx->gfork, s));
  BLWS_TRY_CUDA(ctx, cudaStreamWaitEvent(ctx->gstream, ctx->gfork, 0));
  BLWS_TRY_CUDA(ctx, cudaStreamBeginCapture(ctx->gstream, cudaStreamCaptureModeRelaxed));
  ctx->capturing = true;
  ctx->capture_broken = false;
  drop_capture_events(ctx);
  return BLWS_OK;
}

blws_status graph_capture_end(Ctx* ctx, const GraphKey& key, blws_status phase_status,
                              unsigned long long launches_before, GraphEntry** out) {
  *out = nullptr;
  ctx->capturing = false;
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(ctx->gstream, &g);
  cudaGraphExec_t x = nullptr;
  bool ok = phase_status == BLWS_OK && e == cudaSuccess && g != nullptr;
  if (ok) ok = cudaGraphInstantiateWithFlags(&x, g, 0) == cudaSuccess;
  if (g) cudaGraphDestroy(g);
  if (!ok) {
    // nothing of the phase ran: it runs again directly (a workspace buffer
    // that had to grow grows there; a genuine error is reported there)
    cudaGetLastError();
    drop_capture_events(ctx);
    ctx->capture_broken = false;
    ctx->launches = launches_before;
    return BLWS_OK;
  }
  if (ctx->graphs.size() >= kMaxGraphs) {
    // the least recently used entry goes; its timed products are read first
    BLWS_TRY(graph_harvest(ctx));
    auto lru = std::min_element(ctx->graphs.begin(), ctx->graphs.end(),
                                [](const GraphEntry& a, const GraphEntry& b) { return a.last_use < b.last_use; });
    destroy_entry(*lru);
    ctx->graphs.erase(lru);
  }
  GraphEntry ne;
  ne.key = key.v;
  ne.exec = x;
  ne.nlaunch = ctx->launches - launches_before;
  ne.ev.swap(ctx->cap_ev);
  ctx->graphs.push_back(std::move(ne));
  ctx->launches = launches_before;  // counted again by the replay that follows
  ++ctx->graph_captures;
  *out = &ctx->graphs.back();
  return BLWS_OK;
}

blws_status graph_harvest(Ctx* ctx) {
  for (const TimedPair& t : ctx->pending_ev) {
    BLWS_TRY_CUDA(ctx, cudaEventSynchronize(t.e1));
    float ms = 0.0f;
    BLWS_TRY_CUDA(ctx, cudaEventElapsedTime(&ms, t.e0, t.e1));
    ctx->graph_ms.push_back(ms);
    ctx->graph_w.push_back(t.work);
    ctx->graph_kind.push_back(t.kind);
  }
  ctx->pending_ev.clear();
  return BLWS_OK;
}

void Ctx::free_graphs() {
  graph_harvest(this);
  for (GraphEntry& e : graphs) destroy_entry(e);
  graphs.clear();
  seen.clear();
  drop_capture_events(this);
}

blws_status Ctx::host_eig_get(size_t bytes) {
  if (bytes <= host_eig_cap) return BLWS_OK;
  if (capturing) {  // pinned allocation: outside the capture
    capture_broken = true;
    return fail(BLWS_ECUDA, "pinned host buffer must grow inside a graph capture");
  }
  ++gen;  // graphs copy into the old buffer's address: none may be replayed again
  if (host_eig) {
    cudaFreeHost(host_eig);
    host_eig = nullptr;
    host_eig_cap = 0;
  }
  const size_t want = std::max<size_t>(bytes, 4096);
  if (cudaMallocHost(&host_eig, want) != cudaSuccess) {
    cudaGetLastError();
    host_eig = nullptr;
    return fail(BLWS_ENOMEM, "cudaMallocHost(%zu) for the eigen-solver's host copies", want);
  }
  host_eig_cap = want;
  return BLWS_OK;
}

}  // namespace blws
