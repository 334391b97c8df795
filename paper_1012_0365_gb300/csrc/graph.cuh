// CUDA graphs of the solvers' outer-iteration phases.
//
// An outer iteration of the RPCA solver is two phases that never wait on the
// host (the BLWS block steps up to the device stage of the eigen-solver; the
// Ritz lift, thresholds and fused epilogue), separated by host decisions (the
// eigen-solver's clusters, the rank prediction, the stopping test).  Once the
// rank settles, every iteration launches the same kernels with the same
// arguments: only the scalars mu and eps change, and the kernels read those
// from device memory.  A phase is therefore described by a key (every
// argument its launches depend on, the context's workspace generation
// included); the first time a key is met the phase launches directly, the
// second time it is captured into a graph on the context's graph stream, and
// from then on the graph is replayed with one launch.  The phase runs on the
// graph stream between an event recorded on the caller's stream and one the
// caller's stream waits for, so stream order is what it would be with direct
// launches, and the kernels and their arguments are the same either way:
// results are bit-identical with and without graphs.
#pragma once
#include <string.h>

#include <vector>

#include "common.cuh"

namespace blws {

struct GraphKey {
  std::vector<uint64_t> v;
  GraphKey& u(uint64_t x) {
    v.push_back(x);
    return *this;
  }
  GraphKey& p(const void* x) { return u((uint64_t)(uintptr_t)x); }
  GraphKey& d(double x) {
    uint64_t b;
    memcpy(&b, &x, sizeof b);
    return u(b);
  }
};

// append the context state every phase's launches depend on
void graph_key_ctx(const Ctx* ctx, GraphKey& key);
// the cached graph for key (nullptr: none)
GraphEntry* graph_find(Ctx* ctx, const GraphKey& key);
// true when key was met before (and remembers it otherwise)
bool graph_seen(Ctx* ctx, const GraphKey& key);
// replay e after the work already on s
blws_status graph_replay(Ctx* ctx, cudaStream_t s, GraphEntry* e);
// start capturing on the graph stream, ordered after the work on s
blws_status graph_capture_begin(Ctx* ctx, cudaStream_t s);
// end the capture; on success *e is the new entry (not yet launched), else
// nullptr (the phase must then run directly)
blws_status graph_capture_end(Ctx* ctx, const GraphKey& key, blws_status phase_status,
                              unsigned long long launches_before, GraphEntry** e);
// read the times of the products timed inside replayed graphs (synchronises
// their events; the caller has synchronised the stream already in practice)
blws_status graph_harvest(Ctx* ctx);

// Run phase(stream) for key: replayed, captured or direct (see above).
template <class Phase>
blws_status graph_phase(Ctx* ctx, cudaStream_t s, GraphKey& key, Phase&& phase) {
  if (!ctx->graphs_on) return phase(s);
  graph_key_ctx(ctx, key);
  if (GraphEntry* e = graph_find(ctx, key)) return graph_replay(ctx, s, e);
  if (!graph_seen(ctx, key)) return phase(s);
  BLWS_TRY(graph_capture_begin(ctx, s));
  const unsigned long long l0 = ctx->launches;
  const blws_status st = phase(ctx->gstream);
  GraphEntry* e = nullptr;
  BLWS_TRY(graph_capture_end(ctx, key, st, l0, &e));
  if (!e) return phase(s);  // not capturable this time: launch directly
  return graph_replay(ctx, s, e);
}

}  // namespace blws
