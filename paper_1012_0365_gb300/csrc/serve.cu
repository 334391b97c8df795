// Serving and batching runtime around the solvers (include/blws.h, "Serving
// and batching"): a pool of worker threads, each owning a context and a
// non-blocking CUDA stream, fed from one FIFO queue with admission by device
// memory.  Solves admitted together run concurrently on their streams.
//
// Admission: the head of the queue starts when a worker is idle and the device
// bytes every worker would then hold fit the budget.  A worker holds the
// larger of its running request's estimate and what its context's workspace
// retains from earlier requests (workspace buffers only grow), so memory kept
// by idle workers counts too.  When nothing runs, the head starts anyway (a
// request larger than the whole budget runs alone), taken by the idle worker
// that retains the most workspace, so that it reuses that memory instead of
// adding to it.  A worker that finishes while the workers together hold more
// than the budget frees its workspace.  Requests keep arrival order: a large
// head is not overtaken by smaller ones behind it.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "common.cuh"

namespace {

using Clock = std::chrono::steady_clock;

struct Job {
  uint64_t ticket;
  blws_request req;
  size_t bytes;
  Clock::time_point submitted;
};

struct Done {
  blws_result res;
};

}  // namespace

struct blws_server {
  blws_server_config cfg;
  std::vector<std::thread> threads;
  std::mutex mu;
  std::condition_variable cv_work;   // workers: a job may be admissible
  std::condition_variable cv_done;   // waiters: a result arrived
  std::deque<Job> queue;
  std::unordered_map<uint64_t, Done> done;
  std::unordered_set<uint64_t> outstanding;  // submitted, not yet waited for
  uint64_t next_ticket = 1;
  bool stopping = false;
  size_t in_use = 0;
  int running = 0;
  std::vector<size_t> held;  // per worker: bytes its context's workspace retains
  std::vector<size_t> est;   // per worker: estimate of its running request (0: idle)
  blws_server_stats stats{};
  blws_status start_status = BLWS_OK;
  int started = 0;
};

namespace {

// workspace every solve reserves whatever its size: the split-K partial sums
// of the FP64 GEMMs (16 x SMs x 64 x 64 doubles) and the reduction partials
size_t fixed_bytes(int sms) { return (size_t)16 * sms * 64 * 64 * 8 + (size_t)sms * 8 * 8 + 4096 * 8; }

size_t rpca_bytes(int m, int n, int ld, int k, int k_cold, int sv0, int precision, int sms) {
  const size_t N = (size_t)m + n;
  const int pmin = std::min(m, n);
  // widest Lanczos block the solve is expected to reach: the rank prediction
  // grows by 5% of n per step while counts keep up; capped as the solver caps it
  const size_t bcap = std::max<size_t>(1, std::min<size_t>((size_t)pmin, N / std::max(k, k_cold)));
  const size_t best = std::min<size_t>(bcap, std::max<size_t>((size_t)sv0 * 4, (size_t)pmin / 4 + sv0));
  const size_t kb = (size_t)std::max(k, k_cold) * best;
  size_t b = 3 * (size_t)ld * n * 8;       // Y, W, second E buffer
  b += N * kb * 8 + 2 * N * best * 8;      // Lanczos basis, P, P2
  b += 3 * kb * kb * 8 + 9 * kb * kb * 4;  // T_k, eigen-solver scratch
  b += (m + n) * best * 8;                 // warm-start factors
  if (precision == BLWS_PREC_MIXED) b += (size_t)16 * m * n + 4 * N * best * 4;  // TF32 planes
  if (precision == BLWS_PREC_FP64_TC)  // BF16 digit planes; A as a product
    b += (size_t)28 * m * n + 28 * N * 128 + (size_t)ld * n * 8;
  return b + fixed_bytes(sms);
}

size_t mc_bytes(int m, int n, int nnz, int max_rank, int k, int k_cold, int sms) {
  const size_t N = (size_t)m + n;
  const size_t b = (size_t)std::max(1, max_rank);
  const size_t kb = (size_t)std::max(k, k_cold) * b;
  size_t s = (size_t)nnz * (4 + 4 + 8 + 8) + ((size_t)n + 1) * 4;  // CSC mirror, iterate values
  s += N * kb * 8 + 2 * N * b * 8 + 3 * kb * kb * 8 + 9 * kb * kb * 4;
  s += 2 * N * b * 8;  // factors of the iterate
  return s + fixed_bytes(sms);
}

// the idle worker that retains the most workspace (lowest index on ties)
int largest_idle(const blws_server* srv) {
  int best = -1;
  for (size_t v = 0; v < srv->held.size(); ++v)
    if (srv->est[v] == 0 && (best < 0 || srv->held[v] > srv->held[best])) best = (int)v;
  return best;
}

// device bytes all workers hold if `worker` takes a request of `need` bytes
size_t held_with(const blws_server* srv, int worker, size_t need) {
  size_t t = 0;
  for (size_t v = 0; v < srv->held.size(); ++v)
    t += std::max(srv->held[v], (int)v == worker ? need : srv->est[v]);
  return t;
}

void worker_main(blws_server* srv, int index) {
  blws_ctx* ctx = nullptr;
  cudaStream_t stream = nullptr;
  blws_status st = blws_create(&ctx, &srv->cfg.cfg);
  if (st == BLWS_OK && cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking) != cudaSuccess)
    st = BLWS_ECUDA;
  if (st == BLWS_OK) ctx->sole_stream = stream;  // growth waits for this worker's stream only
  {
    std::lock_guard<std::mutex> lock(srv->mu);
    if (st != BLWS_OK && srv->start_status == BLWS_OK) srv->start_status = st;
    ++srv->started;
  }
  srv->cv_done.notify_all();
  for (;;) {
    Job job;
    {
      std::unique_lock<std::mutex> lock(srv->mu);
      srv->cv_work.wait(lock, [&] {
        if (srv->queue.empty()) return srv->stopping;
        const size_t need = srv->queue.front().bytes;
        if (held_with(srv, index, need) <= srv->cfg.hbm_budget) return true;
        return srv->running == 0 && largest_idle(srv) == index;
      });
      if (srv->queue.empty()) break;  // stopping and drained
      job = srv->queue.front();
      srv->queue.pop_front();
      srv->est[index] = job.bytes;
      srv->in_use = held_with(srv, -1, 0);
      ++srv->running;
      srv->stats.in_use = srv->in_use;
      srv->stats.peak_in_use = std::max(srv->stats.peak_in_use, srv->in_use);
      srv->stats.peak_running = std::max(srv->stats.peak_running, srv->running);
    }
    const Clock::time_point t0 = Clock::now();
    Done d{};
    if (st != BLWS_OK) {
      d.res.status = st;
    } else if (job.req.kind == BLWS_REQ_RPCA) {
      d.res.status = rpca_solve(ctx, job.req.D, job.req.m, job.req.n, job.req.ld, &job.req.rpca,
                                job.req.A, job.req.E, &d.res.rpca, stream);
    } else {
      d.res.status = mc_solve(ctx, job.req.m, job.req.n, job.req.nnz, job.req.rowptr, job.req.colidx,
                              job.req.vals, &job.req.mc, job.req.max_rank, job.req.U, job.req.theta,
                              job.req.V, &d.res.mc, stream);
    }
    if (st == BLWS_OK && cudaStreamSynchronize(stream) != cudaSuccess && d.res.status == BLWS_OK)
      d.res.status = BLWS_ECUDA;
    const Clock::time_point t1 = Clock::now();
    d.res.queue_ms = std::chrono::duration<double, std::milli>(t0 - job.submitted).count();
    d.res.run_ms = std::chrono::duration<double, std::milli>(t1 - t0).count();
    bool over = false;
    {
      std::lock_guard<std::mutex> lock(srv->mu);
      if (ctx) srv->held[index] = ctx->held_bytes();
      srv->stats.peak_in_use = std::max(srv->stats.peak_in_use, held_with(srv, -1, 0));
      srv->est[index] = 0;
      over = held_with(srv, -1, 0) > srv->cfg.hbm_budget;
    }
    // over the budget (other workers' retained workspace included): give this
    // worker's workspace back before taking more work
    if (over && ctx && ctx->trim() != BLWS_OK && d.res.status == BLWS_OK) d.res.status = BLWS_ECUDA;
    {
      std::lock_guard<std::mutex> lock(srv->mu);
      if (ctx) srv->held[index] = ctx->held_bytes();
      srv->in_use = held_with(srv, -1, 0);
      srv->stats.peak_in_use = std::max(srv->stats.peak_in_use, srv->in_use);
      --srv->running;
      srv->stats.in_use = srv->in_use;
      ++srv->stats.completed;
      srv->done[job.ticket] = d;
    }
    srv->cv_done.notify_all();
    srv->cv_work.notify_all();
  }
  if (stream) cudaStreamDestroy(stream);
  if (ctx) blws_destroy(ctx);
}

}  // namespace

extern "C" {

blws_status blws_server_config_default(blws_server_config* cfg) {
  if (!cfg) return BLWS_EINVAL;
  cfg->workers = 8;
  cfg->hbm_budget = 0;
  return blws_config_default(&cfg->cfg);
}

size_t blws_request_bytes(const blws_request* req, int precision) {
  if (!req) return 0;
  blws_config c;
  blws_config_default(&c);
  // SM count of the current device (the split-K reservation scales with it)
  int dev = 0, sms = 152;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    sms = 152;
  }
  if (req->kind == BLWS_REQ_RPCA)
    return rpca_bytes(req->m, req->n, req->ld, c.k, c.k_cold, std::max(req->rpca.sv0, 1), precision, sms);
  return mc_bytes(req->m, req->n, req->nnz, req->max_rank, c.k, c.k_cold, sms);
}

blws_status blws_server_create(blws_server** out, const blws_server_config* cfg) {
  if (!out) return BLWS_EINVAL;
  *out = nullptr;
  blws_server_config c;
  blws_server_config_default(&c);
  if (cfg) c = *cfg;
  if (c.workers < 1 || c.workers > 256) return BLWS_EINVAL;
  if (cudaSetDevice(c.cfg.device) != cudaSuccess) return BLWS_ECUDA;
  if (c.hbm_budget == 0) {
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) return BLWS_ECUDA;
    c.hbm_budget = free_b / 10 * 7;
  }
  blws_server* srv = new (std::nothrow) blws_server();
  if (!srv) return BLWS_ENOMEM;
  srv->cfg = c;
  srv->stats.budget = c.hbm_budget;
  srv->held.assign(c.workers, 0);
  srv->est.assign(c.workers, 0);
  for (int i = 0; i < c.workers; ++i) srv->threads.emplace_back(worker_main, srv, i);
  blws_status st;
  {
    std::unique_lock<std::mutex> lock(srv->mu);
    srv->cv_done.wait(lock, [&] { return srv->started == c.workers; });
    st = srv->start_status;
  }
  if (st != BLWS_OK) {
    blws_server_destroy(srv);
    return st;
  }
  *out = srv;
  return BLWS_OK;
}

blws_status blws_server_submit(blws_server* srv, const blws_request* req, uint64_t* ticket) {
  if (!srv || !req || !ticket) return BLWS_EINVAL;
  if (req->kind == BLWS_REQ_RPCA) {
    if (!req->D || !req->A || !req->E || req->m < 1 || req->n < 1 || req->ld < req->m) return BLWS_EINVAL;
  } else if (req->kind == BLWS_REQ_MC) {
    if (!req->rowptr || !req->U || !req->theta || !req->V || req->m < 1 || req->n < 1 ||
        req->nnz < 0 || req->max_rank < 1)
      return BLWS_EINVAL;
  } else {
    return BLWS_EINVAL;
  }
  Job job;
  job.req = *req;
  job.bytes = blws_request_bytes(req, srv->cfg.cfg.precision);
  job.submitted = Clock::now();
  {
    std::lock_guard<std::mutex> lock(srv->mu);
    if (srv->stopping) return BLWS_EINVAL;
    job.ticket = srv->next_ticket++;
    *ticket = job.ticket;
    srv->outstanding.insert(job.ticket);
    srv->queue.push_back(job);
    ++srv->stats.submitted;
  }
  srv->cv_work.notify_all();
  return BLWS_OK;
}

blws_status blws_server_wait(blws_server* srv, uint64_t ticket, blws_result* out) {
  if (!srv || !out) return BLWS_EINVAL;
  std::unique_lock<std::mutex> lock(srv->mu);
  if (!srv->outstanding.count(ticket)) return BLWS_EINVAL;  // unknown or already waited for
  srv->cv_done.wait(lock, [&] { return srv->done.count(ticket) > 0; });
  *out = srv->done[ticket].res;
  srv->done.erase(ticket);
  srv->outstanding.erase(ticket);
  return BLWS_OK;
}

blws_status blws_server_stats_get(blws_server* srv, blws_server_stats* out) {
  if (!srv || !out) return BLWS_EINVAL;
  std::lock_guard<std::mutex> lock(srv->mu);
  *out = srv->stats;
  return BLWS_OK;
}

blws_status blws_server_destroy(blws_server* srv) {
  if (!srv) return BLWS_OK;
  {
    std::lock_guard<std::mutex> lock(srv->mu);
    srv->stopping = true;
  }
  srv->cv_work.notify_all();
  for (auto& t : srv->threads) t.join();
  delete srv;
  return BLWS_OK;
}

}  // extern "C"
