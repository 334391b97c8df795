// C ABI of the library (include/blws.h): argument checks, context, buffers.
#include <stdarg.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>

#include "mc_kernels.cuh"
#include "graph.cuh"
#include "solver.cuh"

namespace blws {

blws_status Ctx::fail(blws_status code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(last_error, sizeof(last_error), fmt, ap);
  va_end(ap);
  return code;
}

namespace {
std::mutex g_attr_mutex;
constexpr int kAttrDevices = 64;
int g_attr_bytes[kAttrDevices][Ctx::ATTR_COUNT_] = {};
}  // namespace

blws_status Ctx::smem_limit(SmemAttr which, const void* func, int bytes) {
  if (device < 0 || device >= kAttrDevices) return fail(BLWS_ENOTSUP, "device ordinal %d", device);
  std::lock_guard<std::mutex> lock(g_attr_mutex);
  if (bytes <= g_attr_bytes[device][which]) return BLWS_OK;
  const cudaError_t e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e != cudaSuccess)
    return fail(BLWS_ECUDA, "cudaFuncSetAttribute(%d bytes): %s", bytes, cudaGetErrorString(e));
  g_attr_bytes[device][which] = bytes;
  return BLWS_OK;
}

blws_status Ctx::get(Buf b, size_t bytes, void** out) {
  if (bytes == 0) bytes = 256;
  if (bytes > cap[b]) {
    if (capturing) {  // growth would synchronise: the phase runs directly instead
      capture_broken = true;
      return fail(BLWS_ECUDA, "workspace buffer %d must grow inside a graph capture", (int)b);
    }
    ++gen;
    if (buf[b]) {
      // growth happens between solver phases; make sure nothing still uses it
      if (sole_stream)
        BLWS_TRY_CUDA(this, cudaStreamSynchronize(sole_stream));
      else
        BLWS_TRY_CUDA(this, cudaDeviceSynchronize());
      BLWS_TRY_CUDA(this, cudaFree(buf[b]));
      buf[b] = nullptr;
      cap[b] = 0;
    }
    const size_t want = std::max(bytes, cap[b] + cap[b] / 2);
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, want);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(BLWS_ENOMEM, "cudaMalloc(%zu) for workspace buffer %d: %s", want, (int)b,
                  cudaGetErrorString(e));
    }
    buf[b] = p;
    cap[b] = want;
  }
  *out = buf[b];
  return BLWS_OK;
}

blws_status Ctx::time_begin(cudaStream_t s) {
  if (!timing) return BLWS_OK;
  if (capturing) {  // events of the graph: recorded by every replay, read after it
    TimedPair t{nullptr, nullptr, 0.0, 0};
    BLWS_TRY_CUDA(this, cudaEventCreate(&t.e0));
    BLWS_TRY_CUDA(this, cudaEventCreate(&t.e1));
    cap_ev.push_back(t);
    BLWS_TRY_CUDA(this, cudaEventRecordWithFlags(t.e0, s, cudaEventRecordExternal));
    return BLWS_OK;
  }
  if (tused == tcap) {  // grow the event pool (between products, not in a kernel's way)
    const size_t ncap = tcap ? 2 * tcap : 256;
    cudaEvent_t* n = new (std::nothrow) cudaEvent_t[2 * ncap];
    double* w = new (std::nothrow) double[ncap];
    int* kk = new (std::nothrow) int[ncap];
    if (!n || !w || !kk) {
      delete[] n;
      delete[] w;
      delete[] kk;
      return fail(BLWS_ENOMEM, "timing events");
    }
    for (size_t i = 0; i < 2 * tcap; ++i) n[i] = tev[i];
    for (size_t i = 0; i < tcap; ++i) {
      w[i] = tw[i];
      kk[i] = tk[i];
    }
    for (size_t i = 2 * tcap; i < 2 * ncap; ++i) BLWS_TRY_CUDA(this, cudaEventCreate(&n[i]));
    delete[] tev;
    delete[] tw;
    delete[] tk;
    tev = n;
    tw = w;
    tk = kk;
    tcap = ncap;
  }
  BLWS_TRY_CUDA(this, cudaEventRecord(tev[2 * tused], s));
  return BLWS_OK;
}

blws_status Ctx::time_end(cudaStream_t s, double work, int kind) {
  if (!timing) return BLWS_OK;
  if (capturing) {
    cap_ev.back().work = work;
    cap_ev.back().kind = kind;
    BLWS_TRY_CUDA(this, cudaEventRecordWithFlags(cap_ev.back().e1, s, cudaEventRecordExternal));
    return BLWS_OK;
  }
  BLWS_TRY_CUDA(this, cudaEventRecord(tev[2 * tused + 1], s));
  tw[tused] = work;
  tk[tused] = kind;
  ++tused;
  twork += work;
  return BLWS_OK;
}

blws_status Ctx::trim() {
  if (sole_stream)
    BLWS_TRY_CUDA(this, cudaStreamSynchronize(sole_stream));
  else
    BLWS_TRY_CUDA(this, cudaDeviceSynchronize());
  free_graphs();
  ++gen;
  for (int b = 0; b < BUF_COUNT_; ++b) {
    if (b == BUF_SCAL || !buf[b]) continue;
    BLWS_TRY_CUDA(this, cudaFree(buf[b]));
    buf[b] = nullptr;
    cap[b] = 0;
  }
  return BLWS_OK;
}

}  // namespace blws

using blws::Ctx;

namespace {

bool dev_ptr_ok(const void* p) { return p != nullptr; }

blws_status bind_device(blws_ctx* ctx) {
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return ctx->fail(BLWS_ECUDA, "cudaSetDevice(%d): %s", ctx->device, cudaGetErrorString(e));
  return BLWS_OK;
}

// The tensor-core kernels raise SLOT_TCERR when a bounded wait gives up.  Every
// entry point that can launch one clears it first, and the ones that
// synchronise report it (BLWS_ETIMEOUT) from the slots they copy back.
blws_status clear_tc_error(blws_ctx* ctx, cudaStream_t s) {
  double* scal = nullptr;
  BLWS_TRY(ctx->get(blws::BUF_SCAL, blws::SLOT_MAX, &scal));
  BLWS_TRY_CUDA(ctx, cudaMemsetAsync(scal + blws::SLOT_TCERR, 0, sizeof(double), s));
  return BLWS_OK;
}

bool tc_error_seen(const blws_ctx* ctx) {
  return *reinterpret_cast<const int*>(ctx->host_pinned + blws::SLOT_TCERR) != 0;
}

}  // namespace

extern "C" {

blws_status blws_config_default(blws_config* cfg) {
  if (!cfg) return BLWS_EINVAL;
  cfg->k = 3;
  cfg->k_cold = 4;
  cfg->precision = BLWS_PREC_FP64;
  cfg->seed = 0x5eedull;
  cfg->device = 0;
  cfg->start = 0;
  cfg->warm = 1;
  cfg->grid_sms = 0;
  cfg->graphs = 1;
  cfg->tune = 0;
  cfg->guard = 0.0;
  return BLWS_OK;
}

blws_status blws_create(blws_ctx** out, const blws_config* cfg) {
  if (!out) return BLWS_EINVAL;
  *out = nullptr;
  blws_config c;
  blws_config_default(&c);
  if (cfg) c = *cfg;
  if (c.k < 1 || c.k_cold < 1 ||
      (c.precision != BLWS_PREC_FP64 && c.precision != BLWS_PREC_MIXED && c.precision != BLWS_PREC_FP64_TC) ||
      (c.start != 0 && c.start != 1) || (c.warm != 0 && c.warm != 1) || c.grid_sms < 0 ||
      (c.graphs != 0 && c.graphs != 1) || (c.tune != 0 && c.tune != 1) ||
      !(c.guard >= 0.0))
    return BLWS_EINVAL;
  blws_ctx* ctx = new (std::nothrow) blws_ctx();
  if (!ctx) return BLWS_ENOMEM;
  ctx->cfg = c;
  ctx->device = c.device;
  if (const char* ev = std::getenv("BLWS_EIG")) ctx->eig_route = std::strcmp(ev, "jacobi") == 0 ? 1 : 0;
  if (const char* ev = std::getenv("BLWS_TRI")) ctx->tri_route = std::strcmp(ev, "packed") == 0 ? 1 : 0;
  ctx->graphs_on = c.graphs == 1;
  if (const char* ev = std::getenv("BLWS_GRAPH")) ctx->graphs_on = ctx->graphs_on && std::strcmp(ev, "0") != 0;
  blws_status st = bind_device(ctx);
  cudaDeviceProp prop;
  if (st == BLWS_OK && cudaGetDeviceProperties(&prop, ctx->device) != cudaSuccess) st = BLWS_ECUDA;
  if (st == BLWS_OK && prop.major < 10) st = BLWS_ENOTSUP;
  if (st == BLWS_OK) {
    ctx->sms = c.grid_sms > 0 ? std::min(c.grid_sms, prop.multiProcessorCount) : prop.multiProcessorCount;
    ctx->smem_optin = prop.sharedMemPerBlockOptin;
    if (cudaMallocHost(&ctx->host_pinned, 64 * sizeof(double)) != cudaSuccess) st = BLWS_ENOMEM;
  }
  double* scal = nullptr;
  if (st == BLWS_OK) st = ctx->get(blws::BUF_SCAL, blws::SLOT_MAX, &scal);
  if (st == BLWS_OK) {
    double init[blws::SLOT_MAX] = {0};
    init[blws::SLOT_ONE] = 1.0;
    if (cudaMemcpy(scal, init, sizeof(init), cudaMemcpyHostToDevice) != cudaSuccess) st = BLWS_ECUDA;
  }
  if (st != BLWS_OK) {
    cudaGetLastError();
    blws_destroy(ctx);
    return st;
  }
  *out = ctx;
  return BLWS_OK;
}

blws_status blws_destroy(blws_ctx* ctx) {
  if (!ctx) return BLWS_OK;
  cudaSetDevice(ctx->device);
  if (ctx->gstream) cudaStreamSynchronize(ctx->gstream);
  ctx->free_graphs();
  if (ctx->gstream) cudaStreamDestroy(ctx->gstream);
  if (ctx->gfork) cudaEventDestroy(ctx->gfork);
  if (ctx->gjoin) cudaEventDestroy(ctx->gjoin);
  for (int b = 0; b < blws::BUF_COUNT_; ++b)
    if (ctx->buf[b]) cudaFree(ctx->buf[b]);
  if (ctx->host_pinned) cudaFreeHost(ctx->host_pinned);
  if (ctx->host_eig) cudaFreeHost(ctx->host_eig);
  for (size_t i = 0; i < 2 * ctx->tcap; ++i) cudaEventDestroy(ctx->tev[i]);
  delete[] ctx->tev;
  delete[] ctx->tw;
  delete[] ctx->tk;
  delete[] ctx->trec_ms;
  delete[] ctx->trec_w;
  delete[] ctx->trec_k;
  delete ctx;
  return BLWS_OK;
}

const char* blws_status_str(blws_status s) {
  switch (s) {
    case BLWS_OK: return "ok";
    case BLWS_EINVAL: return "invalid argument";
    case BLWS_ENOMEM: return "out of device memory";
    case BLWS_ECUDA: return "CUDA error";
    case BLWS_ENOCONV: return "not converged within max_iter";
    case BLWS_ENONFINITE: return "non-finite value";
    case BLWS_ETIMEOUT: return "device wait timed out";
    case BLWS_ENOTSUP: return "not supported on this device";
    default: return "unknown status";
  }
}

const char* blws_last_error(const blws_ctx* ctx) { return ctx ? ctx->last_error : ""; }

uint64_t blws_launch_count(const blws_ctx* ctx) { return ctx ? ctx->launches : 0; }

blws_status blws_graph_stats(const blws_ctx* ctx, uint64_t* captures, uint64_t* replays) {
  if (!ctx) return BLWS_EINVAL;
  if (captures) *captures = ctx->graph_captures;
  if (replays) *replays = ctx->graph_replays;
  return BLWS_OK;
}

static blws_status make_operator(blws_ctx* ctx, const blws_op* W, cudaStream_t s,
                                 blws::Operator* op) {
  const int m = W->m, n = W->n;
  op->m = m;
  op->n = n;
  if (W->W) {
    if (W->ldw < m) return ctx->fail(BLWS_EINVAL, "operator: ldw < m");
    op->W = W->W;
    op->ldw = W->ldw;
    return BLWS_OK;
  }
  if (W->nnz < 0 || !W->rowptr || (W->nnz > 0 && (!W->colidx || !W->val)))
    return ctx->fail(BLWS_EINVAL, "operator: bad CSR part");
  if (W->rl < 0 || (W->rl > 0 && (!W->Ul || !W->sl || !W->Vl)))
    return ctx->fail(BLWS_EINVAL, "operator: bad low-rank term");
  op->nnz = W->nnz;
  op->rowptr = W->rowptr;
  op->colidx = W->colidx;
  op->val = W->val;
  if (W->colptr && W->rowidx && W->perm) {  // the caller's mirror of this pattern
    op->colptr = W->colptr;
    op->rowidx = W->rowidx;
    op->perm = W->perm;
  } else {
    int *cp, *ri, *pm;
    BLWS_TRY(blws::build_csc(ctx, s, m, n, W->nnz, W->rowptr, W->colidx, &cp, &ri, &pm));
    op->colptr = cp;
    op->rowidx = ri;
    op->perm = pm;
  }
  op->rl = W->rl;
  op->Ul = W->Ul;
  op->sl = W->sl;
  op->Vl = W->Vl;
  return BLWS_OK;
}

// Mixed-precision contexts: TF32 planes of a dense W in both orientations
// (context workspace), so that products with W run on the tensor cores.
static blws_status attach_planes(blws_ctx* ctx, cudaStream_t s, blws::Operator* op,
                                 blws::TcPlanes* Wr, blws::TcPlanes* Wc, blws::OzPlanes* Or,
                                 blws::OzPlanes* Oc) {
  if (!op->W) return BLWS_OK;
  if (ctx->cfg.precision == BLWS_PREC_FP64_TC) {
    BLWS_TRY(blws::oz_alloc(ctx, op->m, op->n, Or, Oc));
    BLWS_TRY(blws::oz_planes_from_rows(ctx, s, op->W, op->ldw, op->m, op->n, *Or));
    BLWS_TRY(blws::oz_planes_from_cols(ctx, s, op->W, op->ldw, 0, op->m, op->n, *Oc));
    op->Or = Or;
    op->Oc = Oc;
    return BLWS_OK;
  }
  if (ctx->cfg.precision != BLWS_PREC_MIXED) return BLWS_OK;
  const int m = op->m, n = op->n;
  const int ldr = blws::tc_ld(n), ldc = blws::tc_ld(m);
  float* wp = nullptr;
  BLWS_TRY(ctx->get(blws::BUF_TC_W, (size_t)2 * m * ldr + (size_t)2 * n * ldc, &wp));
  *Wr = blws::TcPlanes{wp, wp + (size_t)m * ldr, m, n, ldr};
  *Wc = blws::TcPlanes{wp + (size_t)2 * m * ldr, wp + (size_t)2 * m * ldr + (size_t)n * ldc, n, m, ldc};
  BLWS_TRY(blws::tc_planes_from_rows(ctx, s, op->W, op->ldw, m, n, *Wr));
  BLWS_TRY(blws::tc_planes_from_cols(ctx, s, op->W, op->ldw, 0, m, n, *Wc));
  op->Wr = Wr;
  op->Wc = Wc;
  return BLWS_OK;
}

blws_status blws_csc_mirror(blws_ctx* ctx, int m, int n, int nnz, const int* rowptr,
                            const int* colidx, int* colptr, int* rowidx, int* perm, void* stream) {
  if (!ctx) return BLWS_EINVAL;
  if (m < 1 || n < 1 || nnz < 0 || !rowptr || !colptr || (nnz > 0 && (!colidx || !rowidx || !perm)))
    return ctx->fail(BLWS_EINVAL, "blws_csc_mirror: bad arguments");
  BLWS_TRY(bind_device(ctx));
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int *cp, *ri, *pm;
  BLWS_TRY(blws::build_csc(ctx, s, m, n, nnz, rowptr, colidx, &cp, &ri, &pm));
  BLWS_TRY_CUDA(ctx, cudaMemcpyAsync(colptr, cp, sizeof(int) * (n + 1), cudaMemcpyDeviceToDevice, s));
  if (nnz > 0) {
    BLWS_TRY_CUDA(ctx, cudaMemcpyAsync(rowidx, ri, sizeof(int) * nnz, cudaMemcpyDeviceToDevice, s));
    BLWS_TRY_CUDA(ctx, cudaMemcpyAsync(perm, pm, sizeof(int) * nnz, cudaMemcpyDeviceToDevice, s));
  }
  return BLWS_OK;
}

blws_status blws_apply(blws_ctx* ctx, const blws_op* W, const double* X, int ldx, int b,
                       double* P, int ldp, void* stream) {
  if (!ctx) return BLWS_EINVAL;
  if (!W || !X || !P) return ctx->fail(BLWS_EINVAL, "blws_apply: null argument");
  if (W->m < 1 || W->n < 1 || b < 1 || ldx < W->m + W->n || ldp < W->m + W->n)
    return ctx->fail(BLWS_EINVAL, "blws_apply: bad sizes");
  BLWS_TRY(bind_device(ctx));
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  BLWS_TRY(clear_tc_error(ctx, s));
  blws::Operator op;
  BLWS_TRY(make_operator(ctx, W, s, &op));
  BLWS_TRY(blws::blws_reserve(ctx, W->m, W->n, b, 1));
  blws::TcPlanes Wr, Wc;
  blws::OzPlanes Or, Oc;
  BLWS_TRY(attach_planes(ctx, s, &op, &Wr, &Wc, &Or, &Oc));
  return blws::apply_op(ctx, s, op, X, ldx, b, P, ldp);
}

blws_status blws_svt(blws_ctx* ctx, const blws_op* W, double eps, int r, const double* U0,
                     const double* V0, int w, const double* G, int g, double* U, double* V,
                     double* sigma, int* count, void* stream) {
  if (!ctx) return BLWS_EINVAL;
  if (!W || !U || !V || !sigma || !count) return ctx->fail(BLWS_EINVAL, "blws_svt: null argument");
  const int m = W->m, n = W->n;
  if (m < 1 || n < 1) return ctx->fail(BLWS_EINVAL, "blws_svt: empty operator %d x %d", m, n);
  if (!(eps > 0.0) || r < 1 || r > std::min(m, n) || w < 0 || g < 0)
    return ctx->fail(BLWS_EINVAL, "blws_svt: need eps > 0, 1 <= r <= min(m, n), w, g >= 0");
  if (w > 0 && (!dev_ptr_ok(U0) || !dev_ptr_ok(V0)))
    return ctx->fail(BLWS_EINVAL, "blws_svt: warm start pointers missing");
  if (g > 0 && !G) return ctx->fail(BLWS_EINVAL, "blws_svt: g > 0 but G is NULL");
  BLWS_TRY(bind_device(ctx));
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  blws::Operator op;
  BLWS_TRY(make_operator(ctx, W, s, &op));
  blws::BlwsArgs a;
  a.eps = eps;
  a.r = r;
  a.U0 = U0;
  a.ldu0 = m;
  a.V0 = V0;
  a.ldv0 = n;
  a.w = w;
  a.G = g > 0 ? G : nullptr;
  a.ldg = m + n;
  a.g = g;
  a.cold = (w == 0);
  a.standard = ctx->cfg.start == 1;
  a.k = a.cold ? ctx->cfg.k_cold : ctx->cfg.k;
  BLWS_TRY(clear_tc_error(ctx, s));
  blws::TcPlanes Wr, Wc;
  blws::OzPlanes Or, Oc;
  BLWS_TRY(attach_planes(ctx, s, &op, &Wr, &Wc, &Or, &Oc));
  a.mixed = ctx->cfg.precision == BLWS_PREC_MIXED;
  double* scal;
  BLWS_TRY(ctx->get(blws::BUF_SCAL, blws::SLOT_MAX, &scal));
  int* cdev = reinterpret_cast<int*>(scal + blws::SLOT_COUNT);
  BLWS_TRY(blws::blws_run(ctx, s, op, a, U, m, V, n, sigma, cdev));
  BLWS_TRY_CUDA(ctx, cudaMemcpyAsync(ctx->host_pinned, scal, sizeof(double) * blws::SLOT_MAX,
                                     cudaMemcpyDeviceToHost, s));
  BLWS_TRY_CUDA(ctx, cudaStreamSynchronize(s));
  *count = *reinterpret_cast<int*>(ctx->host_pinned + blws::SLOT_COUNT);
  if (tc_error_seen(ctx)) return ctx->fail(BLWS_ETIMEOUT, "blws_svt: a tensor-core wait ran out");
  return BLWS_OK;
}

blws_status blws_evd(blws_ctx* ctx, const double* W, int m, int ldw, double eps, int r,
                     const double* U0, int w, const double* G, int g, double* U, double* lam,
                     int* count, void* stream) {
  if (!ctx) return BLWS_EINVAL;
  if (!W || !U || !lam || !count) return ctx->fail(BLWS_EINVAL, "blws_evd: null argument");
  if (m < 1 || ldw < m) return ctx->fail(BLWS_EINVAL, "blws_evd: need m >= 1, ldw >= m (m=%d ldw=%d)", m, ldw);
  if (!std::isfinite(eps) || r < 1 || r > m || w < 0 || g < 0)
    return ctx->fail(BLWS_EINVAL, "blws_evd: need finite eps, 1 <= r <= m, w, g >= 0");
  if (w > 0 && !dev_ptr_ok(U0)) return ctx->fail(BLWS_EINVAL, "blws_evd: warm start pointer missing");
  if (g > 0 && !G) return ctx->fail(BLWS_EINVAL, "blws_evd: g > 0 but G is NULL");
  BLWS_TRY(bind_device(ctx));
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  blws::Operator op;
  op.m = op.n = m;
  op.sym = true;
  op.W = W;
  op.ldw = ldw;
  blws::BlwsArgs a;
  a.eps = eps;
  a.r = r;
  a.U0 = U0;
  a.ldu0 = m;
  a.w = w;
  a.G = g > 0 ? G : nullptr;
  a.ldg = m;
  a.g = g;
  a.cold = (w == 0);
  a.k = a.cold ? ctx->cfg.k_cold : ctx->cfg.k;
  a.mixed = ctx->cfg.precision == BLWS_PREC_MIXED;
  double* scal;
  BLWS_TRY(ctx->get(blws::BUF_SCAL, blws::SLOT_MAX, &scal));
  int* cdev = reinterpret_cast<int*>(scal + blws::SLOT_COUNT);
  BLWS_TRY(clear_tc_error(ctx, s));
  BLWS_TRY(blws::blws_run(ctx, s, op, a, U, m, nullptr, 0, lam, cdev));
  BLWS_TRY_CUDA(ctx, cudaMemcpyAsync(ctx->host_pinned, scal, sizeof(double) * blws::SLOT_MAX,
                                     cudaMemcpyDeviceToHost, s));
  BLWS_TRY_CUDA(ctx, cudaStreamSynchronize(s));
  *count = *reinterpret_cast<int*>(ctx->host_pinned + blws::SLOT_COUNT);
  if (tc_error_seen(ctx)) return ctx->fail(BLWS_ETIMEOUT, "blws_evd: a tensor-core wait ran out");
  return BLWS_OK;
}

blws_status rpca_params_default(rpca_params* p) {
  if (!p) return BLWS_EINVAL;
  p->lambda = 0.0;
  p->tol = 1e-7;
  p->max_iter = 1000;
  p->rho = 1.5;
  p->mu0 = 0.0;
  p->mu_bar_ratio = 1e7;
  p->sv0 = 10;
  p->trace = nullptr;
  p->trace_len = 0;
  p->mixed_tol = 1e-5;
  return BLWS_OK;
}

blws_status rpca_solve(blws_ctx* ctx, const double* D, int m, int n, int ld, const rpca_params* p,
                       double* A, double* E, rpca_info* info, void* stream) {
  if (!ctx) return BLWS_EINVAL;
  if (!D || !A || !E || !info) return ctx->fail(BLWS_EINVAL, "rpca_solve: null argument");
  if (m < 1 || n < 1 || ld < m) return ctx->fail(BLWS_EINVAL, "rpca_solve: bad size %d x %d ld %d", m, n, ld);
  rpca_params q;
  rpca_params_default(&q);
  if (p) q = *p;
  if (!(q.tol > 0) || q.max_iter < 1 || !(q.rho >= 1.0) || q.sv0 < 1 || !(q.mu_bar_ratio >= 1.0) ||
      !(q.mixed_tol >= 0.0))
    return ctx->fail(BLWS_EINVAL, "rpca_solve: bad parameters");
  BLWS_TRY(bind_device(ctx));
  return blws::rpca_run(ctx, reinterpret_cast<cudaStream_t>(stream), D, m, n, ld, q, A, E, info);
}

blws_status mc_params_default(mc_params* p) {
  if (!p) return BLWS_EINVAL;
  p->variant = 0;
  p->tau = 0.0;
  p->delta = 0.0;
  p->tol = 1e-4;
  p->max_iter = 500;
  p->incr = 5;
  p->eta = 0.25;
  p->tau_min_rel = 1e-4;
  p->xtol = 1e-3;
  return BLWS_OK;
}

blws_status mc_solve(blws_ctx* ctx, int m, int n, int nnz, const int* rowptr, const int* colidx,
                     const double* vals, const mc_params* p, int max_rank, double* U,
                     double* theta, double* V, mc_info* info, void* stream) {
  if (!ctx) return BLWS_EINVAL;
  if (!rowptr || !U || !theta || !V || !info || (nnz > 0 && (!colidx || !vals)))
    return ctx->fail(BLWS_EINVAL, "mc_solve: null argument");
  if (m < 1 || n < 1 || nnz < 0 || (long long)nnz > (long long)m * n || max_rank < 1)
    return ctx->fail(BLWS_EINVAL, "mc_solve: bad sizes");
  mc_params q;
  mc_params_default(&q);
  if (p) q = *p;
  if ((q.variant != 0 && q.variant != 1) || !(q.tol > 0) || q.max_iter < 1)
    return ctx->fail(BLWS_EINVAL, "mc_solve: bad parameters");
  if (q.variant == 1 && !(q.eta > 0 && q.eta < 1)) return ctx->fail(BLWS_EINVAL, "mc_solve: eta");
  BLWS_TRY(bind_device(ctx));
  return blws::mc_run(ctx, reinterpret_cast<cudaStream_t>(stream), m, n, nnz, rowptr, colidx, vals,
                      q, max_rank, U, theta, V, info);
}

blws_status blws_gemm(blws_ctx* ctx, int ta, int tb, int M, int N, int K, double alpha,
                      const double* A, int lda, const double* B, int ldb, double beta, double* C,
                      int ldc, int sym, void* stream) {
  if (!ctx) return BLWS_EINVAL;
  if (!A || !B || !C) return ctx->fail(BLWS_EINVAL, "blws_gemm: null argument");
  if (M < 1 || N < 1 || K < 1 || lda < (ta ? K : M) || ldb < (tb ? N : K) || ldc < M ||
      !std::isfinite(alpha) || !std::isfinite(beta))
    return ctx->fail(BLWS_EINVAL, "blws_gemm: bad sizes or scalars");
  if (sym && (M != N || beta != 0.0))
    return ctx->fail(BLWS_EINVAL, "blws_gemm: a symmetric result needs M == N and beta == 0");
  BLWS_TRY(bind_device(ctx));
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  BLWS_TRY(clear_tc_error(ctx, s));
  const bool f32 = ctx->cfg.precision == BLWS_PREC_MIXED;
  if (sym)
    BLWS_TRY(blws::gemm_sym(ctx, s, ta != 0, tb != 0, N, K, alpha, A, lda, B, ldb, C, ldc, f32));
  else
    BLWS_TRY(blws::gemm(ctx, s, ta != 0, tb != 0, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, f32));
  double* scal;
  BLWS_TRY(ctx->get(blws::BUF_SCAL, blws::SLOT_MAX, &scal));
  BLWS_TRY_CUDA(ctx, cudaMemcpyAsync(ctx->host_pinned, scal, sizeof(double) * blws::SLOT_MAX,
                                     cudaMemcpyDeviceToHost, s));
  BLWS_TRY_CUDA(ctx, cudaStreamSynchronize(s));
  if (tc_error_seen(ctx)) return ctx->fail(BLWS_ETIMEOUT, "blws_gemm: a tensor-core wait ran out");
  return BLWS_OK;
}

blws_status blws_timing_start(blws_ctx* ctx) {
  if (!ctx) return BLWS_EINVAL;
  ctx->timing = true;
  ctx->tused = 0;
  ctx->twork = 0.0;
  ctx->pending_ev.clear();
  ctx->graph_ms.clear();
  ctx->graph_w.clear();
  ctx->graph_kind.clear();
  return BLWS_OK;
}

blws_status blws_timing_stop(blws_ctx* ctx, double* ms, uint64_t* launches, double* work) {
  if (!ctx || !ms || !launches || !work) return BLWS_EINVAL;
  ctx->timing = false;
  BLWS_TRY(bind_device(ctx));
  BLWS_TRY(blws::graph_harvest(ctx));  // products timed inside replayed graphs
  const size_t ng = ctx->graph_ms.size();
  double total = 0.0;
  delete[] ctx->trec_ms;
  delete[] ctx->trec_w;
  delete[] ctx->trec_k;
  ctx->trec_ms = new (std::nothrow) double[ctx->tused + ng + 1];
  ctx->trec_w = new (std::nothrow) double[ctx->tused + ng + 1];
  ctx->trec_k = new (std::nothrow) int[ctx->tused + ng + 1];
  ctx->trec_n = 0;
  if (!ctx->trec_ms || !ctx->trec_w || !ctx->trec_k) return ctx->fail(BLWS_ENOMEM, "timing records");
  for (size_t i = 0; i < ctx->tused; ++i) {
    BLWS_TRY_CUDA(ctx, cudaEventSynchronize(ctx->tev[2 * i + 1]));
    float t = 0.0f;
    BLWS_TRY_CUDA(ctx, cudaEventElapsedTime(&t, ctx->tev[2 * i], ctx->tev[2 * i + 1]));
    total += t;
    ctx->trec_ms[i] = t;
    ctx->trec_w[i] = ctx->tw[i];
    ctx->trec_k[i] = ctx->tk[i];
  }
  double gwork = 0.0;
  for (size_t i = 0; i < ng; ++i) {
    total += ctx->graph_ms[i];
    gwork += ctx->graph_w[i];
    ctx->trec_ms[ctx->tused + i] = ctx->graph_ms[i];
    ctx->trec_w[ctx->tused + i] = ctx->graph_w[i];
    ctx->trec_k[ctx->tused + i] = ctx->graph_kind[i];
  }
  ctx->trec_n = ctx->tused + ng;
  *ms = total;
  *launches = ctx->tused + ng;
  *work = ctx->twork + gwork;
  ctx->tused = 0;
  ctx->twork = 0.0;
  ctx->graph_ms.clear();
  ctx->graph_w.clear();
  ctx->graph_kind.clear();
  return BLWS_OK;
}

size_t blws_timing_records(const blws_ctx* ctx, size_t cap, double* ms, double* work, int* kind) {
  if (!ctx) return 0;
  const size_t k = std::min(cap, ctx->trec_n);
  for (size_t i = 0; i < k; ++i) {
    if (ms) ms[i] = ctx->trec_ms[i];
    if (work) work[i] = ctx->trec_w[i];
    if (kind) kind[i] = ctx->trec_k[i];
  }
  return ctx->trec_n;
}

blws_status blws_wait_probe(blws_ctx* ctx, unsigned polls, void* stream) {
  if (!ctx) return BLWS_EINVAL;
  if (polls < 1 || polls > (1u << 16)) return ctx->fail(BLWS_EINVAL, "blws_wait_probe: polls in [1, 65536]");
  BLWS_TRY(bind_device(ctx));
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  BLWS_TRY(clear_tc_error(ctx, s));
  BLWS_TRY(blws::wait_probe(ctx, s, polls));
  double* scal;
  BLWS_TRY(ctx->get(blws::BUF_SCAL, blws::SLOT_MAX, &scal));
  BLWS_TRY_CUDA(ctx, cudaMemcpyAsync(ctx->host_pinned, scal, sizeof(double) * blws::SLOT_MAX,
                                     cudaMemcpyDeviceToHost, s));
  BLWS_TRY_CUDA(ctx, cudaStreamSynchronize(s));
  if (tc_error_seen(ctx)) return ctx->fail(BLWS_ETIMEOUT, "blws_wait_probe: the wait gave up after %u polls", polls);
  return BLWS_OK;
}

}  // extern "C"
