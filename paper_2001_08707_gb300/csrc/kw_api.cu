// C ABI and host driver of the shifted COCG solver (see include/komega_gb300.h).
//
// The driver validates arguments, sizes the device workspace (kept across
// calls), uploads the shifts and the initial state, enqueues the iteration
// kernels in chunks and polls the device stop flag one chunk behind, so the
// GPU always has the next chunk queued.  Iterations enqueued after the stop
// flag is set return at their first instruction.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "komega_gb300.h"
#include "kw_arith.cuh"
#include "kw_internal.cuh"

namespace {

// Bytes of a complex vector element and of a real projection-row element.
size_t vec_bytes(kw_precision p) { return p == KW_C32V_F64S ? 8 : 16; }
size_t real_bytes(kw_precision p) { return p == KW_C32V_F64S ? 4 : 8; }
int prec_id(kw_precision p) { return p == KW_C32V_F64S ? kw::PREC_C32 : p == KW_DF64 ? kw::PREC_DF : kw::PREC_F64; }

// FP32-pair image of a complex FP64 scalar, computed on the host.
float4 host_pair(double re, double im) {
  const float rh = (float)re, ih = (float)im;
  return make_float4(rh, (float)(re - (double)rh), ih, (float)(im - (double)ih));
}

// Device buffer that only grows.
struct DBuf {
  void* p = nullptr;
  size_t cap = 0;
  cudaError_t ensure(size_t bytes) {
    if (bytes <= cap) return cudaSuccess;
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e == cudaSuccess) cap = bytes;
    return e;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
  }
};

// Events destroyed when the holder goes out of scope (every return path).
struct ScopedEvents {
  std::vector<cudaEvent_t> ev;
  cudaError_t create(size_t n, unsigned flags) {
    ev.assign(n, nullptr);
    for (auto& e : ev) {
      cudaError_t r = cudaEventCreateWithFlags(&e, flags);
      if (r != cudaSuccess) {
        e = nullptr;
        return r;
      }
    }
    return cudaSuccess;
  }
  cudaEvent_t operator[](size_t i) const { return ev[i]; }
  ~ScopedEvents() {
    for (cudaEvent_t e : ev)
      if (e) cudaEventDestroy(e);
  }
};

}  // namespace

struct kw_ctx {
  kw_options opt;
  std::string tune_cache;   // copy of opt.tune_cache (opt.tune_cache points here)
  cudaStream_t stream = nullptr;
  int device = 0;
  int num_sms = 0;
  char err[512];
  // operator
  int64_t m = 0, nnz = 0;
  const int64_t* rowptr = nullptr;
  const int32_t* col = nullptr;
  const double* val = nullptr;
  // operator generated on the fly (kw_set_spin_operator, kw_set_lattice3d)
  int op = kw::OP_CSR;
  DBuf sp_binom, sp_basis, sp_bond, sp_J, sp_h, sp_val, sp_table;
  int sp_nbond = 0, sp_uniform = 0;
  bool sp_table_on = false, sp_table_built = false;
  int lx = 0, ly = 0, lz = 0;
  DBuf g_diag64, g_diag32, g_diagpair;   // diagonal (spin) or on-site energies (lattice)
  int g_kind = 0;                        // storage read by the form (kw::Work::u_kind)
  double g_v = 0.0;                      // uniform off-diagonal value (J/2 or the hopping)
  // operator as a caller's callback (kw_set_matvec); the FP32-pair form hands it kw_c128 copies
  kw_matvec_fn mv_fn = nullptr;
  void* mv_user = nullptr;
  kw_matvec_fn mv_fn_adj = nullptr;   // adjoint product for BiCG (NULL: Hermitian)
  void* mv_user_adj = nullptr;
  DBuf mv_r, mv_q, mv_r2, mv_q2;
  // reverse communication (kw_rci_*)
  bool rci_active = false;
  int64_t rci_iter = 0;
  // solver of Table 1 (kw_set_method) and the BiCG shadow vectors
  int method = KW_METHOD_COCG;
  const double* btilde = nullptr;
  DBuf rtA, rtB, qt;
  DBuf val32;
  DBuf valpair;               // FP32-pair copy of the values (KW_DF64, values not exact in FP32)
  DBuf inexact;
  bool val32_exact = false;   // every value representable in FP32
  DBuf tune_fp;               // fingerprint samples for the persistent tuning cache
  int64_t tune_runs = 0, tune_hits = 0;   // timing runs of the tuner; picks taken from the cache
  int spmv_lanes = 0;         // tuned or forced lanes per row (0 = tune at first use)
  int spmv_val_f32 = 0;       // tuned or forced: FP32 value array in FP64 mode
  int force_lanes = 0, force_val = -1;
  // SELL-32 copy of the operator (built when the tuner tries it or it is forced)
  DBuf sell_perm, sell_len, sell_slen, sell_ptr, sell_col, sell_val;
  bool sell_built = false;
  // uniform off-diagonal copy (built when the tuner tries it or it is forced)
  int u_state = 0;            // 0: not examined, 1: built, -1: off-diagonal values differ
  DBuf u_sptr, u_scol;        // SELL-32 copy of the uniform layout
  int us_state = 0;           // 0: not built, 1: built, -1: not applicable
  double u_v = 0.0;
  int u_kind = 0;             // diagonal/value storage for the context's form (kw::Work::u_kind)
  DBuf u_fm, u_dcount, u_scratch, u_rowptr, u_col, u_diag64, u_diag32, u_diagpair;
  // host-solve copies
  DBuf h_rowptr, h_col, h_val, h_b, h_left, h_x;
  // workspace
  DBuf bil_part, bil_out;     // kw_bilinear scratch and result
  DBuf bil_diag, bil_flag;    // kw_bilinear: the terms' diagonals [nterm][m] and diagonal-only flags
  DBuf rA, rB, q, proj_rows, z, pi1, pi0, active, conv_iter, final_res, coef, coef_pair, Y, U, w, w0, hist, list,
      X, P, part, st, projx, tdot;
  kw::State* st_host = nullptr;   // pinned
  int* flags_host = nullptr;      // pinned, two slots
  cudaEvent_t ev[2] = {nullptr, nullptr};
  // kernel timing: one sampled iteration per chunk, two chunks in flight
  int64_t timing_every = 0;
  cudaEvent_t kev[2][6] = {};
  // second stream of a solve (shift scalars and x/p update) and its ordering events
  cudaStream_t stream2 = nullptr, stream3 = nullptr;
  cudaEvent_t ev_k2 = nullptr, ev_k3 = nullptr, ev_k4[2] = {nullptr, nullptr};
  DBuf part_k1;   // K1's block partials (K1 overlaps K3, which uses part)
  int overlap = 1;
  int bulk = -1;  // kw_set_bulk_copy (-1: auto)
  int xp32 = 0;   // kw_set_shift_storage: full-mode x/p as complex FP32
  int seed_rg = -1;  // kw_set_seed_update: K2 row-group form (-1 auto)
  int force_xp_tile = 0;      // kw_set_update_tile: 0 = timed, else 4, 8 or 16 shifts per K4 tile
  int xp_tile_pick = 0;       // the timed pick and what it was timed on
  long long xp_key[4] = {-1, -1, -1, -1};
  int last_xp_tile = 0;       // the tile of the last full-mode solve
  DBuf xp_st;                 // scratch state of the K4 timing
  DBuf comb_w;                // weights of kw_shift_combine
  kw_stats stats = {};
  // phases of a solve
  kw::Work work;
  int64_t work_K = 0;
  // batched solves: one child context (own stream) per instance
  std::vector<kw_ctx*> children;
  cudaStream_t batch_stream = nullptr;   // capturable stream of kw_solve_batched
  bool owns_stream = false;
  DBuf child_states, done_count;
  int* done_host = nullptr;   // pinned
  // device-side iteration loop (opt.use_graph): a graph whose WHILE node runs
  // chunks of iterations until the stop flag is raised; kept while the
  // descriptor it was captured from is unchanged
  cudaStream_t cap_stream = nullptr;   // capture stream (the caller's may be the legacy stream)
  DBuf loop;                           // device [trips, trip cap]
  unsigned* loop_host = nullptr;       // pinned [2]
  cudaGraph_t loop_graph = nullptr;
  cudaGraphExec_t loop_exec = nullptr;
  kw::Work loop_work;                  // descriptor of the captured iterations
  int loop_parity = -1, loop_chunk = 0;
  int64_t loop_launches = 0;           // kernel launches per trip
  // last solve
  bool resumable = false;     // the last kw_solve stopped at maxiter and its workspace is intact
  int64_t run_maxiter = 0;    // iteration cap of the running solve
  int64_t last_K = 0;
  int64_t last_nrec = 0;
  // Krylov log (kw_set_krylov_log) and the last solve's record of it
  int64_t log_max = 0;
  DBuf klog;
  int64_t last_log_rows = -1;   // -1: the last solve recorded no log
  int64_t last_run = 0;
  int last_log_np = 0;
  double last_thresh = 0.0;
  // kw_recalc buffers
  DBuf rc_log, rc_w0, rc_z, rc_proj, rc_conv, rc_res, rc_flag;
};

static kw_status fail(kw_ctx* c, kw_status s, const char* fmt, ...) {
  if (c) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(c->err, sizeof(c->err), fmt, ap);
    va_end(ap);
  }
  return s;
}

static kw_status cuda_fail(kw_ctx* c, cudaError_t e, const char* where) {
  if (e == cudaErrorMemoryAllocation) return fail(c, KW_ERR_OOM, "%s: %s", where, cudaGetErrorString(e));
  return fail(c, KW_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

#define KW_CUDA(call, where)                          \
  do {                                                \
    cudaError_t e_ = (call);                          \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, where); \
  } while (0)

extern "C" {

int kw_abi_version(void) { return KW_ABI_VERSION; }

void kw_default_options(kw_options* opt) {
  if (!opt) return;
  opt->prec = KW_F64;
  opt->tol = 1e-10;
  opt->maxiter = 100000;
  opt->seed_switch = 1;
  opt->hist_stride = 0;
  opt->hist_max = 0;
  opt->use_graph = 1;
  opt->tune_cache = nullptr;
}

const char* kw_status_string(kw_status s) {
  switch (s) {
    case KW_OK: return "KW_OK";
    case KW_ERR_ARG: return "KW_ERR_ARG";
    case KW_ERR_CUDA: return "KW_ERR_CUDA";
    case KW_ERR_OOM: return "KW_ERR_OOM";
    case KW_ERR_BREAKDOWN: return "KW_ERR_BREAKDOWN";
    case KW_ERR_NONFINITE: return "KW_ERR_NONFINITE";
    case KW_ERR_CALLBACK: return "KW_ERR_CALLBACK";
    case KW_ERR_TIMEOUT: return "KW_ERR_TIMEOUT";
    case KW_NOT_CONVERGED: return "KW_NOT_CONVERGED";
  }
  return "KW_UNKNOWN";
}

kw_status kw_create(kw_ctx** out, const kw_options* opt, void* cuda_stream) {
  if (!out || !opt) return KW_ERR_ARG;
  *out = nullptr;
  if (!(opt->tol >= 0.0) || opt->maxiter < 1 || opt->hist_stride < 0 || opt->hist_max < 0 ||
      (opt->prec != KW_F64 && opt->prec != KW_C32V_F64S && opt->prec != KW_DF64))
    return KW_ERR_ARG;
  kw_ctx* ctx = new kw_ctx();
  ctx->opt = *opt;
  if (opt->tune_cache) ctx->tune_cache = opt->tune_cache;
  ctx->opt.tune_cache = ctx->tune_cache.c_str();
  ctx->stream = (cudaStream_t)cuda_stream;
  ctx->err[0] = 0;
  cudaError_t e = cudaGetDevice(&ctx->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, ctx->device);
  if (e == cudaSuccess) e = cudaMallocHost((void**)&ctx->st_host, sizeof(kw::State));
  if (e == cudaSuccess) e = cudaMallocHost((void**)&ctx->flags_host, 2 * sizeof(int));
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->ev[0], cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->ev[1], cudaEventDisableTiming);
  if (e != cudaSuccess) {
    kw_destroy(ctx);
    return KW_ERR_CUDA;
  }
  *out = ctx;
  return KW_OK;
}

void kw_destroy(kw_ctx* ctx) {
  if (!ctx) return;
  cudaStreamSynchronize(ctx->stream);   // the caller's stream (possibly the legacy one) may hold our work
  DBuf* bufs[] = {&ctx->bil_part, &ctx->bil_out, &ctx->bil_diag, &ctx->bil_flag, &ctx->val32, &ctx->valpair, &ctx->coef_pair, &ctx->inexact, &ctx->sell_perm, &ctx->sell_len,
                  &ctx->sell_slen, &ctx->sell_ptr, &ctx->sell_col, &ctx->sell_val, &ctx->h_rowptr, &ctx->h_col, &ctx->h_val, &ctx->h_b, &ctx->h_left, &ctx->h_x,
                  &ctx->rA, &ctx->rB, &ctx->q, &ctx->proj_rows, &ctx->z, &ctx->pi1, &ctx->pi0, &ctx->active,
                  &ctx->conv_iter, &ctx->final_res, &ctx->coef, &ctx->Y, &ctx->U, &ctx->w, &ctx->w0,
                  &ctx->hist, &ctx->list, &ctx->X, &ctx->P, &ctx->part, &ctx->part_k1, &ctx->st, &ctx->projx, &ctx->tdot,
                  &ctx->mv_r, &ctx->mv_q, &ctx->mv_r2, &ctx->mv_q2, &ctx->rtA, &ctx->rtB, &ctx->qt, &ctx->sp_binom, &ctx->sp_basis, &ctx->sp_bond, &ctx->sp_J,
                  &ctx->sp_h, &ctx->sp_val, &ctx->sp_table, &ctx->g_diag64, &ctx->g_diag32, &ctx->g_diagpair, &ctx->u_fm, &ctx->u_dcount, &ctx->u_scratch, &ctx->u_rowptr,
                  &ctx->u_col, &ctx->u_sptr, &ctx->u_scol, &ctx->u_diag64, &ctx->u_diag32, &ctx->u_diagpair, &ctx->klog, &ctx->rc_log, &ctx->rc_w0, &ctx->rc_z, &ctx->rc_proj, &ctx->rc_conv, &ctx->rc_res,
                  &ctx->rc_flag, &ctx->tune_fp, &ctx->xp_st, &ctx->comb_w};
  for (DBuf* b : bufs) b->release();
  for (kw_ctx* c : ctx->children) kw_destroy(c);
  if (ctx->batch_stream) cudaStreamDestroy(ctx->batch_stream);
  ctx->child_states.release();
  ctx->done_count.release();
  ctx->loop.release();
  if (ctx->loop_exec) cudaGraphExecDestroy(ctx->loop_exec);
  if (ctx->loop_graph) cudaGraphDestroy(ctx->loop_graph);
  if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
  if (ctx->loop_host) cudaFreeHost(ctx->loop_host);
  if (ctx->done_host) cudaFreeHost(ctx->done_host);
  if (ctx->owns_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
  if (ctx->st_host) cudaFreeHost(ctx->st_host);
  if (ctx->flags_host) cudaFreeHost(ctx->flags_host);
  for (int i = 0; i < 2; ++i) {
    if (ctx->ev[i]) cudaEventDestroy(ctx->ev[i]);
    for (int j = 0; j < 6; ++j)
      if (ctx->kev[i][j]) cudaEventDestroy(ctx->kev[i][j]);
  }
  if (ctx->ev_k2) cudaEventDestroy(ctx->ev_k2);
  if (ctx->ev_k3) cudaEventDestroy(ctx->ev_k3);
  for (cudaEvent_t e : ctx->ev_k4)
    if (e) cudaEventDestroy(e);
  if (ctx->stream2) cudaStreamDestroy(ctx->stream2);
  if (ctx->stream3) cudaStreamDestroy(ctx->stream3);
  delete ctx;
}

kw_status kw_last_error(const kw_ctx* ctx, char* buf, size_t n) {
  if (!ctx || !buf || n == 0) return KW_ERR_ARG;
  snprintf(buf, n, "%s", ctx->err);
  return KW_OK;
}

kw_status kw_set_csr(kw_ctx* ctx, int64_t m, int64_t nnz, const int64_t* rowptr_dev, const int32_t* col_dev,
                     const double* val_dev) {
  if (!ctx) return KW_ERR_ARG;
  if (m < 1 || m > KW_MAX_ROWS || nnz < 0 || nnz > KW_MAX_NNZ || !rowptr_dev ||
      (nnz > 0 && (!col_dev || !val_dev)))
    return fail(ctx, KW_ERR_ARG, "kw_set_csr: need 1 <= m <= KW_MAX_ROWS, 0 <= nnz <= KW_MAX_NNZ and non-NULL arrays");
  ctx->mv_fn = nullptr;
  ctx->mv_user = nullptr;
  ctx->mv_fn_adj = nullptr;
  ctx->mv_user_adj = nullptr;
  ctx->op = kw::OP_CSR;
  ctx->resumable = false;
  ctx->m = m;
  ctx->nnz = nnz;
  ctx->rowptr = rowptr_dev;
  ctx->col = col_dev;
  ctx->val = val_dev;
  ctx->val32_exact = false;
  ctx->spmv_lanes = 0;   // re-tune for the new operator
  ctx->sell_built = false;
  ctx->u_state = 0;
  ctx->us_state = 0;
  if (nnz > 0) {
    KW_CUDA(ctx->val32.ensure((size_t)nnz * sizeof(float)), "kw_set_csr: FP32 value copy");
    KW_CUDA(ctx->inexact.ensure(sizeof(unsigned long long)), "kw_set_csr: counter");
    KW_CUDA(cudaMemsetAsync(ctx->inexact.p, 0, sizeof(unsigned long long), ctx->stream), "kw_set_csr: memset");
    KW_CUDA(kw::launch_convert_f64_to_f32(val_dev, (float*)ctx->val32.p, nnz, (unsigned long long*)ctx->inexact.p,
                                          ctx->stream), "kw_set_csr: convert");
    unsigned long long bad = 0;
    KW_CUDA(cudaMemcpyAsync(&bad, ctx->inexact.p, sizeof(bad), cudaMemcpyDeviceToHost, ctx->stream), "kw_set_csr: read");
    KW_CUDA(cudaStreamSynchronize(ctx->stream), "kw_set_csr: sync");
    ctx->val32_exact = bad == 0;
    if (ctx->opt.prec == KW_DF64 && !ctx->val32_exact) {
      KW_CUDA(ctx->valpair.ensure((size_t)nnz * 8), "kw_set_csr: FP32-pair value copy");
      KW_CUDA(kw::launch_convert_f64_to_pair(val_dev, ctx->valpair.p, nnz, ctx->stream), "kw_set_csr: convert");
    }
  }
  return KW_OK;
}

// Storage of a generated operator's diagonal for the context's form: FP32 when
// it and the off-diagonal values are exact in FP32 (always in the FP32 form),
// else FP64 (FP64 form) or FP32 pairs (pair form).  offdiag_exact32: the
// off-diagonal values are exact in FP32.
static kw_status generated_diag(kw_ctx* ctx, int64_t m, bool offdiag_exact32) {
  KW_CUDA(ctx->g_diag32.ensure((size_t)m * 4), "operator allocation");
  KW_CUDA(ctx->inexact.ensure(sizeof(unsigned long long)), "operator allocation");
  KW_CUDA(cudaMemsetAsync(ctx->inexact.p, 0, sizeof(unsigned long long), ctx->stream), "operator memset");
  KW_CUDA(kw::launch_convert_f64_to_f32((const double*)ctx->g_diag64.p, (float*)ctx->g_diag32.p, m,
                                        (unsigned long long*)ctx->inexact.p, ctx->stream), "operator convert");
  unsigned long long bad = 0;
  KW_CUDA(cudaMemcpyAsync(&bad, ctx->inexact.p, sizeof(bad), cudaMemcpyDeviceToHost, ctx->stream), "operator read");
  KW_CUDA(cudaStreamSynchronize(ctx->stream), "operator sync");
  const kw_precision p = ctx->opt.prec;
  if (p == KW_C32V_F64S || (bad == 0 && offdiag_exact32)) {
    ctx->g_kind = 1;
  } else if (p == KW_DF64) {
    ctx->g_kind = 2;
    KW_CUDA(ctx->g_diagpair.ensure((size_t)m * 8), "operator allocation");
    KW_CUDA(kw::launch_convert_f64_to_pair((const double*)ctx->g_diag64.p, ctx->g_diagpair.p, m, ctx->stream),
            "operator convert");
  } else {
    ctx->g_kind = 0;
  }
  return KW_OK;
}

// The context's operator becomes a generated one: forget the CSR and callback.
static void become_generated(kw_ctx* ctx, int op, int64_t m) {
  ctx->op = op;
  ctx->resumable = false;
  ctx->m = m;
  ctx->nnz = 0;
  ctx->rowptr = nullptr;
  ctx->col = nullptr;
  ctx->val = nullptr;
  ctx->mv_fn = nullptr;
  ctx->mv_user = nullptr;
  ctx->mv_fn_adj = nullptr;
  ctx->mv_user_adj = nullptr;
  ctx->val32_exact = false;
  ctx->spmv_lanes = 1;
  ctx->spmv_val_f32 = 0;
  ctx->sell_built = false;
  ctx->u_state = 0;
  ctx->us_state = 0;
}

kw_status kw_set_spin_operator(kw_ctx* ctx, int nsite, int nup, int nbond, const int32_t* bonds_host,
                               const double* J_host, const double* h_host) {
  if (!ctx) return KW_ERR_ARG;
  if (nsite < 2 || nsite > KW_SPIN_MAX_SITES || nup < 1 || nup >= nsite || nbond < 1 || nbond > KW_SPIN_MAX_BONDS ||
      !bonds_host || !J_host)
    return fail(ctx, KW_ERR_ARG, "kw_set_spin_operator: need 1 <= nup < nsite <= %d, 1 <= nbond <= %d, bonds, J",
                KW_SPIN_MAX_SITES, KW_SPIN_MAX_BONDS);
  double M = 1.0;
  for (int k = 0; k < nup; ++k) M = M * (nsite - k) / (k + 1);
  if (M > (double)KW_MAX_ROWS) return fail(ctx, KW_ERR_ARG, "kw_set_spin_operator: C(nsite, nup) > KW_MAX_ROWS");
  const int64_t m = (int64_t)(M + 0.5);
  std::vector<int> bond(nbond);
  bool uniform = true, exact32 = true;
  for (int b = 0; b < nbond; ++b) {
    const int i = bonds_host[2 * b], j = bonds_host[2 * b + 1];
    if (i < 0 || j < 0 || i >= nsite || j >= nsite || i == j || !isfinite(J_host[b]))
      return fail(ctx, KW_ERR_ARG, "kw_set_spin_operator: bond %d (%d, %d) or its J is invalid", b, i, j);
    bond[b] = std::min(i, j) | (std::max(i, j) << 8);
    uniform = uniform && J_host[b] == J_host[0];
    const double v = 0.5 * J_host[b];
    exact32 = exact32 && (double)(float)v == v;
  }
  if (h_host)
    for (int i = 0; i < nsite; ++i)
      if (!isfinite(h_host[i])) return fail(ctx, KW_ERR_ARG, "kw_set_spin_operator: field %d is not finite", i);
  KW_CUDA(cudaStreamSynchronize(ctx->stream), "kw_set_spin_operator: sync");
  KW_CUDA(ctx->sp_binom.ensure((size_t)kw::KW_BINOM_N * kw::KW_BINOM_K * 4), "operator allocation");
  KW_CUDA(ctx->sp_basis.ensure((size_t)m * 4), "operator allocation");
  KW_CUDA(ctx->sp_bond.ensure((size_t)nbond * 4), "operator allocation");
  KW_CUDA(ctx->sp_J.ensure((size_t)nbond * 8), "operator allocation");
  KW_CUDA(ctx->sp_h.ensure((size_t)nsite * 8), "operator allocation");
  KW_CUDA(ctx->g_diag64.ensure((size_t)m * 8), "operator allocation");
  KW_CUDA(cudaMemcpy(ctx->sp_bond.p, bond.data(), (size_t)nbond * 4, cudaMemcpyHostToDevice), "operator upload");
  KW_CUDA(cudaMemcpy(ctx->sp_J.p, J_host, (size_t)nbond * 8, cudaMemcpyHostToDevice), "operator upload");
  if (h_host) KW_CUDA(cudaMemcpy(ctx->sp_h.p, h_host, (size_t)nsite * 8, cudaMemcpyHostToDevice), "operator upload");
  KW_CUDA(kw::launch_spin_setup((int)m, nsite, nup, nbond, (const int*)ctx->sp_bond.p, (const double*)ctx->sp_J.p,
                                h_host ? (const double*)ctx->sp_h.p : nullptr, (int*)ctx->sp_binom.p,
                                (unsigned*)ctx->sp_basis.p, (double*)ctx->g_diag64.p, ctx->stream),
          "kw_set_spin_operator: set-up");
  become_generated(ctx, kw::OP_SPIN, m);
  ctx->sp_table_built = false;
  if (ctx->sp_table_on) {
    KW_CUDA(ctx->sp_table.ensure((size_t)nbond * m * 4), "kw_set_spin_operator: exchange table");
    KW_CUDA(kw::launch_spin_table((int)m, nbond, (const int*)ctx->sp_bond.p, (const int*)ctx->sp_binom.p,
                                  (const unsigned*)ctx->sp_basis.p, (int*)ctx->sp_table.p, ctx->stream),
            "kw_set_spin_operator: exchange table");
    ctx->sp_table_built = true;
  }
  kw_status st = generated_diag(ctx, m, exact32);
  if (st != KW_OK) return st;
  ctx->sp_nbond = nbond;
  ctx->sp_uniform = uniform ? 1 : 0;
  ctx->g_v = 0.5 * J_host[0];
  // per-bond amplitudes J_b/2 in the diagonal's storage (read when the J_b differ)
  KW_CUDA(ctx->sp_val.ensure((size_t)nbond * 8), "operator allocation");
  std::vector<unsigned char> vals((size_t)nbond * 8);
  for (int b = 0; b < nbond; ++b) {
    const double v = 0.5 * J_host[b];
    if (ctx->g_kind == 0) {
      memcpy(&vals[(size_t)b * 8], &v, 8);
    } else if (ctx->g_kind == 1) {
      const float f = (float)v;
      memcpy(&vals[(size_t)b * 4], &f, 4);
    } else {
      const float hi = (float)v, lo = (float)(v - (double)hi);
      memcpy(&vals[(size_t)b * 8], &hi, 4);
      memcpy(&vals[(size_t)b * 8 + 4], &lo, 4);
    }
  }
  KW_CUDA(cudaMemcpy(ctx->sp_val.p, vals.data(), vals.size(), cudaMemcpyHostToDevice), "operator upload");
  return KW_OK;
}

kw_status kw_set_spin_table(kw_ctx* ctx, int on) {
  if (!ctx || (on != 0 && on != 1)) return KW_ERR_ARG;
  ctx->sp_table_on = on == 1;
  if (ctx->op != kw::OP_SPIN) return KW_OK;   // takes effect at the next kw_set_spin_operator
  KW_CUDA(cudaStreamSynchronize(ctx->stream), "kw_set_spin_table: sync");
  if (!on) {
    ctx->sp_table.release();
    ctx->sp_table_built = false;
    return KW_OK;
  }
  if (!ctx->sp_table_built) {
    KW_CUDA(ctx->sp_table.ensure((size_t)ctx->sp_nbond * ctx->m * 4), "kw_set_spin_table: allocation");
    KW_CUDA(kw::launch_spin_table((int)ctx->m, ctx->sp_nbond, (const int*)ctx->sp_bond.p, (const int*)ctx->sp_binom.p,
                                  (const unsigned*)ctx->sp_basis.p, (int*)ctx->sp_table.p, ctx->stream),
            "kw_set_spin_table: build");
    KW_CUDA(cudaStreamSynchronize(ctx->stream), "kw_set_spin_table: sync");
    ctx->sp_table_built = true;
  }
  return KW_OK;
}

kw_status kw_set_lattice3d(kw_ctx* ctx, int64_t nx, int64_t ny, int64_t nz, const double* eps_dev, double hopping) {
  if (!ctx) return KW_ERR_ARG;
  if (nx < 3 || ny < 3 || nz < 3 || !eps_dev || !isfinite(hopping) || (double)nx * ny * nz > (double)KW_MAX_ROWS)
    return fail(ctx, KW_ERR_ARG, "kw_set_lattice3d: need extents >= 3, nx ny nz < 2^31, eps and a finite hopping");
  const int64_t m = nx * ny * nz;
  KW_CUDA(ctx->g_diag64.ensure((size_t)m * 8), "operator allocation");
  KW_CUDA(cudaMemcpyAsync(ctx->g_diag64.p, eps_dev, (size_t)m * 8, cudaMemcpyDeviceToDevice, ctx->stream),
          "kw_set_lattice3d: copy");
  become_generated(ctx, kw::OP_LATTICE, m);
  kw_status st = generated_diag(ctx, m, (double)(float)hopping == hopping);
  if (st != KW_OK) return st;
  ctx->lx = (int)nx;
  ctx->ly = (int)ny;
  ctx->lz = (int)nz;
  ctx->g_v = hopping;
  return KW_OK;
}

kw_status kw_set_matvec(kw_ctx* ctx, int64_t m, kw_matvec_fn fn, void* user) {
  if (!ctx) return KW_ERR_ARG;
  if (m < 1 || m > KW_MAX_ROWS || !fn) return fail(ctx, KW_ERR_ARG, "kw_set_matvec: need 1 <= m <= KW_MAX_ROWS and fn");
  ctx->mv_fn = fn;
  ctx->mv_user = user;
  ctx->mv_fn_adj = nullptr;
  ctx->mv_user_adj = nullptr;
  ctx->op = kw::OP_CALLBACK;
  ctx->resumable = false;
  ctx->m = m;
  ctx->nnz = 0;
  ctx->rowptr = nullptr;
  ctx->col = nullptr;
  ctx->val = nullptr;
  ctx->val32_exact = false;
  ctx->spmv_lanes = 1;   // nothing to tune
  ctx->spmv_val_f32 = 0;
  ctx->sell_built = false;
  return KW_OK;
}

}  // extern "C"

static size_t part_doubles(const kw_ctx* ctx, int64_t K) {
  return std::max<size_t>({(size_t)kw::kMaxBlocksPerSM * ctx->num_sms * (3 + 2 * KW_MAX_PROJ),
                           (size_t)K * 4, (size_t)4 * ctx->num_sms * (KW_MAX_PROJ + 1)});
}

// Work descriptor holding only what the SpMV kernel needs.
static void spmv_work(kw_ctx* ctx, kw::Work& w, int lanes, int val_f32) {
  const kw_precision p = ctx->opt.prec;
  memset(&w, 0, sizeof(w));
  w.prec = prec_id(p);
  w.m = ctx->m;
  w.rowptr = ctx->rowptr;
  w.col = ctx->col;
  if (p == KW_C32V_F64S) w.val_f32 = 1;
  else if (p == KW_DF64) w.val_f32 = ctx->val32_exact ? 1 : 0;
  else w.val_f32 = val_f32;
  w.val = w.val_f32 ? (const void*)ctx->val32.p
                    : (p == KW_DF64 ? (const void*)ctx->valpair.p : (const void*)ctx->val);
  w.spmv_lanes = lanes;
  if (lanes > kw::KW_SPMV_UNIFORM && ctx->u_state == 1) {
    if (lanes == kw::KW_SPMV_UNIFORM_SELL && ctx->us_state == 1) {
      w.u_sptr = (const int*)ctx->u_sptr.p;
      w.u_scol = (const int*)ctx->u_scol.p;
    }
    w.u_rowptr = (const int*)ctx->u_rowptr.p;
    w.u_col = (const int*)ctx->u_col.p;
    w.u_kind = ctx->u_kind;
    w.u_diag = ctx->u_kind == 0 ? ctx->u_diag64.p : ctx->u_kind == 1 ? ctx->u_diag32.p : ctx->u_diagpair.p;
    w.u_v = ctx->u_v;
  }
  w.op = ctx->op;
  if (ctx->op == kw::OP_SPIN || ctx->op == kw::OP_LATTICE) {
    w.u_kind = ctx->g_kind;
    w.u_diag = ctx->g_kind == 0 ? ctx->g_diag64.p : ctx->g_kind == 1 ? ctx->g_diag32.p : ctx->g_diagpair.p;
    w.u_v = ctx->g_v;
    w.sp_basis = (const unsigned*)ctx->sp_basis.p;
    w.sp_binom = (const int*)ctx->sp_binom.p;
    w.sp_bond = (const int*)ctx->sp_bond.p;
    w.sp_val = ctx->sp_val.p;
    w.sp_nbond = ctx->sp_nbond;
    w.sp_uniform = ctx->sp_uniform;
    w.sp_table = (ctx->op == kw::OP_SPIN && ctx->sp_table_built) ? (const int*)ctx->sp_table.p : nullptr;
    w.lx = ctx->lx;
    w.ly = ctx->ly;
    w.lz = ctx->lz;
  }
  w.part_k1 = (double*)ctx->part_k1.p;
  w.mv_fn = ctx->mv_fn;
  w.mv_user = ctx->mv_user;
  w.mv_fn_adj = ctx->mv_fn_adj;
  w.mv_user_adj = ctx->mv_user_adj;
  w.mv_r = ctx->mv_r.p;
  w.mv_q = ctx->mv_q.p;
  w.mv_r2 = ctx->mv_r2.p;
  w.mv_q2 = ctx->mv_q2.p;
  w.rci = ctx->rci_active ? 1 : 0;
  w.rci_phase = ctx->rci_active ? 1 : 0;
  if (lanes == kw::KW_SPMV_SELL) {
    if (p == KW_F64) w.val_f32 = 0;       // the SELL copy keeps FP64 values in the FP64 form
    w.sell_perm = (const int*)ctx->sell_perm.p;
    w.sell_len = (const int*)ctx->sell_len.p;
    w.sell_ptr = (const int64_t*)ctx->sell_ptr.p;
    w.sell_col = (const int*)ctx->sell_col.p;
    w.sell_val = ctx->sell_val.p;
  }
  w.stream = ctx->stream;
  w.num_sms = ctx->num_sms;
  w.part = (double*)ctx->part.p;
  w.part_k1 = (double*)ctx->part_k1.p;
  w.st = (kw::State*)ctx->st.p;
}

// Build the SELL-32 copy of the operator: device sort of each 1024-row window
// by row length, slice offsets by a host prefix sum, device fill.
static kw_status build_sell(kw_ctx* ctx) {
  if (ctx->sell_built) return KW_OK;
  const kw_precision p = ctx->opt.prec;
  const int m = (int)ctx->m;
  const int nslice = (m + 31) / 32;
  KW_CUDA(ctx->sell_perm.ensure((size_t)m * 4), "sell alloc");
  KW_CUDA(ctx->sell_len.ensure((size_t)m * 4), "sell alloc");
  KW_CUDA(ctx->sell_slen.ensure((size_t)nslice * 4), "sell alloc");
  KW_CUDA(ctx->sell_ptr.ensure((size_t)(nslice + 1) * 8), "sell alloc");
  KW_CUDA(kw::launch_sell_order(m, ctx->rowptr, (int*)ctx->sell_perm.p, (int*)ctx->sell_len.p,
                                (int*)ctx->sell_slen.p, ctx->stream), "sell order");
  std::vector<int> slen(nslice);
  std::vector<int64_t> sptr(nslice + 1);
  KW_CUDA(cudaMemcpyAsync(slen.data(), ctx->sell_slen.p, (size_t)nslice * 4, cudaMemcpyDeviceToHost, ctx->stream),
          "sell read");
  KW_CUDA(cudaStreamSynchronize(ctx->stream), "sell sync");
  sptr[0] = 0;
  for (int s = 0; s < nslice; ++s) sptr[s + 1] = sptr[s] + 32 * (int64_t)slen[s];
  KW_CUDA(cudaMemcpyAsync(ctx->sell_ptr.p, sptr.data(), (size_t)(nslice + 1) * 8, cudaMemcpyHostToDevice, ctx->stream),
          "sell upload");
  const int64_t padded = std::max<int64_t>(sptr[nslice], 1);
  // value kind: FP64 form -> double; FP32 form -> float; pair form -> float if exact, else pairs
  const int kind = p == KW_F64 ? 0 : (p == KW_C32V_F64S || ctx->val32_exact) ? 1 : 2;
  const size_t vb = kind == 1 ? 4 : 8;
  KW_CUDA(ctx->sell_col.ensure((size_t)padded * 4), "sell alloc");
  KW_CUDA(ctx->sell_val.ensure((size_t)padded * vb), "sell alloc");
  KW_CUDA(cudaMemsetAsync(ctx->sell_col.p, 0, (size_t)padded * 4, ctx->stream), "sell memset");
  KW_CUDA(cudaMemsetAsync(ctx->sell_val.p, 0, (size_t)padded * vb, ctx->stream), "sell memset");
  if (ctx->nnz > 0) {
    const void* src = kind == 0 ? (const void*)ctx->val : kind == 1 ? ctx->val32.p : ctx->valpair.p;
    cudaError_t e =
        kind == 0 ? kw::launch_sell_fill<double>(m, (const int*)ctx->sell_perm.p, (const int*)ctx->sell_len.p,
                                                 (const int64_t*)ctx->sell_ptr.p, ctx->rowptr, ctx->col, src,
                                                 (int*)ctx->sell_col.p, ctx->sell_val.p, ctx->stream)
        : kind == 1 ? kw::launch_sell_fill<float>(m, (const int*)ctx->sell_perm.p, (const int*)ctx->sell_len.p,
                                                  (const int64_t*)ctx->sell_ptr.p, ctx->rowptr, ctx->col, src,
                                                  (int*)ctx->sell_col.p, ctx->sell_val.p, ctx->stream)
                    : kw::launch_sell_fill<kw::df>(m, (const int*)ctx->sell_perm.p, (const int*)ctx->sell_len.p,
                                                   (const int64_t*)ctx->sell_ptr.p, ctx->rowptr, ctx->col, src,
                                                   (int*)ctx->sell_col.p, ctx->sell_val.p, ctx->stream);
    KW_CUDA(e, "sell fill");
  }
  ctx->sell_built = true;
  return KW_OK;
}

// Uniform off-diagonal copy of the CSR operator: detect (every off-diagonal
// value bitwise equal), then build int32 offsets, the off-diagonal columns and
// the summed diagonal in the storage the context's form reads.
static kw_status build_uniform(kw_ctx* ctx) {
  if (ctx->u_state != 0) return KW_OK;
  const int m = (int)ctx->m;
  KW_CUDA(ctx->u_fm.ensure(2 * sizeof(unsigned long long)), "uniform layout allocation");
  KW_CUDA(ctx->u_dcount.ensure((size_t)m * 4), "uniform layout allocation");
  KW_CUDA(kw::launch_uniform_check(m, ctx->rowptr, ctx->col, ctx->val, (unsigned long long*)ctx->u_fm.p,
                                   (int*)ctx->u_dcount.p, ctx->stream), "uniform layout check");
  unsigned long long fm[2] = {0, 0};
  KW_CUDA(cudaMemcpyAsync(fm, ctx->u_fm.p, sizeof(fm), cudaMemcpyDeviceToHost, ctx->stream), "uniform layout check");
  KW_CUDA(cudaStreamSynchronize(ctx->stream), "uniform layout check");
  if (fm[1] != 0) {
    ctx->u_state = -1;
    return KW_OK;
  }
  double v = 0.0;
  if (fm[0] != ~0ull)
    KW_CUDA(cudaMemcpy(&v, ctx->val + fm[0], sizeof(double), cudaMemcpyDeviceToHost), "uniform layout value");
  const int64_t noff = ctx->nnz;   // upper bound: the diagonal entries are dropped
  KW_CUDA(ctx->u_scratch.ensure((size_t)((m + 1023) / 1024) * 4), "uniform layout allocation");
  KW_CUDA(ctx->u_rowptr.ensure((size_t)(m + 1) * 4), "uniform layout allocation");
  // four entries of padding: K1 reads the columns as aligned groups of four
  KW_CUDA(ctx->u_col.ensure((size_t)(noff + 4) * 4), "uniform layout allocation");
  KW_CUDA(ctx->u_diag64.ensure((size_t)m * 8), "uniform layout allocation");
  KW_CUDA(kw::launch_uniform_build(m, ctx->rowptr, ctx->col, ctx->val, (int*)ctx->u_dcount.p,
                                   (int*)ctx->u_scratch.p, (int*)ctx->u_rowptr.p, (int*)ctx->u_col.p,
                                   (double*)ctx->u_diag64.p, ctx->stream), "uniform layout build");
  // FP32 copy of the diagonal and whether it (and the value) is exact in FP32
  KW_CUDA(ctx->u_diag32.ensure((size_t)m * 4), "uniform layout allocation");
  KW_CUDA(ctx->inexact.ensure(sizeof(unsigned long long)), "uniform layout allocation");
  KW_CUDA(cudaMemsetAsync(ctx->inexact.p, 0, sizeof(unsigned long long), ctx->stream), "uniform layout memset");
  KW_CUDA(kw::launch_convert_f64_to_f32((const double*)ctx->u_diag64.p, (float*)ctx->u_diag32.p, m,
                                        (unsigned long long*)ctx->inexact.p, ctx->stream), "uniform layout convert");
  unsigned long long bad = 0;
  KW_CUDA(cudaMemcpyAsync(&bad, ctx->inexact.p, sizeof(bad), cudaMemcpyDeviceToHost, ctx->stream), "uniform layout");
  KW_CUDA(cudaStreamSynchronize(ctx->stream), "uniform layout sync");
  const bool exact32 = bad == 0 && (double)(float)v == v;
  const kw_precision p = ctx->opt.prec;
  if (p == KW_C32V_F64S || exact32) {
    ctx->u_kind = 1;
  } else if (p == KW_DF64) {
    ctx->u_kind = 2;
    KW_CUDA(ctx->u_diagpair.ensure((size_t)m * 8), "uniform layout allocation");
    KW_CUDA(kw::launch_convert_f64_to_pair((const double*)ctx->u_diag64.p, ctx->u_diagpair.p, m, ctx->stream),
            "uniform layout convert");
  } else {
    ctx->u_kind = 0;
  }
  ctx->u_v = v;
  ctx->u_state = 1;
  return KW_OK;
}

// SELL-32 copy of the uniform layout: the off-diagonal columns of each slice of
// 32 consecutive rows stored slot-major (slot k = each row's k-th column, -1
// past its end), so that K1's index loads are coalesced.  Not built when the
// padding would more than triple the column array (rows of very different
// lengths in one slice) or the slots overflow 32-bit offsets.
static kw_status build_uniform_sell(kw_ctx* ctx) {
  if (ctx->us_state != 0) return KW_OK;
  kw_status us = build_uniform(ctx);
  if (us != KW_OK) return us;
  if (ctx->u_state != 1) {
    ctx->us_state = -1;
    return KW_OK;
  }
  const int m = (int)ctx->m;
  const int nslice = (m + 31) / 32;
  KW_CUDA(ctx->u_sptr.ensure((size_t)(nslice + 1) * 4), "uniform SELL allocation");
  KW_CUDA(ctx->u_fm.ensure(2 * sizeof(unsigned long long)), "uniform SELL allocation");
  KW_CUDA(kw::launch_uniform_sell_count(m, (const int*)ctx->u_rowptr.p, (int*)ctx->u_sptr.p,
                                        (unsigned long long*)ctx->u_fm.p, ctx->stream), "uniform SELL count");
  unsigned long long total = 0;
  int last = 0, noff = 0;
  KW_CUDA(cudaMemcpyAsync(&total, ctx->u_fm.p, sizeof(total), cudaMemcpyDeviceToHost, ctx->stream), "uniform SELL");
  KW_CUDA(cudaMemcpyAsync(&last, (const int*)ctx->u_sptr.p + (nslice - 1), sizeof(int), cudaMemcpyDeviceToHost,
                          ctx->stream), "uniform SELL");
  KW_CUDA(cudaMemcpyAsync(&noff, (const int*)ctx->u_rowptr.p + m, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream),
          "uniform SELL");
  KW_CUDA(cudaStreamSynchronize(ctx->stream), "uniform SELL sync");
  if (total > 0x7fffffffULL || 32ULL * total > 3ULL * (unsigned long long)noff + 32ULL * (unsigned long long)nslice) {
    ctx->us_state = -1;
    return KW_OK;
  }
  KW_CUDA(ctx->u_scol.ensure((size_t)std::max<unsigned long long>(total, 1) * 32 * 4), "uniform SELL allocation");
  KW_CUDA(kw::launch_uniform_sell_fill(m, (const int*)ctx->u_rowptr.p, (const int*)ctx->u_col.p,
                                       (int*)ctx->u_sptr.p, (int*)ctx->u_scratch.p, last, (int*)ctx->u_scol.p,
                                       ctx->stream), "uniform SELL fill");
  ctx->us_state = 1;
  return KW_OK;
}

static void release_uniform_sell(kw_ctx* ctx) {
  ctx->u_scol.release();
  ctx->u_sptr.release();
  ctx->us_state = 0;
}

// kw_c128 staging vectors of the callback operator in the FP32-pair form.
static kw_status ensure_mv_buffers(kw_ctx* ctx) {
  if (!ctx->mv_fn || ctx->opt.prec != KW_DF64) return KW_OK;
  KW_CUDA(ctx->mv_r.ensure((size_t)ctx->m * 16), "callback staging allocation");
  KW_CUDA(ctx->mv_q.ensure((size_t)ctx->m * 16), "callback staging allocation");
  return KW_OK;
}

static cudaError_t spmv_dot_launch(kw::Work& w, const void* r, void* q, double2 zs, double2* t) {
  if (!w.st || !w.part_k1 || !t || (!w.rowptr && !w.mv_fn && w.op < kw::OP_SPIN))
    return cudaErrorInvalidValue;   // workspace and operator must exist
  const float4 zp = host_pair(zs.x, zs.y);
  switch (w.prec) {
    case kw::PREC_C32: return kw::launch_spmv_dot<kw::PREC_C32>(w, r, q, zs, zp, t);
    case kw::PREC_DF: return kw::launch_spmv_dot<kw::PREC_DF>(w, r, q, zs, zp, t);
    default: return kw::launch_spmv_dot<kw::PREC_F64>(w, r, q, zs, zp, t);
  }
}

// Autotuner for K1: time every (lanes per row, value type) candidate on the
// current operator with CUDA events and keep the fastest.
// Operators below this many non-zeros are not timed (launch overhead dominates
// and the pick would be noise); they use one thread per row and FP64 values.
static const int64_t kTuneMinNnz = 1 << 20;

// ---------------------------------------------------------------- persistent tuning cache
// One line per pick: "kwtune1 <prec> <m> <nnz> <fingerprint> <sms> <lanes> <val_f32>".
struct TuneKey {
  int prec;
  long long m, nnz;
  unsigned long long fp;
  int sms;
};

// FNV-1a over sampled rows (row offsets, first column and its value's bits).
static kw_status tune_fingerprint(kw_ctx* ctx, unsigned long long* fp) {
  const int ns = kw::kTuneSamples;
  KW_CUDA(ctx->tune_fp.ensure((size_t)ns * 4 * sizeof(long long)), "tune cache alloc");
  KW_CUDA(kw::launch_fingerprint((int)ctx->m, ctx->rowptr, ctx->col, ctx->val, (long long*)ctx->tune_fp.p,
                                 ctx->stream), "tune fingerprint");
  std::vector<long long> h((size_t)ns * 4);
  KW_CUDA(cudaMemcpyAsync(h.data(), ctx->tune_fp.p, h.size() * sizeof(long long), cudaMemcpyDeviceToHost,
                          ctx->stream), "tune fingerprint copy");
  KW_CUDA(cudaStreamSynchronize(ctx->stream), "tune fingerprint sync");
  unsigned long long x = 1469598103934665603ULL;
  for (long long v : h)
    for (int b = 0; b < 8; ++b) {
      x ^= (unsigned long long)((v >> (8 * b)) & 0xff);
      x *= 1099511628211ULL;
    }
  *fp = x;
  return KW_OK;
}

static bool tune_cache_lookup(const char* path, const TuneKey& k, int* lanes, int* val) {
  FILE* f = fopen(path, "r");
  if (!f) return false;
  char line[256];
  bool found = false;
  while (fgets(line, sizeof(line), f)) {
    int prec = 0, sms = 0, l = 0, v = 0;
    long long m = 0, nnz = 0;
    unsigned long long fp = 0;
    if (sscanf(line, "kwtune1 %d %lld %lld %llx %d %d %d", &prec, &m, &nnz, &fp, &sms, &l, &v) != 7) continue;
    if (prec == k.prec && m == k.m && nnz == k.nnz && fp == k.fp && sms == k.sms) {
      *lanes = l;   // the last matching line wins
      *val = v;
      found = true;
    }
  }
  fclose(f);
  return found;
}

static void tune_cache_store(const char* path, const TuneKey& k, int lanes, int val) {
  FILE* f = fopen(path, "a");
  if (!f) return;   // an unwritable cache only costs the next context a timing run
  char line[256];
  const int n = snprintf(line, sizeof(line), "kwtune1 %d %lld %lld %016llx %d %d %d\n", k.prec, k.m, k.nnz, k.fp,
                         k.sms, lanes, val);
  if (n > 0) fwrite(line, 1, (size_t)n, f);   // one write per line (appends do not interleave within it)
  fclose(f);
}

static bool has_operator(const kw_ctx* ctx) {
  return ctx->rowptr || ctx->mv_fn || ctx->rci_active || ctx->op >= kw::OP_SPIN;
}

static kw_status tune_spmv(kw_ctx* ctx) {
  if (ctx->op != kw::OP_CSR) {   // callback or generated operator: nothing to tune
    ctx->spmv_lanes = 1;
    ctx->spmv_val_f32 = 0;
    return KW_OK;
  }
  if (ctx->spmv_lanes > 0) return KW_OK;
  const kw_precision p = ctx->opt.prec;
  if (ctx->nnz < kTuneMinNnz || ctx->force_lanes == kw::KW_SPMV_SELL || ctx->force_lanes > kw::KW_SPMV_UNIFORM) {
    ctx->spmv_lanes = ctx->force_lanes > 0 ? ctx->force_lanes : 1;
    ctx->spmv_val_f32 = (p == KW_F64 && ctx->force_val == 1 && ctx->val32_exact) ? 1 : 0;
    if (ctx->spmv_lanes > kw::KW_SPMV_UNIFORM) {
      kw_status us = build_uniform(ctx);
      if (us != KW_OK) return us;
      if (ctx->u_state != 1) {
        ctx->spmv_lanes = 0;
        return fail(ctx, KW_ERR_ARG, "uniform off-diagonal layout requested, but the off-diagonal values differ");
      }
      if (ctx->spmv_lanes == kw::KW_SPMV_UNIFORM_SELL) {
        if ((us = build_uniform_sell(ctx)) != KW_OK) return us;
        if (ctx->us_state != 1) {
          ctx->spmv_lanes = 0;
          return fail(ctx, KW_ERR_ARG, "uniform SELL-32 layout requested, but its padding would exceed 3x");
        }
      }
      ctx->spmv_val_f32 = ctx->u_kind == 1 ? 1 : 0;
      return KW_OK;
    }
    if (ctx->spmv_lanes == kw::KW_SPMV_SELL) {
      if (p == KW_F64) ctx->spmv_val_f32 = 0;   // the SELL copy keeps FP64 values in the FP64 form
      return build_sell(ctx);
    }
    return KW_OK;
  }
  // persistent cache: a pick stored for this operator and device is applied without timing
  const bool use_cache = ctx->opt.tune_cache && ctx->opt.tune_cache[0] && ctx->force_lanes == 0 &&
                         ctx->force_val < 0;
  TuneKey key = {(int)p, (long long)ctx->m, (long long)ctx->nnz, 0ULL, ctx->num_sms};
  if (use_cache) {
    kw_status fs = tune_fingerprint(ctx, &key.fp);
    if (fs != KW_OK) return fs;
    int cl = 0, cv = 0;
    if (tune_cache_lookup(ctx->opt.tune_cache, key, &cl, &cv)) {
      const bool lanes_ok = (cl >= 1 && cl <= 16 && (cl & (cl - 1)) == 0) || cl == kw::KW_SPMV_SELL ||
                            (cl > kw::KW_SPMV_UNIFORM && cl <= kw::KW_SPMV_UNIFORM + 16 &&
                             ((cl - kw::KW_SPMV_UNIFORM) & (cl - kw::KW_SPMV_UNIFORM - 1)) == 0) ||
                            cl == kw::KW_SPMV_UNIFORM_SELL;
      const bool val_ok = cv == 0 || (cv == 1 && (p != KW_F64 || ctx->val32_exact));
      bool ok = lanes_ok && val_ok;
      if (ok && cl > kw::KW_SPMV_UNIFORM) {
        kw_status us = build_uniform(ctx);
        if (us != KW_OK) return us;
        ok = ctx->u_state == 1;   // the values may differ from the operator the pick was timed on
        if (ok && cl == kw::KW_SPMV_UNIFORM_SELL) {
          if ((us = build_uniform_sell(ctx)) != KW_OK) return us;
          ok = ctx->us_state == 1;
        }
      }
      if (ok && cl == kw::KW_SPMV_SELL) {
        kw_status bs = build_sell(ctx);
        if (bs != KW_OK) return bs;
      }
      if (ok) {
        ctx->spmv_lanes = cl;
        ctx->spmv_val_f32 = cl > kw::KW_SPMV_UNIFORM ? (ctx->u_kind == 1 ? 1 : 0)
                            : cl == kw::KW_SPMV_SELL ? (p == KW_F64 ? 0 : cv)
                                                     : cv;
        ctx->tune_hits += 1;
        return KW_OK;
      }
    }
  }
  const size_t vs = vec_bytes(p);
  KW_CUDA(ctx->rA.ensure(ctx->m * vs), "tune alloc");
  KW_CUDA(ctx->q.ensure(ctx->m * vs), "tune alloc");
  KW_CUDA(ctx->part_k1.ensure(part_doubles(ctx, 1) * 8), "tune alloc");
  KW_CUDA(ctx->st.ensure(sizeof(kw::State)), "tune alloc");
  KW_CUDA(ctx->tdot.ensure(16), "tune alloc");
  KW_CUDA(cudaMemsetAsync(ctx->rA.p, 0, ctx->m * vs, ctx->stream), "tune memset");
  KW_CUDA(cudaMemsetAsync(ctx->st.p, 0, sizeof(kw::State), ctx->stream), "tune memset");
  const int lane_opts[] = {1, 2, 4, 8, 16, kw::KW_SPMV_SELL, kw::KW_SPMV_UNIFORM + 1, kw::KW_SPMV_UNIFORM + 2,
                           kw::KW_SPMV_UNIFORM + 4, kw::KW_SPMV_UNIFORM + 8, kw::KW_SPMV_UNIFORM_SELL};
  // value storage candidates: only the FP64 form has a choice (FP64 or exact FP32 values)
  int vals[2] = {0, 1}, nvals = 1;
  if (p == KW_F64 && ctx->val32_exact) nvals = 2;
  if (p == KW_F64 && ctx->force_val >= 0) {
    vals[0] = (ctx->force_val && ctx->val32_exact) ? 1 : 0;
    nvals = 1;
  }
  ScopedEvents tev;
  KW_CUDA(tev.create(2, cudaEventDefault), "tune events");
  cudaEvent_t e0 = tev[0], e1 = tev[1];
  float best = 1e30f;
  int best_l = 4, best_v = vals[0];
  // Candidates are visited in a fixed order; a later one replaces the current
  // pick only if it is more than 5% faster, so near-ties resolve the same way.
  for (int vi = 0; vi < nvals; ++vi) {
    for (int l : lane_opts) {
      if (ctx->force_lanes > 0 && l != ctx->force_lanes) continue;
      if (l == kw::KW_SPMV_SELL) {
        if (vi > 0) continue;   // the SELL copy has one value type per form
        kw_status bs = build_sell(ctx);
        if (bs != KW_OK) return bs;
      }
      if (l > kw::KW_SPMV_UNIFORM) {
        if (vi > 0) continue;   // one storage per form, chosen when the copy is built
        kw_status us = build_uniform(ctx);
        if (us != KW_OK) return us;
        if (ctx->u_state != 1) continue;
        if (l == kw::KW_SPMV_UNIFORM_SELL) {
          if ((us = build_uniform_sell(ctx)) != KW_OK) return us;
          if (ctx->us_state != 1) continue;
        }
      }
      kw::Work w;
      spmv_work(ctx, w, l, vals[vi]);
      const double2 zs = make_double2(0.5, 0.5);
      if (spmv_dot_launch(w, ctx->rA.p, ctx->q.p, zs, (double2*)ctx->tdot.p) != cudaSuccess) break;
      cudaEventRecord(e0, ctx->stream);
      for (int rep = 0; rep < 3; ++rep) spmv_dot_launch(w, ctx->rA.p, ctx->q.p, zs, (double2*)ctx->tdot.p);
      cudaEventRecord(e1, ctx->stream);
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < 0.95f * best) {
        best = ms;
        best_l = l;
        best_v = vals[vi];
      }
    }
  }
  KW_CUDA(cudaGetLastError(), "tune launches");
  ctx->spmv_lanes = best_l;
  ctx->spmv_val_f32 = best_l == kw::KW_SPMV_SELL ? (p == KW_F64 ? 0 : best_v) : best_v;
  if (best_l > kw::KW_SPMV_UNIFORM) ctx->spmv_val_f32 = ctx->u_kind == 1 ? 1 : 0;
  if (best_l != kw::KW_SPMV_UNIFORM_SELL && ctx->us_state == 1) release_uniform_sell(ctx);
  if (best_l != kw::KW_SPMV_SELL && ctx->sell_built) {   // not chosen: give the memory back
    ctx->sell_col.release();
    ctx->sell_val.release();
    ctx->sell_built = false;
  }
  ctx->tune_runs += 1;
  if (use_cache) tune_cache_store(ctx->opt.tune_cache, key, ctx->spmv_lanes, ctx->spmv_val_f32);
  return KW_OK;
}

// Allocate the workspace of one solve and fill the Work descriptor.
static kw_status prepare(kw_ctx* ctx, kw::Work& w, const double* b_dev, int64_t K, const kw_c128* z_host,
                         int64_t nleft, const double* left_dev, void* x_out_dev) {
  const size_t vs = vec_bytes(ctx->opt.prec), rs = real_bytes(ctx->opt.prec);
  const int64_t m = ctx->m;
  spmv_work(ctx, w, ctx->spmv_lanes, ctx->spmv_val_f32);
  w.m = m;
  w.K = (int)K;
  w.full = x_out_dev != nullptr;
  w.nout = (int)nleft + 1;
  // FP32 shift storage (full mode, FP64 and FP32-pair forms): the projections come from the
  // projected recurrences run beside the x/p update, so K2 forms P r_{n+1} in full mode too
  w.xp32 = (w.full && ctx->xp32 && ctx->opt.prec != KW_C32V_F64S) ? 1 : 0;
  w.nproj = (w.full && !w.xp32) ? 0 : (int)nleft + 1;
  w.tol = ctx->opt.tol;
  w.proj_ld = (m + kw::KW_PROJ_ALIGN - 1) / kw::KW_PROJ_ALIGN * kw::KW_PROJ_ALIGN;
  w.bulk = ctx->bulk;
  w.seed_rg = ctx->seed_rg;
  w.b = b_dev;
  w.left = left_dev;
  w.stream = ctx->stream;
  w.num_sms = ctx->num_sms;
  const int npw = std::max(w.nproj, 1);
  const int64_t nrecmax = ctx->opt.hist_stride > 0 ? ctx->opt.hist_max : 0;
  const size_t part_d = part_doubles(ctx, K);
  const size_t Ks = (size_t)K, Ms = (size_t)m;
  struct {
    DBuf* b;
    size_t bytes;
  } plan[] = {
      {&ctx->rA, Ms * vs},
      {&ctx->rB, Ms * vs},
      {&ctx->q, Ms * vs},
      {&ctx->proj_rows, (size_t)std::max(w.nproj, 1) * (size_t)w.proj_ld * rs},
      {&ctx->z, Ks * 16},
      {&ctx->pi1, Ks * 16},
      {&ctx->pi0, Ks * 16},
      {&ctx->active, Ks * 4},
      {&ctx->conv_iter, Ks * 8},
      {&ctx->final_res, Ks * 8},
      {&ctx->coef, 2 * Ks * 48},        // two parity slots: K4(n) reads one while K3(n+1) writes the other
      {&ctx->coef_pair, 2 * Ks * 48},
      {&ctx->Y, Ks * npw * 16},
      {&ctx->U, Ks * npw * 16},
      {&ctx->w, (size_t)KW_MAX_PROJ * 16},
      {&ctx->w0, (size_t)KW_MAX_PROJ * 16},
      {&ctx->hist, std::max<size_t>((size_t)nrecmax * Ks, 1) * 8},
      {&ctx->list, 2 * Ks * 4},
      {&ctx->P, w.full ? Ks * Ms * (w.xp32 ? 8 : vs) : 16},
      {&ctx->part, part_d * 8},
      {&ctx->part_k1, part_d * 8},
      {&ctx->st, sizeof(kw::State)},
      {&ctx->projx, Ks * w.nout * 16},
  };
  for (auto& pl : plan) KW_CUDA(pl.b->ensure(pl.bytes), "workspace allocation");
  w.method = ctx->method;
  w.btilde = ctx->method == KW_METHOD_BICG ? ctx->btilde : nullptr;
  w.rtA = w.rtB = w.qt = nullptr;
  if (ctx->method == KW_METHOD_BICG) {
    KW_CUDA(ctx->rtA.ensure(Ms * vs), "workspace allocation");
    KW_CUDA(ctx->rtB.ensure(Ms * vs), "workspace allocation");
    KW_CUDA(ctx->qt.ensure(Ms * vs), "workspace allocation");
    w.rtA = ctx->rtA.p;
    w.rtB = ctx->rtB.p;
    w.qt = ctx->qt.p;
  }
  w.log = nullptr;
  w.log_max = 0;
  if (ctx->log_max > 0) {
    KW_CUDA(ctx->klog.ensure((size_t)ctx->log_max * (KW_LOG_FIXED + w.nproj) * 16), "Krylov log allocation");
    w.log = (double2*)ctx->klog.p;
    w.log_max = ctx->log_max;
  }
  w.rA = ctx->rA.p;
  w.rB = ctx->rB.p;
  w.q = ctx->q.p;
  w.proj_rows = ctx->proj_rows.p;
  w.z = (double2*)ctx->z.p;
  w.pi1 = (double2*)ctx->pi1.p;
  w.pi0 = (double2*)ctx->pi0.p;
  w.active = (int*)ctx->active.p;
  w.conv_iter = (long long*)ctx->conv_iter.p;
  w.final_res = (double*)ctx->final_res.p;
  w.coef = (double2*)ctx->coef.p;
  w.coef_pair = (float4*)ctx->coef_pair.p;
  w.Y = (double2*)ctx->Y.p;
  w.U = (double2*)ctx->U.p;
  w.w = (double2*)ctx->w.p;
  w.w0 = (double2*)ctx->w0.p;
  w.hist = (double*)ctx->hist.p;
  w.list = (int*)ctx->list.p;
  w.X = x_out_dev;
  w.P = ctx->P.p;
  w.part = (double*)ctx->part.p;
  w.part_k1 = (double*)ctx->part_k1.p;
  w.st = (kw::State*)ctx->st.p;
  if (!ctx->stream2) {   // highest priority: K3's few blocks are placed before the concurrent K1's
    int lo = 0, hi = 0;
    KW_CUDA(cudaDeviceGetStreamPriorityRange(&lo, &hi), "stream priorities");
    KW_CUDA(cudaStreamCreateWithPriority(&ctx->stream2, cudaStreamNonBlocking, hi), "second stream");
  }
  if (!ctx->stream3) {   // lowest priority: K4 fills the SMs that the next iteration's K2 and K1 leave free
    int lo = 0, hi = 0;
    KW_CUDA(cudaDeviceGetStreamPriorityRange(&lo, &hi), "stream priorities");
    KW_CUDA(cudaStreamCreateWithPriority(&ctx->stream3, cudaStreamNonBlocking, lo), "third stream");
  }
  if (!ctx->ev_k2) KW_CUDA(cudaEventCreateWithFlags(&ctx->ev_k2, cudaEventDisableTiming), "stream events");
  if (!ctx->ev_k3) KW_CUDA(cudaEventCreateWithFlags(&ctx->ev_k3, cudaEventDisableTiming), "stream events");
  for (cudaEvent_t& e : ctx->ev_k4)
    if (!e) KW_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "stream events");
  w.stream2 = ctx->stream2;
  w.stream3 = ctx->stream3;
  w.ev_k2 = ctx->ev_k2;
  w.ev_k3 = ctx->ev_k3;
  w.ev_k4[0] = ctx->ev_k4[0];
  w.ev_k4[1] = ctx->ev_k4[1];
  w.k4_mask = 0;
  w.overlap = ctx->rci_active ? 0 : ctx->overlap;   // one step per call under reverse communication

  KW_CUDA(cudaMemcpyAsync(w.z, z_host, K * 16, cudaMemcpyHostToDevice, ctx->stream), "upload shifts");
  kw::State& s = *ctx->st_host;
  memset(&s, 0, sizeof(s));
  s.zs = make_double2(z_host[0].re, z_host[0].im);
  s.zs_k1 = s.zs;
  s.p_zs_k1 = host_pair(z_host[0].re, z_host[0].im);
  s.boa = make_double2(0.0, 0.0);
  s.bscale[0] = s.bscale[1] = make_double2(1.0, 0.0);
  s.p_zs = host_pair(z_host[0].re, z_host[0].im);
  s.seed = 0;
  s.seed_switch = ctx->opt.seed_switch ? 1 : 0;
  s.status = KW_NOT_CONVERGED;
  s.n_active = (int)K;
  s.maxiter = ctx->opt.maxiter;
  s.hist_stride = ctx->opt.hist_stride;
  s.hist_max = nrecmax;
  KW_CUDA(cudaMemcpyAsync(w.st, &s, sizeof(s), cudaMemcpyHostToDevice, ctx->stream), "upload state");
  return KW_OK;
}

// Accumulate the sampled kernel times of one chunk (its events are complete):
// kernel_ms[0] K1 (ev 1-2), [1] K2 (ev 0-1), [2] K3 (ev 3-4), [3] K4 (ev 4-5).
static void collect_times(kw_ctx* ctx, int slot, bool full) {
  static const int from[4] = {1, 0, 3, 4}, to[4] = {2, 1, 4, 5};
  float ms[4] = {0, 0, 0, 0};
  for (int i = 0; i < 4; ++i) {
    if (i == 3 && !full) break;
    if (cudaEventElapsedTime(&ms[i], ctx->kev[slot][from[i]], ctx->kev[slot][to[i]]) != cudaSuccess) return;
  }
  for (int i = 0; i < 4; ++i) ctx->stats.kernel_ms[i] += ms[i];
  ctx->stats.timed_iters += 1;
}

static cudaError_t init_launch(kw::Work& w) {
  switch (w.prec) {
    case kw::PREC_C32: return kw::launch_init<kw::PREC_C32>(w);
    case kw::PREC_DF: return kw::launch_init<kw::PREC_DF>(w);
    default: return kw::launch_init<kw::PREC_F64>(w);
  }
}

static cudaError_t iteration_launch(kw::Work& w, int parity, int first, cudaEvent_t* ev, int64_t* launches) {
  switch (w.prec) {
    case kw::PREC_C32: return kw::launch_iteration<kw::PREC_C32>(w, parity, first, ev, launches);
    case kw::PREC_DF: return kw::launch_iteration<kw::PREC_DF>(w, parity, first, ev, launches);
    default: return kw::launch_iteration<kw::PREC_F64>(w, parity, first, ev, launches);
  }
}

// K4's shift tile (4, 8 or 16 shifts per block item): timed once per form,
// storage, K and M, on the solve's own x/p buffers before they are initialised
// (the tile only decides which block updates which (shift, element) pair, so
// every pick gives the same bits).  A scratch state marks the update pending
// for all K shifts (the list is the identity, the coefficients zero); each
// pick runs once untimed and three times timed, and a later pick replaces the
// current one only if it is more than 5% faster.
static kw_status tune_xp_tile(kw_ctx* ctx, kw::Work& w) {
  if (!w.full) return KW_OK;
  if (ctx->force_xp_tile > 0) {
    w.xp_tile = ctx->force_xp_tile;
    return KW_OK;
  }
  const long long key[4] = {w.prec, w.xp32, w.K, (long long)w.m};
  if (ctx->xp_tile_pick > 0 && std::equal(key, key + 4, ctx->xp_key)) {
    w.xp_tile = ctx->xp_tile_pick;
    return KW_OK;
  }
  KW_CUDA(ctx->xp_st.ensure(sizeof(kw::State)), "update tile: scratch");
  kw::State hs;
  memset(&hs, 0, sizeof(hs));
  hs.xp_pending[0] = 1;
  hs.n_list[0] = w.K;
  std::vector<int> iota((size_t)w.K);
  for (int k = 0; k < w.K; ++k) iota[k] = k;
  cudaStream_t st = ctx->stream;
  KW_CUDA(cudaMemcpyAsync(w.list, iota.data(), (size_t)w.K * 4, cudaMemcpyHostToDevice, st), "update tile: list");
  KW_CUDA(cudaMemsetAsync(w.coef, 0, (size_t)w.K * 48, st), "update tile: coefficients");
  KW_CUDA(cudaMemsetAsync(w.coef_pair, 0, (size_t)w.K * 48, st), "update tile: coefficients");
  ScopedEvents tev;
  KW_CUDA(tev.create(2, cudaEventDefault), "update tile: events");
  kw::State* sst = (kw::State*)ctx->xp_st.p;
  const int opts[3] = {4, 8, 16};
  float best = 1e30f;
  int best_ts = 8;
  for (int ts : opts) {
    w.xp_tile = ts;
    float tot = 0.f;
    for (int rep = 0; rep < 4; ++rep) {   // every launch clears the pending flag: set it again first
      KW_CUDA(cudaMemcpyAsync(sst, &hs, sizeof(hs), cudaMemcpyHostToDevice, st), "update tile: state");
      KW_CUDA(cudaEventRecord(tev[0], st), "update tile: event");
      cudaError_t e = w.prec == kw::PREC_C32 ? kw::launch_update_xp<kw::PREC_C32>(w, w.rA, sst, 0, st)
                      : w.prec == kw::PREC_DF ? kw::launch_update_xp<kw::PREC_DF>(w, w.rA, sst, 0, st)
                                              : kw::launch_update_xp<kw::PREC_F64>(w, w.rA, sst, 0, st);
      KW_CUDA(e, "update tile: launch");
      KW_CUDA(cudaEventRecord(tev[1], st), "update tile: event");
      KW_CUDA(cudaEventSynchronize(tev[1]), "update tile: sync");
      float ms = 0.f;
      KW_CUDA(cudaEventElapsedTime(&ms, tev[0], tev[1]), "update tile: time");
      if (rep > 0) tot += ms;
    }
    if (tot < 0.95f * best) {
      best = tot;
      best_ts = ts;
    }
  }
  w.xp_tile = best_ts;
  ctx->xp_tile_pick = best_ts;
  std::copy(key, key + 4, ctx->xp_key);
  return KW_OK;
}

// Phase 1 of a solve: validate, tune, allocate, upload and enqueue the
// initialisation (no synchronisation).  The descriptor is kept in ctx->work.
static kw_status solve_begin(kw_ctx* ctx, const double* b_dev, int64_t nshift, const kw_c128* z_host, int64_t nleft,
                             const double* left_dev, void* x_out_dev) {
  if (!has_operator(ctx)) return fail(ctx, KW_ERR_ARG, "kw_solve: no operator has been set");
  if (ctx->rci_active && ctx->rci_iter > 0)
    return fail(ctx, KW_ERR_ARG, "kw_solve: a reverse-communication solve is in progress (kw_rci_finalize first)");
  if (!b_dev || !z_host || nshift < 1 || nshift > 0x7fffffffLL)
    return fail(ctx, KW_ERR_ARG, "kw_solve: need b, z and 1 <= nshift < 2^31");
  if (nleft < 0 || nleft >= KW_MAX_PROJ || (nleft > 0 && !left_dev))
    return fail(ctx, KW_ERR_ARG, "kw_solve: need 0 <= nleft < %d and left vectors when nleft > 0", KW_MAX_PROJ);
  for (int64_t k = 0; k < nshift; ++k)
    if (!isfinite(z_host[k].re) || !isfinite(z_host[k].im))
      return fail(ctx, KW_ERR_ARG, "kw_solve: shift %lld is not finite", (long long)k);
  if (ctx->method == KW_METHOD_CG)
    for (int64_t k = 0; k < nshift; ++k)
      if (z_host[k].im != 0.0)
        return fail(ctx, KW_ERR_ARG, "kw_solve: the CG solver needs real shifts (shift %lld is complex)", (long long)k);
  memset(&ctx->stats, 0, sizeof(ctx->stats));
  ctx->resumable = false;
  ctx->run_maxiter = ctx->opt.maxiter;
  kw_status s = tune_spmv(ctx);
  if (s != KW_OK) return s;
  s = ensure_mv_buffers(ctx);
  if (s != KW_OK) return s;
  s = prepare(ctx, ctx->work, b_dev, nshift, z_host, nleft, left_dev, x_out_dev);
  if (s != KW_OK) return s;
  s = tune_xp_tile(ctx, ctx->work);
  if (s != KW_OK) return s;
  if (ctx->work.full) ctx->last_xp_tile = ctx->work.xp_tile;
  ctx->work_K = nshift;
  cudaError_t ie = init_launch(ctx->work);   // ends with the first K1, which may call the callback
  if (ie != cudaSuccess) {
    if (ctx->work.mv_failed) {
      cudaStreamSynchronize(ctx->stream);
      return fail(ctx, KW_ERR_CALLBACK, "kw_solve: the matrix-vector callback returned nonzero");
    }
    return cuda_fail(ctx, ie, "init kernels");
  }
  ctx->stats.launches += ctx->work.full ? 6 : 5;
  return KW_OK;
}

static const int kChunk = 16;   // iterations per chunk (even: buffer parity repeats)

// Phase 2 for one context: enqueue chunks and poll the device stop flag one
// chunk behind; returns after the stream has drained.
static kw_status run_loop(kw_ctx* ctx, int64_t start = 0) {
  kw::Work& w = ctx->work;
  const bool timing = ctx->timing_every > 0;
  int64_t launched = start;   // iteration number of the next launch (its parity selects the buffers)
  int slot = 0;
  bool have_prev = false;
  int64_t sampled_at[2] = {-1, -1};
  for (;;) {
    sampled_at[slot] = -1;
    for (int i = 0; i < kChunk; ++i) {
      cudaEvent_t* ev = nullptr;
      if (timing && i == 0 && (launched / kChunk) % ctx->timing_every == 0) {
        ev = ctx->kev[slot];
        sampled_at[slot] = launched;
      }
      cudaError_t le = iteration_launch(w, (int)(launched & 1), i == 0, ev, &ctx->stats.launches);
      if (le != cudaSuccess) {
        if (w.mv_failed) {
          cudaStreamSynchronize(ctx->stream);   // let the iterations already enqueued finish
          return fail(ctx, KW_ERR_CALLBACK, "kw_solve: the matrix-vector callback returned nonzero");
        }
        return cuda_fail(ctx, le, "iteration launch");
      }
      ++launched;
    }
    KW_CUDA(kw::join_streams(w), "join streams");
    KW_CUDA(cudaMemcpyAsync(ctx->flags_host + slot, &w.st->done, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream),
            "flag copy");
    KW_CUDA(cudaEventRecord(ctx->ev[slot], ctx->stream), "event record");
    if (have_prev) {
      KW_CUDA(cudaEventSynchronize(ctx->ev[slot ^ 1]), "event sync");
      if (ctx->flags_host[slot ^ 1]) break;
      // the previous chunk ran entirely before the stop flag: its sample is a real iteration
      if (sampled_at[slot ^ 1] >= 0) collect_times(ctx, slot ^ 1, w.full);
    }
    have_prev = true;
    slot ^= 1;
    if (launched > ctx->run_maxiter + 2 * kChunk) break;   // the device stops at maxiter; never loop forever
  }
  KW_CUDA(cudaStreamSynchronize(ctx->stream), "solve sync");
  return KW_OK;
}

// Iterations per trip of the device-side loop (even).  Each trip ends with a
// join of the streams and the loop-condition kernel; 32 against 8 cut the small
// Anderson workload's iteration by 4% and the N=24 chain's by 0.6%; at most 31
// iterations after the stop then launch and return at once.
static const int kGraphChunk = 32;

// Iterations per trip of the device-side loop: 0 when the host loop runs (the
// option is off, kernel timing samples events per chunk, or a callback's work
// may not be capturable).
static int graph_chunk(const kw_ctx* ctx) {
  if (ctx->opt.use_graph <= 0 || ctx->timing_every > 0 || ctx->work.op == kw::OP_CALLBACK || ctx->work.mv_fn)
    return 0;
  const int n = ctx->opt.use_graph == 1 ? kGraphChunk : std::min(ctx->opt.use_graph, 1 << 12);
  return (n + 1) & ~1;
}

// Capture one trip of the device-side loop into the body of a WHILE node:
// `chunk` iterations from parity `parity`, the join of the two streams, and
// the loop condition (stop flag clear, trip cap not reached).
static cudaError_t capture_loop(kw_ctx* ctx, int parity, int chunk, cudaGraph_t* out, int64_t* launches) {
  kw::Work& w = ctx->work;
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaGraphCreate(&g, 0);
  if (e != cudaSuccess) return e;
  cudaGraphConditionalHandle h;
  e = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault);
  cudaGraphNodeParams np = {};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = h;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t node;
  if (e == cudaSuccess) e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np);
  if (e != cudaSuccess) {
    cudaGraphDestroy(g);
    return e;
  }
  cudaGraph_t body = np.conditional.phGraph_out[0];
  const cudaStream_t user = w.stream;
  w.stream = ctx->cap_stream;
  e = cudaStreamBeginCaptureToGraph(w.stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
  if (e == cudaSuccess) {
    int64_t n = 0;
    for (int i = 0; i < chunk && e == cudaSuccess; ++i) e = iteration_launch(w, (parity + i) & 1, i == 0, nullptr, &n);
    if (e == cudaSuccess) e = kw::join_streams(w);
    if (e == cudaSuccess) e = kw::launch_loop_cond(&w.st->done, 1, (unsigned*)ctx->loop.p, h, w.stream);
    *launches = n + 1;
    cudaGraph_t captured = nullptr;   // the body graph itself, owned by the node
    const cudaError_t ee = cudaStreamEndCapture(w.stream, &captured);
    if (e == cudaSuccess) e = ee;
  }
  w.stream = user;
  if (e != cudaSuccess) {
    cudaGraphDestroy(g);
    return e;
  }
  *out = g;
  return cudaSuccess;
}

// Phase 2 on the device: one launch of the loop graph (captured again only
// when the descriptor, the starting parity or the chunk changed); returns
// after the stream has drained.
static kw_status run_graph_loop(kw_ctx* ctx, int64_t start, int chunk) {
  kw::Work& w = ctx->work;
  const int parity = (int)(start & 1);
  if (!ctx->cap_stream) KW_CUDA(cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking), "loop stream");
  if (!ctx->loop_host) KW_CUDA(cudaMallocHost((void**)&ctx->loop_host, 2 * sizeof(unsigned)), "loop alloc");
  if (!ctx->loop.p) {
    KW_CUDA(ctx->loop.ensure(2 * sizeof(unsigned)), "loop alloc");
    if (ctx->loop_exec) cudaGraphExecDestroy(ctx->loop_exec);   // captured with another counter
    ctx->loop_exec = nullptr;
  }
  const bool same = ctx->loop_exec && ctx->loop_parity == parity && ctx->loop_chunk == chunk &&
                    memcmp(&ctx->loop_work, &w, sizeof(kw::Work)) == 0;
  if (!same) {
    if (ctx->loop_exec) cudaGraphExecDestroy(ctx->loop_exec);
    if (ctx->loop_graph) cudaGraphDestroy(ctx->loop_graph);
    ctx->loop_exec = nullptr;
    ctx->loop_graph = nullptr;
    int64_t per_trip = 0;
    KW_CUDA(capture_loop(ctx, parity, chunk, &ctx->loop_graph, &per_trip), "loop graph capture");
    cudaError_t e = cudaGraphInstantiate(&ctx->loop_exec, ctx->loop_graph, 0);
    if (e != cudaSuccess) {
      ctx->loop_exec = nullptr;
      return cuda_fail(ctx, e, "loop graph instantiate");
    }
    memcpy(&ctx->loop_work, &w, sizeof(kw::Work));
    ctx->loop_parity = parity;
    ctx->loop_chunk = chunk;
    ctx->loop_launches = per_trip;
  }
  // trip cap: the device stops at run_maxiter; two trips of slack
  const int64_t left = std::max<int64_t>(ctx->run_maxiter - start, 0);
  ctx->loop_host[0] = 0;
  ctx->loop_host[1] = (unsigned)std::min<int64_t>(left / chunk + 3, 0x7fffffff);
  KW_CUDA(cudaMemcpyAsync(ctx->loop.p, ctx->loop_host, 2 * sizeof(unsigned), cudaMemcpyHostToDevice, ctx->stream),
          "loop counter");
  KW_CUDA(cudaGraphLaunch(ctx->loop_exec, ctx->stream), "loop graph launch");
  KW_CUDA(cudaMemcpyAsync(ctx->loop_host, ctx->loop.p, sizeof(unsigned), cudaMemcpyDeviceToHost, ctx->stream),
          "loop counter");
  KW_CUDA(cudaStreamSynchronize(ctx->stream), "solve sync");
  ctx->stats.launches += (int64_t)ctx->loop_host[0] * ctx->loop_launches;
  return KW_OK;
}

// Phase 2: the device-side loop when it applies, else the host loop.
static kw_status run_iterations(kw_ctx* ctx, int64_t start = 0) {
  const int chunk = graph_chunk(ctx);
  return chunk ? run_graph_loop(ctx, start, chunk) : run_loop(ctx, start);
}

// Phase 3 (the context's stream has drained): outputs and summary.
static kw_status solve_end(kw_ctx* ctx, kw_c128* proj_out_host, kw_solve_info* info) {
  kw::Work& w = ctx->work;
  const int64_t nshift = ctx->work_K;
  if (w.full && w.prec == kw::PREC_DF && !w.xp32) {   // FP32-pair x is converted to FP64 in place (the caller's buffer holds kw_c128)
    KW_CUDA(kw::launch_finish_x<kw::PREC_DF>(w), "finish x");
  }
  KW_CUDA(cudaMemcpyAsync(ctx->st_host, w.st, sizeof(kw::State), cudaMemcpyDeviceToHost, ctx->stream), "read state");
  KW_CUDA(cudaStreamSynchronize(ctx->stream), "state sync");
  const kw::State& st = *ctx->st_host;
  ctx->last_K = nshift;
  ctx->last_nrec = st.n_rec;
  ctx->resumable = st.status == KW_NOT_CONVERGED;
  ctx->last_run = st.iter;
  ctx->last_log_rows = w.log ? std::min<int64_t>(st.iter, w.log_max) : -1;
  ctx->last_log_np = w.nproj;
  ctx->last_thresh = st.thresh;
  if (proj_out_host) {
    if (w.full && !w.xp32) {
      cudaError_t e = w.prec == kw::PREC_C32 ? kw::launch_project_x<kw::PREC_C32>(w, (double2*)ctx->projx.p)
                      : w.prec == kw::PREC_DF ? kw::launch_project_x<kw::PREC_DF>(w, (double2*)ctx->projx.p)
                                              : kw::launch_project_x<kw::PREC_F64>(w, (double2*)ctx->projx.p);
      KW_CUDA(e, "projection of x");
      KW_CUDA(cudaMemcpyAsync(proj_out_host, ctx->projx.p, (size_t)nshift * w.nout * 16, cudaMemcpyDeviceToHost,
                              ctx->stream), "copy projections");
    } else {
      KW_CUDA(cudaMemcpyAsync(proj_out_host, w.Y, (size_t)nshift * w.nout * 16, cudaMemcpyDeviceToHost, ctx->stream),
              "copy projections");
    }
    KW_CUDA(cudaStreamSynchronize(ctx->stream), "projection sync");
  }
  if (info) {
    std::vector<double> res(nshift);
    std::vector<long long> ci(nshift);
    KW_CUDA(cudaMemcpy(res.data(), w.final_res, nshift * 8, cudaMemcpyDeviceToHost), "read residuals");
    KW_CUDA(cudaMemcpy(ci.data(), w.conv_iter, nshift * 8, cudaMemcpyDeviceToHost), "read convergence");
    info->iters = st.iter;
    info->n_seed_switch = st.n_seed_switch;
    info->updates = st.updates;
    info->seed = st.seed;
    info->status = (kw_status)st.status;
    int64_t nc = 0;
    double mx = 0.0;
    for (int64_t k = 0; k < nshift; ++k) {
      nc += ci[k] >= 0;
      mx = std::max(mx, res[k]);
    }
    info->n_converged = nc;
    info->max_res = mx;
  }
  if (st.status != KW_OK) {
    fail(ctx, (kw_status)st.status, "kw_solve: %s after %lld iterations", kw_status_string((kw_status)st.status),
         (long long)st.iter);
  }
  return (kw_status)st.status;
}

extern "C" {

kw_status kw_solve(kw_ctx* ctx, const double* b_dev, int64_t nshift, const kw_c128* z_host, int64_t nleft,
                   const double* left_dev, void* x_out_dev, kw_c128* proj_out_host, kw_solve_info* info) {
  if (!ctx) return KW_ERR_ARG;
  kw_status s = solve_begin(ctx, b_dev, nshift, z_host, nleft, left_dev, x_out_dev);
  if (s != KW_OK) return s;
  s = run_iterations(ctx);
  if (s != KW_OK) return s;
  return solve_end(ctx, proj_out_host, info);
}

static void rci_io(kw_ctx* ctx, kw_rci_io* io) {
  if (!io) return;
  const kw::Work& w = ctx->work;
  io->r = w.rci_r;
  io->q = w.rci_q;
  io->rt = w.method == KW_METHOD_BICG ? w.rci_rt : nullptr;
  io->qt = w.method == KW_METHOD_BICG ? w.rci_qt : nullptr;
  io->elem = ctx->opt.prec == KW_C32V_F64S ? KW_ELEM_C64 : KW_ELEM_C128;
}

kw_status kw_rci_init(kw_ctx* ctx, int64_t m, const double* b_dev, int64_t nshift, const kw_c128* z_host,
                      int64_t nleft, const double* left_dev, void* x_out_dev, kw_rci_io* io) {
  if (!ctx) return KW_ERR_ARG;
  if (m < 1 || m > KW_MAX_ROWS || !io) return fail(ctx, KW_ERR_ARG, "kw_rci_init: need 1 <= m <= KW_MAX_ROWS and io");
  // the caller is the operator from now on
  ctx->op = kw::OP_CALLBACK;
  ctx->m = m;
  ctx->nnz = 0;
  ctx->rowptr = nullptr;
  ctx->col = nullptr;
  ctx->val = nullptr;
  ctx->mv_fn = nullptr;
  ctx->mv_user = nullptr;
  ctx->mv_fn_adj = nullptr;
  ctx->mv_user_adj = nullptr;
  ctx->spmv_lanes = 1;
  ctx->u_state = 0;
  ctx->us_state = 0;
  ctx->sell_built = false;
  ctx->resumable = false;
  ctx->rci_active = true;
  if (ctx->opt.prec == KW_DF64) {
    KW_CUDA(ctx->mv_r.ensure((size_t)m * 16), "kw_rci_init: staging");
    KW_CUDA(ctx->mv_q.ensure((size_t)m * 16), "kw_rci_init: staging");
    if (ctx->method == KW_METHOD_BICG) {
      KW_CUDA(ctx->mv_r2.ensure((size_t)m * 16), "kw_rci_init: staging");
      KW_CUDA(ctx->mv_q2.ensure((size_t)m * 16), "kw_rci_init: staging");
    }
  }
  kw_status s = solve_begin(ctx, b_dev, nshift, z_host, nleft, left_dev, x_out_dev);
  if (s != KW_OK) {
    ctx->rci_active = false;
    return s;
  }
  KW_CUDA(cudaStreamSynchronize(ctx->stream), "kw_rci_init: sync");
  ctx->rci_iter = 0;
  rci_io(ctx, io);
  return KW_OK;
}

kw_status kw_rci_update(kw_ctx* ctx, int* done, kw_rci_io* io) {
  if (!ctx || !done) return KW_ERR_ARG;
  if (!ctx->rci_active) return fail(ctx, KW_ERR_ARG, "kw_rci_update: no kw_rci_init");
  kw::Work& w = ctx->work;
  const int64_t n = ctx->rci_iter;
  // finish iteration n's products (the caller wrote them), then K2, K3, K4 and the staging of r_{n+1}
  w.rci_phase = 2;
  void* rn = (n & 1) ? w.rB : w.rA;
  void* rtn = (n & 1) ? w.rtB : w.rtA;
  cudaError_t e = w.prec == kw::PREC_C32 ? kw::launch_k1<kw::PREC_C32>(w, rn, rtn)
                  : w.prec == kw::PREC_DF ? kw::launch_k1<kw::PREC_DF>(w, rn, rtn)
                                          : kw::launch_k1<kw::PREC_F64>(w, rn, rtn);
  w.rci_phase = 1;
  KW_CUDA(e, "kw_rci_update: products");
  KW_CUDA(iteration_launch(w, (int)(n & 1), 1, nullptr, &ctx->stats.launches), "kw_rci_update: iteration");
  int d = 0;
  KW_CUDA(cudaMemcpyAsync(&d, &w.st->done, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream), "kw_rci_update");
  KW_CUDA(cudaStreamSynchronize(ctx->stream), "kw_rci_update: sync");
  ctx->rci_iter = n + 1;
  *done = d;
  rci_io(ctx, io);
  return KW_OK;
}

kw_status kw_rci_get_residual(kw_ctx* ctx, double* res_host) {
  if (!ctx || !res_host) return KW_ERR_ARG;
  if (!ctx->rci_active) return fail(ctx, KW_ERR_ARG, "kw_rci_get_residual: no kw_rci_init");
  KW_CUDA(cudaMemcpy(res_host, ctx->work.final_res, (size_t)ctx->work_K * 8, cudaMemcpyDeviceToHost),
          "kw_rci_get_residual");
  return KW_OK;
}

kw_status kw_rci_finalize(kw_ctx* ctx, kw_c128* proj_out_host, kw_solve_info* info) {
  if (!ctx) return KW_ERR_ARG;
  if (!ctx->rci_active) return fail(ctx, KW_ERR_ARG, "kw_rci_finalize: no kw_rci_init");
  ctx->rci_active = false;
  kw_status s = solve_end(ctx, proj_out_host, info);
  ctx->resumable = false;
  ctx->op = kw::OP_CSR;   // no operator until the next kw_set_*
  ctx->m = 0;
  return s;
}

kw_status kw_resume(kw_ctx* ctx, int64_t more_iters, kw_c128* proj_out_host, kw_solve_info* info) {
  if (!ctx) return KW_ERR_ARG;
  if (more_iters < 1) return fail(ctx, KW_ERR_ARG, "kw_resume: more_iters < 1");
  if (!ctx->resumable)
    return fail(ctx, KW_ERR_ARG, "kw_resume: the last kw_solve of this context did not stop at maxiter, or its "
                                 "operator, method or workspace has changed since");
  kw::Work& w = ctx->work;
  const kw::State& sh = *ctx->st_host;   // read back by the last solve_end
  const int64_t it = sh.iter;
  ctx->resumable = false;
  ctx->run_maxiter = it + more_iters;
  memset(&ctx->stats, 0, sizeof(ctx->stats));
  if (w.full && w.prec == kw::PREC_DF && !w.xp32) {   // x was handed out as kw_c128: back to FP32 pairs
    KW_CUDA(kw::launch_unfinish_x<kw::PREC_DF>(w), "kw_resume: x to pairs");
  }
  // restart the device loop: new cap, stop flag cleared, K1 counter reset
  long long maxit = (long long)ctx->run_maxiter;
  const int zero = 0, notconv = KW_NOT_CONVERGED;
  const unsigned int uzero = 0;
  KW_CUDA(cudaMemcpyAsync(&w.st->maxiter, &maxit, sizeof(maxit), cudaMemcpyHostToDevice, ctx->stream), "kw_resume");
  KW_CUDA(cudaMemcpyAsync(&w.st->done, &zero, sizeof(int), cudaMemcpyHostToDevice, ctx->stream), "kw_resume");
  KW_CUDA(cudaMemcpyAsync(&w.st->status, &notconv, sizeof(int), cudaMemcpyHostToDevice, ctx->stream), "kw_resume");
  KW_CUDA(cudaMemcpyAsync(&w.st->cnt_spmv, &uzero, sizeof(uzero), cudaMemcpyHostToDevice, ctx->stream), "kw_resume");
  // K1 of iteration `it` again: the one queued after the last K2 may have seen the stop flag
  void* rn = (it & 1) ? w.rB : w.rA;
  void* rtn = (it & 1) ? w.rtB : w.rtA;
  cudaError_t e = w.prec == kw::PREC_C32 ? kw::launch_k1<kw::PREC_C32>(w, rn, rtn)
                  : w.prec == kw::PREC_DF ? kw::launch_k1<kw::PREC_DF>(w, rn, rtn)
                                          : kw::launch_k1<kw::PREC_F64>(w, rn, rtn);
  if (e != cudaSuccess) {
    if (w.mv_failed) {
      cudaStreamSynchronize(ctx->stream);
      return fail(ctx, KW_ERR_CALLBACK, "kw_resume: the matrix-vector callback returned nonzero");
    }
    return cuda_fail(ctx, e, "kw_resume: first product");
  }
  kw_status s = run_iterations(ctx, it);
  if (s != KW_OK) return s;
  return solve_end(ctx, proj_out_host, info);
}

kw_status kw_solve_batched(kw_ctx* ctx, int64_t n, const kw_instance* inst, kw_solve_info* info) {
  if (!ctx) return KW_ERR_ARG;
  if (n < 1 || n > 65536 || !inst) return fail(ctx, KW_ERR_ARG, "kw_solve_batched: need 1 <= n <= 65536 instances");
  // the caller's stream may be the legacy default stream, which cannot be
  // captured: the batch runs on an own stream ordered after the caller's work
  if (!ctx->batch_stream)
    KW_CUDA(cudaStreamCreateWithFlags(&ctx->batch_stream, cudaStreamNonBlocking), "kw_solve_batched: stream");
  cudaStream_t bs = ctx->batch_stream;
  ctx->last_log_rows = -1;   // the instances run on child contexts, which keep no log
  ctx->resumable = false;
  {
    cudaEvent_t e0;
    KW_CUDA(cudaEventCreateWithFlags(&e0, cudaEventDisableTiming), "kw_solve_batched: event");
    cudaError_t e = cudaEventRecord(e0, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(bs, e0, 0);
    cudaEventDestroy(e0);
    KW_CUDA(e, "kw_solve_batched: order after the caller's stream");
  }
  // child contexts, one stream each
  while ((int64_t)ctx->children.size() < n) {
    cudaStream_t s = nullptr;
    KW_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking), "kw_solve_batched: stream");
    kw_ctx* c = nullptr;
    kw_status cs = kw_create(&c, &ctx->opt, s);
    if (cs != KW_OK) {
      cudaStreamDestroy(s);
      return fail(ctx, cs, "kw_solve_batched: child context");
    }
    c->owns_stream = true;
    ctx->children.push_back(c);
  }
  // begin every instance on its own stream; the batch stream waits for all initialisations
  ScopedEvents ev;
  KW_CUDA(ev.create((size_t)n + 1, cudaEventDisableTiming), "batch events");
  kw_status result = KW_OK;
  KW_CUDA(cudaEventRecord(ev[n], bs), "batch event");   // instances start after the caller's work
  for (int64_t i = 0; i < n; ++i) {
    kw_ctx* c = ctx->children[i];
    c->opt = ctx->opt;
    c->method = ctx->method;   // BiCG instances start their shadow from b
    c->btilde = nullptr;
    c->overlap = ctx->overlap;
    c->bulk = ctx->bulk;
    c->xp32 = ctx->xp32;
    c->seed_rg = ctx->seed_rg;
    c->force_xp_tile = ctx->force_xp_tile;
    if (inst[i].tol > 0.0) c->opt.tol = inst[i].tol;
    c->run_maxiter = c->opt.maxiter;
    KW_CUDA(cudaStreamWaitEvent(c->stream, ev[n], 0), "batch wait");
    kw_status s = kw_set_csr(c, inst[i].m, inst[i].nnz, inst[i].rowptr_dev, inst[i].col_dev, inst[i].val_dev);
    if (s == KW_OK)
      s = solve_begin(c, inst[i].b_dev, inst[i].nshift, inst[i].z_host, inst[i].nleft, inst[i].left_dev,
                      inst[i].x_out_dev);
    if (s != KW_OK) {
      return fail(ctx, s, "kw_solve_batched: instance %lld: %s", (long long)i, c->err);
    }
    KW_CUDA(cudaEventRecord(ev[i], c->stream), "batch event");
    KW_CUDA(cudaStreamWaitEvent(bs, ev[i], 0), "batch wait");
  }
  // device list of the instances' states for the done counter
  std::vector<kw::State*> sts(n);
  for (int64_t i = 0; i < n; ++i) sts[i] = ctx->children[i]->work.st;
  KW_CUDA(ctx->child_states.ensure((size_t)n * sizeof(void*)), "batch alloc");
  KW_CUDA(ctx->done_count.ensure(sizeof(int)), "batch alloc");
  if (!ctx->done_host) KW_CUDA(cudaMallocHost((void**)&ctx->done_host, 2 * sizeof(int)), "batch alloc");
  KW_CUDA(cudaMemcpyAsync(ctx->child_states.p, sts.data(), (size_t)n * sizeof(void*), cudaMemcpyHostToDevice,
                          bs), "batch upload");
  KW_CUDA(cudaStreamSynchronize(bs), "batch sync");
  // One graph: a chunk of iterations of every instance (fork/join over the
  // instance streams), then the count of finished instances.  With the
  // device-side loop the chunk is the body of a WHILE node that repeats until
  // every instance has stopped; otherwise the host relaunches it per chunk.
  const int gchunk = graph_chunk(ctx);
  const int chunk = gchunk ? gchunk : kChunk;
  int64_t maxit = ctx->opt.maxiter;
  for (int64_t i = 0; i < n; ++i) maxit = std::max<int64_t>(maxit, ctx->children[i]->opt.maxiter);
  if (gchunk) {
    if (!ctx->loop_host) KW_CUDA(cudaMallocHost((void**)&ctx->loop_host, 2 * sizeof(unsigned)), "loop alloc");
    if (!ctx->loop.p) {
      KW_CUDA(ctx->loop.ensure(2 * sizeof(unsigned)), "loop alloc");
      if (ctx->loop_exec) cudaGraphExecDestroy(ctx->loop_exec);   // captured with another counter
      ctx->loop_exec = nullptr;
    }
  }
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaGraph_t body = nullptr;
  cudaGraphConditionalHandle h = 0;
  cudaError_t ce = cudaSuccess;
  if (gchunk) {
    ce = cudaGraphCreate(&graph, 0);
    if (ce == cudaSuccess) ce = cudaGraphConditionalHandleCreate(&h, graph, 1, cudaGraphCondAssignDefault);
    cudaGraphNodeParams np = {};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    if (ce == cudaSuccess) ce = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &np);
    if (ce == cudaSuccess) body = np.conditional.phGraph_out[0];
    if (ce == cudaSuccess) ce = cudaStreamBeginCaptureToGraph(bs, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
  } else {
    ce = cudaStreamBeginCapture(bs, cudaStreamCaptureModeRelaxed);
  }
  if (ce != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return cuda_fail(ctx, ce, "kw_solve_batched: graph capture");
  }
  ce = cudaEventRecord(ev[n], bs);
  int64_t per_trip = 0;
  for (int64_t i = 0; i < n && ce == cudaSuccess; ++i) {
    kw_ctx* c = ctx->children[i];
    ce = cudaStreamWaitEvent(c->stream, ev[n], 0);
    for (int it = 0; it < chunk && ce == cudaSuccess; ++it)
      ce = iteration_launch(c->work, it & 1, it == 0, nullptr, &per_trip);
    if (ce == cudaSuccess) ce = kw::join_streams(c->work);
    if (ce == cudaSuccess) ce = cudaEventRecord(ev[i], c->stream);
    if (ce == cudaSuccess) ce = cudaStreamWaitEvent(bs, ev[i], 0);
  }
  if (ce == cudaSuccess) ce = kw::launch_count_done((int)n, (kw::State* const*)ctx->child_states.p,
                                                   (int*)ctx->done_count.p, bs);
  if (gchunk) {
    if (ce == cudaSuccess) ce = kw::launch_loop_cond((const int*)ctx->done_count.p, (int)n, (unsigned*)ctx->loop.p, h, bs);
    cudaGraph_t captured = nullptr;   // the body graph itself, owned by the node
    const cudaError_t ee = cudaStreamEndCapture(bs, &captured);
    if (ce == cudaSuccess) ce = ee;
  } else {
    if (ce == cudaSuccess)
      ce = cudaMemcpyAsync(ctx->done_host, ctx->done_count.p, sizeof(int), cudaMemcpyDeviceToHost, bs);
    const cudaError_t ee = cudaStreamEndCapture(bs, &graph);
    if (ce == cudaSuccess) ce = ee;
  }
  if (ce == cudaSuccess) ce = cudaGraphInstantiate(&exec, graph, 0);
  if (ce != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return cuda_fail(ctx, ce, "kw_solve_batched: graph capture");
  }
  int64_t trips = 0;
  if (gchunk) {   // one launch; the trip cap stops the loop even if an instance never raises its flag
    ctx->loop_host[0] = 0;
    ctx->loop_host[1] = (unsigned)std::min<int64_t>(maxit / chunk + 3, 0x7fffffff);
    ce = cudaMemcpyAsync(ctx->loop.p, ctx->loop_host, 2 * sizeof(unsigned), cudaMemcpyHostToDevice, bs);
    if (ce == cudaSuccess) ce = cudaGraphLaunch(exec, bs);
    if (ce == cudaSuccess)
      ce = cudaMemcpyAsync(ctx->loop_host, ctx->loop.p, sizeof(unsigned), cudaMemcpyDeviceToHost, bs);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(bs);
    if (ce == cudaSuccess) trips = ctx->loop_host[0];
  } else {
    for (;;) {
      ce = cudaGraphLaunch(exec, bs);
      if (ce != cudaSuccess) break;
      ++trips;
      ce = cudaStreamSynchronize(bs);   // one chunk of the whole batch per graph launch
      if (ce != cudaSuccess) break;
      if (*(volatile int*)ctx->done_host >= n) break;
      if (trips * chunk > maxit + 2 * chunk) break;   // every instance stops at its maxiter
    }
  }
  cudaGraphExecDestroy(exec);
  cudaGraphDestroy(graph);
  if (ce != cudaSuccess) return cuda_fail(ctx, ce, "kw_solve_batched: graph launch");
  for (int64_t i = 0; i < n; ++i) {
    kw_ctx* c = ctx->children[i];
    c->stats.launches += trips * chunk * (c->work.full ? 4 : 3);   // per iteration: K2, K1, K3 (+K4)
    kw_status s = solve_end(c, inst[i].proj_out_host, info ? &info[i] : nullptr);
    if (s != KW_OK && result == KW_OK) {
      result = s;
      fail(ctx, s, "kw_solve_batched: instance %lld: %s", (long long)i, c->err);
    }
  }
  ctx->stats.launches = trips * (per_trip + (gchunk ? 2 : 1));   // every instance's kernels, the count (+ condition)
  {   // the caller's stream is ordered after the batch
    cudaEvent_t e1;
    KW_CUDA(cudaEventCreateWithFlags(&e1, cudaEventDisableTiming), "kw_solve_batched: event");
    cudaError_t e = cudaEventRecord(e1, bs);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->stream, e1, 0);
    cudaEventDestroy(e1);
    KW_CUDA(e, "kw_solve_batched: order the caller's stream");
  }
  return result;
}

kw_status kw_solve_host(kw_ctx* ctx, int64_t m, int64_t nnz, const int64_t* rowptr_host, const int32_t* col_host,
                        const double* val_host, const double* b_host, int64_t nshift, const kw_c128* z_host,
                        int64_t nleft, const double* left_host, void* x_out_host, kw_c128* proj_out_host,
                        kw_solve_info* info) {
  if (!ctx) return KW_ERR_ARG;
  if (m < 1 || nnz < 0 || !rowptr_host || (nnz > 0 && (!col_host || !val_host)) || !b_host || nshift < 1 ||
      nleft < 0 || (nleft > 0 && !left_host))
    return fail(ctx, KW_ERR_ARG, "kw_solve_host: invalid sizes or NULL host arrays");
  // x element: complex FP32 under FP32 shift storage (or in the FP32 form), else 16 bytes
  const size_t vs = (ctx->xp32 && ctx->opt.prec != KW_C32V_F64S) ? 8 : vec_bytes(ctx->opt.prec);
  KW_CUDA(ctx->h_rowptr.ensure((m + 1) * 8), "alloc rowptr");
  KW_CUDA(ctx->h_col.ensure(std::max<int64_t>(nnz, 1) * 4), "alloc col");
  KW_CUDA(ctx->h_val.ensure(std::max<int64_t>(nnz, 1) * 8), "alloc val");
  KW_CUDA(ctx->h_b.ensure(m * 8), "alloc b");
  KW_CUDA(ctx->h_left.ensure(std::max<int64_t>(nleft * m, 1) * 8), "alloc left");
  if (x_out_host) KW_CUDA(ctx->h_x.ensure((size_t)nshift * m * vs), "alloc x");
  cudaStream_t s = ctx->stream;
  KW_CUDA(cudaMemcpyAsync(ctx->h_rowptr.p, rowptr_host, (m + 1) * 8, cudaMemcpyHostToDevice, s), "copy rowptr");
  if (nnz > 0) {
    KW_CUDA(cudaMemcpyAsync(ctx->h_col.p, col_host, nnz * 4, cudaMemcpyHostToDevice, s), "copy col");
    KW_CUDA(cudaMemcpyAsync(ctx->h_val.p, val_host, nnz * 8, cudaMemcpyHostToDevice, s), "copy val");
  }
  KW_CUDA(cudaMemcpyAsync(ctx->h_b.p, b_host, m * 8, cudaMemcpyHostToDevice, s), "copy b");
  if (nleft > 0) KW_CUDA(cudaMemcpyAsync(ctx->h_left.p, left_host, nleft * m * 8, cudaMemcpyHostToDevice, s), "copy left");
  kw_status st = kw_set_csr(ctx, m, nnz, (const int64_t*)ctx->h_rowptr.p, (const int32_t*)ctx->h_col.p,
                            (const double*)ctx->h_val.p);
  if (st != KW_OK) return st;
  st = kw_solve(ctx, (const double*)ctx->h_b.p, nshift, z_host, nleft, nleft > 0 ? (const double*)ctx->h_left.p : nullptr,
                x_out_host ? ctx->h_x.p : nullptr, proj_out_host, info);
  ctx->resumable = false;   // its outputs went to host memory: kw_resume is for kw_solve
  if (x_out_host && (st == KW_OK || st == KW_NOT_CONVERGED || st == KW_ERR_BREAKDOWN || st == KW_ERR_NONFINITE))
    KW_CUDA(cudaMemcpy(x_out_host, ctx->h_x.p, (size_t)nshift * m * vs, cudaMemcpyDeviceToHost), "copy x");
  return st;
}

kw_status kw_get_shift_status(kw_ctx* ctx, int64_t* conv_iter_host, double* final_res_host) {
  if (!ctx) return KW_ERR_ARG;
  if (ctx->last_K == 0) return fail(ctx, KW_ERR_ARG, "kw_get_shift_status: no solve yet");
  if (conv_iter_host)
    KW_CUDA(cudaMemcpy(conv_iter_host, ctx->conv_iter.p, ctx->last_K * 8, cudaMemcpyDeviceToHost), "read conv_iter");
  if (final_res_host)
    KW_CUDA(cudaMemcpy(final_res_host, ctx->final_res.p, ctx->last_K * 8, cudaMemcpyDeviceToHost), "read final_res");
  return KW_OK;
}

kw_status kw_get_residual_history(kw_ctx* ctx, double* hist_host, int64_t* n_rec) {
  if (!ctx || !n_rec) return KW_ERR_ARG;
  *n_rec = ctx->last_nrec;
  if (hist_host && ctx->last_nrec > 0)
    KW_CUDA(cudaMemcpy(hist_host, ctx->hist.p, (size_t)ctx->last_nrec * ctx->last_K * 8, cudaMemcpyDeviceToHost),
            "read history");
  return KW_OK;
}

static kw_status bilinear(kw_ctx* ctx, const char* name, int64_t m, int64_t nterm, const kw_csr_term* terms,
                          int64_t nshift, const void* X_dev, const void* Y_dev, int x32, kw_c128* out_host) {
  if (!ctx) return KW_ERR_ARG;
  if (m < 1 || m > KW_MAX_ROWS || nterm < 1 || nshift < 1 || nshift > KW_BILINEAR_MAX_SHIFTS || !terms || !X_dev ||
      !out_host)
    return fail(ctx, KW_ERR_ARG, "%s: invalid sizes or NULL pointer", name);
  for (int64_t t = 0; t < nterm; ++t)
    if (!terms[t].rowptr_dev || terms[t].nnz < 0 || terms[t].nnz > KW_MAX_NNZ ||
        (terms[t].nnz > 0 && (!terms[t].col_dev || !terms[t].val_dev)))
      return fail(ctx, KW_ERR_ARG, "%s: term %lld is invalid", name, (long long)t);
  const int nblk = 2 * ctx->num_sms;
  const int64_t ntile = (nshift + kw::kBilinearTile - 1) / kw::kBilinearTile;
  // diagonal path: blocks per shift so that all shifts together fill the device about four times
  const int dblk = (int)std::max<int64_t>(1, std::min<int64_t>((m + 255) / 256, (4 * ctx->num_sms + nshift - 1) / nshift));
  const size_t part_bytes = std::max((size_t)ntile * nblk * kw::kBilinearTile, (size_t)nshift * dblk * kw::kDiagGroup) * 16;
  KW_CUDA(ctx->bil_part.ensure(part_bytes), "kw_bilinear: scratch");
  KW_CUDA(ctx->bil_out.ensure((size_t)nshift * nterm * 16), "kw_bilinear: result");
  KW_CUDA(ctx->bil_diag.ensure((size_t)nterm * m * 8), "kw_bilinear: diagonals");
  KW_CUDA(ctx->bil_flag.ensure((size_t)nterm * 4), "kw_bilinear: flags");
  // which terms hold only diagonal entries (each such term then costs one FMA pair per shift and row
  // in a shared pass over X and Y, instead of a pass of its own)
  KW_CUDA(cudaMemsetAsync(ctx->bil_flag.p, 1, (size_t)nterm * 4, ctx->stream), "kw_bilinear: flags");
  double* dg = (double*)ctx->bil_diag.p;
  int* flag = (int*)ctx->bil_flag.p;
  for (int64_t t = 0; t < nterm; ++t)
    KW_CUDA(kw::launch_diag_scan((int)m, terms[t].rowptr_dev, terms[t].col_dev, terms[t].val_dev, dg + t * m,
                                 flag + t, ctx->num_sms, ctx->stream),
            "kw_bilinear: structure");
  std::vector<int> is_diag((size_t)nterm);
  KW_CUDA(cudaMemcpyAsync(is_diag.data(), flag, (size_t)nterm * 4, cudaMemcpyDeviceToHost, ctx->stream),
          "kw_bilinear: flags");
  KW_CUDA(cudaStreamSynchronize(ctx->stream), "kw_bilinear: flags");
  const void* Y = Y_dev ? Y_dev : X_dev;
  kw::DiagGroup g;
  g.n = 0;
  auto flush = [&]() -> cudaError_t {
    if (g.n == 0) return cudaSuccess;
    cudaError_t e = kw::launch_bilinear_diag((int)m, (int)nshift, dg, g, X_dev, Y, x32, dblk,
                                             (double2*)ctx->bil_part.p, (int)nterm, (double2*)ctx->bil_out.p,
                                             ctx->stream);
    g.n = 0;
    return e;
  };
  for (int64_t t = 0; t < nterm; ++t) {
    if (is_diag[(size_t)t]) {
      g.idx[g.n++] = (int)t;
      if (g.n == kw::kDiagGroup) KW_CUDA(flush(), "kw_bilinear launch");
      continue;
    }
    KW_CUDA(kw::launch_bilinear((int)m, (int)nshift, terms[t].rowptr_dev, terms[t].col_dev, terms[t].val_dev, X_dev,
                                Y, x32, nblk, (double2*)ctx->bil_part.p, (int)t, (int)nterm,
                                (double2*)ctx->bil_out.p, ctx->stream),
            "kw_bilinear launch");
  }
  KW_CUDA(flush(), "kw_bilinear launch");
  KW_CUDA(cudaMemcpyAsync(out_host, ctx->bil_out.p, (size_t)nshift * nterm * 16, cudaMemcpyDeviceToHost, ctx->stream),
          "kw_bilinear read");
  KW_CUDA(cudaStreamSynchronize(ctx->stream), "kw_bilinear sync");
  return KW_OK;
}

kw_status kw_bilinear(kw_ctx* ctx, int64_t m, int64_t nterm, const kw_csr_term* terms, int64_t nshift,
                      const kw_c128* X_dev, const kw_c128* Y_dev, kw_c128* out_host) {
  return bilinear(ctx, "kw_bilinear", m, nterm, terms, nshift, X_dev, Y_dev, 0, out_host);
}

kw_status kw_bilinear_c64(kw_ctx* ctx, int64_t m, int64_t nterm, const kw_csr_term* terms, int64_t nshift,
                          const void* X_dev, const void* Y_dev, kw_c128* out_host) {
  return bilinear(ctx, "kw_bilinear_c64", m, nterm, terms, nshift, X_dev, Y_dev, 1, out_host);
}

kw_status kw_shift_combine(kw_ctx* ctx, int64_t m, int64_t nshift, const void* X_dev, int x_elem, int64_t nk,
                           const kw_c128* W_host, kw_c128* S_dev) {
  if (!ctx) return KW_ERR_ARG;
  if (m < 1 || m > KW_MAX_ROWS || nshift < 1 || nshift > 0x7fffffffLL || nk < 1 || nk > kw::kMaxCombine || !X_dev ||
      !W_host || !S_dev || (x_elem != KW_ELEM_C128 && x_elem != KW_ELEM_C64))
    return fail(ctx, KW_ERR_ARG, "kw_shift_combine: invalid sizes, element type or NULL pointer");
  KW_CUDA(ctx->comb_w.ensure((size_t)nk * nshift * 16), "kw_shift_combine: weights");
  KW_CUDA(cudaMemcpyAsync(ctx->comb_w.p, W_host, (size_t)nk * nshift * 16, cudaMemcpyHostToDevice, ctx->stream),
          "kw_shift_combine: upload");
  KW_CUDA(kw::launch_shift_combine((int)m, (int)nshift, (int)nk, X_dev, x_elem == KW_ELEM_C64 ? 1 : 0,
                                   (const double2*)ctx->comb_w.p, (double2*)S_dev, ctx->num_sms, ctx->stream),
          "kw_shift_combine: launch");
  KW_CUDA(cudaStreamSynchronize(ctx->stream), "kw_shift_combine: sync");
  return KW_OK;
}

kw_status kw_set_krylov_log(kw_ctx* ctx, int64_t max_iters) {
  if (!ctx) return KW_ERR_ARG;
  if (max_iters < 0) return fail(ctx, KW_ERR_ARG, "kw_set_krylov_log: max_iters < 0");
  ctx->log_max = max_iters;
  if (max_iters == 0) {
    KW_CUDA(cudaStreamSynchronize(ctx->stream), "kw_set_krylov_log: sync");
    ctx->klog.release();
    ctx->last_log_rows = -1;
  }
  return KW_OK;
}

kw_status kw_get_krylov_log(kw_ctx* ctx, int64_t* n_iter, int64_t* n_run, int64_t* nproj, double* thresh,
                            kw_c128* log_host, kw_c128* w0_host) {
  if (!ctx) return KW_ERR_ARG;
  if (ctx->last_log_rows < 0) return fail(ctx, KW_ERR_ARG, "kw_get_krylov_log: the last solve recorded no log");
  const int64_t rows = ctx->last_log_rows;
  const int np = ctx->last_log_np;
  if (n_iter) *n_iter = rows;
  if (n_run) *n_run = ctx->last_run;
  if (nproj) *nproj = np;
  if (thresh) *thresh = ctx->last_thresh;
  if (log_host && rows > 0)
    KW_CUDA(cudaMemcpy(log_host, ctx->klog.p, (size_t)rows * (KW_LOG_FIXED + np) * 16, cudaMemcpyDeviceToHost),
            "kw_get_krylov_log: read log");
  if (w0_host && np > 0)
    KW_CUDA(cudaMemcpy(w0_host, ctx->w0.p, (size_t)np * 16, cudaMemcpyDeviceToHost), "kw_get_krylov_log: read w0");
  return KW_OK;
}

kw_status kw_recalc(kw_ctx* ctx, int64_t n_iter, int64_t nproj, double thresh, const kw_c128* log_host,
                    const kw_c128* w0_host, int64_t nshift, const kw_c128* z_host, kw_c128* proj_out_host,
                    int64_t* conv_iter_host, double* final_res_host, kw_solve_info* info) {
  if (!ctx) return KW_ERR_ARG;
  if (!z_host || nshift < 1 || nshift > 0x7fffffffLL)
    return fail(ctx, KW_ERR_ARG, "kw_recalc: need z and 1 <= nshift < 2^31");
  for (int64_t k = 0; k < nshift; ++k)
    if (!isfinite(z_host[k].re) || !isfinite(z_host[k].im))
      return fail(ctx, KW_ERR_ARG, "kw_recalc: shift %lld is not finite", (long long)k);
  if (isnan(thresh)) return fail(ctx, KW_ERR_ARG, "kw_recalc: thresh is NaN");
  int64_t rows;
  int np;
  const double2* dlog;
  const double2* dw0;
  if (log_host) {
    if (n_iter < 0 || nproj < 0 || nproj > KW_MAX_PROJ || (nproj > 0 && !w0_host))
      return fail(ctx, KW_ERR_ARG, "kw_recalc: need n_iter >= 0, 0 <= nproj <= %d and w0 when nproj > 0",
                  KW_MAX_PROJ);
    rows = n_iter;
    np = (int)nproj;
    const size_t lb = (size_t)rows * (KW_LOG_FIXED + np) * 16;
    KW_CUDA(ctx->rc_log.ensure(std::max<size_t>(lb, 16)), "kw_recalc: allocation");
    KW_CUDA(ctx->rc_w0.ensure((size_t)std::max(np, 1) * 16), "kw_recalc: allocation");
    if (lb) KW_CUDA(cudaMemcpyAsync(ctx->rc_log.p, log_host, lb, cudaMemcpyHostToDevice, ctx->stream), "kw_recalc: upload");
    if (np)
      KW_CUDA(cudaMemcpyAsync(ctx->rc_w0.p, w0_host, (size_t)np * 16, cudaMemcpyHostToDevice, ctx->stream),
              "kw_recalc: upload");
    dlog = (const double2*)ctx->rc_log.p;
    dw0 = (const double2*)ctx->rc_w0.p;
  } else {
    if (ctx->last_log_rows < 0) return fail(ctx, KW_ERR_ARG, "kw_recalc: no log given and the last solve recorded none");
    rows = (n_iter < 0 || n_iter > ctx->last_log_rows) ? ctx->last_log_rows : n_iter;
    np = ctx->last_log_np;
    dlog = (const double2*)ctx->klog.p;
    dw0 = (const double2*)ctx->w0.p;
  }
  const size_t K = (size_t)nshift;
  KW_CUDA(ctx->rc_z.ensure(K * 16), "kw_recalc: allocation");
  KW_CUDA(ctx->rc_proj.ensure(K * std::max(np, 1) * 16), "kw_recalc: allocation");
  KW_CUDA(ctx->rc_conv.ensure(K * 8), "kw_recalc: allocation");
  KW_CUDA(ctx->rc_res.ensure(K * 8), "kw_recalc: allocation");
  KW_CUDA(ctx->rc_flag.ensure(4), "kw_recalc: allocation");
  KW_CUDA(cudaMemcpyAsync(ctx->rc_z.p, z_host, K * 16, cudaMemcpyHostToDevice, ctx->stream), "kw_recalc: upload");
  KW_CUDA(cudaMemsetAsync(ctx->rc_flag.p, 0, 4, ctx->stream), "kw_recalc: memset");
  KW_CUDA(kw::launch_recalc((int)nshift, np, (long long)rows, dlog, dw0, (const double2*)ctx->rc_z.p,
                            thresh > 0.0 ? thresh : -1.0, (double2*)ctx->rc_proj.p, (long long*)ctx->rc_conv.p,
                            (double*)ctx->rc_res.p, (int*)ctx->rc_flag.p, ctx->num_sms, ctx->stream),
          "kw_recalc: launch");
  ctx->stats.launches += 1;
  std::vector<long long> ci(K);
  std::vector<double> res(K);
  int flag = 0;
  KW_CUDA(cudaMemcpyAsync(ci.data(), ctx->rc_conv.p, K * 8, cudaMemcpyDeviceToHost, ctx->stream), "kw_recalc: read");
  KW_CUDA(cudaMemcpyAsync(res.data(), ctx->rc_res.p, K * 8, cudaMemcpyDeviceToHost, ctx->stream), "kw_recalc: read");
  KW_CUDA(cudaMemcpyAsync(&flag, ctx->rc_flag.p, 4, cudaMemcpyDeviceToHost, ctx->stream), "kw_recalc: read");
  if (proj_out_host && np > 0)
    KW_CUDA(cudaMemcpyAsync(proj_out_host, ctx->rc_proj.p, K * np * 16, cudaMemcpyDeviceToHost, ctx->stream),
            "kw_recalc: read");
  KW_CUDA(cudaStreamSynchronize(ctx->stream), "kw_recalc: sync");
  int64_t nc = 0, upd = 0;
  double mx = 0.0;
  for (size_t k = 0; k < K; ++k) {
    nc += ci[k] >= 0;
    upd += ci[k] >= 0 ? ci[k] : rows;
    mx = std::max(mx, res[k]);
  }
  if (conv_iter_host) memcpy(conv_iter_host, ci.data(), K * 8);
  if (final_res_host) memcpy(final_res_host, res.data(), K * 8);
  const kw_status st = flag ? KW_ERR_BREAKDOWN : nc == (int64_t)K ? KW_OK : KW_NOT_CONVERGED;
  if (info) {
    info->iters = rows;
    info->n_converged = nc;
    info->max_res = mx;
    info->n_seed_switch = 0;
    info->updates = upd;
    info->seed = -1;
    info->status = st;
  }
  if (st == KW_ERR_BREAKDOWN) return fail(ctx, st, "kw_recalc: pi_{n+1} = 0 for some shift");
  if (st == KW_NOT_CONVERGED)
    fail(ctx, st, "kw_recalc: %lld of %lld shifts did not freeze within %lld rows", (long long)(nshift - nc),
         (long long)nshift, (long long)rows);
  return st;
}

kw_status kw_set_method(kw_ctx* ctx, int method, const double* btilde_dev) {
  if (!ctx) return KW_ERR_ARG;
  if (method != KW_METHOD_COCG && method != KW_METHOD_CG && method != KW_METHOD_BICG)
    return fail(ctx, KW_ERR_ARG, "kw_set_method: unknown method %d", method);
  if (btilde_dev && method != KW_METHOD_BICG)
    return fail(ctx, KW_ERR_ARG, "kw_set_method: a shadow start vector is for BiCG only");
  ctx->method = method;
  ctx->btilde = btilde_dev;
  ctx->resumable = false;
  return KW_OK;
}

kw_status kw_set_matvec_adjoint(kw_ctx* ctx, kw_matvec_fn fn, void* user) {
  if (!ctx) return KW_ERR_ARG;
  if (!ctx->mv_fn) return fail(ctx, KW_ERR_ARG, "kw_set_matvec_adjoint: set the product with kw_set_matvec first");
  ctx->mv_fn_adj = fn;
  ctx->mv_user_adj = fn ? user : nullptr;
  return KW_OK;
}

kw_status kw_set_stream_overlap(kw_ctx* ctx, int on) {
  if (!ctx || (on != 0 && on != 1)) return KW_ERR_ARG;
  ctx->overlap = on;
  return KW_OK;
}

kw_status kw_set_update_tile(kw_ctx* ctx, int shifts) {
  if (!ctx || !(shifts == 0 || shifts == 4 || shifts == 8 || shifts == 16)) return KW_ERR_ARG;
  ctx->force_xp_tile = shifts;
  return KW_OK;
}

kw_status kw_get_update_tile(kw_ctx* ctx, int* shifts) {
  if (!ctx || !shifts) return KW_ERR_ARG;
  *shifts = ctx->last_xp_tile;
  return KW_OK;
}

kw_status kw_set_seed_update(kw_ctx* ctx, int mode) {
  if (!ctx || mode < -1 || mode > 1) return KW_ERR_ARG;
  ctx->seed_rg = mode;
  return KW_OK;
}

kw_status kw_set_shift_storage(kw_ctx* ctx, int fp32) {
  if (!ctx || (fp32 != 0 && fp32 != 1)) return KW_ERR_ARG;
  ctx->xp32 = fp32;
  ctx->resumable = false;   // a stopped solve keeps its own storage
  return KW_OK;
}

kw_status kw_set_bulk_copy(kw_ctx* ctx, int on) {
  if (!ctx || on < -1 || on > 2) return KW_ERR_ARG;
  ctx->bulk = on;
  return KW_OK;
}

kw_status kw_set_kernel_timing(kw_ctx* ctx, int64_t every) {
  if (!ctx || every < 0) return KW_ERR_ARG;
  if (every > 0 && !ctx->kev[0][0]) {
    for (int i = 0; i < 2; ++i)
      for (int j = 0; j < 6; ++j) KW_CUDA(cudaEventCreate(&ctx->kev[i][j]), "kernel timing events");
  }
  ctx->timing_every = every;
  return KW_OK;
}

kw_status kw_set_spmv_config(kw_ctx* ctx, int lanes, int val_f32) {
  if (!ctx ||
      !(lanes == 0 || lanes == 1 || lanes == 2 || lanes == 4 || lanes == 8 || lanes == 16 ||
        lanes == kw::KW_SPMV_SELL || lanes == kw::KW_SPMV_UNIFORM + 1 || lanes == kw::KW_SPMV_UNIFORM + 2 ||
        lanes == kw::KW_SPMV_UNIFORM + 4 || lanes == kw::KW_SPMV_UNIFORM + 8 || lanes == kw::KW_SPMV_UNIFORM + 16 ||
        lanes == kw::KW_SPMV_UNIFORM_SELL) ||
      val_f32 < -1 || val_f32 > 1)
    return KW_ERR_ARG;
  ctx->force_lanes = lanes;
  ctx->force_val = val_f32;
  ctx->spmv_lanes = 0;
  return KW_OK;
}

kw_status kw_get_spmv_config(kw_ctx* ctx, int* lanes, int* val_f32) {
  if (!ctx || !lanes || !val_f32) return KW_ERR_ARG;
  if (!ctx->rowptr) return fail(ctx, KW_ERR_ARG, "kw_get_spmv_config: kw_set_csr has not been called");
  kw_status s = tune_spmv(ctx);
  if (s != KW_OK) return s;
  *lanes = ctx->spmv_lanes;
  if (ctx->spmv_lanes > kw::KW_SPMV_UNIFORM) *val_f32 = ctx->u_kind == 1 ? 1 : 0;
  else *val_f32 = ctx->opt.prec == KW_F64 ? ctx->spmv_val_f32 : (ctx->opt.prec == KW_C32V_F64S ? 1 : (ctx->val32_exact ? 1 : 0));
  return KW_OK;
}

kw_status kw_get_stats(kw_ctx* ctx, kw_stats* out) {
  if (!ctx || !out) return KW_ERR_ARG;
  *out = ctx->stats;
  out->tune_runs = ctx->tune_runs;
  out->tune_hits = ctx->tune_hits;
  return KW_OK;
}

kw_status kw_spmv_dot(kw_ctx* ctx, kw_c128 zs, const void* r_dev, void* q_dev, kw_c128* t_host) {
  if (!ctx) return KW_ERR_ARG;
  if (!has_operator(ctx)) return fail(ctx, KW_ERR_ARG, "kw_spmv_dot: no operator has been set");
  if (!r_dev || !q_dev || !t_host) return fail(ctx, KW_ERR_ARG, "kw_spmv_dot: NULL pointer");
  kw_status ts = tune_spmv(ctx);
  if (ts != KW_OK) return ts;
  ts = ensure_mv_buffers(ctx);
  if (ts != KW_OK) return ts;
  KW_CUDA(ctx->part_k1.ensure(part_doubles(ctx, 1) * 8), "alloc partials");
  KW_CUDA(ctx->st.ensure(sizeof(kw::State)), "alloc state");
  KW_CUDA(ctx->tdot.ensure(16), "alloc dot");
  ctx->resumable = false;   // shares the solve's state buffer
  kw::Work w;
  spmv_work(ctx, w, ctx->spmv_lanes, ctx->spmv_val_f32);
  KW_CUDA(cudaMemsetAsync(&w.st->cnt_spmv, 0, sizeof(unsigned int), ctx->stream), "reset counter");
  const double2 z2 = make_double2(zs.re, zs.im);
  cudaError_t e = spmv_dot_launch(w, r_dev, q_dev, z2, (double2*)ctx->tdot.p);
  if (e != cudaSuccess && w.mv_failed) {
    cudaStreamSynchronize(ctx->stream);
    return fail(ctx, KW_ERR_CALLBACK, "kw_spmv_dot: the matrix-vector callback returned nonzero");
  }
  KW_CUDA(e, "kw_spmv_dot launch");
  KW_CUDA(cudaMemcpyAsync(t_host, ctx->tdot.p, 16, cudaMemcpyDeviceToHost, ctx->stream), "read dot");
  KW_CUDA(cudaStreamSynchronize(ctx->stream), "kw_spmv_dot sync");
  return KW_OK;
}

}  // extern "C"
