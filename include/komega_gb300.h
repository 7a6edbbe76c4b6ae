/*
 * komega_gb300.h - C ABI of the GB300 shifted Krylov (shifted COCG) solver.
 *
 * Problem (Komega paper, arXiv:2001.08707, Sec. 1, Eq. 4-5):
 *     (z_k I - H) x^(k) = b,   k = 0 .. nshift-1,
 * with H real symmetric (M x M, CSR), b real, z_k complex.  The matrix
 * z_k I - H is complex symmetric, so the method is shifted COCG (Table 1,
 * Appendix A): one seed Krylov iteration (sparse H r, unconjugated dots,
 * three-term recurrence Eq. 16-17) drives every shift through the
 * collinearity factors pi_k (Eq. 19-22).  Outputs are the full x^(k)
 * (Eq. 23-24) or only the projections a_l^T x^(k) (Eq. 25-26, Sec. 2.2.3),
 * with seed switching after every update (Sec. 2.2.4).
 *
 * Conventions used by every call:
 *   - "_dev" pointers are CUDA device pointers on the context's device; "_host"
 *     pointers are ordinary host memory.  The caller owns every buffer passed
 *     in and keeps it alive until the call returns.
 *   - Complex vectors are interleaved (re, im): kw_c128 / double2 in KW_F64,
 *     float2 (8 bytes) in KW_C32V_F64S.
 *   - All device work is issued on the context's stream.  Calls that return
 *     results return after synchronising that stream.
 *   - Errors are status codes only.  No call exits, aborts or traps; a failed
 *     call leaves the context usable.  kw_last_error() gives a message.
 *   - A context is not thread-safe; separate contexts are independent.
 */
#ifndef KOMEGA_GB300_H
#define KOMEGA_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define KW_ABI_VERSION 2
/* Largest number of projection rows (b plus left vectors) in projected mode. */
#define KW_MAX_PROJ 32
/* Largest operator dimension M and largest nnz any call accepts: 2^31 - 2^22.
 * Row and entry counters on the device are 32-bit; a grid-stride step is at
 * most 2^22, so no counter passes 2^31 - 1. */
#define KW_MAX_ROWS 2143289344LL
#define KW_MAX_NNZ 2143289344LL

typedef struct kw_ctx kw_ctx;

typedef enum {
    KW_OK = 0,
    KW_ERR_ARG = 1,          /* invalid argument (null pointer, size, non-finite shift) */
    KW_ERR_CUDA = 2,         /* a CUDA runtime call failed */
    KW_ERR_OOM = 3,          /* device allocation failed */
    KW_ERR_BREAKDOWN = 4,    /* rho_n = 0, zero alpha denominator (Eq. 17) or pi_{n+1} = 0 (Eq. 20) */
    KW_ERR_NONFINITE = 5,    /* a seed scalar became Inf/NaN */
    KW_ERR_CALLBACK = 6,     /* the matrix-vector callback returned nonzero */
    KW_ERR_TIMEOUT = 7,      /* a bounded device wait expired (a staged copy did not complete) */
    KW_NOT_CONVERGED = 8     /* maxiter reached; outputs hold the last iterates */
} kw_status;

typedef enum {
    KW_F64 = 0,         /* complex FP64 vectors, FP64 matrix values, FP64 scalars */
    KW_C32V_F64S = 1,   /* complex FP32 vectors and FP32 matrix values; dots
                           accumulated in FP64 over FP32 chunk partials; every
                           seed and shift scalar (alpha, beta, rho, pi) and the
                           convergence test in FP64 */
    KW_DF64 = 2         /* complex vectors as FP32 pairs (hi, lo): a 48-bit
                           significand computed with error-free FP32 operations
                           (TwoSum, TwoProd) on the FP32 pipes; matrix values
                           FP32 when exact, else FP32 pairs; FP64 scalars and
                           convergence test.  Element layout in device memory:
                           4 floats (re.hi, re.lo, im.hi, im.lo), 16 bytes.
                           Values below about 1e-30 lose precision (FP32
                           exponent range). */
} kw_precision;

typedef struct { double re, im; } kw_c128;

typedef struct {
    kw_precision prec;
    double tol;          /* per shift: stop updating shift k once ||r_n|| / |pi_n^k| <= tol * ||b||
                            (the convergence criterion of Sec. 3.2.2, read per shift and relative) */
    int64_t maxiter;     /* seed iterations (matrix-vector products) at most */
    int seed_switch;     /* 1: switch the seed after every update (Sec. 2.2.4); 0: fixed seed z_0 */
    int64_t hist_stride; /* record the per-shift residual every hist_stride iterations (0 = never) */
    int64_t hist_max;    /* records kept at most */
    int use_graph;       /* 0: the host enqueues the iterations in chunks and polls the stop flag;
                            1: the iterations loop on the device in one CUDA graph (a WHILE node whose
                            body runs a chunk of 32 iterations and then tests the stop flag), with no host
                            work per chunk; n >= 2: the same with n iterations per body (rounded up to
                            even).  The graph is kept and relaunched while the solve's descriptor is
                            unchanged.  Solves with a matrix-vector callback, or with kernel timing on
                            (kw_set_kernel_timing), use the host loop whatever this says. */
    const char* tune_cache; /* NULL or "": the product kernel's layout is timed once per context.  A
                            file path: the pick is looked up there first, keyed by the precision, M,
                            nnz, a fingerprint of sampled rows (offsets, first column and value) and
                            the device's SM count, and appended after a timing run.  One text line per
                            pick; unreadable or foreign lines are skipped.  The string is copied by
                            kw_create. */
} kw_options;

typedef struct {
    int64_t iters;          /* seed iterations performed */
    int64_t n_converged;    /* shifts that met the tolerance */
    double max_res;         /* max over shifts of the last residual estimate ||r||/|pi| */
    int64_t n_seed_switch;  /* seed switches performed */
    int64_t updates;        /* sum over iterations of the active shift count; x M = shift-row updates */
    int64_t seed;           /* index of the seed shift at exit */
    kw_status status;
} kw_solve_info;

/* ABI version of the loaded library (KW_ABI_VERSION it was built with); no
 * paper counterpart.  Never fails. */
int kw_abi_version(void);

/* Fill *opt with defaults: KW_F64, tol 1e-10, maxiter 100000, seed_switch 1
 * (Sec. 2.2.4), hist_stride 0, hist_max 0, use_graph 1, tune_cache NULL.  The
 * tolerance is the per-shift criterion of Sec. 3.2.2.  Errors: none (a NULL
 * opt is ignored). */
void kw_default_options(kw_options* opt);

/* No paper counterpart.  Human-readable name of a status code (static string,
 * never NULL; unknown codes give "KW_UNKNOWN").  Errors: none. */
const char* kw_status_string(kw_status s);

/* Create a context on the current CUDA device: the solver state of one
 * shifted system family (Eq. 4-5), with no operator yet.  cuda_stream is a
 * cudaStream_t (NULL = legacy default stream) on which all work is issued; the
 * options are copied (tune_cache included).  Errors:
 * KW_ERR_ARG (out or opt NULL, tol < 0, maxiter < 1, hist_stride < 0, bad
 * precision), KW_ERR_CUDA. */
kw_status kw_create(kw_ctx** out, const kw_options* opt, void* cuda_stream);

/* No paper counterpart.  Release the context and every device buffer it owns,
 * after synchronising its stream.  Buffers the caller lent (kw_set_csr,
 * outputs) are not freed. Errors: none (NULL is ignored). */
void kw_destroy(kw_ctx* ctx);

/* No paper counterpart.  Copy the last error message (NUL-terminated,
 * truncated to n) into buf. Errors: KW_ERR_ARG (ctx or buf NULL, n = 0). */
kw_status kw_last_error(const kw_ctx* ctx, char* buf, size_t n);

/* Set the operator H of Eq. 4 (real symmetric, M x M) as a device CSR matrix:
 * rowptr_dev int64 [m+1] (rowptr[0] = 0, nondecreasing, rowptr[m] = nnz),
 * col_dev int32 [nnz] in [0, m), val_dev float64 [nnz].  The pointers are
 * borrowed in KW_F64 mode (they must stay valid until the next kw_set_csr or
 * kw_destroy); in KW_C32V_F64S mode the context keeps its own FP32 copy of the
 * values (and, in KW_F64 mode, uses an FP32 copy only if every value is
 * exactly representable in FP32).  Symmetry is the caller's promise and is
 * not checked.  Errors:
 * KW_ERR_ARG (m < 1, m > KW_MAX_ROWS, nnz < 0, nnz > KW_MAX_NNZ, NULL pointer),
 * KW_ERR_OOM. */
kw_status kw_set_csr(kw_ctx* ctx, int64_t m, int64_t nnz, const int64_t* rowptr_dev,
                     const int32_t* col_dev, const double* val_dev);

/* Solvers of Table 1: COCG (the default) for complex symmetric A + sigma I
 * (real symmetric or complex symmetric H, complex shifts); CG for Hermitian
 * A + sigma I (real symmetric or Hermitian H, real shifts); BiCG otherwise
 * (Appendix B: a shadow residual driven by A^dagger). */
typedef enum { KW_METHOD_COCG = 0, KW_METHOD_CG = 1, KW_METHOD_BICG = 2 } kw_method;

/* Element types of the vectors handed to a matrix-vector callback. */
#define KW_ELEM_C128 0   /* kw_c128 */
#define KW_ELEM_C64 1    /* complex FP32: {float re, im} */

/* Matrix-vector callback: enqueue on cuda_stream (a cudaStream_t) the work
 * that writes q = H r into all m entries of q_dev, reading r_dev, both device
 * vectors of element type elem; return 0, or nonzero to stop the solve with
 * KW_ERR_CALLBACK.  The pointers are valid only for the work enqueued by this
 * call. */
typedef int (*kw_matvec_fn)(void* user, const void* r_dev, void* q_dev, int64_t m, int elem, void* cuda_stream);

/* Set the operator H (M x M) as a caller-supplied product instead of a matrix
 * (Sec. 3.1 (i): the library leaves "q = H r" to the application, which may
 * generate the matrix elements on the fly, as HPhi does).  H must be symmetric
 * (H^T = H; real, or complex symmetric, since COCG only needs A = zI - H to be
 * complex symmetric).  Until the next kw_set_csr, kw_solve and kw_spmv_dot
 * call fn once per iteration from the calling thread while they enqueue work
 * (the host runs up to 32 iterations ahead of the GPU, so fn may be called for
 * iterations after the solve has converged; their products are ignored).
 * elem is KW_ELEM_C64 in the KW_C32V_F64S form and KW_ELEM_C128 otherwise (the
 * KW_DF64 form converts its FP32-pair vectors to and from kw_c128 around the
 * call).  r_dev holds the seed residual, possibly still in the previous seed's
 * normalisation (the library applies the seed-switch factor to q itself, which
 * is exact by linearity).  kw_solve_batched and kw_bilinear take their own
 * matrices and ignore the callback; kw_solve_host sets its matrix as the
 * operator (as kw_set_csr does), which ends the callback.  Errors: KW_ERR_ARG
 * (m < 1, m > KW_MAX_ROWS, fn NULL). */
kw_status kw_set_matvec(kw_ctx* ctx, int64_t m, kw_matvec_fn fn, void* user);

/* Most bonds and sites of a spin operator (kw_set_spin_operator). */
#define KW_SPIN_MAX_BONDS 256
#define KW_SPIN_MAX_SITES 31

/* Set the operator H to a spin-1/2 Hamiltonian generated on the fly (matrix-
 * free, Sec. 3.1 (i): the matrix elements are produced inside the product and
 * never stored, the paper's route to large M):
 *   H = sum_b J_b S_{i_b} . S_{j_b} + sum_i h_i S^z_i
 * on the basis of all nsite-bit words with nup set bits (bit i set = spin i up;
 * fixed S^z_total sector), in increasing order, so M = C(nsite, nup) and the
 * row of a word is its rank in the combinatorial number system.  A bond
 * contributes J_b/4 (parallel spins) or -J_b/4 (antiparallel) to the diagonal
 * and J_b/2 between two words that differ by exchanging its two spins; h_i
 * contributes +h_i/2 (up) or -h_i/2 (down).  bonds_host int32 [nbond][2] (site
 * pairs, i != j, each < nsite), J_host [nbond], h_host [nsite] or NULL (no
 * field).  The context builds the basis table (4 bytes per row) and the
 * diagonal (4 or 8 bytes per row) on the device; a product then reads only
 * these, r and q.  Ends any CSR matrix or callback.  Errors: KW_ERR_ARG
 * (1 <= nup < nsite <= KW_SPIN_MAX_SITES, 1 <= nbond <= KW_SPIN_MAX_BONDS, bad
 * bond, M > KW_MAX_ROWS, non-finite J or h), KW_ERR_OOM. */
kw_status kw_set_spin_operator(kw_ctx* ctx, int nsite, int nup, int nbond, const int32_t* bonds_host,
                               const double* J_host, const double* h_host);

/* Spin operator storage (the matrix-free product of Sec. 3.1 (i) for the
 * Heisenberg-type Hamiltonians of Eq. 41).  on = 0 (default): every product regenerates the
 * exchanged words' rows from the combinatorial number system (4 + 4 bytes per
 * row: basis word and diagonal).  on = 1: the context also keeps an exchange
 * table of nbond * M int32 (the row of each bond's exchanged word, -1 for
 * parallel spins), stored bond by bond so that a warp's rows read each bond
 * together, and the product only gathers.  Applies to the current spin
 * operator at once and to later ones.  Errors: KW_ERR_ARG, KW_ERR_OOM. */
kw_status kw_set_spin_table(kw_ctx* ctx, int on);

/* Set the operator H to a tight-binding model on a periodic nx x ny x nz
 * lattice, generated on the fly: H_ii = eps_i, H_ij = hopping for the six
 * nearest neighbours j of site i = x + nx (y + ny z) (the Anderson model of
 * Sec. 4 with eps_i the disorder).  eps_dev float64 [nx ny nz] (device; the
 * context keeps its own copy in the form's precision).  Each extent must be at
 * least 3 (six distinct neighbours).  Ends any CSR matrix or callback.  Errors:
 * KW_ERR_ARG (extent < 3, nx ny nz > KW_MAX_ROWS, eps_dev NULL, hopping not finite),
 * KW_ERR_OOM. */
kw_status kw_set_lattice3d(kw_ctx* ctx, int64_t nx, int64_t ny, int64_t nz, const double* eps_dev, double hopping);

/* Solve (z_k I - H) x_k = b for all nshift shifts (Eq. 4) by shifted COCG.
 *   b_dev       float64 [m], real right-hand side (||b|| > 0).
 *   z_host      kw_c128 [nshift], finite shifts; the initial seed is z_0 (Eq. 6).
 *   nleft       number of left vectors a_l (0 .. KW_MAX_PROJ-1).
 *   left_dev    float64 [nleft][m] row-major, or NULL when nleft = 0.
 *   x_out_dev   full mode: [nshift][m] complex in the context precision
 *               (kw_c128 for KW_F64 and KW_DF64, float2 for KW_C32V_F64S),
 *               receives x_k.
 *               NULL selects projected mode (Eq. 25-26): no x_k is formed.
 *   proj_out_host kw_c128 [nshift][nleft+1] or NULL; column 0 = b^T x_k,
 *               column l = a_{l-1}^T x_k (a real, so a^dagger = a^T).
 *   info        optional summary.
 * Returns KW_OK when every shift met the tolerance, KW_NOT_CONVERGED at
 * maxiter (outputs then hold the last iterates), KW_ERR_BREAKDOWN /
 * KW_ERR_NONFINITE with the outputs of the last completed iteration, or an
 * argument/CUDA error.  A right-hand side with ||b|| = 0 (where rho_0 = 0 and
 * Eq. 17 has no alpha_0) or a non-finite norm is found on the device before the
 * first iteration and returns KW_ERR_ARG with 0 iterations and x = 0.
 * kw_set_csr must have been called. */
kw_status kw_solve(kw_ctx* ctx, const double* b_dev, int64_t nshift, const kw_c128* z_host,
                   int64_t nleft, const double* left_dev, void* x_out_dev,
                   kw_c128* proj_out_host, kw_solve_info* info);

/* kw_solve (Eq. 4-5, Eqs. 23-26) with every array in host memory: copies H
 * (CSR as in kw_set_csr), b and the left vectors to the device, solves, and
 * copies x (if x_out_host is not NULL; same layout as x_out_dev) and the
 * projections back.  The device copies are owned by the context and reused by
 * later calls.  Errors: those of kw_set_csr and kw_solve, KW_ERR_ARG (NULL
 * host arrays, m < 1, nshift < 1), KW_ERR_OOM. */
kw_status kw_solve_host(kw_ctx* ctx, int64_t m, int64_t nnz, const int64_t* rowptr_host,
                        const int32_t* col_host, const double* val_host, const double* b_host,
                        int64_t nshift, const kw_c128* z_host, int64_t nleft,
                        const double* left_host, void* x_out_host, kw_c128* proj_out_host,
                        kw_solve_info* info);

/* One problem of a batch: an operator, a right-hand side and its shifts. */
typedef struct {
    int64_t m, nnz;
    const int64_t* rowptr_dev;     /* as in kw_set_csr */
    const int32_t* col_dev;
    const double* val_dev;
    const double* b_dev;           /* [m] */
    int64_t nshift;
    const kw_c128* z_host;         /* [nshift] */
    int64_t nleft;
    const double* left_dev;        /* [nleft][m] or NULL */
    void* x_out_dev;               /* full mode: [nshift][m] as in kw_solve; NULL: projected */
    kw_c128* proj_out_host;        /* [nshift][nleft+1] or NULL */
    double tol;                    /* > 0 overrides the context's tolerance for this problem */
} kw_instance;

/* ---------------------------------------------------------------------------
 * Reverse communication (Sec. 3.1 (iii), Algorithm 1): the caller computes
 * every product itself, between calls, as the paper's *_init / *_update /
 * *_getresidual / *_finalize flow does.  Each kw_rci_update runs one iteration
 * synchronously (no host run-ahead, one stream), so it is slower than
 * kw_set_matvec, which it otherwise matches bit for bit.
 * --------------------------------------------------------------------------- */
typedef struct {
    const void* r;   /* device [m]: the vector to multiply (elem type below) */
    void* q;         /* device [m]: where the caller writes H r */
    const void* rt;  /* BiCG: the shadow vector r~ (else NULL) */
    void* qt;        /* BiCG: where the caller writes H^dagger r~ (else NULL) */
    int elem;        /* KW_ELEM_C128, or KW_ELEM_C64 in the KW_C32V_F64S form */
} kw_rci_io;

/* Reverse communication (Sec. 3.1 (iii), Algorithm 1: the library's _init,
 * _update, _getresidual and _finalize steps).  Start a solve of
 * (z_k I - H) x_k = b of size m (arguments as kw_solve) with
 * the caller as the operator: any CSR matrix, callback or generated operator of
 * ctx is dropped.  *io receives the first vectors.  The solver of
 * kw_set_method is used (COCG by default).  Errors: those of kw_solve. */
kw_status kw_rci_init(kw_ctx* ctx, int64_t m, const double* b_dev, int64_t nshift, const kw_c128* z_host,
                      int64_t nleft, const double* left_dev, void* x_out_dev, kw_rci_io* io);

/* The update step of Algorithm 1 (Sec. 3.1 (iii)).  After the caller has
 * written q = H r (and, for BiCG, qt = H^dagger rt) for
 * the vectors of the last *io: finish the iteration; *done = 1 when every
 * shift has converged or the iteration cap or a breakdown was reached, else 0
 * with the next vectors in *io (their addresses change between iterations).
 * The vectors may still carry a pending seed-switch scale, which the library
 * applies by linearity.  Errors: KW_ERR_ARG (no kw_rci_init), KW_ERR_CUDA. */
kw_status kw_rci_update(kw_ctx* ctx, int* done, kw_rci_io* io);

/* Current residual estimate ||r_n||/|pi_n^k| of every shift (Sec. 3.2.2; host,
 * [nshift]).  Errors: KW_ERR_ARG (no reverse-communication solve, NULL res),
 * KW_ERR_CUDA. */
kw_status kw_rci_get_residual(kw_ctx* ctx, double* res_host);

/* End the solve: outputs and status as kw_solve returns them (x^(k) of
 * Eq. 23-24 or the projections of Eq. 25-26).  ctx then has no operator until
 * the next kw_set_csr, kw_set_matvec or generated operator.  Errors:
 * KW_ERR_ARG (no reverse-communication solve), the solve's own status
 * (KW_NOT_CONVERGED, KW_ERR_BREAKDOWN, KW_ERR_NONFINITE), KW_ERR_CUDA. */
kw_status kw_rci_finalize(kw_ctx* ctx, kw_c128* proj_out_host, kw_solve_info* info);

/* Continue the last kw_solve of ctx for up to more_iters further iterations
 * (the "restart" mode of Sec. 3.3: a solve stopped by its iteration cap goes on
 * from where it stopped, on the device state the context kept).  Valid only
 * when that solve ended with KW_NOT_CONVERGED and nothing has since changed
 * the context's operator, method or workspace (kw_set_csr, kw_set_matvec, the
 * generated operators, kw_set_method, kw_spmv_dot, kw_solve_batched and other
 * solves end it).  b, the shifts, the left vectors and, in full mode, the
 * caller's x buffer must still be valid: they are read and updated in place.
 * The result is the one a single solve with the larger cap would give (the
 * pair form's x is converted back from kw_c128 to pairs first, which keeps
 * its value).  proj_out_host and info as for kw_solve (iteration counts are
 * totals); the same residual history and Krylov log continue.  Errors:
 * KW_ERR_ARG (more_iters < 1, nothing to resume), the kw_solve errors. */
kw_status kw_resume(kw_ctx* ctx, int64_t more_iters, kw_c128* proj_out_host, kw_solve_info* info);

/* Solve n independent problems (uneven sizes and shift counts; each one
 * Eq. 4-5) together.  Each instance runs the kw_solve iteration on its own
 * stream and workspace, owned by the context and reused by later calls; one
 * CUDA graph holds a trip of iterations of every instance, repeated on the
 * device by a WHILE node until every instance has stopped (use_graph 0: the
 * host relaunches it per chunk); instances that stop early return from their
 * kernels at the first instruction.  Results are those kw_solve gives for each instance
 * alone.  info: [n] or NULL.  Returns KW_OK if every instance converged, else
 * the first other status (per-instance status in info).  Errors: KW_ERR_ARG
 * (n < 1, NULL pointer, an instance's own argument errors), KW_ERR_CUDA. */
kw_status kw_solve_batched(kw_ctx* ctx, int64_t n, const kw_instance* inst, kw_solve_info* info);

/* Per-shift results of the last solve: the iteration at which shift k met the
 * tolerance of Sec. 3.2.2 (-1 if never) and its last residual estimate
 * ||r_n||/|pi_n^k| (Eq. 19).  Either pointer may be NULL.  Arrays have the
 * last solve's nshift entries.  Errors: KW_ERR_ARG (no solve yet), KW_ERR_CUDA. */
kw_status kw_get_shift_status(kw_ctx* ctx, int64_t* conv_iter_host, double* final_res_host);

/* Residual history of the last solve (the per-shift ||r_n||/|pi_n^k| of
 * Sec. 3.2.2 over the iterations): *n_rec records of nshift doubles, record i
 * taken after iteration (i+1)*hist_stride.  hist_host may be NULL to query
 * *n_rec; otherwise it must hold hist_max * nshift doubles.  Before any solve
 * *n_rec is 0.  Errors: KW_ERR_ARG (ctx or n_rec NULL), KW_ERR_CUDA. */
kw_status kw_get_residual_history(kw_ctx* ctx, double* hist_host, int64_t* n_rec);

/* ---------------------------------------------------------------------------
 * Recalculation at new shifts (Sec. 3.3 (iv)).  A solve can record, per
 * iteration, what the shift recurrences consume; the projections a_l^T x at
 * shifts that were not in the solve then follow from Eqs. 20-22 and 25-26
 * alone, with no product with H.
 *
 * Log row n (iteration n, 0-based) holds KW_LOG_FIXED + nproj kw_c128 values:
 *   [0] z_s   the seed shift used by iteration n
 *   [1] alpha_n, [2] c_n = alpha_n beta_{n-1}/alpha_{n-1}, [3] beta_n   (Eq. 17)
 *   [4] (||r_{n+1}||_2^2, 0)
 *   [5] pi^j_{n+1}, [6] pi^j_n: the factors of a seed switch to shift j after
 *       iteration n (Sec. 2.2.4), both 1 when the seed was kept
 *   [7 + l] (P r_{n+1})_l, l < nproj: row 0 of P is b, rows 1.. the left
 *       vectors; taken before the switch of that iteration.
 * w0 holds P r_0 = P b (nproj values).  A projected-mode solve logs nproj =
 * nleft + 1 columns; a full-mode solve logs nproj = 0 (the seed scalars only).
 * --------------------------------------------------------------------------- */
#define KW_LOG_FIXED 7

/* Krylov log for recalculation at new shifts (Sec. 3.3 (iv): the seed scalars
 * and projections a run needs to replay Eqs. 20-22 and 25-26 without products).
 * Record the log in the next solves of ctx (kw_solve, kw_solve_host), at most
 * max_iters rows (0 = off, the default).  The device log takes
 * max_iters * (KW_LOG_FIXED + nproj) * 16 bytes, allocated at the next solve.
 * Errors: KW_ERR_ARG (max_iters < 0). */
kw_status kw_set_krylov_log(kw_ctx* ctx, int64_t max_iters);

/* The log of the last solve (Sec. 3.3 (iv)).  *n_iter = rows recorded (fewer than *n_run, the
 * solve's iteration count, when max_iters cut it short), *nproj = columns of
 * P, *thresh = the solve's absolute threshold tol*||b||_2.  log_host (NULL to
 * query sizes) receives n_iter rows of KW_LOG_FIXED + nproj values; w0_host
 * (may be NULL) receives nproj values.  Any output pointer may be NULL.
 * Errors: KW_ERR_ARG (the last solve recorded no log). */
kw_status kw_get_krylov_log(kw_ctx* ctx, int64_t* n_iter, int64_t* n_run, int64_t* nproj, double* thresh,
                            kw_c128* log_host, kw_c128* w0_host);

/* Projections at nshift new shifts z_host from a log, on the GPU (one thread
 * per shift replays Eq. 20, Eqs. 21-22 and Eqs. 25-26 row by row, then the
 * seed-switch rescale of pi).  A shift freezes at the first row where
 * ||r_{n+1}|| / |pi_{n+1}| <= thresh (thresh <= 0: never).
 *   log_host != NULL: a log of n_iter rows and nproj columns (0..KW_MAX_PROJ)
 *       in the layout above, and w0_host its P b; both are copied to the
 *       device.
 *   log_host == NULL: the device log of the last solve of ctx (nproj and
 *       w0_host are ignored; n_iter < 0 or above the recorded rows means all
 *       recorded rows).
 *   proj_out_host: [nshift][nproj] (column 0 = b^T x) or NULL;
 *   conv_iter_host: [nshift], the row count at which the shift froze, -1 if
 *       never, or NULL;  final_res_host: [nshift] last residual estimate or NULL.
 *   info (may be NULL): iters = rows replayed, n_converged, max_res,
 *       updates = shift-rows replayed, status.
 * Returns KW_OK when every shift froze, else KW_NOT_CONVERGED, with every
 * output filled (a shift that did not freeze has its last iterate).  Errors:
 * KW_ERR_ARG (bad sizes, NULL log without a logged solve, non-finite shift),
 * KW_ERR_BREAKDOWN (pi_{n+1} = 0 for some shift), KW_ERR_OOM, KW_ERR_CUDA. */
kw_status kw_recalc(kw_ctx* ctx, int64_t n_iter, int64_t nproj, double thresh, const kw_c128* log_host,
                    const kw_c128* w0_host, int64_t nshift, const kw_c128* z_host, kw_c128* proj_out_host,
                    int64_t* conv_iter_host, double* final_res_host, kw_solve_info* info);

/* Per-solve statistics for measurement.  kernel_ms[i] sums the device time
 * of kernel i (0: SpMV + r^T q, 1: three-term update + dots, 2: shift
 * scalars, 3: x/p update) over timed_iters iterations sampled by
 * kw_set_kernel_timing; launches counts every kernel the last solve enqueued
 * (including iterations enqueued after the device stop flag, which return at
 * once). */
typedef struct {
    int64_t launches;
    int64_t timed_iters;
    double kernel_ms[4];
    int64_t tune_runs;      /* timing runs of the product-kernel tuner in this context */
    int64_t tune_hits;      /* picks taken from the persistent tuning cache (kw_options.tune_cache) */
} kw_stats;

/* Measurement only (no paper counterpart): bracket the kernels of one
 * iteration in every `every` with CUDA events on the context stream (0 turns it
 * off; the default).  While it is on, solves run the host-driven loop (events
 * cannot sit inside the device loop); kw_get_stats reports the times.
 * Errors: KW_ERR_ARG (ctx NULL, every < 0), KW_ERR_CUDA. */
kw_status kw_set_kernel_timing(kw_ctx* ctx, int64_t every);

/* Select the solver of Table 1 for the next solves of ctx (kw_solve,
 * kw_solve_host, kw_solve_batched):
 *   KW_METHOD_COCG (default): unconjugated inner products (Appendix A).
 *   KW_METHOD_CG: conjugated inner products, rho = ||r||^2; for Hermitian
 *     A + sigma I, i.e. a real symmetric or Hermitian H (Hermitian through
 *     kw_set_matvec) and real shifts (a complex shift fails with KW_ERR_ARG).
 *   KW_METHOD_BICG: Appendix B; a shadow residual r~ (start btilde_dev, real
 *     [m] device vector, or NULL for b; kw_solve_batched always uses b) is
 *     advanced with A^dagger and the conjugated coefficients, rho = r~^dagger r.
 *     A^dagger r~ = conj(z_s) r~ - H^dagger r~, with H^dagger = H for the CSR and
 *     generated operators (real symmetric) and, for a callback, the adjoint
 *     callback (kw_set_matvec_adjoint) or the same callback when none is set.
 *     Each iteration then makes two products and one more pass over r~ and q.
 * The shifted recurrences (Eqs. 20-26), seed switching and outputs are those of
 * COCG for every method.  btilde_dev is borrowed until the next kw_set_method.
 * Errors: KW_ERR_ARG (unknown method, btilde_dev with a method other than BiCG). */
kw_status kw_set_method(kw_ctx* ctx, int method, const double* btilde_dev);

/* Adjoint product q = H^dagger r (the A^dagger of Appendix B) for BiCG with a
 * callback operator that is not Hermitian (same calling rules as kw_matvec_fn;
 * NULL: H is Hermitian).  A later kw_set_matvec or kw_set_csr clears it.
 * Errors: KW_ERR_ARG (no callback set). */
kw_status kw_set_matvec_adjoint(kw_ctx* ctx, kw_matvec_fn fn, void* user);

/* Schedule of an iteration (the steps of Sec. 2.2: Eq. 16-17, then Eq. 20-26).
 * on = 1 (the default): the shift scalars of iteration n run on a second stream
 * while the product of iteration n+1 runs, since neither needs the other's
 * results (a seed switch reaches that product through the next three-term
 * update, by linearity), and the full-mode x/p update of iteration n runs on a
 * third stream beside the next three-term update (its coefficients and shift
 * list sit in slots of the iteration's parity); on = 0: one stream, in the
 * order K2(n), K1(n+1), K3(n), K4(n).  Both give the same numbers.  Errors:
 * KW_ERR_ARG. */
kw_status kw_set_stream_overlap(kw_ctx* ctx, int on);

/* Loads of the three-term update (Eq. 16) in the FP32 and FP32-pair forms.
 * on = 1: the tiles of r_n, q_n, r_{n-1} and the projection rows are staged in
 * shared memory by TMA bulk copies (cp.async.bulk) completed on mbarriers, up to
 * three tiles ahead of the arithmetic; on = 0: plain coalesced loads; on = -1
 * (the default): staged when the update carries more than 9 projection rows.
 * Each thread sums the same elements in the same order either way; the results
 * agree to rounding (the two kernels are compiled separately).  Measured on
 * GB300: with 17 projection rows (Anderson L=160) staging takes the update from
 * 281 to 256 us (pairs) and 133 to 110 us (FP32); with 5 rows (Heisenberg N=24)
 * plain loads are faster (67 vs 74 us, pairs).  A staged copy that does not
 * complete within about a second ends the solve with KW_ERR_TIMEOUT.  The FP64
 * form and BiCG always use plain loads.  on = 2 exercises that bound: each
 * stage is armed for 16 bytes more than its copies bring, so the first staged
 * wait of every block runs out and the solve ends with KW_ERR_TIMEOUT after a
 * few seconds (the context stays usable).  Errors: KW_ERR_ARG. */
kw_status kw_set_bulk_copy(kw_ctx* ctx, int on);

/* Tile of the full-mode x/p update (Eq. 23-24): the number of shifts one block
 * item updates for a chunk of 256 rows, reading r_{n+1} once for them.
 * shifts = 4, 8 or 16 forces that tile; 0 (default) times the three on the
 * solve's own x/p buffers before they are initialised, once per form, shift
 * storage, K and M, and keeps the fastest (every tile gives the same results).
 * Applies from the next full-mode solve (kw_solve_batched instances
 * included).  Errors: KW_ERR_ARG. */
kw_status kw_set_update_tile(kw_ctx* ctx, int shifts);

/* The x/p update tile of the last full-mode solve (0 before any).  Errors:
 * KW_ERR_ARG (NULL pointer). */
kw_status kw_get_update_tile(kw_ctx* ctx, int* shifts);

/* Form of the three-term update kernel (Eq. 16 with rho, nu and P r_{n+1} of
 * Eq. 26) in the KW_DF64 form with the COCG or CG solver.  mode 1: two phases
 * per 256-element tile, r_{n+1} of each element first, then four thread groups
 * each forming every fourth projection row from shared memory (few
 * accumulators per thread, for many projection rows); 0: one element per
 * thread with every projection accumulated by that thread (kw_set_bulk_copy
 * then selects plain or staged loads); -1 (default): mode 1 above nine
 * projection rows (b plus the left vectors), else 0.  Results agree to
 * rounding, not bit for bit (different summation order).  Applies from the next
 * solve.  Errors: KW_ERR_ARG. */
kw_status kw_set_seed_update(kw_ctx* ctx, int mode);

/* Storage of the shifted vectors in full mode (Eq. 23-24; the K*M-sized part of
 * the state, Sec. 2.2.3).  fp32 = 1: x^(k) and p^(k) are stored and updated as
 * complex FP32 (8 bytes per element) in the KW_F64 and KW_DF64 forms, while
 * the seed vectors, the seed and shift scalars and the convergence test keep
 * the form's precision; r_{n+1} enters the update rounded to FP32 and the
 * scalars alpha^k, beta^k, 1/pi^k as their FP32 roundings.  The full-mode
 * x_out buffer is then [nshift][m] complex FP32 ({float re, im}), and proj_out
 * (b^T x_k and a_l^T x_k) comes from the projected recurrences of Eq. 25-26,
 * which run in the same solve (FP64 y/u, P r_{n+1} formed by the seed update
 * in the form's precision), not from the stored x.  Errors in x/p never feed
 * back into the seed recurrence, so the iteration is the form's; x carries
 * FP32 storage error.  fp32 = 0 (default): x/p in the form's vector type.  No
 * effect in KW_C32V_F64S (already FP32) or in projected mode.  Applies from
 * the next solve (kw_solve_batched instances included).  Errors: KW_ERR_ARG. */
kw_status kw_set_shift_storage(kw_ctx* ctx, int fp32);

/* Configuration of the sparse product kernel (the "q = H r" of Algorithm 1).
 * lanes = threads per matrix
 * row of the CSR kernel (1, 2, 4, 8 or 16), or 32 = the SELL-32 layout (an
 * internal sliced-ELLPACK copy: rows sorted by length within windows of 1024
 * rows, 32 rows per slice, column-major inside a slice, one thread per row);
 * 64 + G (G = 1, 2, 4, 8, 16) = the uniform off-diagonal layout with G threads
 * per row, for operators whose off-diagonal entries all have one value (lattice
 * hoppings, spin-flip amplitudes): an internal copy holding int32 row offsets,
 * the off-diagonal columns only and the summed diagonal, so that
 * H r = d_i r_i + v * (sum of r over the row's off-diagonal columns); forcing
 * it on another operator fails with KW_ERR_ARG at the next solve; 96 = the
 * same uniform layout stored as SELL-32: the off-diagonal columns of each slice
 * of 32 consecutive rows (rows not reordered) slot-major, -1 past a row's end,
 * one thread per row, so that a warp's index loads are contiguous (not built,
 * and forcing it fails with KW_ERR_ARG, when the padding would exceed three
 * times the columns);
 * 0 = choose by timing every candidate on the current operator at the next
 * solve, the default (operators with fewer than 2^20 non-zeros are not timed
 * and use 1).  val_f32 (KW_F64 mode only): 1 =
 * read the matrix values from an FP32 copy, allowed only when every value is
 * exactly representable in FP32 (checked by kw_set_csr; otherwise FP64 is
 * used); 0 = FP64 values; -1 = choose by timing.  Errors: KW_ERR_ARG. */
kw_status kw_set_spmv_config(kw_ctx* ctx, int lanes, int val_f32);

/* The configuration the next solve will use (tunes first if needed; the layout
 * of the product of Algorithm 1).  Errors: KW_ERR_ARG (a NULL pointer, no CSR
 * operator set), KW_ERR_CUDA, KW_ERR_OOM (tuning copies). */
kw_status kw_get_spmv_config(kw_ctx* ctx, int* lanes, int* val_f32);

/* Statistics of the last kw_solve / kw_solve_host (measurement only; no paper
 * counterpart).  Errors: KW_ERR_ARG (ctx or out NULL). */
kw_status kw_get_stats(kw_ctx* ctx, kw_stats* out);

/* One seed matrix-vector step (Alg. 1 "q = H r" combined with the seed shift,
 * and the first dot of Eq. 17): q = zs r - H r and t = r^T q (unconjugated),
 * with the context's operator and precision.  r_dev, q_dev: [m] complex in the
 * context precision (KW_DF64: the 4-float pair layout), not overlapping;
 * t_host receives the FP64 dot.  Errors: KW_ERR_ARG (no operator, NULL
 * pointer), KW_ERR_CALLBACK, KW_ERR_CUDA, KW_ERR_OOM. */
kw_status kw_spmv_dot(kw_ctx* ctx, kw_c128 zs, const void* r_dev, void* q_dev, kw_c128* t_host);

/* One parameter matrix H_t of H(theta) = sum_t theta_t H_t, as a device CSR
 * matrix with the layout of kw_set_csr (int64 rowptr [m+1], int32 col, f64 val). */
typedef struct {
    int64_t nnz;
    const int64_t* rowptr_dev;
    const int32_t* col_dev;
    const double* val_dev;
} kw_csr_term;

/* Most shifts of one kw_bilinear call (65535 tiles of 8 shifts). */
#define KW_BILINEAR_MAX_SHIFTS 524280LL

/* Adjoint bilinear forms for the parameter derivative of the Green's function.
 * With G(z) = (z I - H)^{-1} (Eq. 2) and H = sum_t theta_t H_t,
 * dG/dtheta_t = G H_t G, and G^T = G for real symmetric H, so
 *     d(a^T G(z_k) b)/dtheta_t = y_k^T H_t x_k,  x_k = G(z_k) b,  y_k = G(z_k) a
 * (y_k = x_k when a = b).  This call forms out[k][t] = y_k^T H_t x_k
 * (unconjugated) for every shift k and term t.
 *   m: rows; terms_host: nterm term descriptors (device arrays, m x m each);
 *   X_dev, Y_dev: [nshift][m] kw_c128 device arrays (x_k from kw_solve in full
 *   mode with KW_F64 or KW_DF64); Y_dev NULL means Y = X.
 *   out_host: kw_c128 [nshift][nterm].
 * Terms whose every row holds at most one entry, on the diagonal (field and
 * on-site terms), are found by a scan of their structure and handled together:
 * y_k[i] x_k[i] is formed once per shift and row and applied to up to 16 such
 * terms in one pass over X and Y; the other terms take a pass each.
 * FP64 arithmetic; uses the context's stream and workspace (nterm x m doubles
 * for the diagonals).  Errors: KW_ERR_ARG (sizes, nshift > KW_BILINEAR_MAX_SHIFTS,
 * NULL pointers), KW_ERR_OOM, KW_ERR_CUDA. */
kw_status kw_bilinear(kw_ctx* ctx, int64_t m, int64_t nterm, const kw_csr_term* terms_host, int64_t nshift,
                      const kw_c128* X_dev, const kw_c128* Y_dev, kw_c128* out_host);

/* kw_bilinear for complex FP32 solution vectors (full-mode x from the
 * KW_C32V_F64S form or from FP32 shift storage, kw_set_shift_storage): X_dev,
 * Y_dev are [nshift][m] {float re, im} device arrays (Y_dev NULL means Y = X),
 * widened to FP64 on load; the sums and out_host are FP64 as in kw_bilinear
 * (the same bilinear forms y_k^T H_t x_k of Eq. 2's derivative).  Errors: as
 * kw_bilinear. */
kw_status kw_bilinear_c64(kw_ctx* ctx, int64_t m, int64_t nterm, const kw_csr_term* terms_host, int64_t nshift,
                          const void* X_dev, const void* Y_dev, kw_c128* out_host);

/* Linear combinations of the full-mode solutions over the shifts:
 *     S[k][i] = sum_j W[k][j] x_j[i],   k < nk, j < nshift,
 * the form of the contour moments of Sec. 4.1, s_k = sum_j w_j (z_j - gamma)^k x_j
 * (trapezoid rule on the circle), formed on the device so that only the nk
 * moment vectors, not the nshift solutions, need to leave it.
 *   X_dev: [nshift][m] device solutions, element x_elem (KW_ELEM_C128, or
 *   KW_ELEM_C64 for complex FP32 from the FP32 form or FP32 shift storage);
 *   W_host: kw_c128 [nk][nshift] weights (1 <= nk <= 16);
 *   S_dev: kw_c128 [nk][m] device output.
 * FP64 sums in a fixed order; returns after synchronising the context's
 * stream.  Errors: KW_ERR_ARG (sizes, element type, NULL pointers), KW_ERR_OOM,
 * KW_ERR_CUDA. */
kw_status kw_shift_combine(kw_ctx* ctx, int64_t m, int64_t nshift, const void* X_dev, int x_elem, int64_t nk,
                           const kw_c128* W_host, kw_c128* S_dev);

/* Most thread blocks kw_spmv_dot_noalloc launches; its static scratch holds
 * one FP64 complex partial per block (64 KiB) plus a counter and the result. */
#define KW_NOALLOC_MAX_BLOCKS 4096

/* kw_spmv_dot for callers that cannot allocate device memory: code whose GPU
 * memory is entirely owned by another allocator (for example a framework's
 * caching pool, or a fixed budget) and latency-critical loops that cannot pay
 * for the implicit synchronisation of cudaMalloc.  The paper has no
 * counterpart for this entry point.  It computes q = zs r - H r and
 * t = r^T q (unconjugated) in FP64, as kw_spmv_dot does in the KW_F64 form,
 * without a context.
 *   m, nnz, rowptr_dev, col_dev, val_dev: the operator as in kw_set_csr.
 *   r_dev, q_dev: [m] kw_c128 device arrays (input r, output q).
 *   t_host: receives t.  cuda_stream: the stream to run on (NULL = default).
 * Nothing is allocated: the scratch is one static device array of about 66 KiB
 * that every GPU loading this library keeps until the process exits, and the
 * launch uses at most KW_NOALLOC_MAX_BLOCKS blocks (grid-stride loops cover any
 * m up to KW_MAX_ROWS).  The first call on a device resolves the array's device
 * address for that device and keeps it for the life of the process (make that
 * first call before any stream capture).  The address belongs to the device's
 * primary context: do not call this entry point again on a device after
 * cudaDeviceReset or after its primary context was destroyed.  All calls share
 * the array and each call leaves its last contents there, so calls that
 * overlap on the GPU (other streams, other threads) race: serialise them.
 * Returns after synchronising cuda_stream.  Errors: KW_ERR_ARG (m < 1,
 * m > KW_MAX_ROWS, nnz > KW_MAX_NNZ, NULL pointer), KW_ERR_CUDA. */
kw_status kw_spmv_dot_noalloc(int64_t m, int64_t nnz, const int64_t* rowptr_dev, const int32_t* col_dev,
                              const double* val_dev, kw_c128 zs, const kw_c128* r_dev, kw_c128* q_dev,
                              kw_c128* t_host, void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* KOMEGA_GB300_H */
