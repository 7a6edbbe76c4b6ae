// Internal definitions shared by the kernels and the host driver.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "komega_gb300.h"

namespace kw {

// Iteration state kept in device memory for the whole solve.  Every scalar of
// the seed recurrence (Eq. 16-17) and of the seed switch lives here in FP64,
// in both precision modes.
struct State {
  double2 zs;        // current seed shift z_s (Eq. 6)
  double2 rho;       // rho_n = r_n^T r_n (unconjugated, Appendix A)
  double2 rho1;      // rho_{n+1}
  double2 boa;       // beta_{n-1} / alpha_{n-1}
  double2 alpha;     // alpha_n (Eq. 17)
  double2 c;         // alpha_n beta_{n-1} / alpha_{n-1}
  double2 beta;      // beta_n = rho_{n+1} / rho_n
  double2 t;         // r_n^T A r_n
  double2 u;         // K1's r^T (z r - H r) for its seed zs_k1, before any pending seed switch
  double2 zs_k1;     // the seed shift K1 uses: the one current when the previous K2 ended
  float4 p_zs_k1;    // its FP32-pair image
  // Scalars of Eq. 17 formed by K1's last block for the case that the seed is
  // kept (K2 uses them unless a seed switch is pending)
  double2 k1_alpha, k1_c, k1_inv_rho, k1_inv_rho_alpha, k1_t;
  int k1_status;     // 0, KW_ERR_BREAKDOWN or KW_ERR_NONFINITE
  int pad2;
  double2 inv_rho;   // 1 / rho_n
  double2 inv_rho_alpha;  // 1 / (rho_n alpha_n)
  double nu;         // ||r_{n+1}||_2^2
  double thresh;     // tol * ||b||
  double norm_b;
  // Seed switch without touching the vectors: bscale[b] is the pending factor
  // of residual buffer b (0: rA, 1: rB) that K2 folds into its coefficients;
  // switched: the last K3 switched the seed (K2 then re-forms alpha_n).
  double2 bscale[2];
  double2 inv_pj1, inv_pj0;  // 1/pi^j_{n+1}, 1/pi^j_n for the lazy pi rescale in K3
  // FP32-pair images (re.hi, re.lo, im.hi, im.lo) of the scalars the vector
  // kernels use, written next to their FP64 values; the FP32 form uses the .hi parts.
  float4 p_zs, p_alpha, p_c, p_opc;
  int switched;
  int pi_rescale_pending;
  int new_seed;
  int seed;
  int seed_switch;
  int done;
  int status;
  int n_active;
  // shifts processed in an iteration (compacted list length) and whether its
  // full-mode x/p update is pending, by iteration parity: K4(n) may still run
  // while K2(n+1) and K3(n+1) use the other slot
  int n_list[2];
  int xp_pending[2];
  int n_seed_switch;
  int pad0;
  long long iter, maxiter, updates;
  long long hist_stride, hist_max, n_rec;
  unsigned int cnt_spmv, cnt_seed, cnt_shift, cnt_xp, cnt_init;
  unsigned int pad1;
};

enum Prec { PREC_F64 = 0, PREC_C32 = 1, PREC_DF = 2 };
enum OpKind { OP_CSR = 0, OP_CALLBACK = 1, OP_SPIN = 2, OP_LATTICE = 3 };
// Binomial table of the spin operator: C(n, k) for n < KW_BINOM_N, k < KW_BINOM_K.
constexpr int KW_BINOM_N = 32;
constexpr int KW_BINOM_K = 34;

// Device buffers of one solve.  Vector buffers are void* and typed by precision.
struct Work {
  int prec;
  int64_t m;
  int K;           // shifts
  int nproj;       // projection rows used by the iteration incl. b (0 in full mode)
  int nout;        // output columns: b plus the left vectors
  double tol;
  bool full;
  // operator
  const int64_t* rowptr;
  const int32_t* col;
  const void* val;   // double* (F64) or float* (C32)
  int spmv_lanes;    // lanes per row in K1 (1 = one thread per row); KW_SPMV_SELL = SELL-32 layout
  // SELL-32 copy of the operator (used when spmv_lanes == KW_SPMV_SELL)
  const int* sell_perm;      // [m] sorted position -> row
  const int* sell_len;       // [m] row length at each sorted position
  const int64_t* sell_ptr;   // [nslice + 1] start of each slice
  const int* sell_col;       // [padded nnz]
  const void* sell_val;      // [padded nnz] in the SpMV value type
  // Uniform off-diagonal copy of the operator (spmv_lanes >= KW_SPMV_UNIFORM):
  // H r = diag * r + u_v * (sum of r over the off-diagonal columns of the row).
  const int* u_rowptr;       // [m + 1] int32 offsets into u_col
  const int* u_col;          // off-diagonal columns only
  const void* u_diag;        // [m] diagonal: double, float (u_kind 1) or FP32 pair (u_kind 2)
  int u_kind;                // 0: FP64 diagonal and value, 1: FP32 (exact), 2: FP32 pair
  double u_v;                // the off-diagonal value
  const int* u_sptr = nullptr;   // SELL-32 copy: [nslice + 1] first slot of each 32-row slice
  const int* u_scol = nullptr;   // [slots * 32] slot-major off-diagonal columns, -1 = none
  int val_f32;       // matrix values stored as FP32 (always in C32 mode; in F64 mode when lossless)
  // seed vectors
  void* rA;          // two rotating residual buffers and q
  void* rB;
  void* q;
  const double* b;   // caller's b (FP64)
  const double* left;  // caller's left vectors (FP64) [nproj-1][m]
  void* proj_rows;   // [nproj][proj_ld] real, vector precision (b then left vectors)
  int64_t proj_ld;   // row stride of proj_rows: m rounded up to KW_PROJ_ALIGN elements (16-byte aligned rows)
  int bulk = -1;     // K2 tile staging by TMA bulk copies: -1 auto (more than 9 projection rows), 0 off, 1 on, 2 test
  int seed_rg = -1;  // K2 row-group form (pair form): -1 auto (more than 9 projection rows), 0 off, 1 on
  // shift state
  double2* z;
  double2* pi1;      // pi_n
  double2* pi0;      // pi_{n-1}
  int* active;
  long long* conv_iter;
  double* final_res;
  double2* coef;     // full mode: [K][3] = alpha^k, beta^k, 1/pi^k_{n+1}
  float4* coef_pair; // the same as FP32 pairs
  double2* Y;        // projected: [K][nproj]
  double2* U;
  double2* w;        // [nproj] = P r_{n+1}
  double2* w0;       // [nproj] = P b
  double* hist;
  int* list;
  void* X;           // full mode [K][m]
  void* P;           // full mode [K][m]
  int xp_tile = 8;   // shifts per tile of K4 (4, 8 or 16; picked by the autotuner)
  int xp32 = 0;      // full mode: X and P stored as complex FP32 (float2) whatever the form; the
                     // projections then come from the projected recurrences (nproj = nout)
  // operator kind: CSR arrays (spmv_lanes picks the layout), callback, or generated on the fly
  int op = 0;             // OP_CSR, OP_CALLBACK, OP_SPIN, OP_LATTICE
  // spin operator (kw_set_spin_operator); diagonal in u_diag/u_kind, uniform J/2 in u_v
  const unsigned* sp_basis = nullptr;   // [m] basis words, increasing
  const int* sp_binom = nullptr;        // [KW_BINOM_N][KW_BINOM_K] binomial coefficients
  const int* sp_bond = nullptr;         // [nbond] a | (c << 8), a < c
  const void* sp_val = nullptr;         // [nbond] J_b/2 in the diagonal's storage (when not uniform)
  int sp_nbond = 0;
  int sp_uniform = 0;                   // every J_b equal: one value u_v
  const int* sp_table = nullptr;        // optional [nbond][m] exchange columns (-1: parallel spins)
  // lattice operator (kw_set_lattice3d): eps in u_diag/u_kind, hopping in u_v
  int lx = 0, ly = 0, lz = 0;
  // solver of Table 1 and the BiCG shadow vectors (rotating like rA/rB) and A^dagger r~
  int method = KW_METHOD_COCG;
  void* rtA = nullptr;
  void* rtB = nullptr;
  void* qt = nullptr;
  const double* btilde = nullptr;   // BiCG r~_0 (NULL: b)
  // operator given as a callback (kw_set_matvec) instead of the CSR arrays
  kw_matvec_fn mv_fn = nullptr;
  void* mv_user = nullptr;
  kw_matvec_fn mv_fn_adj = nullptr;   // q = H^dagger r (BiCG; NULL: H Hermitian)
  void* mv_user_adj = nullptr;
  int mv_adjoint = 0;                 // set while K1 forms the adjoint product
  void* mv_r2 = nullptr;              // FP32-pair form, BiCG under reverse communication:
  void* mv_q2 = nullptr;              // staging of the shadow product (both are outstanding)
  // reverse communication (kw_rci_*): the caller computes the products between calls.
  // rci_phase 1: stage the vectors and record them (no product); 2: finish the products
  int rci = 0;
  int rci_phase = 0;
  const void* rci_r = nullptr;
  void* rci_q = nullptr;
  const void* rci_rt = nullptr;
  void* rci_qt = nullptr;
  void* mv_r = nullptr;   // FP32-pair form: kw_c128 copy of r handed to the callback
  void* mv_q = nullptr;   // FP32-pair form: the callback's H r (kw_c128)
  int mv_failed = 0;      // set when the callback returned nonzero
  // Krylov log for recalculation (NULL = off): rows [log_max][KW_LOG_FIXED + nproj]
  double2* log = nullptr;
  long long log_max = 0;
  // reduction scratch (part_k1: K1's own, since K1 overlaps K3)
  double* part;
  double* part_k1 = nullptr;
  // second stream for K3/K4 and the events that order the two streams
  cudaStream_t stream2 = nullptr;
  cudaEvent_t ev_k2 = nullptr, ev_k3 = nullptr;
  // K4 on a third stream: K4(n) overlaps K2(n+1), K1(n+2) and K3(n+1);
  // ev_k4[n & 1] marks K4(n)'s end.  k4_mask: the parities whose ev_k4 was
  // recorded since the last join (a wait only ever names an event recorded
  // in the same launch sequence, which a stream capture requires).
  cudaStream_t stream3 = nullptr;
  cudaEvent_t ev_k4[2] = {nullptr, nullptr};
  int k4_mask = 0;
  int overlap = 1;   // 0: K3/K4 on the work stream after K1(n+1), no events
  State* st;
  cudaStream_t stream;
  int num_sms;
};

// Make the work stream wait for the shift and update streams (end of a chunk of iterations).
inline cudaError_t join_streams(Work& w) {
  if (!w.overlap) return cudaSuccess;
  cudaError_t e = cudaStreamWaitEvent(w.stream, w.ev_k3, 0);
  for (int i = 0; i < 2 && e == cudaSuccess; ++i)
    if (w.k4_mask & (1 << i)) e = cudaStreamWaitEvent(w.stream, w.ev_k4[i], 0);
  w.k4_mask = 0;
  return e;
}

// Launchers implemented per precision (kw_kernels_f64.cu / kw_kernels_c32.cu).
template <int P> cudaError_t launch_init(Work& w);
// first: the first iteration after launch_init or after join_streams (no wait for K3).
template <int P> cudaError_t launch_iteration(Work& w, int parity, int first, cudaEvent_t* ev, int64_t* launches);
template <int P> cudaError_t launch_finish_x(Work& w);
template <int P> cudaError_t launch_unfinish_x(Work& w);
template <int P> cudaError_t launch_k1(Work& w, void* r, void* rt);
// K4 on the Work's X, P for the compacted list of iteration parity `parity`
// (its coefficient and list slots), with the given state (the solve's, or a
// scratch state when the autotuner times the tiles).
template <int P> cudaError_t launch_update_xp(Work& w, const void* r1, State* st, int parity, cudaStream_t s);
template <int P> cudaError_t launch_project_x(Work& w, double2* out);
template <int P>
cudaError_t launch_spmv_dot(Work& w, const void* r, void* q, double2 zs, float4 zs_pair, double2* t_dev);
cudaError_t launch_convert_f64_to_f32(const double* in, float* out, int64_t n, unsigned long long* inexact,
                                      cudaStream_t s);
cudaError_t launch_convert_f64_to_pair(const double* in, void* out, int64_t n, cudaStream_t s);

// spmv_lanes value that selects the SELL-32 layout.
constexpr int KW_SPMV_SELL = 32;
// spmv_lanes = KW_SPMV_UNIFORM + G selects the uniform off-diagonal layout with
// G lanes per row (G = 1, 2, 4, 8, 16); KW_SPMV_UNIFORM_SELL selects the same
// layout stored as SELL-32 (slot-major columns of 32-row slices, one lane per row).
constexpr int KW_SPMV_UNIFORM = 64;
constexpr int KW_SPMV_UNIFORM_SELL = KW_SPMV_UNIFORM + 32;
// Uniform off-diagonal layout: find the first off-diagonal entry and count the
// off-diagonal values that differ from it (bitwise) and the diagonal entries
// per row (dcount [m]); then build u_rowptr, u_col and the FP64 diagonal.
// scratch: [nblk] ints for the scan, nblk = ceil(m / 1024).
cudaError_t launch_uniform_check(int m, const int64_t* rowptr, const int* col, const double* val,
                                 unsigned long long* first_and_mismatch, int* dcount, cudaStream_t s);
cudaError_t launch_uniform_build(int m, const int64_t* rowptr, const int* col, const double* val, int* dcount,
                                 int* scratch, int* u_rowptr, int* u_col, double* diag, cudaStream_t s);
// SELL-32 copy of the uniform layout (spmv_lanes == KW_SPMV_UNIFORM_SELL):
// count: cnt[s] = slots of slice s (its longest row), *total = their sum;
// fill: cnt becomes the slice offsets sptr [nslice + 1] (in place; scratch
// [ceil(nslice / 1024)] ints; last_cnt = cnt[nslice - 1] before the call) and
// scol [total * 32] receives the slot-major columns, -1 past a row's end.
cudaError_t launch_uniform_sell_count(int m, const int* u_rowptr, int* cnt, unsigned long long* total,
                                      cudaStream_t s);
cudaError_t launch_uniform_sell_fill(int m, const int* u_rowptr, const int* u_col, int* sptr, int* scratch,
                                     int last_cnt, int* scol, cudaStream_t s);
cudaError_t launch_sell_order(int m, const int64_t* rowptr, int* perm, int* rlen, int* slen, cudaStream_t s);
template <class RV>
cudaError_t launch_sell_fill(int m, const int* perm, const int* rlen, const int64_t* sptr, const int64_t* rowptr,
                             const int* col, const void* val, int* scol, void* sval, cudaStream_t s);

// Spin operator set-up: binomial table, basis words of rank 0..m-1 (nsite bits,
// nup set), and the FP64 diagonal (bond terms +-J/4, field terms +-h/2).
cudaError_t launch_spin_setup(int m, int nsite, int nup, int nbond, const int* bond, const double* J, const double* h,
                              int* binom, unsigned* basis, double* diag, cudaStream_t s);
// Exchange table of a spin operator: table[b*m + row] = the row of the word with
// bond b's spins exchanged, or -1 when they are parallel.
cudaError_t launch_spin_table(int m, int nbond, const int* bond, const int* binom, const unsigned* basis, int* table,
                              cudaStream_t s);

// Fingerprint of a CSR operator for the persistent tuning cache: for kTuneSamples
// rows spread over [0, m), out[4s..4s+3] = row, rowptr[row+1] - rowptr[row], the
// row's first column (or -1) and its value's bits (or 0).
constexpr int kTuneSamples = 256;
cudaError_t launch_fingerprint(int m, const int64_t* rowptr, const int* col, const double* val, long long* out,
                               cudaStream_t s);

// Batched solves: count of instances whose solve has stopped (written to *out).
cudaError_t launch_count_done(int n, State* const* states, int* out, cudaStream_t s);
// Loop condition of a CUDA graph WHILE node: continue while *count < target and
// loop[0] (trips so far, incremented here) < loop[1].
cudaError_t launch_loop_cond(const int* count, int target, unsigned* loop, cudaGraphConditionalHandle h,
                             cudaStream_t s);

// Adjoint bilinear forms (kw_bilinear): shifts per tile and the launcher.
constexpr int kBilinearTile = 8;
// Combinations over the shifts (kw_shift_combine): S [nk][m] = W [nk][K] X [K][m],
// X kw_c128 (x32 = 0) or complex FP32 (x32 = 1), W and S FP64 complex; nk <= kMaxCombine.
constexpr int kMaxCombine = 16;
cudaError_t launch_shift_combine(int m, int K, int nk, const void* X, int x32, const double2* W, double2* S,
                                 int num_sms, cudaStream_t s);
// X, Y: [K][m] kw_c128 (x32 = 0) or complex FP32 (x32 = 1).
cudaError_t launch_bilinear(int m, int K, const int64_t* rowptr, const int* col, const double* val, const void* X,
                            const void* Y, int x32, int nblk, double2* part, int term, int nterm, double2* out,
                            cudaStream_t s);
// Diagonal terms of kw_bilinear.  launch_diag_scan: d[i] = the row's diagonal
// entry (0 for an empty row); *flag is cleared if some row holds anything else
// (an entry off the diagonal, or more than one entry).  launch_bilinear_diag:
// out[k * nterm + idx[t]] = sum_i d_t[i] y_k[i] x_k[i] for the n <= kDiagGroup
// terms of one group (d_t = d + idx[t] * m), all shifts in one pass over X and
// Y; part holds K * nblk * kDiagGroup double2.
constexpr int kDiagGroup = 16;
struct DiagGroup {
  int n;
  int idx[kDiagGroup];
};
cudaError_t launch_diag_scan(int m, const int64_t* rowptr, const int* col, const double* val, double* d, int* flag,
                             int num_sms, cudaStream_t s);
cudaError_t launch_bilinear_diag(int m, int K, const double* d, const DiagGroup& g, const void* X, const void* Y,
                                 int x32, int nblk, double2* part, int nterm, double2* out, cudaStream_t s);

// Recalculation at new shifts (kw_recalc): threads per block, log rows per
// shared-memory chunk, and the launcher (flag: set to 1 on breakdown).
constexpr int KW_PROJ_ALIGN = 64;   // elements; projection rows start 16-byte aligned in every form
constexpr int kRecalcThreads = 32;
constexpr int kRecalcChunk = 16;
cudaError_t launch_recalc(int K, int np, long long n_iter, const double2* log, const double2* w0, const double2* z,
                          double thresh, double2* proj, long long* conv_iter, double* final_res, int* flag,
                          int num_sms, cudaStream_t s);

// Upper bound on resident 256-thread blocks per SM (2048 threads per SM).
constexpr int kMaxBlocksPerSM = 8;

// Scratch needed by the reduction kernels (doubles).
int64_t part_doubles(const Work& w);
void choose_grids(Work& w);

}  // namespace kw
