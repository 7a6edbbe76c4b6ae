// FP64 instantiation of the iteration kernels (complex FP64 vectors and values).
#include "kw_kernels.cuh"

namespace kw {
template cudaError_t launch_init<PREC_F64>(Work&);
template cudaError_t launch_iteration<PREC_F64>(Work&, int, cudaEvent_t*, int64_t*);
template cudaError_t launch_finish_x<PREC_F64>(Work&);
template cudaError_t launch_project_x<PREC_F64>(Work&, double2*);
template cudaError_t launch_spmv_dot<PREC_F64>(Work&, const void*, void*, double2, float4, double2*);

cudaError_t launch_convert_f64_to_f32(const double* in, float* out, int64_t n, unsigned long long* inexact,
                                      cudaStream_t s) {
  k_f64_to_f32<<<1024, 256, 0, s>>>(in, out, n, inexact);
  return cudaGetLastError();
}

cudaError_t launch_convert_f64_to_pair(const double* in, void* out, int64_t n, cudaStream_t s) {
  k_f64_to_pair<<<1024, 256, 0, s>>>(in, (df*)out, n);
  return cudaGetLastError();
}
// SELL-32 construction, step 1: sorted order, row lengths, slice lengths.
cudaError_t launch_sell_order(int m, const int64_t* rowptr, int* perm, int* rlen, int* slen,
                                     cudaStream_t s) {
  const int nwin = (m + 1023) / 1024, nslice = (m + 31) / 32;
  k_sell_sort<<<nwin, 1024, 0, s>>>(m, rowptr, perm, rlen);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_sell_slicelen<<<(nslice + 255) / 256, 256, 0, s>>>(m, nslice, rlen, slen);
  return cudaGetLastError();
}

// Step 2 (after the host has formed the slice offsets): copy the entries.
template <class RV>
cudaError_t launch_sell_fill(int m, const int* perm, const int* rlen, const int64_t* sptr, const int64_t* rowptr,
                             const int* col, const void* val, int* scol, void* sval, cudaStream_t s) {
  const int nslice = (m + 31) / 32;
  k_sell_fill<RV><<<(nslice + 7) / 8, 256, 0, s>>>(m, nslice, perm, rlen, sptr, rowptr, col, (const RV*)val, scol,
                                                   (RV*)sval);
  return cudaGetLastError();
}

template cudaError_t launch_sell_fill<double>(int, const int*, const int*, const int64_t*, const int64_t*,
                                               const int*, const void*, int*, void*, cudaStream_t);
template cudaError_t launch_sell_fill<float>(int, const int*, const int*, const int64_t*, const int64_t*,
                                              const int*, const void*, int*, void*, cudaStream_t);
template cudaError_t launch_sell_fill<df>(int, const int*, const int*, const int64_t*, const int64_t*, const int*,
                                           const void*, int*, void*, cudaStream_t);

// Number of instances of a batch whose solve has stopped.
static __global__ void k_count_done(int n, State* const* states, int* out) {
  int c = 0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) c += states[i]->done ? 1 : 0;
  c = warp_sum((unsigned long long)c);
  __shared__ int sh[32];
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
    *out = t;
  }
}

cudaError_t launch_count_done(int n, State* const* states, int* out, cudaStream_t s) {
  k_count_done<<<1, 256, 0, s>>>(n, states, out);
  return cudaGetLastError();
}

// Bilinear forms y_k^T H x_k of one term for every shift; partials need
// kBilinearTile * nblk * ceil(K / kBilinearTile) double2.
cudaError_t launch_bilinear(int m, int K, const int64_t* rowptr, const int* col, const double* val,
                            const double2* X, const double2* Y, int nblk, double2* part, int term, int nterm,
                            double2* out, cudaStream_t s) {
  const int ntile = (K + kBilinearTile - 1) / kBilinearTile;
  k_bilinear<kBilinearTile><<<dim3(nblk, ntile), 256, 0, s>>>(m, K, rowptr, col, val, X, Y, part);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_bilinear_reduce<kBilinearTile><<<(K + 127) / 128, 128, 0, s>>>(K, nblk, term, nterm, part, out);
  return cudaGetLastError();
}

template <int LPS, int NPL>
static cudaError_t recalc_launch(int K, int np, long long n_iter, const double2* log, const double2* w0,
                                 const double2* z, double thresh, double2* proj, long long* conv_iter,
                                 double* final_res, int* flag, cudaStream_t s) {
  const size_t smem = (size_t)kRecalcChunk * (KW_LOG_FIXED + np) * sizeof(double2);
  constexpr int spb = kRecalcThreads / LPS;
  const int grid = (K + spb - 1) / spb;
  k_recalc<LPS, NPL><<<grid, kRecalcThreads, smem, s>>>(K, np, n_iter, log, w0, z, thresh, proj, conv_iter,
                                                        final_res, flag);
  return cudaGetLastError();
}

// Columns per lane, rounded up to a power of two, for LPS lanes per shift.
template <int LPS>
static cudaError_t recalc_npl(int K, int np, long long n_iter, const double2* log, const double2* w0,
                              const double2* z, double thresh, double2* proj, long long* conv_iter, double* final_res,
                              int* flag, cudaStream_t s) {
  const int per_lane = (np + LPS - 1) / LPS;
#define KW_RC(NPL) recalc_launch<LPS, NPL>(K, np, n_iter, log, w0, z, thresh, proj, conv_iter, final_res, flag, s)
  if (per_lane <= 1) return KW_RC(1);
  if constexpr (LPS <= 16) {
    if (per_lane <= 2) return KW_RC(2);
  }
  if constexpr (LPS <= 8) {
    if (per_lane <= 4) return KW_RC(4);
  }
  if constexpr (LPS <= 4) {
    if (per_lane <= 8) return KW_RC(8);
  }
  if constexpr (LPS <= 2) {
    if (per_lane <= 16) return KW_RC(16);
  }
  if constexpr (LPS == 1) return KW_RC(32);
#undef KW_RC
  return cudaErrorInvalidValue;
}

cudaError_t launch_recalc(int K, int np, long long n_iter, const double2* log, const double2* w0, const double2* z,
                          double thresh, double2* proj, long long* conv_iter, double* final_res, int* flag,
                          int num_sms, cudaStream_t s) {
  if (K < 1 || np < 0 || np > KW_MAX_PROJ || n_iter < 0 || !z || !proj || !conv_iter || !final_res || !flag ||
      (n_iter > 0 && !log) || (np > 0 && !w0))
    return cudaErrorInvalidValue;
  // Lanes per shift: double while there are fewer than two warps per SM and
  // a shift still has more than one column per lane.
  int lps = 1;
  while (lps < 32 && lps < np && (long long)K * lps < 2LL * 32 * num_sms) lps *= 2;
#define KW_RL(L) recalc_npl<L>(K, np, n_iter, log, w0, z, thresh, proj, conv_iter, final_res, flag, s)
  switch (lps) {
    case 1: return KW_RL(1);
    case 2: return KW_RL(2);
    case 4: return KW_RL(4);
    case 8: return KW_RL(8);
    case 16: return KW_RL(16);
    default: return KW_RL(32);
  }
#undef KW_RL
}
}  // namespace kw
