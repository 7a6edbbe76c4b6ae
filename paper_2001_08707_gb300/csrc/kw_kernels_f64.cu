// FP64 instantiation of the iteration kernels (complex FP64 vectors and values).
#include "kw_kernels.cuh"

namespace kw {
template cudaError_t launch_init<PREC_F64>(Work&);
template cudaError_t launch_iteration<PREC_F64>(Work&, int, int, cudaEvent_t*, int64_t*);
template cudaError_t launch_finish_x<PREC_F64>(Work&);
template cudaError_t launch_unfinish_x<PREC_F64>(Work&);
template cudaError_t launch_k1<PREC_F64>(Work&, void*, void*);
template cudaError_t launch_update_xp<PREC_F64>(Work&, const void*, State*, int, cudaStream_t);
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

static __global__ void k_fingerprint(int m, const int64_t* __restrict__ rowptr, const int* __restrict__ col,
                                     const double* __restrict__ val, long long* out) {
  for (int t = threadIdx.x; t < kTuneSamples; t += blockDim.x) {
    const long long row = m > 1 ? (long long)t * (m - 1) / (kTuneSamples - 1) : 0;
    const int64_t b = rowptr[row], e = rowptr[row + 1];
    out[4 * t] = row;
    out[4 * t + 1] = (long long)(e - b);
    out[4 * t + 2] = e > b ? (long long)col[b] : -1;
    out[4 * t + 3] = e > b ? __double_as_longlong(val[b]) : 0;
  }
}

cudaError_t launch_fingerprint(int m, const int64_t* rowptr, const int* col, const double* val, long long* out,
                               cudaStream_t s) {
  k_fingerprint<<<1, kTuneSamples, 0, s>>>(m, rowptr, col, val, out);
  return cudaGetLastError();
}

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

// Last node of a device-side loop body: one more trip while *count < target
// and fewer than loop[1] trips have run (loop[0] counts them, so the loop ends
// even if the stop flag is never raised).
static __global__ void k_loop_cond(const int* count, int target, unsigned* loop, cudaGraphConditionalHandle h) {
  const unsigned trips = loop[0] + 1;
  loop[0] = trips;
  cudaGraphSetConditional(h, (*count < target && trips < loop[1]) ? 1u : 0u);
}

cudaError_t launch_loop_cond(const int* count, int target, unsigned* loop, cudaGraphConditionalHandle h,
                             cudaStream_t s) {
  k_loop_cond<<<1, 1, 0, s>>>(count, target, loop, h);
  return cudaGetLastError();
}

// Bilinear forms y_k^T H x_k of one term for every shift; partials need
// kBilinearTile * nblk * ceil(K / kBilinearTile) double2.
cudaError_t launch_bilinear(int m, int K, const int64_t* rowptr, const int* col, const double* val, const void* X,
                            const void* Y, int x32, int nblk, double2* part, int term, int nterm, double2* out,
                            cudaStream_t s) {
  const int ntile = (K + kBilinearTile - 1) / kBilinearTile;
  if (x32)
    k_bilinear<kBilinearTile, float2><<<dim3(nblk, ntile), 256, 0, s>>>(m, K, rowptr, col, val, (const float2*)X,
                                                                        (const float2*)Y, part);
  else
    k_bilinear<kBilinearTile, double2><<<dim3(nblk, ntile), 256, 0, s>>>(m, K, rowptr, col, val, (const double2*)X,
                                                                         (const double2*)Y, part);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_bilinear_reduce<kBilinearTile><<<(K + 127) / 128, 128, 0, s>>>(K, nblk, term, nterm, part, out);
  return cudaGetLastError();
}

cudaError_t launch_diag_scan(int m, const int64_t* rowptr, const int* col, const double* val, double* d, int* flag,
                             int num_sms, cudaStream_t s) {
  const int grid = std::max(1, std::min(4 * num_sms, (m + 255) / 256));
  k_diag_scan<<<grid, 256, 0, s>>>(m, rowptr, col, val, d, flag);
  return cudaGetLastError();
}

cudaError_t launch_bilinear_diag(int m, int K, const double* d, const DiagGroup& g, const void* X, const void* Y,
                                 int x32, int nblk, double2* part, int nterm, double2* out, cudaStream_t s) {
  for (int k0 = 0; k0 < K; k0 += 65535) {   // the grid's y extent
    const dim3 grid(nblk, std::min(K - k0, 65535));
    if (x32)
      k_bilinear_diag<kDiagGroup, float2><<<grid, 256, 0, s>>>(m, k0, d, g, (const float2*)X, (const float2*)Y, part);
    else
      k_bilinear_diag<kDiagGroup, double2><<<grid, 256, 0, s>>>(m, k0, d, g, (const double2*)X, (const double2*)Y,
                                                                 part);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  k_bilinear_diag_reduce<kDiagGroup><<<(K * g.n + 127) / 128, 128, 0, s>>>(K, nblk, g, nterm, part, out);
  return cudaGetLastError();
}

cudaError_t launch_shift_combine(int m, int K, int nk, const void* X, int x32, const double2* W, double2* S,
                                 int num_sms, cudaStream_t s) {
  const int grid = std::max(1, std::min(8 * num_sms, (m + 255) / 256));
  if (nk <= 8) {
    if (x32) k_shift_combine<8, float2><<<grid, 256, 0, s>>>(m, K, nk, (const float2*)X, W, S);
    else k_shift_combine<8, double2><<<grid, 256, 0, s>>>(m, K, nk, (const double2*)X, W, S);
  } else {
    if (x32) k_shift_combine<kMaxCombine, float2><<<grid, 256, 0, s>>>(m, K, nk, (const float2*)X, W, S);
    else k_shift_combine<kMaxCombine, double2><<<grid, 256, 0, s>>>(m, K, nk, (const double2*)X, W, S);
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------- uniform off-diagonal layout
// fm[0]: smallest index of an off-diagonal entry (ULLONG_MAX if none);
// fm[1]: off-diagonal entries whose value differs bitwise from that entry's.
static __global__ void k_u_first(int m, const int64_t* __restrict__ rowptr, const int* __restrict__ col,
                                 unsigned long long* fm) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
    for (int64_t j = rowptr[i]; j < rowptr[i + 1]; ++j) {
      if (col[j] != i) {
        atomicMin(fm, (unsigned long long)j);
        break;
      }
    }
  }
}

static __global__ void k_u_count(int m, const int64_t* __restrict__ rowptr, const int* __restrict__ col,
                                 const double* __restrict__ val, unsigned long long* fm, int* __restrict__ dcount) {
  const unsigned long long first = fm[0];
  const long long v0 = first == ~0ull ? 0 : __double_as_longlong(val[first]);
  unsigned long long bad = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
    int d = 0;
    for (int64_t j = rowptr[i]; j < rowptr[i + 1]; ++j) {
      if (col[j] == i) ++d;
      else bad += __double_as_longlong(val[j]) != v0;
    }
    dcount[i] = d;
  }
  bad = warp_sum(bad);
  if ((threadIdx.x & 31) == 0 && bad) atomicAdd(fm + 1, bad);
}

cudaError_t launch_uniform_check(int m, const int64_t* rowptr, const int* col, const double* val,
                                 unsigned long long* fm, int* dcount, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(fm, 0xff, sizeof(unsigned long long), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(fm + 1, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  const int grid = std::max(1, std::min(4096, (m + 255) / 256));
  k_u_first<<<grid, 256, 0, s>>>(m, rowptr, col, fm);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_u_count<<<grid, 256, 0, s>>>(m, rowptr, col, val, fm, dcount);
  return cudaGetLastError();
}

// Exclusive scan of dcount in blocks of 1024 (in place), block totals to tot.
static __global__ void __launch_bounds__(1024) k_scan_blocks(int m, int* __restrict__ v, int* __restrict__ tot) {
  __shared__ int ws[32];
  const int i = blockIdx.x * 1024 + threadIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int x = i < m ? v[i] : 0;
  int inc = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(KW_FULL_MASK, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) ws[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    int w = ws[lane], wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(KW_FULL_MASK, wi, o);
      if (lane >= o) wi += y;
    }
    ws[lane] = wi - w;   // exclusive prefix of the warp totals
    if (lane == 31) tot[blockIdx.x] = wi;
  }
  __syncthreads();
  if (i < m) v[i] = ws[warp] + inc - x;
}

// Exclusive scan of the nb block totals in place (one block of 1024 threads,
// each owning a contiguous segment).
static __global__ void __launch_bounds__(1024) k_scan_tops(int nb, int* __restrict__ tot) {
  __shared__ int ws[32];
  const int seg = (nb + 1023) / 1024, t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int b0 = min(nb, t * seg), b1 = min(nb, b0 + seg);
  int local = 0;
  for (int b = b0; b < b1; ++b) local += tot[b];
  int inc = local;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(KW_FULL_MASK, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) ws[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    int w = ws[lane], wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(KW_FULL_MASK, wi, o);
      if (lane >= o) wi += y;
    }
    ws[lane] = wi - w;
  }
  __syncthreads();
  int run = ws[warp] + inc - local;
  for (int b = b0; b < b1; ++b) {
    const int x = tot[b];
    tot[b] = run;
    run += x;
  }
}

// Row i: its off-diagonal columns start at rowptr[i] minus the diagonal entries
// of the rows before it; the diagonal entries of the row are summed.
static __global__ void k_u_fill(int m, const int64_t* __restrict__ rowptr, const int* __restrict__ col,
                                const double* __restrict__ val, const int* __restrict__ dpre,
                                const int* __restrict__ tops, int* __restrict__ u_rowptr, int* __restrict__ u_col,
                                double* __restrict__ diag) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
    const int64_t b = rowptr[i] - (dpre[i] + tops[i >> 10]);
    int k = 0;
    double d = 0.0;
    for (int64_t j = rowptr[i]; j < rowptr[i + 1]; ++j) {
      if (col[j] == i) d += val[j];
      else u_col[b + k++] = col[j];
    }
    u_rowptr[i] = (int)b;
    diag[i] = d;
    if (i == m - 1) u_rowptr[m] = (int)(b + k);
  }
}

cudaError_t launch_uniform_build(int m, const int64_t* rowptr, const int* col, const double* val, int* dcount,
                                 int* scratch, int* u_rowptr, int* u_col, double* diag, cudaStream_t s) {
  const int nb = (m + 1023) / 1024;
  k_scan_blocks<<<nb, 1024, 0, s>>>(m, dcount, scratch);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_scan_tops<<<1, 1024, 0, s>>>(nb, scratch);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const int grid = std::max(1, std::min(4096, (m + 255) / 256));
  k_u_fill<<<grid, 256, 0, s>>>(m, rowptr, col, val, dcount, scratch, u_rowptr, u_col, diag);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- SELL-32 copy of the uniform layout
// Slots of each 32-row slice (its longest row) into cnt, and their sum over
// all slices (64-bit) into *total.
static __global__ void __launch_bounds__(256) k_us_count(int m, int nslice, const int* __restrict__ u_rowptr,
                                                         int* __restrict__ cnt, unsigned long long* total) {
  unsigned long long acc = 0;
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < nslice; s += gridDim.x * blockDim.x) {
    const int r0 = s * 32, r1 = min(r0 + 32, m);
    int mx = 0;
    for (int r = r0; r < r1; ++r) mx = max(mx, u_rowptr[r + 1] - u_rowptr[r]);
    cnt[s] = mx;
    acc += (unsigned long long)mx;
  }
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0 && acc) atomicAdd(total, acc);
}

// sptr[s] = block-local exclusive prefix + the prefix of the block totals;
// sptr[nslice] = the total.
static __global__ void k_us_ptr(int nslice, int* __restrict__ sptr, const int* __restrict__ tops, int last_cnt) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < nslice; s += gridDim.x * blockDim.x) {
    const int v = sptr[s] + tops[s >> 10];
    sptr[s] = v;
    if (s == nslice - 1) sptr[nslice] = v + last_cnt;
  }
}

// One warp per slice: slot k of lane t = the k-th off-diagonal column of row
// 32 s + t, or -1 past the row's end (or past m).
static __global__ void __launch_bounds__(256) k_us_fill(int m, int nslice, const int* __restrict__ u_rowptr,
                                                        const int* __restrict__ u_col, const int* __restrict__ sptr,
                                                        int* __restrict__ scol) {
  const int lane = threadIdx.x & 31;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int s = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; s < nslice; s += nw) {
    const int row = s * 32 + lane;
    int beg = 0, len = 0;
    if (row < m) {
      beg = u_rowptr[row];
      len = u_rowptr[row + 1] - beg;
    }
    const int k0 = sptr[s], n = sptr[s + 1] - k0;
    for (int k = 0; k < n; ++k) scol[(size_t)(k0 + k) * 32 + lane] = k < len ? u_col[beg + k] : -1;
  }
}

cudaError_t launch_uniform_sell_count(int m, const int* u_rowptr, int* cnt, unsigned long long* total,
                                      cudaStream_t s) {
  const int nslice = (m + 31) / 32;
  cudaError_t e = cudaMemsetAsync(total, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  const int grid = std::max(1, std::min(1024, (nslice + 255) / 256));
  k_us_count<<<grid, 256, 0, s>>>(m, nslice, u_rowptr, cnt, total);
  return cudaGetLastError();
}

cudaError_t launch_uniform_sell_fill(int m, const int* u_rowptr, const int* u_col, int* sptr, int* scratch,
                                     int last_cnt, int* scol, cudaStream_t s) {
  const int nslice = (m + 31) / 32;
  const int nb = (nslice + 1023) / 1024;
  k_scan_blocks<<<nb, 1024, 0, s>>>(nslice, sptr, scratch);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_scan_tops<<<1, 1024, 0, s>>>(nb, scratch);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_us_ptr<<<std::max(1, std::min(1024, (nslice + 255) / 256)), 256, 0, s>>>(nslice, sptr, scratch, last_cnt);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_us_fill<<<std::max(1, std::min(4096, (nslice + 7) / 8)), 256, 0, s>>>(m, nslice, u_rowptr, u_col, sptr, scol);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- spin operator set-up
static __global__ void k_binom(int* binom) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  for (int n = 0; n < KW_BINOM_N; ++n)
    for (int k = 0; k < KW_BINOM_K; ++k)
      binom[n * KW_BINOM_K + k] =
          k == 0 ? 1 : (n == 0 || k > n) ? 0 : binom[(n - 1) * KW_BINOM_K + k - 1] + binom[(n - 1) * KW_BINOM_K + k];
}

// Word of rank `row` among the nsite-bit words with nup set bits (increasing
// order): greedily take, for t = nup .. 1, the highest position p with
// C(p, t) <= the remaining rank (the combinatorial number system).
static __global__ void k_spin_basis(int m, int nsite, int nup, const int* __restrict__ binom, unsigned* basis) {
  for (int row = blockIdx.x * blockDim.x + threadIdx.x; row < m; row += gridDim.x * blockDim.x) {
    int rem = row;
    unsigned wd = 0;
    int p = nsite - 1;
    for (int t = nup; t >= 1; --t) {
      while (binom[p * KW_BINOM_K + t] > rem) --p;
      wd |= 1u << p;
      rem -= binom[p * KW_BINOM_K + t];
      --p;
    }
    basis[row] = wd;
  }
}

static __global__ void k_spin_diag(int m, int nsite, int nbond, const int* __restrict__ bond,
                                   const double* __restrict__ J, const double* __restrict__ h,
                                   const unsigned* __restrict__ basis, double* __restrict__ diag) {
  for (int row = blockIdx.x * blockDim.x + threadIdx.x; row < m; row += gridDim.x * blockDim.x) {
    const unsigned wd = basis[row];
    double d = 0.0;
    for (int b = 0; b < nbond; ++b) {
      const int a = bond[b] & 255, c = bond[b] >> 8;
      d += ((((wd >> a) ^ (wd >> c)) & 1u) ? -0.25 : 0.25) * J[b];
    }
    if (h)
      for (int i = 0; i < nsite; ++i) d += (((wd >> i) & 1u) ? 0.5 : -0.5) * h[i];
    diag[row] = d;
  }
}

static __global__ void k_spin_table(int m, int nbond, const int* __restrict__ bond, const int* __restrict__ binom_g,
                                    const unsigned* __restrict__ basis, int* __restrict__ table) {
  __shared__ int binom[KW_BINOM_N * KW_BINOM_K];
  for (int i = threadIdx.x; i < KW_BINOM_N * KW_BINOM_K; i += blockDim.x) binom[i] = binom_g[i];
  __syncthreads();
  for (int row = blockIdx.x * blockDim.x + threadIdx.x; row < m; row += gridDim.x * blockDim.x) {
    const unsigned sw = basis[row];
    for (int b = 0; b < nbond; ++b) {
      const int a = bond[b] & 255, c = bond[b] >> 8;
      table[(size_t)b * m + row] = (((sw >> a) ^ (sw >> c)) & 1u) ? spin_exchange_row(sw, row, a, c, binom) : -1;
    }
  }
}

cudaError_t launch_spin_table(int m, int nbond, const int* bond, const int* binom, const unsigned* basis, int* table,
                              cudaStream_t s) {
  const int grid = std::max(1, std::min(8192, (m + 255) / 256));
  k_spin_table<<<grid, 256, 0, s>>>(m, nbond, bond, binom, basis, table);
  return cudaGetLastError();
}

cudaError_t launch_spin_setup(int m, int nsite, int nup, int nbond, const int* bond, const double* J, const double* h,
                              int* binom, unsigned* basis, double* diag, cudaStream_t s) {
  k_binom<<<1, 1, 0, s>>>(binom);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int grid = std::max(1, std::min(8192, (m + 255) / 256));
  k_spin_basis<<<grid, 256, 0, s>>>(m, nsite, nup, binom, basis);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_spin_diag<<<grid, 256, 0, s>>>(m, nsite, nbond, bond, J, h, basis, diag);
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
