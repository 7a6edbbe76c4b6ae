// Kernels of one shifted-COCG iteration (Komega paper, Sec. 2.2, Appendix A).
//
//   K1 k_spmv_dot     q = A r_n = z_s r_n - H r_n and t_n = r_n^T q (Alg. 1 "q = H r",
//                     Eq. 17); last block: alpha_n, c_n = alpha_n beta_{n-1}/alpha_{n-1}.
//   K2 k_seed_update  r_{n+1} = (1+c_n) r_n - alpha_n q - c_n r_{n-1} (Eq. 16), with
//                     rho_{n+1} = r^T r, nu = r^dagger r and w_l = a_l^T r_{n+1} (the
//                     P r_{n+1} of Eq. 26); last block: beta_n = rho_{n+1}/rho_n.
//                     With more than 9 projection rows (FP32 and pair forms) its tiles
//                     are staged in shared memory by TMA bulk copies on mbarriers.
//   K3 k_shift        per active shift: pi_{n+1} (Eq. 20), alpha^k, beta^k (Eq. 21-22),
//                     projected y/u update (Eq. 25-26), residual ||r||/|pi|, freeze,
//                     compaction; last block: seed switch (Sec. 2.2.4), stop flag.
//   K4 k_update_xp    full mode: x^k += alpha^k p^k; p^k = r_{n+1}/pi^k + beta^k p^k
//                     (Eq. 23-24) for the compacted active shifts.
//
// Three vector forms share these kernels through kw_arith.cuh: FP64 (double2),
// FP32 (float2; FP32 partials over at most 16 terms per lane, FP64 across
// chunks, warps and blocks) and FP32 pairs (dfc, 48-bit significand on the FP32
// pipes).  Every seed and shift scalar is FP64 in all three; kernels read the
// FP32 / FP32-pair images of the scalars they need from the State, written by
// the reduction tails, so no kernel converts FP64 scalars per thread.
//
// Every kernel reads the iteration state from device memory, so the host only
// enqueues launches; no host synchronisation happens inside the loop.
// Reductions are deterministic: fixed per-block partials summed in a fixed
// order by the last block to finish (arrival counter, no spin-wait).  The only
// waits are the staged K2's mbarrier waits, each bounded by a poll limit after
// which the solve stops with KW_ERR_TIMEOUT.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <utility>
#include <type_traits>

#include "kw_arith.cuh"
#include "kw_bulk.cuh"
#include "kw_internal.cuh"

namespace kw {

template <int P> struct PT;
template <> struct PT<PREC_F64> {
  typedef double2 V;   // complex vector element
  typedef double R;    // projection-row element
  typedef double A;    // in-block accumulator
  static const int CHUNK = 1 << 30;  // no chunking in FP64
};
template <> struct PT<PREC_C32> {
  typedef float2 V;
  typedef float R;
  typedef float A;
  static const int CHUNK = 16;       // FP32 partial over at most 16 terms per lane
};
template <> struct PT<PREC_DF> {
  typedef dfc V;
  typedef df R;
  typedef df A;
  static const int CHUNK = 1 << 30;
};

// ---------------------------------------------------------------- FP64 scalar helpers
// Complex division a/b in FP64 (Smith's algorithm).
__device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
  if (fabs(b.x) >= fabs(b.y)) {
    double r = b.y / b.x, d = b.x + b.y * r;
    return make_double2((a.x + a.y * r) / d, (a.y - a.x * r) / d);
  } else {
    double r = b.x / b.y, d = b.x * r + b.y;
    return make_double2((a.x * r + a.y) / d, (a.y * r - a.x) / d);
  }
}
// 1/b = conj(b) / |b|^2, evaluated on b scaled by a power of two (exact) so that
// |b|^2 neither overflows nor underflows; one division.  b must be nonzero.
__device__ __forceinline__ double2 crecip(double2 b) {
  const int e = ilogb(fmax(fabs(b.x), fabs(b.y)));
  const double bx = scalbn(b.x, -e), by = scalbn(b.y, -e);
  const double r = 1.0 / (bx * bx + by * by);
  return make_double2(scalbn(bx * r, -e), scalbn(-by * r, -e));
}
__device__ __forceinline__ bool cfinite(double2 a) { return isfinite(a.x) && isfinite(a.y); }
// FP32-pair image of a complex FP64 scalar (x = re.hi, y = re.lo, z = im.hi, w = im.lo).
__device__ __forceinline__ float4 pair_of(double2 a) {
  const df r = df_from_double(a.x), i = df_from_double(a.y);
  return make_float4(r.hi, r.lo, i.hi, i.lo);
}

// ---------------------------------------------------------------- reductions
// Sum N per-thread accumulators over the block: warp trees in the accumulator
// type, then the warps combined in FP64 in a fixed order.  Result valid in
// `out` (shared).  Requires blockDim.x a multiple of 32, <= 1024.
template <int N, class T>
__device__ __forceinline__ void block_sum(const T (&v)[N], int n, double* out) {
  __shared__ double sh[32][N > 0 ? N : 1];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int i = 0; i < N; ++i) {
    if (i < n) {
      const T s = warp_sum(anorm(v[i]));
      if (lane == 0) sh[warp][i] = ato_double(s);
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double s = 0.0;
    for (int k = 0; k < nw; ++k) s += sh[k][i];
    out[i] = s;
  }
  __syncthreads();
}

// FP32-pair form: the same block sum kept in pairs (FP32 pipe) across the
// warps; out[i] receives the pair.  Converting to FP64 once per value at the
// very end keeps the FP64 pipe, 1/64 of the FP32 rate on this GPU, out of the
// reduction.
template <int N>
__device__ __forceinline__ void block_sum_df(const df (&v)[N], int n, df* out) {
  __shared__ df sh[32][N > 0 ? N : 1];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int i = 0; i < N; ++i) {
    if (i < n) {
      const df s = warp_sum(anorm(v[i]));
      if (lane == 0) sh[warp][i] = s;
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    df s = sh[0][i];
    for (int k = 1; k < nw; ++k) s = df_add(s, sh[k][i]);
    out[i] = s;
  }
  __syncthreads();
}

// Arrival counter: true in the one block that finishes last.  Every block's
// partials are fenced before it arrives, so the last block sees all of them.
__device__ __forceinline__ bool arrive_last(unsigned int* cnt) {
  __shared__ int last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned int prev = atomicAdd(cnt, 1u);
    last = (prev == gridDim.x - 1);
  }
  __syncthreads();
  if (last) __threadfence();
  return last != 0;
}

// In the last block: out[i] = sum over blocks b of part[b*stride + i], FP64, fixed order.
template <int N>
__device__ __forceinline__ void reduce_partials(const double* part, int nblk, int stride, int n, double* out) {
  double acc[N];
#pragma unroll
  for (int i = 0; i < N; ++i) acc[i] = 0.0;
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) {
#pragma unroll
    for (int i = 0; i < N; ++i)
      if (i < n) acc[i] += __ldcg(part + (size_t)b * stride + i);
  }
  block_sum<N, double>(acc, n, out);
}

__device__ __forceinline__ void set_fail(State* st, int status) {
  if (st->status == KW_OK || st->status == KW_NOT_CONVERGED) st->status = status;
  st->done = 1;
}

// Programmatic dependent launch for small problems: K1 and K2 follow each
// other on the work stream; when their grids are small (less than one block
// per SM, where the iteration is bound by launch latency) they are launched
// with programmatic stream serialization, so that the next one's blocks are
// placed while this one's last blocks still reduce.  Each waits at entry for
// its predecessor's completion and memory before touching anything, then lets
// its own successor launch; both instructions are no-ops for an ordinary
// launch.  (On large grids the early blocks cost more than they save.)
__device__ __forceinline__ void pdl_entry() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// ================================================================ K1: SpMV + first dot
struct SpmvMode {
  int solver;        // 1: inside the solve (reads z_s, computes alpha)
  double2 zs;        // standalone: seed shift
  float4 zs_pair;    // standalone: its FP32-pair image
  double2* t_out;    // standalone: result
  int conj_zs = 0;   // use the conjugate seed shift (BiCG: the adjoint product A^dagger r~ for real H)
  int conj_dot = 0;  // r^dagger q instead of r^T q (CG)
  int dot = 1;       // 0: only q, no r^T q and no K1 tail (BiCG forms its dot separately)
};

// End of K1 (every layout): block sum of r^T q; the last block stores it for
// the next K2, which forms alpha_n and c_n (Eq. 17), or returns it standalone.
template <class A>
__device__ __forceinline__ void spmv_finish(A c_re, A c_im, double t_re, double t_im, int lane, State* st,
                                            double* __restrict__ part, const SpmvMode& mode) {
  if (!mode.dot) return;   // uniform: no block takes part, the counter is untouched
  t_re += ato_double(warp_sum(anorm(c_re)));
  t_im += ato_double(warp_sum(anorm(c_im)));
  __shared__ double red[2];
  {
    double v2[2] = {lane == 0 ? t_re : 0.0, lane == 0 ? t_im : 0.0};
    block_sum<2, double>(v2, 2, red);
  }
  if (threadIdx.x < 2) part[blockIdx.x * 2 + threadIdx.x] = red[threadIdx.x];
  if (!arrive_last(&st->cnt_spmv)) return;

  __shared__ double tot[2];
  reduce_partials<2>(part, gridDim.x, 2, 2, tot);
  if (threadIdx.x == 0) {
    st->cnt_spmv = 0;
    const double2 t = make_double2(tot[0], tot[1]);
    if (!mode.solver) {
      *mode.t_out = t;
      return;
    }
    st->u = t;
    // alpha_{n+1} for the case that the concurrent K3 keeps the seed (the next
    // K2 recomputes it after a switch): rho = rho_{n+1}, beta_n/alpha_n =
    // rho_{n+1} / (rho_n alpha_n), both from the K2 that produced r_{n+1}
    const double2 rho = st->rho1, boa = cmul(rho, st->inv_rho_alpha);
    const double2 denom = csub(t, cmul(boa, rho));   // Eq. 17
    int status = ((rho.x == 0.0 && rho.y == 0.0) || (denom.x == 0.0 && denom.y == 0.0)) ? KW_ERR_BREAKDOWN : 0;
    double2 alpha = make_double2(0.0, 0.0), c = alpha, inv_rho = alpha;
    if (!status) {
      inv_rho = crecip(rho);
      alpha = cmul(rho, crecip(denom));
      c = cmul(alpha, boa);
      if (!cfinite(alpha) || !cfinite(c)) status = KW_ERR_NONFINITE;
    }
    st->k1_status = status;
    st->k1_alpha = alpha;
    st->k1_c = c;
    st->k1_inv_rho = inv_rho;
    st->k1_inv_rho_alpha = cmul(denom, cmul(inv_rho, inv_rho));
    st->k1_t = t;
    st->p_alpha = pair_of(alpha);
    st->p_c = pair_of(c);
    st->p_opc = pair_of(make_double2(1.0 + c.x, c.y));
  }
}

template <int P, class RV, int G>
__global__ void __launch_bounds__(256)
k_spmv_dot(int m, const int64_t* __restrict__ rowptr, const int* __restrict__ col,
           const RV* __restrict__ val, const typename PT<P>::V* __restrict__ r,
           typename PT<P>::V* __restrict__ q, State* st, double* __restrict__ part, SpmvMode mode) {
  typedef typename PT<P>::V V;
  typedef typename PT<P>::A A;
  pdl_entry();
  V zsv;
  if (mode.solver) {
    if (st->done) return;
    zsv = vscalar<V>(st->zs_k1, st->p_zs_k1);
    if (mode.conj_zs) zsv = vconj(zsv);
  } else {
    zsv = vscalar<V>(mode.zs, mode.zs_pair);
  }
  const int lane = threadIdx.x & 31, sub = lane % G, gw = lane / G;
  const int RPW = 32 / G;
  const int warp_global = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;

  A c_re = azero<A>(), c_im = azero<A>();  // partial over <= CHUNK rows
  double t_re = 0, t_im = 0;               // FP64 total
  int in_chunk = 0;
  for (int base = warp_global * RPW; base < m; base += nwarps * RPW) {
    const int row = base + gw;
    V acc = vzero<V>();
    if (row < m) {
      const int beg = (int)rowptr[row], end = (int)rowptr[row + 1];
      if (G == 1) {
        int j = beg;
        for (; j + 3 < end; j += 4) {        // four independent gathers in flight
          const int c0 = col[j], c1 = col[j + 1], c2 = col[j + 2], c3 = col[j + 3];
          const RV v0 = val[j], v1 = val[j + 1], v2 = val[j + 2], v3 = val[j + 3];
          const V x0 = r[c0], x1 = r[c1], x2 = r[c2], x3 = r[c3];
          mac(acc, v0, x0);
          mac(acc, v1, x1);
          mac(acc, v2, x2);
          mac(acc, v3, x3);
        }
        for (; j < end; ++j) mac(acc, val[j], r[col[j]]);
      } else {
        for (int j = beg + sub; j < end; j += G) mac(acc, val[j], r[col[j]]);
      }
    }
#pragma unroll
    for (int off = G / 2; off > 0; off >>= 1) vshfl_add(acc, off);
    if (sub == 0 && row < m) {
      acc = normalize(acc);
      V ri = r[row];
      V qi = csub(cmul(zsv, ri), acc);        // z_s r - H r
      q[row] = qi;
      acc_cplx(c_re, c_im, cmul(mode.conj_dot ? vconj(ri) : ri, qi));   // r^T q (COCG) or r^dagger q (CG)
    }
    if (++in_chunk == PT<P>::CHUNK) {   // uniform across the warp
      t_re += ato_double(warp_sum(anorm(c_re)));
      t_im += ato_double(warp_sum(anorm(c_im)));
      c_re = c_im = azero<A>();
      in_chunk = 0;
    }
  }
  spmv_finish<A>(c_re, c_im, t_re, t_im, lane, st, part, mode);
}

// K1 on the SELL-32 layout (sliced ELLPACK): rows sorted by length inside
// 1024-row windows, 32 rows per slice, each slice's entries stored column-major
// so that one warp reads 32 consecutive indices and values per step.  One warp
// per slice, one lane per row; perm maps a sorted position to its row.
template <int P, class RV>
__global__ void __launch_bounds__(256)
k_spmv_sell(int m, int nslice, const int* __restrict__ perm, const int* __restrict__ rlen,
            const int64_t* __restrict__ sptr, const int* __restrict__ scol, const RV* __restrict__ sval,
            const typename PT<P>::V* __restrict__ r, typename PT<P>::V* __restrict__ q, State* st,
            double* __restrict__ part, SpmvMode mode) {
  typedef typename PT<P>::V V;
  typedef typename PT<P>::A A;
  V zsv;
  if (mode.solver) {
    if (st->done) return;
    zsv = vscalar<V>(st->zs_k1, st->p_zs_k1);
    if (mode.conj_zs) zsv = vconj(zsv);
  } else {
    zsv = vscalar<V>(mode.zs, mode.zs_pair);
  }
  const int lane = threadIdx.x & 31;
  const int warp_global = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  A c_re = azero<A>(), c_im = azero<A>();
  double t_re = 0, t_im = 0;
  int in_chunk = 0;
  for (int s = warp_global; s < nslice; s += nwarps) {   // uniform across the warp
    const int p = s * 32 + lane;
    if (p < m) {
      const int row = perm[p], len = rlen[p];
      const int* __restrict__ cp = scol + sptr[s] + lane;
      const RV* __restrict__ vp = sval + sptr[s] + lane;
      V acc = vzero<V>();
      int j = 0;
      for (; j + 3 < len; j += 4) {
        const int c0 = cp[32 * j], c1 = cp[32 * (j + 1)], c2 = cp[32 * (j + 2)], c3 = cp[32 * (j + 3)];
        const RV v0 = vp[32 * j], v1 = vp[32 * (j + 1)], v2 = vp[32 * (j + 2)], v3 = vp[32 * (j + 3)];
        const V x0 = r[c0], x1 = r[c1], x2 = r[c2], x3 = r[c3];
        mac(acc, v0, x0);
        mac(acc, v1, x1);
        mac(acc, v2, x2);
        mac(acc, v3, x3);
      }
      for (; j < len; ++j) mac(acc, vp[32 * j], r[cp[32 * j]]);
      acc = normalize(acc);
      V ri = r[row];
      V qi = csub(cmul(zsv, ri), acc);        // z_s r - H r
      q[row] = qi;
      acc_cplx(c_re, c_im, cmul(mode.conj_dot ? vconj(ri) : ri, qi));   // r^T q (COCG) or r^dagger q (CG)
    }
    if (++in_chunk == PT<P>::CHUNK) {
      t_re += ato_double(warp_sum(anorm(c_re)));
      t_im += ato_double(warp_sum(anorm(c_im)));
      c_re = c_im = azero<A>();
      in_chunk = 0;
    }
  }
  spmv_finish<A>(c_re, c_im, t_re, t_im, lane, st, part, mode);
}

// K1 on the uniform off-diagonal layout: every off-diagonal entry of H has the
// same value u_v (lattice hoppings, spin-flip amplitudes), so a row needs only
// its off-diagonal columns and its diagonal: H r = d_i r_i + u_v sum_j r_{c_j}.
// G lanes per row as in k_spmv_dot; the sum is taken in the vector type (the
// pair form with one normalisation per row), then scaled once.
template <int P, class DV, int G>
__global__ void __launch_bounds__(256)
k_spmv_u(int m, const int* __restrict__ rowptr, const int* __restrict__ col, const DV* __restrict__ diag, DV uv,
         const typename PT<P>::V* __restrict__ r, typename PT<P>::V* __restrict__ q, State* st,
         double* __restrict__ part, SpmvMode mode) {
  typedef typename PT<P>::V V;
  typedef typename PT<P>::A A;
  V zsv;
  if (mode.solver) {
    if (st->done) return;
    zsv = vscalar<V>(st->zs_k1, st->p_zs_k1);
    if (mode.conj_zs) zsv = vconj(zsv);
  } else {
    zsv = vscalar<V>(mode.zs, mode.zs_pair);
  }
  const int lane = threadIdx.x & 31, sub = lane % G, gw = lane / G;
  const int RPW = 32 / G;
  const int warp_global = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;

  A c_re = azero<A>(), c_im = azero<A>();
  double t_re = 0, t_im = 0;
  int in_chunk = 0;
  for (int base = warp_global * RPW; base < m; base += nwarps * RPW) {
    const int row = base + gw;
    V sum = vzero<V>();
    if (row < m) {
      const int beg = rowptr[row], end = rowptr[row + 1];
      if (G == 1) {
        int j = beg;
        for (; j + 3 < end; j += 4) {        // four independent gathers in flight
          const int c0 = col[j], c1 = col[j + 1], c2 = col[j + 2], c3 = col[j + 3];
          const V x0 = r[c0], x1 = r[c1], x2 = r[c2], x3 = r[c3];
          vacc(sum, x0);
          vacc(sum, x1);
          vacc(sum, x2);
          vacc(sum, x3);
        }
        for (; j < end; ++j) vacc(sum, r[col[j]]);
      } else {
        for (int j = beg + sub; j < end; j += G) vacc(sum, r[col[j]]);
      }
    }
    sum = normalize(sum);
#pragma unroll
    for (int off = G / 2; off > 0; off >>= 1) vshfl_add(sum, off);
    if (sub == 0 && row < m) {
      V ri = r[row];
      V hr = vzero<V>();
      mac(hr, diag[row], ri);
      mac(hr, uv, sum);
      hr = normalize(hr);
      V qi = csub(cmul(zsv, ri), hr);         // z_s r - H r
      q[row] = qi;
      acc_cplx(c_re, c_im, cmul(mode.conj_dot ? vconj(ri) : ri, qi));   // r^T q (COCG) or r^dagger q (CG)
    }
    if (++in_chunk == PT<P>::CHUNK) {   // uniform across the warp
      t_re += ato_double(warp_sum(anorm(c_re)));
      t_im += ato_double(warp_sum(anorm(c_im)));
      c_re = c_im = azero<A>();
      in_chunk = 0;
    }
  }
  spmv_finish<A>(c_re, c_im, t_re, t_im, lane, st, part, mode);
}

// Shared tail of the generated-operator K1 kernels: q = z_s r - H r for one
// row, the store and the r^T q partial.
template <class V, class A>
__device__ __forceinline__ void k1_emit(int row, V ri, V hr, V zsv, V* __restrict__ q, A& c_re, A& c_im,
                                        int conj_dot) {
  const V qi = csub(cmul(zsv, ri), hr);
  q[row] = qi;
  acc_cplx(c_re, c_im, cmul(conj_dot ? vconj(ri) : ri, qi));
}

// Seed shift of K1 (inside the solve: the one current when the previous K2
// ended; standalone: the caller's).  False when the solve has stopped.
template <class V>
__device__ __forceinline__ bool k1_seed(const State* st, const SpmvMode& mode, V& zsv) {
  if (mode.solver) {
    if (st->done) return false;
    zsv = vscalar<V>(st->zs_k1, st->p_zs_k1);
    if (mode.conj_zs) zsv = vconj(zsv);
  } else {
    zsv = vscalar<V>(mode.zs, mode.zs_pair);
  }
  return true;
}

// K1 on the uniform off-diagonal layout stored as SELL-32: one warp per slice of
// 32 consecutive rows (rows are not reordered), one lane per row; the slice's
// off-diagonal columns are slot-major (slot k holds each row's k-th column, -1
// past the row's end), so every index load of the warp reads 128 contiguous
// bytes.  sptr[s] is the first slot of slice s (in units of 32 columns).  The
// sum over a row's columns runs in the row's column order, as in k_spmv_u.
template <int P, class DV>
__global__ void __launch_bounds__(256)
k_spmv_us(int m, int nslice, const int* __restrict__ sptr, const int* __restrict__ scol,
          const DV* __restrict__ diag, DV uv, const typename PT<P>::V* __restrict__ r,
          typename PT<P>::V* __restrict__ q, State* st, double* __restrict__ part, SpmvMode mode) {
  typedef typename PT<P>::V V;
  typedef typename PT<P>::A A;
  V zsv;
  if (!k1_seed(st, mode, zsv)) return;
  const int lane = threadIdx.x & 31;
  const int warp_global = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  A c_re = azero<A>(), c_im = azero<A>();
  double t_re = 0, t_im = 0;
  int in_chunk = 0;
  for (int s = warp_global; s < nslice; s += nwarps) {   // uniform across the warp
    const int row = s * 32 + lane;
    const int k0 = sptr[s], k1 = sptr[s + 1];
    const int* cp = scol + (size_t)k0 * 32 + lane;
    V sum = vzero<V>();
    int k = k0;
    for (; k + 3 < k1; k += 4, cp += 128) {   // four slots: four coalesced index loads, four gathers
      const int c0 = cp[0], c1 = cp[32], c2 = cp[64], c3 = cp[96];
      const V x0 = c0 >= 0 ? r[c0] : vzero<V>(), x1 = c1 >= 0 ? r[c1] : vzero<V>();
      const V x2 = c2 >= 0 ? r[c2] : vzero<V>(), x3 = c3 >= 0 ? r[c3] : vzero<V>();
      vacc(sum, x0);
      vacc(sum, x1);
      vacc(sum, x2);
      vacc(sum, x3);
    }
    for (; k < k1; ++k, cp += 32) {
      const int c0 = cp[0];
      if (c0 >= 0) vacc(sum, r[c0]);
    }
    sum = normalize(sum);
    if (row < m) {
      V ri = r[row];
      V hr = vzero<V>();
      mac(hr, diag[row], ri);
      mac(hr, uv, sum);
      hr = normalize(hr);
      V qi = csub(cmul(zsv, ri), hr);         // z_s r - H r
      q[row] = qi;
      acc_cplx(c_re, c_im, cmul(mode.conj_dot ? vconj(ri) : ri, qi));   // r^T q (COCG) or r^dagger q (CG)
    }
    if (++in_chunk == PT<P>::CHUNK) {   // uniform across the warp
      t_re += ato_double(warp_sum(anorm(c_re)));
      t_im += ato_double(warp_sum(anorm(c_im)));
      c_re = c_im = azero<A>();
      in_chunk = 0;
    }
  }
  spmv_finish<A>(c_re, c_im, t_re, t_im, lane, st, part, mode);
}

// Row of the word sw (row `row`) with the spins of bond (a, c), a < c, exchanged
// (they differ): the combinatorial-number-system rank change described below.
__device__ __forceinline__ int spin_exchange_row(unsigned sw, int row, int a, int c, const int* binom) {
  const int t = __popc(sw & ((1u << a) - 1u));
  unsigned mid = sw & ((1u << c) - 1u) & ~((2u << a) - 1u);   // set bits strictly between a and c
  const int mc = __popc(mid);
  int d = binom[c * KW_BINOM_K + t + mc + 1] - binom[a * KW_BINOM_K + t + 1];
  for (int u = 1; mid; ++u) {
    const int qb = __ffs(mid) - 1;
    d += binom[qb * KW_BINOM_K + t + u] - binom[qb * KW_BINOM_K + t + u + 1];
    mid &= mid - 1u;
  }
  return ((sw >> a) & 1u) ? row + d : row - d;
}

// K1 for a spin operator with a precomputed exchange table (slot-major: the
// rows of a warp read slot b together, coalesced, and gather bond b's
// exchanged words together, which lie close to each other).
template <int P, class DV, bool UNI>
__global__ void __launch_bounds__(256)
k_spmv_spin_tab(int m, const int* __restrict__ table, const DV* __restrict__ val_g, int nbond,
                const DV* __restrict__ diag, DV uv, const typename PT<P>::V* __restrict__ r,
                typename PT<P>::V* __restrict__ q, State* st, double* __restrict__ part, SpmvMode mode) {
  typedef typename PT<P>::V V;
  typedef typename PT<P>::A A;
  __shared__ DV bval[UNI ? 1 : KW_SPIN_MAX_BONDS];
  if constexpr (!UNI) {
    for (int i = threadIdx.x; i < nbond; i += blockDim.x) bval[i] = val_g[i];
    __syncthreads();
  }
  V zsv;
  if (!k1_seed<V>(st, mode, zsv)) return;
  const int lane = threadIdx.x & 31;
  A c_re = azero<A>(), c_im = azero<A>();
  double t_re = 0, t_im = 0;
  int in_chunk = 0;
  const int stride = gridDim.x * blockDim.x;
  for (int base = blockIdx.x * blockDim.x; base < m; base += stride) {   // uniform trip count per warp
    const int row = base + (int)threadIdx.x;
    if (row < m) {
      V sum = vzero<V>();
      int b = 0;
      for (; b + 3 < nbond; b += 4) {        // four slots' columns, then their gathers
        const int c0 = table[(size_t)b * m + row], c1 = table[(size_t)(b + 1) * m + row];
        const int c2 = table[(size_t)(b + 2) * m + row], c3 = table[(size_t)(b + 3) * m + row];
        if constexpr (UNI) {
          if (c0 >= 0) vacc(sum, r[c0]);
          if (c1 >= 0) vacc(sum, r[c1]);
          if (c2 >= 0) vacc(sum, r[c2]);
          if (c3 >= 0) vacc(sum, r[c3]);
        } else {
          if (c0 >= 0) mac(sum, bval[b], r[c0]);
          if (c1 >= 0) mac(sum, bval[b + 1], r[c1]);
          if (c2 >= 0) mac(sum, bval[b + 2], r[c2]);
          if (c3 >= 0) mac(sum, bval[b + 3], r[c3]);
        }
      }
      for (; b < nbond; ++b) {
        const int cb = table[(size_t)b * m + row];
        if (cb >= 0) {
          if constexpr (UNI) vacc(sum, r[cb]);
          else mac(sum, bval[b], r[cb]);
        }
      }
      V hr = vzero<V>();
      const V ri = r[row];
      mac(hr, diag[row], ri);
      if constexpr (UNI) mac(hr, uv, normalize(sum));
      else vacc(hr, normalize(sum));
      hr = normalize(hr);
      k1_emit(row, ri, hr, zsv, q, c_re, c_im, mode.conj_dot);
    }
    if (++in_chunk == PT<P>::CHUNK) {
      t_re += ato_double(warp_sum(anorm(c_re)));
      t_im += ato_double(warp_sum(anorm(c_im)));
      c_re = c_im = azero<A>();
      in_chunk = 0;
    }
  }
  spmv_finish<A>(c_re, c_im, t_re, t_im, lane, st, part, mode);
}

// K1 for a spin-1/2 operator generated on the fly (kw_set_spin_operator).  One
// thread per basis word s (row = its rank).  For every bond (a, c), a < c, whose
// spins differ, the exchanged word s' is s with the up spin moved across the
// bond; its rank follows from the combinatorial number system without a
// search: moving the set bit of index t (t set bits below a) from a up to c
// past m set bits q_1 < .. < q_m lying between them changes the rank by
//   C(c, t+m+1) - C(a, t+1) + sum_u [C(q_u, t+u) - C(q_u, t+u+1)],
// added when the up spin sits at a and subtracted when it sits at c.  All
// lanes of a warp visit bond b together, so the gathers of 32 neighbouring
// words land close together.  UNI: every J_b equal (sum first, scale once).
template <int P, class DV, bool UNI>
__global__ void __launch_bounds__(256)
k_spmv_spin(int m, const unsigned* __restrict__ basis, const int* __restrict__ binom_g,
            const int* __restrict__ bond_g, const DV* __restrict__ val_g, int nbond, const DV* __restrict__ diag,
            DV uv, const typename PT<P>::V* __restrict__ r, typename PT<P>::V* __restrict__ q, State* st,
            double* __restrict__ part, SpmvMode mode) {
  typedef typename PT<P>::V V;
  typedef typename PT<P>::A A;
  __shared__ int binom[KW_BINOM_N * KW_BINOM_K];
  __shared__ int bond[KW_SPIN_MAX_BONDS];
  __shared__ DV bval[UNI ? 1 : KW_SPIN_MAX_BONDS];
  for (int i = threadIdx.x; i < KW_BINOM_N * KW_BINOM_K; i += blockDim.x) binom[i] = binom_g[i];
  for (int i = threadIdx.x; i < nbond; i += blockDim.x) {
    bond[i] = bond_g[i];
    if constexpr (!UNI) bval[i] = val_g[i];
  }
  __syncthreads();
  V zsv;
  if (!k1_seed<V>(st, mode, zsv)) return;
  const int lane = threadIdx.x & 31;
  A c_re = azero<A>(), c_im = azero<A>();
  double t_re = 0, t_im = 0;
  int in_chunk = 0;
  const int stride = gridDim.x * blockDim.x;
  for (int base = blockIdx.x * blockDim.x; base < m; base += stride) {   // uniform trip count per warp
    const int row = base + (int)threadIdx.x;
    if (row < m) {
      const unsigned sw = basis[row];
      V sum = vzero<V>();
      for (int b = 0; b < nbond; ++b) {
        const int a = bond[b] & 255, c = bond[b] >> 8;
        if ((((sw >> a) ^ (sw >> c)) & 1u) == 0) continue;   // parallel spins: no exchange
        const int colx = spin_exchange_row(sw, row, a, c, binom);
        if constexpr (UNI) vacc(sum, r[colx]);
        else mac(sum, bval[b], r[colx]);
      }
      V hr = vzero<V>();
      const V ri = r[row];
      mac(hr, diag[row], ri);
      if constexpr (UNI) mac(hr, uv, normalize(sum));
      else vacc(hr, normalize(sum));
      hr = normalize(hr);
      k1_emit(row, ri, hr, zsv, q, c_re, c_im, mode.conj_dot);
    }
    if (++in_chunk == PT<P>::CHUNK) {
      t_re += ato_double(warp_sum(anorm(c_re)));
      t_im += ato_double(warp_sum(anorm(c_im)));
      c_re = c_im = azero<A>();
      in_chunk = 0;
    }
  }
  spmv_finish<A>(c_re, c_im, t_re, t_im, lane, st, part, mode);
}

// K1 for the periodic nx x ny x nz tight-binding lattice (kw_set_lattice3d):
// H r_i = eps_i r_i + hopping * (sum of r over the six neighbours); one thread
// per site, so the neighbour loads of a warp are contiguous runs.
template <int P, class DV>
__global__ void __launch_bounds__(256)
k_spmv_lattice(int m, int nx, int ny, int nz, const DV* __restrict__ eps, DV hop,
               const typename PT<P>::V* __restrict__ r, typename PT<P>::V* __restrict__ q, State* st,
               double* __restrict__ part, SpmvMode mode) {
  typedef typename PT<P>::V V;
  typedef typename PT<P>::A A;
  V zsv;
  if (!k1_seed<V>(st, mode, zsv)) return;
  const int lane = threadIdx.x & 31;
  const int nxy = nx * ny;
  A c_re = azero<A>(), c_im = azero<A>();
  double t_re = 0, t_im = 0;
  int in_chunk = 0;
  const int stride = gridDim.x * blockDim.x;
  for (int base = blockIdx.x * blockDim.x; base < m; base += stride) {
    const int row = base + (int)threadIdx.x;
    if (row < m) {
      const int x = row % nx, yz = row / nx, y = yz % ny, z = yz / ny;
      const int xm = x == 0 ? row + nx - 1 : row - 1, xp = x == nx - 1 ? row - nx + 1 : row + 1;
      const int ym = y == 0 ? row + nxy - nx : row - nx, yp = y == ny - 1 ? row - nxy + nx : row + nx;
      const int zm = z == 0 ? row + m - nxy : row - nxy, zp = z == nz - 1 ? row - m + nxy : row + nxy;
      const V n0 = r[xp], n1 = r[xm], n2 = r[yp], n3 = r[ym], n4 = r[zp], n5 = r[zm];
      const V ri = r[row];
      V sum = n0;
      vacc(sum, n1);
      vacc(sum, n2);
      vacc(sum, n3);
      vacc(sum, n4);
      vacc(sum, n5);
      V hr = vzero<V>();
      mac(hr, eps[row], ri);
      mac(hr, hop, normalize(sum));
      hr = normalize(hr);
      k1_emit(row, ri, hr, zsv, q, c_re, c_im, mode.conj_dot);
    }
    if (++in_chunk == PT<P>::CHUNK) {
      t_re += ato_double(warp_sum(anorm(c_re)));
      t_im += ato_double(warp_sum(anorm(c_im)));
      c_re = c_im = azero<A>();
      in_chunk = 0;
    }
  }
  spmv_finish<A>(c_re, c_im, t_re, t_im, lane, st, part, mode);
}

// K1 for an operator given as a callback (kw_set_matvec).  The caller's work
// has left H r in hq (kw_c128 in the FP64 and FP32-pair forms, complex FP32 in
// the FP32 form; in place in q except in the pair form); this pass forms
// q = z_s r - H r with the lazy seed-switch scale and r^T q exactly as
// k_spmv_dot does, then the same K1 tail.
template <int P> struct MvT;
template <> struct MvT<PREC_F64> { typedef double2 H; };
template <> struct MvT<PREC_C32> { typedef float2 H; };
template <> struct MvT<PREC_DF> { typedef double2 H; };
__device__ __forceinline__ double2 mv_in(double2 h, double2*) { return h; }
__device__ __forceinline__ float2 mv_in(float2 h, float2*) { return h; }
__device__ __forceinline__ dfc mv_in(double2 h, dfc*) { return {df_from_double(h.x), df_from_double(h.y)}; }

template <int P>
__global__ void __launch_bounds__(256)
k_matvec_finish(int m, const typename PT<P>::V* r, const typename MvT<P>::H* hq, typename PT<P>::V* q, State* st,
                double* __restrict__ part, SpmvMode mode) {
  typedef typename PT<P>::V V;
  typedef typename PT<P>::A A;
  V zsv;
  if (mode.solver) {
    if (st->done) return;
    zsv = vscalar<V>(st->zs_k1, st->p_zs_k1);
    if (mode.conj_zs) zsv = vconj(zsv);
  } else {
    zsv = vscalar<V>(mode.zs, mode.zs_pair);
  }
  const int lane = threadIdx.x & 31;
  A c_re = azero<A>(), c_im = azero<A>();
  double t_re = 0, t_im = 0;
  int in_chunk = 0;
  const int stride = gridDim.x * blockDim.x;
  // the trip count is uniform across a warp (rows past m do no work)
  for (int base = blockIdx.x * blockDim.x; base < m; base += stride) {
    const int row = base + (int)threadIdx.x;
    if (row < m) {
      V ri = r[row];
      V qi = csub(cmul(zsv, ri), mv_in(hq[row], (V*)nullptr));   // z_s r - H r
      q[row] = qi;
      acc_cplx(c_re, c_im, cmul(mode.conj_dot ? vconj(ri) : ri, qi));   // r^T q (COCG) or r^dagger q (CG)
    }
    if (++in_chunk == PT<P>::CHUNK) {
      t_re += ato_double(warp_sum(anorm(c_re)));
      t_im += ato_double(warp_sum(anorm(c_im)));
      c_re = c_im = azero<A>();
      in_chunk = 0;
    }
  }
  spmv_finish<A>(c_re, c_im, t_re, t_im, lane, st, part, mode);
}

// BiCG's first dot, r~_n^dagger (A r_n), over the two vectors K1 left (r~ and
// q), followed by the same K1 tail (the seed scalars of Eq. 17 for the case
// that the seed is kept).
template <int P>
__global__ void __launch_bounds__(256)
k_dot_tail(int m, const typename PT<P>::V* __restrict__ x, const typename PT<P>::V* __restrict__ y, State* st,
           double* __restrict__ part, SpmvMode mode) {
  typedef typename PT<P>::V V;
  typedef typename PT<P>::A A;
  if (st->done) return;
  const int lane = threadIdx.x & 31;
  A c_re = azero<A>(), c_im = azero<A>();
  double t_re = 0, t_im = 0;
  int in_chunk = 0;
  const int stride = gridDim.x * blockDim.x;
  for (int base = blockIdx.x * blockDim.x; base < m; base += stride) {
    const int i = base + (int)threadIdx.x;
    if (i < m) acc_cplx(c_re, c_im, cmul(vconj(x[i]), y[i]));
    if (++in_chunk == PT<P>::CHUNK) {
      t_re += ato_double(warp_sum(anorm(c_re)));
      t_im += ato_double(warp_sum(anorm(c_im)));
      c_re = c_im = azero<A>();
      in_chunk = 0;
    }
  }
  spmv_finish<A>(c_re, c_im, t_re, t_im, lane, st, part, mode);
}

// FP32-pair form: r as kw_c128 for the callback (skipped once the solve stopped).
static __global__ void k_pairs_to_c128(int m, const dfc* __restrict__ r, double2* __restrict__ out,
                                       const State* st, int solver) {
  if (solver && st->done) return;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
    const dfc v = r[i];
    out[i] = make_double2((double)v.re.hi + (double)v.re.lo, (double)v.im.hi + (double)v.im.lo);
  }
}

// ---------------------------------------------------------------- SELL-32 construction
// One block of 1024 threads per window of 1024 rows: bitonic sort of
// (descending length, row) keys; writes the sorted order and lengths.
static __global__ void __launch_bounds__(1024) k_sell_sort(int m, const int64_t* __restrict__ rowptr, int* perm,
                                                         int* rlen) {
  __shared__ unsigned int key[1024];
  const int i = threadIdx.x, base = blockIdx.x * 1024, row = base + i;
  const unsigned int LMAX = (1u << 21) - 1;
  unsigned int kk = 0xffffffffu;
  if (row < m) {
    const long long len = rowptr[row + 1] - rowptr[row];
    const unsigned int l = (unsigned int)(len < (long long)LMAX ? len : (long long)LMAX);
    kk = ((LMAX - l) << 10) | (unsigned int)i;
  }
  key[i] = kk;
  __syncthreads();
  for (int size = 2; size <= 1024; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      const int j = i ^ stride;
      if (j > i) {
        const unsigned int a = key[i], b = key[j];
        const bool up = (i & size) == 0;
        if ((a > b) == up) {
          key[i] = b;
          key[j] = a;
        }
      }
      __syncthreads();
    }
  }
  if (base + i < m) {
    const int r0 = base + (int)(key[i] & 1023u);
    perm[base + i] = r0;
    rlen[base + i] = (int)(rowptr[r0 + 1] - rowptr[r0]);
  }
}

// Length of each 32-row slice = its longest row.
static __global__ void k_sell_slicelen(int m, int nslice, const int* __restrict__ rlen, int* slen) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < nslice; s += gridDim.x * blockDim.x) {
    int mx = 0;
    for (int p = s * 32; p < min(m, s * 32 + 32); ++p) mx = max(mx, rlen[p]);
    slen[s] = mx;
  }
}

// One warp per slice: copy every row's entries into the column-major slice.
template <class RV>
__global__ void k_sell_fill(int m, int nslice, const int* __restrict__ perm, const int* __restrict__ rlen,
                            const int64_t* __restrict__ sptr, const int64_t* __restrict__ rowptr,
                            const int* __restrict__ col, const RV* __restrict__ val, int* scol, RV* sval) {
  const int lane = threadIdx.x & 31;
  const int warp_global = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int s = warp_global; s < nslice; s += nwarps) {
    const int p = s * 32 + lane;
    if (p >= m) continue;
    const int row = perm[p], len = rlen[p];
    const int64_t src = rowptr[row], dst = sptr[s] + lane;
    for (int j = 0; j < len; ++j) {
      scol[dst + 32 * (int64_t)j] = col[src + j];
      sval[dst + 32 * (int64_t)j] = val[src + j];
    }
  }
}

// ================================================================ K2: three-term update + dots
// Values per block: [rho.re, rho.im, nu, w_0.re, w_0.im, ..., w_{np-1}.re, w_{np-1}.im]
// METHOD (Table 1): COCG rho = r^T r; CG rho = r^dagger r = nu; BiCG also
// advances the shadow residual (Appendix B: conjugated coefficients, A^dagger)
// and rho = r~^dagger r.
//
// BULK (kw_set_bulk_copy): the tiles of r_n, q, r_{n-1} and the projection
// rows are staged in shared memory by TMA bulk copies, nstage tiles ahead, so
// the loads of later tiles are in flight while the pair arithmetic of this one
// runs.  The tile is the block (one element per thread) and tile t of a block
// is the element set of its t-th grid-stride trip, so each thread sums the
// same elements in the same order as without staging.  The ragged last tile
// is read with plain loads.
// K2's head (thread 0): the seed scalars of Eq. 17 and the three coefficients
// of Eq. 16 into shared memory (s_sc = c_n, 1/rho_n; s_cf = the coefficients
// in FP64; s_pp = their FP32-pair images; *s_fail = a breakdown status); block
// 0 also records the scalars in the state.  The two residual buffers carry
// pending scales (bscale) from seed switches (Sec. 2.2.4: r_{n+1} <-
// r_{n+1}/pi^j_{n+1}, r_n <- r_n/pi^j_n), and K1 ran concurrently with the last
// K3, i.e. with the seed before its switch (q_raw = z_K1 r_raw - H r_raw).  With
// s_n, s_{n-1} the buffers' scales and dz = z_s - z_K1, by linearity
// r_n = s_n r_raw, q = s_n (q_raw + dz r_raw), r_n^T A r_n = s_n^2 (u + dz rho_raw), so that
//   r_{n+1} = [s_n (1 + c - alpha dz)] r_raw - [alpha s_n] q_raw - [c s_{n-1}] r_{n-1,raw}:
// a switch changes the coefficients, not the per-element work.
__device__ __forceinline__ void seed_coefficients(State* st, int parity, double2* s_sc, double2* s_cf, float4* s_pp,
                                                  int* s_fail) {
  if (threadIdx.x == 0) {
    const double2 one = make_double2(1.0, 0.0), zero = make_double2(0.0, 0.0);
    const double2 sn = st->bscale[parity], sm = st->bscale[1 - parity];
    const int switched = st->switched;
    double2 alpha, c, inv_rho, inv_rho_alpha, t, dz = zero;
    int fail = 0;
    if (!switched) {           // seed kept: K1's last block already formed the scalars
      fail = st->k1_status;
      alpha = st->k1_alpha;
      c = st->k1_c;
      inv_rho = st->k1_inv_rho;
      inv_rho_alpha = st->k1_inv_rho_alpha;
      t = st->k1_t;
    } else {
      dz = csub(st->zs, st->zs_k1);
      t = cmul(cmul(sn, sn), cadd(st->u, cmul(dz, st->rho1)));
      const double2 rho = st->rho, boa = st->boa;
      // alpha_n = rho_n / (r_n^T A r_n - (beta_{n-1}/alpha_{n-1}) rho_n)   (Eq. 17)
      const double2 denom = csub(t, cmul(boa, rho));
      alpha = c = inv_rho = inv_rho_alpha = zero;
      if ((rho.x == 0.0 && rho.y == 0.0) || (denom.x == 0.0 && denom.y == 0.0)) {
        fail = KW_ERR_BREAKDOWN;
      } else {
        inv_rho = crecip(rho);
        alpha = cmul(rho, crecip(denom));
        c = cmul(alpha, boa);
        inv_rho_alpha = cmul(denom, cmul(inv_rho, inv_rho));
        if (!cfinite(alpha) || !cfinite(c)) fail = KW_ERR_NONFINITE;
      }
    }
    const bool plain = !switched && sn.x == 1.0 && sn.y == 0.0 && sm.x == 1.0 && sm.y == 0.0;
    if (plain) {               // 1 + c, alpha, c as K1 converted them
      s_pp[0] = st->p_opc;
      s_pp[1] = st->p_alpha;
      s_pp[2] = st->p_c;
    } else {
      s_pp[0] = pair_of(cmul(sn, csub(make_double2(1.0 + c.x, c.y), cmul(alpha, dz))));
      s_pp[1] = pair_of(cmul(alpha, sn));
      s_pp[2] = pair_of(cmul(c, sm));
    }
    s_sc[0] = c;
    s_sc[1] = inv_rho;
    *s_fail = fail;
    if (blockIdx.x == 0) {
      if (fail) {
        set_fail(st, fail);
      } else {
        st->t = t;
        st->alpha = alpha;
        st->c = c;
        st->inv_rho = inv_rho;                   // beta_n = rho_{n+1} / rho_n below
        st->inv_rho_alpha = inv_rho_alpha;       // 1/(rho_n alpha_n): beta_n/alpha_n in K3 and the next K1
        st->n_list[parity] = 0;
      }
    }
    // FP64 form: the coefficients themselves (the pair images carry them otherwise)
    s_cf[0] = plain ? make_double2(1.0 + c.x, c.y) : cmul(sn, csub(make_double2(1.0 + c.x, c.y), cmul(alpha, dz)));
    s_cf[1] = plain ? alpha : cmul(alpha, sn);
    s_cf[2] = plain ? c : cmul(c, sm);
  }
}

// K2's tail (last block, after the grid reduction): P r_{n+1} to w_out, and
// rho_{n+1} (r^T r for COCG, ||r||^2 for CG, r~^dagger r for BiCG), beta_n,
// nu = ||r_{n+1}||^2 into the state.  all = [rho.re, rho.im, nu, w...];
// inv_rho = this block's 1/rho_n.
template <int METHOD>
__device__ __forceinline__ void seed_finish(const double* all, int np, int parity, State* st, double2* w_out,
                                            double2 inv_rho) {
  for (int l = threadIdx.x; l < np; l += blockDim.x) w_out[l] = make_double2(all[3 + 2 * l], all[4 + 2 * l]);
  if (threadIdx.x == 0) {
    st->cnt_seed = 0;
    st->bscale[1 - parity] = make_double2(1.0, 0.0);   // r_{n+1} was just written
    st->switched = 0;
    st->zs_k1 = st->zs;                                // the seed the next K1 uses
    st->p_zs_k1 = st->p_zs;
    // rho_{n+1}: r^T r (COCG), ||r||^2 (CG), r~^dagger r (BiCG)
    const double2 rho1 = METHOD == KW_METHOD_CG ? make_double2(all[2], 0.0) : make_double2(all[0], all[1]);
    // beta_n = rho_{n+1} / rho_n, with this block's own 1/rho_n (block 0's copy in
    // the state was written during this kernel and may not be visible here)
    const double2 beta = cmul(rho1, inv_rho);
    st->rho1 = rho1;
    st->beta = beta;
    st->nu = all[2];
    if (!cfinite(beta) || !isfinite(all[2])) set_fail(st, KW_ERR_NONFINITE);
  }
}

constexpr int kSeedTile = 256;

// Bytes of one stage: a tile of r_n, q, r_{n-1} and of the np projection rows.
template <class V, class R>
__host__ __device__ constexpr uint32_t seed_stage_bytes(int np) {
  return (uint32_t)((3 * kSeedTile * sizeof(V) + np * kSeedTile * sizeof(R) + 127) / 128 * 128);
}

template <int P, int NP, int METHOD, bool BULK>
__global__ void __launch_bounds__(256, (P == PREC_DF && NP <= 5 && METHOD != KW_METHOD_BICG) ? 3 : 1)
k_seed_update(int m, const typename PT<P>::V* __restrict__ rn_buf, const typename PT<P>::V* __restrict__ q,
              typename PT<P>::V* __restrict__ rm_buf, const typename PT<P>::R* __restrict__ proj, int64_t ld,
              int np, int parity, State* st, double* __restrict__ part, double2* __restrict__ w_out,
              const typename PT<P>::V* __restrict__ rtn_buf, const typename PT<P>::V* __restrict__ qt,
              typename PT<P>::V* __restrict__ rtm_buf, int nstage, uint32_t tx_pad) {
  typedef typename PT<P>::V V;
  typedef typename PT<P>::R R;
  typedef typename PT<P>::A A;
  constexpr int N = 3 + 2 * NP;
  constexpr bool CHUNKED = PT<P>::CHUNK < (1 << 30);
  pdl_entry();
  if (st->done) return;
  __shared__ double2 s_sc[2];   // c_n, 1/rho_n
  __shared__ double2 s_cf[3];   // the three coefficients in FP64
  __shared__ float4 s_pp[3];    // FP32-pair images of the three coefficients
  __shared__ int s_fail;
  seed_coefficients(st, parity, s_sc, s_cf, s_pp, &s_fail);
  __syncthreads();
  if (s_fail) return;
  // the coefficients are re-read from shared memory at each element (the pair
  // form would otherwise hold 12 more registers through the loop)
  const volatile float4* vpp = s_pp;
  const int n = 3 + 2 * np;

  A chunk[N], tot[N];
#pragma unroll
  for (int i = 0; i < N; ++i) chunk[i] = tot[i] = azero<A>();
  int in_chunk = 0;
  const int stride = gridDim.x * blockDim.x;
  // The pair form (COCG, CG) runs the update in packed FP32x2 pair arithmetic:
  // Eq. 16 as one six-product sum with one normalisation, (re^2, im^2) for rho
  // and nu, re*im for Im rho, and (re, im) of every projection at once.  The
  // coefficients' packed forms sit in shared memory and are re-read per element.
  constexpr bool PK = P == PREC_DF && METHOD != KW_METHOD_BICG;
  __shared__ float4 s_ck[PK ? 6 : 1];     // cpk_coef of a, -b, -c: (re.hi, re.lo, im.hi, im.lo) per part
  if constexpr (PK) {
    if (threadIdx.x < 3) {
      const cpk_coef ck = cpk_coef_of(s_pp[threadIdx.x], threadIdx.x == 0 ? 1.f : -1.f);
      s_ck[2 * threadIdx.x] = make_float4(ck.re.hi.x, ck.re.hi.y, ck.re.lo.x, ck.re.lo.y);
      s_ck[2 * threadIdx.x + 1] = make_float4(ck.im.hi.x, ck.im.hi.y, ck.im.lo.x, ck.im.lo.y);
    }
    __syncthreads();
  }
  const volatile float4* vck = s_ck;
  cpk sq = cpk_zero();            // packed: (sum re^2, sum im^2)
  df x2 = azero<df>();            // sum re * im
  cpk pp[PK && NP > 0 ? NP : 1];  // packed (re, im) of each projection
#pragma unroll
  for (int l = 0; l < (PK && NP > 0 ? NP : 1); ++l) pp[l] = cpk_zero();
  auto element_pk = [&](const V& rnv, const V& qvv, const V& rmv, const R* av, int i, bool has) {
    if constexpr (PK) {
      cpk_coef ck[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const float4 a = make_float4(vck[2 * c].x, vck[2 * c].y, vck[2 * c].z, vck[2 * c].w);
        const float4 b = make_float4(vck[2 * c + 1].x, vck[2 * c + 1].y, vck[2 * c + 1].z, vck[2 * c + 1].w);
        ck[c] = {{make_float2(a.x, a.y), make_float2(a.z, a.w)}, {make_float2(b.x, b.y), make_float2(b.z, b.w)}};
      }
      const cpk r1 = three_term_pk(ck[0], ck[1], ck[2], cpk_of(rnv), cpk_of(qvv), cpk_of(rmv));   // Eq. 16
      if (has) rm_buf[i] = dfc_of(r1);
      acc_sq_pk(sq, r1);
      if constexpr (METHOD != KW_METHOD_CG) acc_prod(x2, df{r1.hi.x, r1.lo.x}, df{r1.hi.y, r1.lo.y});
#pragma unroll
      for (int l = 0; l < NP; ++l)
        if (l < np) acc_proj_pk(pp[l], av[l], r1);
    }
  };
  // Eq. 16 for element i and its contributions to the dots (nothing stored when !has).
  auto element = [&](const V& rnv, const V& qvv, const V& rmv, const R* av, int i, bool has) {
    if constexpr (PK) {
      element_pk(rnv, qvv, rmv, av, i, has);
      return;
    }
    float4 pa, pb, pc;
    if constexpr (P == PREC_DF) {
      pa = make_float4(vpp[0].x, vpp[0].y, vpp[0].z, vpp[0].w);
      pb = make_float4(vpp[1].x, vpp[1].y, vpp[1].z, vpp[1].w);
      pc = make_float4(vpp[2].x, vpp[2].y, vpp[2].z, vpp[2].w);
    } else {
      pa = s_pp[0];
      pb = s_pp[1];
      pc = s_pp[2];
    }
    const V ca = vscalar<V>(s_cf[0], pa), cb = vscalar<V>(s_cf[1], pb), cc = vscalar<V>(s_cf[2], pc);
    const V r1 = csub(csub(cmul(ca, rnv), cmul(cb, qvv)), cmul(cc, rmv));   // Eq. 16; zero when !has
    if (has) rm_buf[i] = r1;
    if constexpr (METHOD == KW_METHOD_BICG) {
      // shadow: the conjugated coefficients (their folded scales are the conjugate ones)
      const V rtn = has ? rtn_buf[i] : vzero<V>(), rtm = has ? rtm_buf[i] : vzero<V>();
      const V qtv = has ? qt[i] : vzero<V>();
      const V rt1 = csub(csub(cmul(vconj(ca), rtn), cmul(vconj(cb), qtv)), cmul(vconj(cc), rtm));
      if (has) rtm_buf[i] = rt1;
      acc_cdot(chunk[0], chunk[1], rt1, r1);
      acc_nrm(chunk[2], r1);
    } else {
      acc_rho_nrm(chunk[0], chunk[1], chunk[2], r1);
    }
#pragma unroll
    for (int l = 0; l < NP; ++l)
      if (l < np) acc_proj(chunk[3 + 2 * l], chunk[4 + 2 * l], av[l], r1);
  };
  auto close_chunk = [&](int count) {
    if (CHUNKED && (in_chunk += count) >= PT<P>::CHUNK) {
#pragma unroll
      for (int k = 0; k < N; ++k) {
        aadd(tot[k], chunk[k]);
        chunk[k] = azero<A>();
      }
      in_chunk = 0;
    }
  };
  if constexpr (BULK) {
    extern __shared__ __align__(128) unsigned char kw_stage[];
    __shared__ __align__(8) uint64_t bars[3];
    constexpr uint32_t SV = kSeedTile * sizeof(V), SR = kSeedTile * sizeof(R);
    // tx_pad > 0 (a test of the bounded wait) arms each stage for bytes that never arrive
    const uint32_t stage_bytes = seed_stage_bytes<V, R>(np), tx = 3 * SV + (uint32_t)np * SR + tx_pad;
    const int nfull = m / kSeedTile, ntiles = (m + kSeedTile - 1) / kSeedTile, G = gridDim.x;
    if (threadIdx.x == 0) {
      for (int s = 0; s < nstage; ++s) mbar_init(&bars[s], 1);
      mbar_init_fence();
    }
    __syncthreads();
    auto issue = [&](int t, int s) {   // thread 0: tile t into stage s
      unsigned char* base = kw_stage + (size_t)s * stage_bytes;
      const size_t e0 = (size_t)t * kSeedTile;
      mbar_arrive_expect(&bars[s], tx);
      bulk_load(base, rn_buf + e0, SV, &bars[s]);
      bulk_load(base + SV, q + e0, SV, &bars[s]);
      bulk_load(base + 2 * SV, rm_buf + e0, SV, &bars[s]);
      for (int l = 0; l < np; ++l) bulk_load(base + 3 * SV + l * SR, proj + (size_t)l * ld + e0, SR, &bars[s]);
    };
    if (threadIdx.x == 0)
      for (int s = 0; s < nstage; ++s)
        if (blockIdx.x + s * G < nfull) issue(blockIdx.x + s * G, s);
    int k = 0;
    bool failed = false;
    for (int t = blockIdx.x; t < ntiles; t += G, ++k) {
      const int i = t * kSeedTile + (int)threadIdx.x;
      V rnv, qvv, rmv;
      R av[NP > 0 ? NP : 1];
      bool late = false, has = true;
      if (t < nfull) {
        const int s = k % nstage;
        late = !mbar_wait(&bars[s], (uint32_t)(k / nstage) & 1u);
        const unsigned char* base = kw_stage + (size_t)s * stage_bytes;
        rnv = reinterpret_cast<const V*>(base)[threadIdx.x];
        qvv = reinterpret_cast<const V*>(base + SV)[threadIdx.x];
        rmv = reinterpret_cast<const V*>(base + 2 * SV)[threadIdx.x];
#pragma unroll
        for (int l = 0; l < NP; ++l)
          av[l] = l < np ? reinterpret_cast<const R*>(base + 3 * SV + l * SR)[threadIdx.x] : rfrom_double<R>(0.0);
      } else {   // the ragged last tile
        has = i < m;
        rnv = has ? rn_buf[i] : vzero<V>();
        qvv = has ? q[i] : vzero<V>();
        rmv = has ? rm_buf[i] : vzero<V>();
#pragma unroll
        for (int l = 0; l < NP; ++l) av[l] = (l < np && has) ? proj[(size_t)l * ld + i] : rfrom_double<R>(0.0);
      }
      element(rnv, qvv, rmv, av, i, has);
      close_chunk(1);
      if (__syncthreads_or(late)) {   // every thread is done with stage k % nstage
        failed = true;
        break;
      }
      if (threadIdx.x == 0 && t + nstage * G < nfull) {
        fence_async_smem();
        issue(t + nstage * G, k % nstage);
      }
    }
    if (failed) {   // a copy did not land in time: report it, and let in-flight copies finish before leaving
      if (threadIdx.x == 0) {
        set_fail(st, KW_ERR_TIMEOUT);
        for (int j = 0; j < nstage; ++j)
          if (blockIdx.x + (k + j) * G < nfull) mbar_wait(&bars[(k + j) % nstage], (uint32_t)((k + j) / nstage) & 1u);
      }
      __syncthreads();
    }
  } else {
    // ILP elements per trip, all loads issued before any store: two for the FP64
    // and FP32 forms; one for FP32 pairs, whose arithmetic already fills the
    // pipes and whose registers would otherwise limit occupancy.
    constexpr int ILP = (P == PREC_DF) ? 1 : 2;
    for (int i0 = blockIdx.x * blockDim.x + threadIdx.x; i0 < m; i0 += ILP * stride) {
      V rn[ILP], rm[ILP], qv[ILP];
      R a[ILP][NP > 0 ? NP : 1];
      bool has[ILP];
#pragma unroll
      for (int u = 0; u < ILP; ++u) {
        const int i = i0 + u * stride;
        has[u] = i < m;
        rn[u] = has[u] ? rn_buf[i] : vzero<V>();
        rm[u] = has[u] ? rm_buf[i] : vzero<V>();
        qv[u] = has[u] ? q[i] : vzero<V>();
#pragma unroll
        for (int l = 0; l < NP; ++l) a[u][l] = (l < np && has[u]) ? proj[(size_t)l * ld + i] : rfrom_double<R>(0.0);
      }
#pragma unroll
      for (int u = 0; u < ILP; ++u) element(rn[u], qv[u], rm[u], a[u], i0 + u * stride, has[u]);
      close_chunk(ILP);
    }
  }
  if constexpr (PK) {   // the packed sums in the layout of the reduction below
    const df re2 = anorm(df{sq.hi.x, sq.lo.x}), im2 = anorm(df{sq.hi.y, sq.lo.y});
    chunk[0] = df_sub(re2, im2);                       // Re r^T r
    chunk[1] = df{2.f * x2.hi, 2.f * x2.lo};           // Im r^T r
    chunk[2] = df_add(re2, im2);                       // ||r||^2
#pragma unroll
    for (int l = 0; l < NP; ++l) {
      chunk[3 + 2 * l] = df{pp[l].hi.x, pp[l].lo.x};
      chunk[4 + 2 * l] = df{pp[l].hi.y, pp[l].lo.y};
    }
  }
#pragma unroll
  for (int k = 0; k < N; ++k) {
    if (CHUNKED) aadd(tot[k], chunk[k]);
    else tot[k] = chunk[k];
  }

  __shared__ double all[N];
  if constexpr (P == PREC_DF) {
    // block and grid sums in FP32 pairs (part holds one pair per value)
    __shared__ df red[N];
    block_sum_df<N>(tot, n, red);
    df* partd = reinterpret_cast<df*>(part);
    for (int k = threadIdx.x; k < n; k += blockDim.x) partd[(size_t)blockIdx.x * n + k] = red[k];
    if (!arrive_last(&st->cnt_seed)) return;
    df acc[N];
#pragma unroll
    for (int i = 0; i < N; ++i) acc[i] = azero<df>();
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
#pragma unroll
      for (int i = 0; i < N; ++i)
        if (i < n) {
          const float2 v = __ldcg(reinterpret_cast<const float2*>(partd + (size_t)b * n + i));
          acc[i] = df_add(acc[i], df{v.x, v.y});
        }
    }
    block_sum_df<N>(acc, n, red);
    for (int k = threadIdx.x; k < n; k += blockDim.x) all[k] = df_to_double(red[k]);
    __syncthreads();
  } else {
    __shared__ double red[N];
    block_sum<N, A>(tot, n, red);
    for (int k = threadIdx.x; k < n; k += blockDim.x) part[(size_t)blockIdx.x * n + k] = red[k];
    if (!arrive_last(&st->cnt_seed)) return;
    reduce_partials<N>(part, gridDim.x, n, n, all);
  }
  seed_finish<METHOD>(all, np, parity, st, w_out, s_sc[1]);
}

// K2 for many projection rows in the FP32-pair form.  The plain kernel keeps
// 3 + 2 NP pair accumulators per thread (rho, nu and every P r_{n+1} entry),
// which above nine rows limits it to one or two blocks per SM.  Here each
// 256-element tile goes through two phases: (A) every thread forms r_{n+1} for
// one element (Eq. 16), stores it, accumulates rho and nu, and leaves it in
// shared memory; (B) the block's four 64-thread groups each take every fourth
// projection row over all 256 elements (four per thread), reading r_{n+1} from
// shared memory, for w_l = a_l^T r_{n+1} (the P r_{n+1} of Eq. 26).  A thread
// holds 3 + 2 ceil(NP / 4) accumulators.  The tile of the np projection rows
// (np x 2 KB) is copied into shared memory by TMA bulk copies two tiles ahead
// (full tiles; the ragged last tile reads the rows directly), on the same
// bounded mbarrier protocol as the staged kernel above: a wait that runs out
// ends the solve with KW_ERR_TIMEOUT after the block's copies have landed.
// Sums run in a fixed order (deterministic), with pair block and grid
// reductions.
constexpr int kRowGroups = 4;
constexpr int kRgStages = 2;

__host__ __device__ constexpr uint32_t rg_stage_bytes(int np) { return (uint32_t)(np * kSeedTile * sizeof(df)); }

template <int NP, int METHOD>
__global__ void __launch_bounds__(256, 3)
k_seed_update_rg(int m, const dfc* __restrict__ rn_buf, const dfc* __restrict__ q, dfc* __restrict__ rm_buf,
                 const df* __restrict__ proj, int64_t ld, int np, int parity, State* st, double* __restrict__ part,
                 double2* __restrict__ w_out, uint32_t tx_pad) {
  constexpr int RPG = (NP + kRowGroups - 1) / kRowGroups;
  constexpr int N = 3 + 2 * NP;
  static_assert(kSeedTile == 256, "four 64-thread row groups per 256-element tile");
  extern __shared__ __align__(128) unsigned char kw_rg_stage[];
  __shared__ __align__(8) uint64_t bars[kRgStages];
  if (st->done) return;
  __shared__ double2 s_sc[2];
  __shared__ double2 s_cf[3];
  __shared__ float4 s_pp[3];
  __shared__ int s_fail;
  __shared__ cpk s_r1[kSeedTile];   // r_{n+1} of the tile, packed (re, im) layout
  __shared__ df sw[N][8];
  __shared__ df red[N];
  __shared__ double all[N];
  seed_coefficients(st, parity, s_sc, s_cf, s_pp, &s_fail);
  __syncthreads();
  if (s_fail) return;
  // packed forms of the three coefficients a, -b, -c (cpk_coef), in registers
  const cpk_coef na = cpk_coef_of(s_pp[0], 1.f), nb = cpk_coef_of(s_pp[1], -1.f), nc = cpk_coef_of(s_pp[2], -1.f);
  const int n = 3 + 2 * np;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = threadIdx.x / 64, e0 = threadIdx.x % 64;
  cpk sq = cpk_zero();            // packed (sum re^2, sum im^2)
  df x2 = azero<df>();            // sum re * im
  cpk pacc[RPG];   // (w_l.re, w_l.im) of this group's rows, packed pairs
#pragma unroll
  for (int j = 0; j < RPG; ++j) pacc[j] = cpk_zero();
  const int ntiles = (m + kSeedTile - 1) / kSeedTile, nfull = m / kSeedTile, G = gridDim.x;
  const uint32_t sbytes = rg_stage_bytes(np), tx = sbytes + tx_pad;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kRgStages; ++s) mbar_init(&bars[s], 1);
    mbar_init_fence();
  }
  __syncthreads();
  auto issue = [&](int t, int s) {   // thread 0: the projection rows of tile t into stage s
    unsigned char* dst = kw_rg_stage + (size_t)s * sbytes;
    const size_t e = (size_t)t * kSeedTile;
    mbar_arrive_expect(&bars[s], tx);
    for (int l = 0; l < np; ++l)
      bulk_load(dst + (size_t)l * kSeedTile * sizeof(df), proj + (size_t)l * ld + e, kSeedTile * sizeof(df), &bars[s]);
  };
  if (threadIdx.x == 0)
    for (int s = 0; s < kRgStages; ++s)
      if (blockIdx.x + s * G < nfull) issue(blockIdx.x + s * G, s);
  int k = 0;
  for (int t = blockIdx.x; t < ntiles; t += G, ++k) {
    const int base = t * kSeedTile;
    const int i = base + (int)threadIdx.x;
    cpk r1 = cpk_zero();
    if (i < m) {                                      // phase A: Eq. 16 for one element (packed pairs)
      r1 = three_term_pk(na, nb, nc, cpk_of(rn_buf[i]), cpk_of(q[i]), cpk_of(rm_buf[i]));
      rm_buf[i] = dfc_of(r1);
      acc_sq_pk(sq, r1);
      if constexpr (METHOD != KW_METHOD_CG) acc_prod(x2, df{r1.hi.x, r1.lo.x}, df{r1.hi.y, r1.lo.y});
    }
    s_r1[threadIdx.x] = r1;
    const bool staged = t < nfull;
    const int s = k % kRgStages;
    const bool late = staged && !mbar_wait(&bars[s], (uint32_t)(k / kRgStages) & 1u);
    if (__syncthreads_or(late)) {   // a copy did not land in time: report, let copies in flight finish, stop
      if (threadIdx.x == 0) {
        set_fail(st, KW_ERR_TIMEOUT);
        for (int j = 0; j < kRgStages; ++j)
          if (blockIdx.x + (k + j) * G < nfull)
            mbar_wait(&bars[(k + j) % kRgStages], (uint32_t)((k + j) / kRgStages) & 1u);
      }
      __syncthreads();
      break;
    }
    const df* sa = reinterpret_cast<const df*>(kw_rg_stage + (size_t)s * sbytes);
#pragma unroll
    for (int jj = 0; jj < kSeedTile / 64; ++jj) {    // phase B: this group's rows over the tile
      const int e = e0 + 64 * jj, ie = base + e;
      if (ie < m) {
        const cpk rv = s_r1[e];
#pragma unroll
        for (int j = 0; j < RPG; ++j) {
          const int l = g + kRowGroups * j;
          if (l < np) {
            const df a = staged ? sa[l * kSeedTile + e] : proj[(size_t)l * ld + ie];
            acc_proj_pk(pacc[j], a, rv);
          }
        }
      }
    }
    __syncthreads();                                  // stage s and s_r1 are free
    if (threadIdx.x == 0 && t + kRgStages * G < nfull) {
      fence_async_smem();
      issue(t + kRgStages * G, s);
    }
  }
  // block sums: one pair per warp and value (a warp lies in one row group; it
  // contributes zero to the other groups' rows), then the eight warps in order
  {
    const df re2 = anorm(df{sq.hi.x, sq.lo.x}), im2 = anorm(df{sq.hi.y, sq.lo.y});
    const df r0 = warp_sum(anorm(df_sub(re2, im2))), r1v = warp_sum(anorm(df{2.f * x2.hi, 2.f * x2.lo}));
    const df r2 = warp_sum(anorm(df_add(re2, im2)));
    if (lane == 0) {
      sw[0][warp] = r0;
      sw[1][warp] = r1v;
      sw[2][warp] = r2;
    }
  }
#pragma unroll
  for (int j = 0; j < RPG; ++j) {
    const df a = warp_sum(anorm(df{pacc[j].hi.x, pacc[j].lo.x})), b = warp_sum(anorm(df{pacc[j].hi.y, pacc[j].lo.y}));
#pragma unroll
    for (int gg = 0; gg < kRowGroups; ++gg) {
      const int l = gg + kRowGroups * j;
      if (l < NP && lane == 0) {
        sw[3 + 2 * l][warp] = gg == g ? a : azero<df>();
        sw[4 + 2 * l][warp] = gg == g ? b : azero<df>();
      }
    }
  }
  __syncthreads();
  df* partd = reinterpret_cast<df*>(part);
  for (int kk = threadIdx.x; kk < n; kk += blockDim.x) {
    df sum = sw[kk][0];
    for (int w = 1; w < 8; ++w) sum = df_add(sum, sw[kk][w]);
    partd[(size_t)blockIdx.x * n + kk] = sum;
  }
  if (!arrive_last(&st->cnt_seed)) return;
  // last block: value kk by warp kk mod 8, its lanes striding over the blocks
  for (int kk = warp; kk < n; kk += 8) {
    df a = azero<df>();
    for (int b = lane; b < (int)gridDim.x; b += 32) {
      const float2 v = __ldcg(reinterpret_cast<const float2*>(partd + (size_t)b * n + kk));
      a = df_add(a, df{v.x, v.y});
    }
    a = warp_sum(anorm(a));
    if (lane == 0) red[kk] = a;
  }
  __syncthreads();
  for (int kk = threadIdx.x; kk < n; kk += blockDim.x) all[kk] = df_to_double(red[kk]);
  __syncthreads();
  seed_finish<METHOD>(all, np, parity, st, w_out, s_sc[1]);   // CG reads rho = ||r||^2 from all[2]
}

// ================================================================ K3: shift scalars
struct ShiftArgs {
  int K, np, full;
  int parity;        // iteration parity: the slots of coef, coef_pair, list, n_list, xp_pending
  const double2* z;
  double2* pi1;      // pi_n on entry, pi_{n+1} on exit
  double2* pi0;      // pi_{n-1} on entry, pi_n on exit
  int* active;
  long long* conv_iter;
  double* final_res;
  double2* coef;     // this parity's slot, full mode [K][3]: alpha^k, beta^k, 1/pi^k_{n+1}
  float4* coef_pair; // the same as FP32 pairs (read by K4 in the FP32 and FP32-pair forms)
  double2* Y;
  double2* U;
  const double2* w;  // P r_{n+1}
  double* hist;
  int* list;
  double* part;      // per block: [best |pi|^2, best index, n still active]
  double2* log;      // Krylov log rows [log_max][KW_LOG_FIXED + np], or NULL
  long long log_max;
};

// One warp per block, LPS lanes per shift (the launcher picks 1 in full mode,
// else the projection count rounded up to a power of two, at most 4): the lanes
// of a shift compute its scalars redundantly and update every LPS-th projection
// row, so the FP64 work spreads over many SMs without recomputing the scalars
// on many lanes.
template <int LPS>
__global__ void __launch_bounds__(32) k_shift(ShiftArgs a, State* st) {
  if (st->done) return;
  constexpr int SPW = 32 / LPS;   // shifts per warp
  const int lane = threadIdx.x, sub = lane % LPS;
  const int k = blockIdx.x * SPW + lane / LPS;
  const double2 alpha = st->alpha, c = st->c, beta = st->beta, zs = st->zs;
  const double nu = st->nu, thresh = st->thresh;
  const int pend = st->pi_rescale_pending, jnew = st->new_seed;
  const double2 i1 = st->inv_pj1, i0 = st->inv_pj0;
  const long long iter = st->iter;
  const bool rec = st->hist_stride > 0 && ((iter + 1) % st->hist_stride) == 0 && st->n_rec < st->hist_max;
  const long long rec_row = st->n_rec;
  const bool inK = k < a.K;
  const bool act = inK && a.active[k];

  double best = INFINITY;
  int best_k = 0x7fffffff, still = 0, brk = 0, in_list = 0;
  if (act) {
    double2 p1 = a.pi1[k], p0 = a.pi0[k];
    const double2 zk = a.z[k];
    if (pend) {                       // lazy rescale after a seed switch
      if (k == jnew) {
        p1 = p0 = make_double2(1.0, 0.0);
      } else {
        p1 = cmul(p1, i1);
        p0 = cmul(p0, i0);
      }
    }
    const double2 sigma = csub(zk, zs);
    // pi_{n+1} = (1 + c_n + alpha_n sigma) pi_n - c_n pi_{n-1}          (Eq. 20)
    const double2 f = cadd(make_double2(1.0 + c.x, c.y), cmul(alpha, sigma));
    const double2 pn = csub(cmul(f, p1), cmul(c, p0));
    in_list = (sub == 0);
    if (pn.x == 0.0 && pn.y == 0.0) {
      brk = 1;
    } else {
      const double2 ipn = crecip(pn);                 // 1 / pi_{n+1}
      const double2 ratio = cmul(p1, ipn);            // pi_n / pi_{n+1}
      const double2 ak = cmul(ratio, alpha);          // Eq. 21
      const double2 bk = cmul(cmul(ratio, ratio), beta);  // Eq. 22
      if (sub == 0) a.coef[3 * k + 2] = ipn;       // read by the seed switch and by K4
      if (a.full && sub == 0) {
        a.coef[3 * k + 0] = ak;
        a.coef[3 * k + 1] = bk;
        a.coef[3 * k + 2] = ipn;
        a.coef_pair[3 * k + 0] = pair_of(ak);
        a.coef_pair[3 * k + 1] = pair_of(bk);
        a.coef_pair[3 * k + 2] = pair_of(ipn);
      }
      {   // projected mode, and full mode with FP32 shift storage: a.np > 0
        for (int l = sub; l < a.np; l += LPS) {       // Eq. 25-26
          const size_t o = (size_t)k * a.np + l;
          const double2 u = a.U[o], y = a.Y[o], wl = a.w[l];
          a.Y[o] = cadd(y, cmul(ak, u));
          a.U[o] = cadd(cmul(wl, ipn), cmul(bk, u));
        }
      }
      const double res = sqrt(nu * (ipn.x * ipn.x + ipn.y * ipn.y));   // ||r|| / |pi_{n+1}|
      if (sub == 0) {
        a.pi0[k] = p1;
        a.pi1[k] = pn;
        a.final_res[k] = res;
        if (rec) a.hist[(size_t)rec_row * a.K + k] = res;
        if (res <= thresh) {
          a.active[k] = 0;
          a.conv_iter[k] = iter + 1;
        } else {
          still = 1;
          best = __dadd_rn(__dmul_rn(pn.x, pn.x), __dmul_rn(pn.y, pn.y));
          best_k = k;
        }
      }
    }
  } else if (rec && inK && sub == 0) {
    a.hist[(size_t)rec_row * a.K + k] = a.final_res[k];
  }
  // compacted list of the shifts updated this iteration (one slot per shift)
  {
    const unsigned bal = __ballot_sync(KW_FULL_MASK, in_list);
    int basepos = 0;
    if (lane == 0 && bal) basepos = atomicAdd(&st->n_list[a.parity], __popc(bal));
    basepos = __shfl_sync(KW_FULL_MASK, basepos, 0);
    if (in_list) a.list[basepos + __popc(bal & ((1u << lane) - 1))] = k;
  }

  // warp argmin of |pi_{n+1}|^2 over still-active shifts (ties: lowest index), count, breakdown
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const double ob = __shfl_xor_sync(KW_FULL_MASK, best, off);
    const int ok = __shfl_xor_sync(KW_FULL_MASK, best_k, off);
    if (ob < best || (ob == best && ok < best_k)) { best = ob; best_k = ok; }
    still += __shfl_xor_sync(KW_FULL_MASK, still, off);
    brk |= __shfl_xor_sync(KW_FULL_MASK, brk, off);
  }
  if (lane == 0) {
    a.part[4 * blockIdx.x + 0] = best;
    a.part[4 * blockIdx.x + 1] = (double)best_k;
    a.part[4 * blockIdx.x + 2] = (double)still;
    a.part[4 * blockIdx.x + 3] = (double)brk;
  }
  if (!arrive_last(&st->cnt_shift)) return;

  // last block: the lanes reduce the block partials in parallel
  double gb = INFINITY;
  int gk = 0x7fffffff, any_brk = 0;
  long long n_still = 0;
  for (int b = lane; b < (int)gridDim.x; b += 32) {
    const double vb = __ldcg(a.part + 4 * b);
    const int vk = (int)__ldcg(a.part + 4 * b + 1);
    if (vb < gb || (vb == gb && vk < gk)) { gb = vb; gk = vk; }
    n_still += (long long)__ldcg(a.part + 4 * b + 2);
    any_brk |= (int)__ldcg(a.part + 4 * b + 3);
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const double ob = __shfl_xor_sync(KW_FULL_MASK, gb, off);
    const int ok = __shfl_xor_sync(KW_FULL_MASK, gk, off);
    if (ob < gb || (ob == gb && ok < gk)) { gb = ob; gk = ok; }
    n_still += __shfl_xor_sync(KW_FULL_MASK, n_still, off);
    any_brk |= __shfl_xor_sync(KW_FULL_MASK, any_brk, off);
  }
  // Krylov log row of this iteration (Sec. 3.3 (iv)): P r_{n+1} by the lanes,
  // the scalars by lane 0 once the seed switch is decided.
  double2* lrow = (a.log && iter < a.log_max) ? a.log + (size_t)iter * (KW_LOG_FIXED + a.np) : nullptr;
  if (lrow)
    for (int l = lane; l < a.np; l += 32) lrow[KW_LOG_FIXED + l] = a.w[l];
  if (lane != 0) return;
  const int nl = *((volatile int*)&st->n_list[a.parity]);
  const bool do_switch = st->seed_switch && n_still > 0 && gb < 1.0;
  const double2 rho1_in = st->rho1;
  const long long upd = st->updates, maxiter = st->maxiter;
  const int nsw = st->n_seed_switch;
  double2 ipj1 = make_double2(1.0, 0.0), pj0 = ipj1, zj = ipj1;
  if (do_switch) {
    ipj1 = __ldcg(a.coef + 3 * gk + 2);   // 1/pi^j_{n+1}, computed by the shift's owner lane
    pj0 = __ldcg(a.pi0 + gk);
    zj = a.z[gk];
  }
  st->cnt_shift = 0;
  st->pi_rescale_pending = 0;
  if (rec) st->n_rec = rec_row + 1;
  st->updates = upd + nl;
  st->xp_pending[a.parity] = (a.full && nl > 0 && !any_brk) ? 1 : 0;
  st->n_active = (int)n_still;
  if (any_brk) {                                        // pi_{n+1} = 0 (Eq. 20)
    set_fail(st, KW_ERR_BREAKDOWN);
    return;
  }
  if (lrow) {
    const double2 one = make_double2(1.0, 0.0);
    lrow[0] = zs;
    lrow[1] = alpha;
    lrow[2] = c;
    lrow[3] = beta;
    lrow[4] = make_double2(nu, 0.0);
    lrow[5] = do_switch ? __ldcg(a.pi1 + gk) : one;   // pi^j_{n+1}, written by the shift's owner lane
    lrow[6] = do_switch ? pj0 : one;
  }
  double2 rho1 = rho1_in;
  double2 boa = cmul(rho1_in, st->inv_rho_alpha);       // beta_n / alpha_n
  if (do_switch) {                                      // Sec. 2.2.4
    const double2 ii1 = ipj1, ii0 = crecip(pj0);
    // r_{n+1} <- r_{n+1} / pi^j_{n+1}, r_n <- r_n / pi^j_n, pending on their
    // buffers: iteration n (parity n & 1) wrote r_{n+1} into buffer 1 - (n & 1)
    const int par = (int)(iter & 1);
    st->bscale[1 - par] = cmul(st->bscale[1 - par], ii1);
    st->bscale[par] = cmul(st->bscale[par], ii0);
    st->p_zs = pair_of(zj);
    st->switched = 1;
    rho1 = cmul(rho1, cmul(ii1, ii1));   // rho_{n+1} of the rescaled residual
    boa = cmul(boa, cmul(pj0, ii1));     // beta^j_n / alpha^j_n
    st->inv_pj1 = ii1;
    st->inv_pj0 = ii0;
    st->pi_rescale_pending = 1;
    st->new_seed = gk;
    st->seed = gk;
    st->zs = zj;
    st->n_seed_switch = nsw + 1;
  }
  st->rho = rho1;
  st->boa = boa;
  st->iter = iter + 1;
  if (n_still == 0) {
    st->status = KW_OK;
    st->done = 1;
  } else if (iter + 1 >= maxiter) {
    st->status = KW_NOT_CONVERGED;
    st->done = 1;
  }
}

// ================================================================ recalculation at new shifts
// Sec. 3.3 (iv): the logged iterations are replayed for each new shift with
// the same arithmetic as K3 (Eq. 20, Eqs. 21-22, Eqs. 25-26, the pi rescale of
// a seed switch).  LPS lanes per shift: they compute the shift's scalars
// redundantly (one warp instruction for all of them) and each updates the
// projection columns l = sub, sub + LPS, ... (at most NPL).  The host picks
// LPS so that there are enough warps to spread over the SMs.  Log rows are
// staged through shared memory in chunks of kRecalcChunk rows, loaded by the
// whole block at once.
template <int LPS, int NPL>
__global__ void __launch_bounds__(kRecalcThreads)
    k_recalc(int K, int np, long long n_iter, const double2* __restrict__ log, const double2* __restrict__ w0,
             const double2* __restrict__ z, double thresh, double2* __restrict__ proj,
             long long* __restrict__ conv_iter, double* __restrict__ final_res, int* __restrict__ flag) {
  extern __shared__ double2 srows[];   // [kRecalcChunk][KW_LOG_FIXED + np]
  constexpr int SPB = kRecalcThreads / LPS;   // shifts per block
  const int R = KW_LOG_FIXED + np;
  const int sub = threadIdx.x % LPS;
  const int k = blockIdx.x * SPB + threadIdx.x / LPS;
  double2 y[NPL], u[NPL];
#pragma unroll
  for (int i = 0; i < NPL; ++i) {
    const int l = sub + i * LPS;
    y[i] = make_double2(0.0, 0.0);
    u[i] = l < np ? w0[l] : make_double2(0.0, 0.0);   // u_0 = P b
  }
  double2 p1 = make_double2(1.0, 0.0), p0 = p1;
  const double2 zk = k < K ? z[k] : make_double2(0.0, 0.0);
  bool act = k < K;
  long long ci = -1;
  double fr = INFINITY;
  for (long long n0 = 0; n0 < n_iter; n0 += kRecalcChunk) {
    if (!__syncthreads_or(act)) break;
    const int rows = (int)min((long long)kRecalcChunk, n_iter - n0);
    for (int i = threadIdx.x; i < rows * R; i += blockDim.x) srows[i] = log[(size_t)n0 * R + i];
    __syncthreads();
    for (int j = 0; act && j < rows; ++j) {
      const double2* row = srows + j * R;
      const double2 zs = row[0], alpha = row[1], c = row[2], beta = row[3];
      const double nu = row[4].x;
      const double2 f = cadd(make_double2(1.0 + c.x, c.y), cmul(alpha, csub(zk, zs)));
      const double2 pn = csub(cmul(f, p1), cmul(c, p0));               // Eq. 20
      if (pn.x == 0.0 && pn.y == 0.0) {
        if (sub == 0) atomicOr(flag, 1);
        act = false;
        break;
      }
      const double2 ipn = crecip(pn);
      const double2 ratio = cmul(p1, ipn);
      const double2 ak = cmul(ratio, alpha);                            // Eq. 21
      const double2 bk = cmul(cmul(ratio, ratio), beta);                // Eq. 22
#pragma unroll
      for (int i = 0; i < NPL; ++i) {
        const int l = sub + i * LPS;
        if (l < np) {                                                   // Eqs. 25-26
          y[i] = cadd(y[i], cmul(ak, u[i]));
          u[i] = cadd(cmul(row[KW_LOG_FIXED + l], ipn), cmul(bk, u[i]));
        }
      }
      fr = sqrt(nu * (ipn.x * ipn.x + ipn.y * ipn.y));
      p0 = p1;
      p1 = pn;
      if (fr <= thresh) {
        act = false;
        ci = n0 + j + 1;
        break;
      }
      const double2 s1 = row[5], s0 = row[6];
      if (s1.x != 1.0 || s1.y != 0.0 || s0.x != 1.0 || s0.y != 0.0) {  // seed switch (Sec. 2.2.4)
        p1 = cmul(p1, crecip(s1));
        p0 = cmul(p0, crecip(s0));
      }
    }
    __syncthreads();
  }
  if (k >= K) return;
#pragma unroll
  for (int i = 0; i < NPL; ++i) {
    const int l = sub + i * LPS;
    if (l < np) proj[(size_t)k * np + l] = y[i];
  }
  if (sub == 0) {
    conv_iter[k] = ci;
    final_res[k] = fr;
  }
}

// ================================================================ K4: fused x/p update
// The shifted vectors' element type: the form's vector type, or complex FP32
// when the shift storage is FP32 (XP32); r_{n+1} is then rounded to FP32 once
// per element (the leading part of an FP32 pair is its FP32 rounding) and the
// update runs in FP32 with the scalars' leading parts.
template <int P, bool XP32> struct XT { typedef typename PT<P>::V V; };
template <int P> struct XT<P, true> { typedef float2 V; };
__device__ __forceinline__ double2 to_x(double2 v, double2*) { return v; }
__device__ __forceinline__ float2 to_x(float2 v, float2*) { return v; }
__device__ __forceinline__ dfc to_x(dfc v, dfc*) { return v; }
__device__ __forceinline__ float2 to_x(dfc v, float2*) { return make_float2(v.re.hi, v.im.hi); }
__device__ __forceinline__ float2 to_x(double2 v, float2*) { return make_float2((float)v.x, (float)v.y); }

template <int P, int TS, bool XP32 = false>
__global__ void __launch_bounds__(256)
k_update_xp(int m, const int* __restrict__ list, const double2* __restrict__ coef,
            const float4* __restrict__ coef_pair, typename XT<P, XP32>::V* __restrict__ X,
            typename XT<P, XP32>::V* __restrict__ Pv, const typename PT<P>::V* __restrict__ r1, State* st,
            int parity, int pairs) {
  typedef typename XT<P, XP32>::V V;
  if (!st->xp_pending[parity]) return;
  const int nl = st->n_list[parity];
  const int ntile = (nl + TS - 1) / TS;
  // pairs (complex FP32 x and p, both 16-byte aligned): thread t of a chunk
  // takes pair t, elements 2t - o and 2t - o + 1 of a row whose offset k m has
  // parity o, so that the pair starts 16-byte aligned, with one 16-byte load
  // and store per row of x and p; an element whose partner falls outside the
  // row (element 0 of an odd row, element m - 1 of an even row when m is odd)
  // is taken alone.  Pair indices 0 .. m/2 cover every element of both parities.
  const int nunit = pairs ? m / 2 + 1 : m;
  const int nchunk = (nunit + (int)blockDim.x - 1) / (int)blockDim.x;
  __shared__ V cs[TS][3];
  __shared__ int ks[TS];
  const long long nitem = (long long)ntile * nchunk;
  for (long long item = blockIdx.x; item < nitem; item += gridDim.x) {
    const int tile = (int)(item % ntile), chunk = (int)(item / ntile);
    const int t0 = tile * TS, nts = min(TS, nl - t0);
    __syncthreads();
    if (threadIdx.x < nts) {
      const int k = list[t0 + threadIdx.x];
      ks[threadIdx.x] = k;
#pragma unroll
      for (int j = 0; j < 3; ++j) cs[threadIdx.x][j] = vscalar<V>(coef[3 * k + j], coef_pair[3 * k + j]);
    }
    __syncthreads();
    if constexpr (std::is_same<V, float2>::value) {
      if (pairs) {
        const int e = 2 * (chunk * (int)blockDim.x + (int)threadIdx.x);   // first element of pair t when o = 0
        if (e <= m) {
          // r_{n+1} at e - 1, e, e + 1 (inside the row): the pair's elements for either parity
          const V rm1 = e >= 1 ? to_x(r1[e - 1], (V*)nullptr) : V{};
          const V r0 = e < m ? to_x(r1[e], (V*)nullptr) : V{};
          const V rp1 = e + 1 < m ? to_x(r1[e + 1], (V*)nullptr) : V{};
#pragma unroll TS
          for (int s = 0; s < nts; ++s) {
            const size_t base = (size_t)ks[s] * m;
            const int par = (int)(base & 1);
            const int e0 = e - par;                          // base + e0 is even
            const V ra = par ? rm1 : r0, rb = par ? r0 : rp1;
            if (e0 >= 0 && e0 + 1 < m) {
              const size_t o = base + e0;
              float4 xx = *reinterpret_cast<const float4*>(X + o), pp = *reinterpret_cast<const float4*>(Pv + o);
              V xa = make_float2(xx.x, xx.y), xb = make_float2(xx.z, xx.w);
              V pa = make_float2(pp.x, pp.y), pb = make_float2(pp.z, pp.w);
              xa = cadd(xa, cmul(cs[s][0], pa));                   // Eq. 23
              xb = cadd(xb, cmul(cs[s][0], pb));
              pa = cadd(cmul(ra, cs[s][2]), cmul(cs[s][1], pa));   // Eq. 24
              pb = cadd(cmul(rb, cs[s][2]), cmul(cs[s][1], pb));
              *reinterpret_cast<float4*>(X + o) = make_float4(xa.x, xa.y, xb.x, xb.y);
              *reinterpret_cast<float4*>(Pv + o) = make_float4(pa.x, pa.y, pb.x, pb.y);
            } else {
              // the element of this pair that lies in the row (if any) alone
              const int i = e0 < 0 ? e0 + 1 : e0;
              if (i >= 0 && i < m) {
                const V ri = e0 < 0 ? rb : ra;
                const size_t o = base + i;
                V x = X[o], p = Pv[o];
                x = cadd(x, cmul(cs[s][0], p));
                p = cadd(cmul(ri, cs[s][2]), cmul(cs[s][1], p));
                X[o] = x;
                Pv[o] = p;
              }
            }
          }
        }
        continue;
      }
    }
    const int i = chunk * blockDim.x + threadIdx.x;
    if (i < m) {
      const V ri = to_x(r1[i], (V*)nullptr);
#pragma unroll (XP32 ? TS : 4)
      for (int s = 0; s < nts; ++s) {
        const size_t o = (size_t)ks[s] * m + i;
        V x = X[o], p = Pv[o];
        x = cadd(x, cmul(cs[s][0], p));                        // Eq. 23
        p = cadd(cmul(ri, cs[s][2]), cmul(cs[s][1], p));       // Eq. 24
        X[o] = x;
        Pv[o] = p;
      }
    }
  }
  if (!arrive_last(&st->cnt_xp)) return;
  if (threadIdx.x == 0) {
    st->cnt_xp = 0;
    st->xp_pending[parity] = 0;
  }
}

// ================================================================ adjoint bilinear forms
// out[k] = y_k^T H x_k (unconjugated) for a tile of BT shifts: one thread per
// row reads the row's indices and values once and applies them to every shift
// of the tile.  X, Y: [K][m] complex, shift-major, FP64 (XV = double2) or FP32
// (XV = float2, widened to FP64 on load); the sums are FP64.  Per-block
// partials part[(tile * gridDim.x + block) * BT + t] are summed by
// k_bilinear_reduce.
__device__ __forceinline__ double2 wide(double2 v) { return v; }
__device__ __forceinline__ double2 wide(float2 v) { return make_double2(v.x, v.y); }

template <int BT, class XV>
__global__ void __launch_bounds__(256)
k_bilinear(int m, int K, const int64_t* __restrict__ rowptr, const int* __restrict__ col,
           const double* __restrict__ val, const XV* __restrict__ X, const XV* __restrict__ Y,
           double2* __restrict__ part) {
  const int tile = blockIdx.y, k0 = tile * BT;
  const int nt = min(BT, K - k0);
  double re[BT], im[BT];
#pragma unroll
  for (int t = 0; t < BT; ++t) re[t] = im[t] = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
    const int beg = (int)rowptr[i], end = (int)rowptr[i + 1];
#pragma unroll
    for (int t = 0; t < BT; ++t) {
      if (t < nt) {
        const XV* xk = X + (size_t)(k0 + t) * m;
        double2 s = make_double2(0.0, 0.0);
        for (int j = beg; j < end; ++j) {
          const double v = val[j];
          const double2 x = wide(xk[col[j]]);
          s.x = fma(v, x.x, s.x);
          s.y = fma(v, x.y, s.y);
        }
        const double2 y = wide(Y[(size_t)(k0 + t) * m + i]);
        re[t] = fma(y.x, s.x, fma(-y.y, s.y, re[t]));
        im[t] = fma(y.x, s.y, fma(y.y, s.x, im[t]));
      }
    }
  }
  __shared__ double red[2 * BT];
  double v[2 * BT];
#pragma unroll
  for (int t = 0; t < BT; ++t) {
    v[2 * t] = re[t];
    v[2 * t + 1] = im[t];
  }
  block_sum<2 * BT, double>(v, 2 * BT, red);
  if (threadIdx.x < BT) {
    const size_t o = ((size_t)tile * gridDim.x + blockIdx.x) * BT + threadIdx.x;
    part[o] = make_double2(red[2 * threadIdx.x], red[2 * threadIdx.x + 1]);
  }
}

// Structure of one term for the diagonal path: d[i] = its entry in row i if
// that is the row's only entry and sits on the diagonal, 0 for an empty row;
// any other row clears *flag (several threads may store the same 0).
static __global__ void k_diag_scan(int m, const int64_t* __restrict__ rowptr, const int* __restrict__ col,
                            const double* __restrict__ val, double* __restrict__ d, int* flag) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
    const int64_t b = rowptr[i], e = rowptr[i + 1];
    double v = 0.0;
    if (e - b == 1 && col[b] == i) v = val[b];
    else if (e != b) *flag = 0;
    d[i] = v;
  }
}

// out[k][idx[t]] = sum_i d_t[i] y_k[i] x_k[i] for a group of diagonal terms:
// block (bx, k - k0) takes shift k over a grid-stride share of the rows, forms
// y_k[i] x_k[i] once per row and applies it to every term of the group (the
// diagonals, a few MB, are re-read from L2 for each shift).  FP64 sums; the
// per-block partials part[(k * gridDim.x + bx) * DT + t] are summed by
// k_bilinear_diag_reduce.
template <int DT, class XV>
__global__ void __launch_bounds__(256)
k_bilinear_diag(int m, int k0, const double* __restrict__ d, DiagGroup g, const XV* __restrict__ X,
                const XV* __restrict__ Y, double2* __restrict__ part) {
  const int k = k0 + (int)blockIdx.y;
  const XV* xk = X + (size_t)k * m;
  const XV* yk = Y + (size_t)k * m;
  double re[DT], im[DT];
#pragma unroll
  for (int t = 0; t < DT; ++t) re[t] = im[t] = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
    const double2 x = wide(xk[i]), y = wide(yk[i]);
    const double pr = fma(y.x, x.x, -y.y * x.y), pi = fma(y.x, x.y, y.y * x.x);   // y_k[i] x_k[i]
#pragma unroll
    for (int t = 0; t < DT; ++t)
      if (t < g.n) {
        const double dv = d[(size_t)g.idx[t] * m + i];
        re[t] = fma(dv, pr, re[t]);
        im[t] = fma(dv, pi, im[t]);
      }
  }
  __shared__ double red[2 * DT];
  double v[2 * DT];
#pragma unroll
  for (int t = 0; t < DT; ++t) {
    v[2 * t] = re[t];
    v[2 * t + 1] = im[t];
  }
  block_sum<2 * DT, double>(v, 2 * DT, red);
  if (threadIdx.x < g.n) {
    const size_t o = ((size_t)k * gridDim.x + blockIdx.x) * DT + threadIdx.x;
    part[o] = make_double2(red[2 * threadIdx.x], red[2 * threadIdx.x + 1]);
  }
}

// out[k * nterm + idx[t]] = sum over the nblk blocks of shift k, fixed order.
template <int DT>
__global__ void k_bilinear_diag_reduce(int K, int nblk, DiagGroup g, int nterm, const double2* __restrict__ part,
                                       double2* __restrict__ out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= K * g.n) return;
  const int k = j / g.n, t = j % g.n;
  double2 s = make_double2(0.0, 0.0);
  for (int b = 0; b < nblk; ++b) {
    const double2 p = part[((size_t)k * nblk + b) * DT + t];
    s.x += p.x;
    s.y += p.y;
  }
  out[(size_t)k * nterm + g.idx[t]] = s;
}

// out[k * nterm + term] = sum over blocks of the partials, fixed order.
template <int BT>
__global__ void k_bilinear_reduce(int K, int nblk, int term, int nterm, const double2* __restrict__ part,
                                  double2* __restrict__ out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= K) return;
  const int tile = k / BT, t = k % BT;
  double2 s = make_double2(0.0, 0.0);
  for (int b = 0; b < nblk; ++b) {
    const double2 p = part[((size_t)tile * nblk + b) * BT + t];
    s.x += p.x;
    s.y += p.y;
  }
  out[(size_t)k * nterm + term] = s;
}

// ================================================================ combinations over the shifts
// S[k][i] = sum_j W[k][j] x_j[i] for k < nk <= NK (the contour moments of
// Sec. 4.1 are such combinations): one thread per element i (grid-stride),
// the weights staged in shared memory 64 shifts at a time, x_j[i] read
// coalesced and widened to FP64, FP64 complex sums in a fixed order.
constexpr int kCombineChunk = 64;

template <int NK, class XV>
__global__ void __launch_bounds__(256)
k_shift_combine(int m, int K, int nk, const XV* __restrict__ X, const double2* __restrict__ W,
                double2* __restrict__ S) {
  __shared__ double2 sw[NK][kCombineChunk];
  for (long long base = (long long)blockIdx.x * blockDim.x; base < m; base += (long long)gridDim.x * blockDim.x) {
    const long long i = base + threadIdx.x;
    double2 acc[NK];
#pragma unroll
    for (int k = 0; k < NK; ++k) acc[k] = make_double2(0.0, 0.0);
    for (int j0 = 0; j0 < K; j0 += kCombineChunk) {
      const int nj = min(kCombineChunk, K - j0);
      __syncthreads();
      for (int t = threadIdx.x; t < NK * kCombineChunk; t += blockDim.x) {
        const int k = t / kCombineChunk, j = t % kCombineChunk;
        sw[k][j] = (k < nk && j < nj) ? W[(size_t)k * K + j0 + j] : make_double2(0.0, 0.0);
      }
      __syncthreads();
      if (i < m) {
        for (int j = 0; j < nj; ++j) {
          const double2 x = wide(X[(size_t)(j0 + j) * m + i]);
#pragma unroll
          for (int k = 0; k < NK; ++k) {
            const double2 w = sw[k][j];
            acc[k].x = fma(w.x, x.x, fma(-w.y, x.y, acc[k].x));
            acc[k].y = fma(w.x, x.y, fma(w.y, x.x, acc[k].y));
          }
        }
      }
    }
    if (i < m)
#pragma unroll
      for (int k = 0; k < NK; ++k)
        if (k < nk) S[(size_t)k * m + i] = acc[k];
  }
}

// ================================================================ initialisation
template <int P>
__global__ void k_init_vectors(int m, int np, const double* __restrict__ b, const double* __restrict__ left,
                               typename PT<P>::V* rn, typename PT<P>::V* rm, typename PT<P>::R* proj,
                               int64_t ld) {
  typedef typename PT<P>::V V;
  typedef typename PT<P>::R R;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
    const double bi = b[i];
    rn[i] = vreal<V>(bi);
    rm[i] = vzero<V>();
    if (np > 0) {
      proj[i] = rfrom_double<R>(bi);
      for (int l = 1; l < np; ++l) proj[(size_t)l * ld + i] = rfrom_double<R>(left[(size_t)(l - 1) * m + i]);
    }
  }
}

// x_k = 0, p_k = b for every shift (full mode, Eq. 23-24 initialisation).
template <class V>
__global__ void k_init_xp(int m, int K, const double* __restrict__ b, V* X, V* Pv) {
  const long long total = (long long)K * m;
  for (long long o = blockIdx.x * (long long)blockDim.x + threadIdx.x; o < total;
       o += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(o % m);
    X[o] = vzero<V>();
    Pv[o] = vreal<V>(b[i]);
  }
}

// FP64 dots of b with b and with each left vector (from the caller's FP64 arrays):
// last block writes rho_0 = b^T b, ||b||, the threshold and w0 = P b.
template <int NPM>
__global__ void __launch_bounds__(256)
k_init_dots(int m, int np, const double* __restrict__ b, const double* __restrict__ left, double tol,
            State* st, double* part, double2* w0) {
  double acc[NPM + 1];
#pragma unroll
  for (int l = 0; l <= NPM; ++l) acc[l] = 0.0;
  const int n = 1 + (np > 1 ? np - 1 : 0);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
    const double bi = b[i];
    acc[0] += bi * bi;
#pragma unroll
    for (int l = 1; l <= NPM; ++l)
      if (l < n) acc[l] += left[(size_t)(l - 1) * m + i] * bi;
  }
  __shared__ double red[NPM + 1];
  block_sum<NPM + 1, double>(acc, n, red);
  for (int k = threadIdx.x; k < n; k += blockDim.x) part[(size_t)blockIdx.x * n + k] = red[k];
  if (!arrive_last(&st->cnt_init)) return;
  __shared__ double all[NPM + 1];
  reduce_partials<NPM + 1>(part, gridDim.x, n, n, all);
  if (threadIdx.x == 0) {
    st->cnt_init = 0;
    st->rho = make_double2(all[0], 0.0);
    st->rho1 = st->rho;             // the first K1 forms alpha_0 from rho1 and inv_rho_alpha = 0 (beta_{-1} = 0)
    st->inv_rho_alpha = make_double2(0.0, 0.0);
    st->norm_b = sqrt(all[0]);
    st->thresh = tol * st->norm_b;
    if (np > 0) w0[0] = make_double2(all[0], 0.0);
    for (int l = 1; l < np; ++l) w0[l] = make_double2(all[l], 0.0);
    if (!(all[0] > 0.0) || !isfinite(all[0])) set_fail(st, KW_ERR_ARG);
  }
}

// BiCG start: r~_0 = b~, r~_{-1} = 0, and rho_0 = b~^T b (b, b~ real) by the last block.
template <int P>
__global__ void __launch_bounds__(256) k_init_shadow(int m, const double* __restrict__ bt, const double* __restrict__ b,
                                                     typename PT<P>::V* rt0, typename PT<P>::V* rtm, State* st,
                                                     double* __restrict__ part) {
  typedef typename PT<P>::V V;
  double acc = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
    rt0[i] = vreal<V>(bt[i]);
    rtm[i] = vzero<V>();
    acc = fma(bt[i], b[i], acc);
  }
  __shared__ double red[1];
  {
    double v1[1] = {acc};
    block_sum<1, double>(v1, 1, red);
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
  if (!arrive_last(&st->cnt_init)) return;
  __shared__ double tot[1];
  reduce_partials<1>(part, gridDim.x, 1, 1, tot);
  if (threadIdx.x == 0) {
    st->cnt_init = 0;
    st->rho = make_double2(tot[0], 0.0);
    st->rho1 = st->rho;
    if (tot[0] == 0.0) set_fail(st, KW_ERR_BREAKDOWN);
  }
}

static __global__ void k_init_shifts(int K, int np, double2* pi1, double2* pi0, int* active, long long* conv_iter,
                                     double* final_res, double2* Y, double2* U, const double2* w0) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= K) return;
  pi1[k] = pi0[k] = make_double2(1.0, 0.0);
  active[k] = 1;
  conv_iter[k] = -1;
  final_res[k] = INFINITY;
  for (int l = 0; l < np; ++l) {
    Y[(size_t)k * np + l] = make_double2(0.0, 0.0);
    U[(size_t)k * np + l] = w0[l];
  }
}

// out[k][l] = a_l^T x_k (a_0 = b), FP64 from the caller's FP64 vectors; one block per shift.
template <int P, int NPM>
__global__ void __launch_bounds__(256)
k_project_x(int m, int np, const double* __restrict__ b, const double* __restrict__ left,
            const typename PT<P>::V* __restrict__ X, double2* out) {
  typedef typename PT<P>::V V;
  const int k = blockIdx.x;
  double acc[2 * NPM];
#pragma unroll
  for (int l = 0; l < 2 * NPM; ++l) acc[l] = 0.0;
  const V* xk = X + (size_t)k * m;
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    const double2 x = vto_double(xk[i]);
#pragma unroll
    for (int l = 0; l < NPM; ++l) {
      if (l < np) {
        const double a = (l == 0) ? b[i] : left[(size_t)(l - 1) * m + i];
        acc[2 * l] = fma(a, x.x, acc[2 * l]);
        acc[2 * l + 1] = fma(a, x.y, acc[2 * l + 1]);
      }
    }
  }
  __shared__ double red[2 * NPM];
  block_sum<2 * NPM, double>(acc, 2 * np, red);
  for (int l = threadIdx.x; l < np; l += blockDim.x) out[(size_t)k * np + l] = make_double2(red[2 * l], red[2 * l + 1]);
}

// In-place conversion of FP32-pair complex vectors to FP64 complex (same 16 bytes):
// hi + lo is exact in FP64.
// In place: kw_c128 back to FP32 pairs (a resumed pair-form solve continues
// from the x that the previous solve converted for the caller).
static __global__ void k_double_to_pairs(dfc* x, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double2 d = reinterpret_cast<const double2*>(x)[i];
    x[i] = {df_from_double(d.x), df_from_double(d.y)};
  }
}

static __global__ void k_pairs_to_double(dfc* x, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const dfc v = x[i];
    reinterpret_cast<double2*>(x)[i] = vto_double(v);
  }
}

// out = (float)in; *inexact counts the values that FP32 does not represent exactly.
static __global__ void k_f64_to_f32(const double* __restrict__ in, float* __restrict__ out, int64_t n,
                                    unsigned long long* inexact) {
  unsigned long long bad = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float f = (float)in[i];
    out[i] = f;
    bad += ((double)f != in[i]);
  }
  bad = warp_sum(bad);
  if ((threadIdx.x & 31) == 0 && bad) atomicAdd(inexact, bad);
}

static __global__ void k_f64_to_pair(const double* __restrict__ in, df* __restrict__ out, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = df_from_double(in[i]);
}

// ================================================================ launchers
// Blocks that fit on the device at once for a kernel with the given block size.
// per_sm caches the occupancy of the kernel (a property of the kernel and the
// architecture); the SM count is the current context's.
// Launch of K1 or K2 on the work stream, with programmatic stream
// serialization when the grid is below one block per SM (see pdl_entry).
template <typename... KArgs, typename... Args>
static cudaError_t launch_k12(void (*kernel)(KArgs...), int grid, int num_sms, cudaStream_t s, Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = grid < num_sms ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

template <class F>
static int resident_blocks(int& per_sm, F kernel, int threads, int num_sms) {
  if (per_sm == 0) {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kernel, threads, 0) != cudaSuccess || b < 1) b = 1;
    per_sm = b;
  }
  return per_sm * num_sms;
}

template <int P, class RV, int G>
static cudaError_t spmv_launch(Work& w, const void* r, void* q, SpmvMode mode) {
  typedef typename PT<P>::V V;
  static int nblk_per_sm = 0;
  const int nblk = resident_blocks(nblk_per_sm, k_spmv_dot<P, RV, G>, 256, w.num_sms);
  const int need = (int)((w.m * G + 255) / 256);   // no more blocks than rows need
  const int grid = std::max(1, std::min(nblk, need));
  return launch_k12(k_spmv_dot<P, RV, G>, grid, w.num_sms, w.stream, (int)w.m, w.rowptr, w.col, (const RV*)w.val,
                    (const V*)r, (V*)q, w.st, w.part_k1, mode);
}

template <int P, class RV>
static cudaError_t sell_launch(Work& w, const void* r, void* q, SpmvMode mode) {
  typedef typename PT<P>::V V;
  static int nblk_per_sm = 0;
  const int nblk = resident_blocks(nblk_per_sm, k_spmv_sell<P, RV>, 256, w.num_sms);
  const int nslice = (int)((w.m + 31) / 32);
  const int grid = std::max(1, std::min(nblk, (nslice + 7) / 8));
  k_spmv_sell<P, RV><<<grid, 256, 0, w.stream>>>((int)w.m, nslice, w.sell_perm, w.sell_len, w.sell_ptr,
                                                 w.sell_col, (const RV*)w.sell_val, (const V*)r, (V*)q, w.st,
                                                 w.part_k1, mode);
  return cudaGetLastError();
}

template <int P, class RV>
static cudaError_t spmv_dispatch_v(Work& w, const void* r, void* q, SpmvMode mode) {
  if (w.spmv_lanes == KW_SPMV_SELL) {
    if (!w.sell_perm || !w.sell_len || !w.sell_ptr || !w.sell_col || !w.sell_val) return cudaErrorInvalidValue;
    return sell_launch<P, RV>(w, r, q, mode);
  }
  switch (w.spmv_lanes) {
    case 1: return spmv_launch<P, RV, 1>(w, r, q, mode);
    case 2: return spmv_launch<P, RV, 2>(w, r, q, mode);
    case 4: return spmv_launch<P, RV, 4>(w, r, q, mode);
    case 8: return spmv_launch<P, RV, 8>(w, r, q, mode);
    default: return spmv_launch<P, RV, 16>(w, r, q, mode);
  }
}

template <int P, class DV, int G>
static cudaError_t uniform_launch(Work& w, const void* r, void* q, SpmvMode mode) {
  typedef typename PT<P>::V V;
  static int nblk_per_sm = 0;
  const int nblk = resident_blocks(nblk_per_sm, k_spmv_u<P, DV, G>, 256, w.num_sms);
  const int need = (int)((w.m * G + 255) / 256);
  const int grid = std::max(1, std::min(nblk, need));
  DV uv;
  if constexpr (std::is_same<DV, double>::value) uv = w.u_v;
  else if constexpr (std::is_same<DV, float>::value) uv = (float)w.u_v;
  else {
    uv.hi = (float)w.u_v;
    uv.lo = (float)(w.u_v - (double)uv.hi);
  }
  k_spmv_u<P, DV, G><<<grid, 256, 0, w.stream>>>((int)w.m, w.u_rowptr, w.u_col, (const DV*)w.u_diag, uv,
                                                 (const V*)r, (V*)q, w.st, w.part_k1, mode);
  return cudaGetLastError();
}

template <int P, class DV>
static cudaError_t uniform_sell_launch(Work& w, const void* r, void* q, SpmvMode mode) {
  typedef typename PT<P>::V V;
  if (!w.u_sptr || !w.u_scol) return cudaErrorInvalidValue;
  static int nblk_per_sm = 0;
  const int nblk = resident_blocks(nblk_per_sm, k_spmv_us<P, DV>, 256, w.num_sms);
  const int nslice = (int)((w.m + 31) / 32);
  const int grid = std::max(1, std::min(nblk, (nslice + 7) / 8));   // one warp per slice, eight per block
  DV uv;
  if constexpr (std::is_same<DV, double>::value) uv = w.u_v;
  else if constexpr (std::is_same<DV, float>::value) uv = (float)w.u_v;
  else {
    uv.hi = (float)w.u_v;
    uv.lo = (float)(w.u_v - (double)uv.hi);
  }
  k_spmv_us<P, DV><<<grid, 256, 0, w.stream>>>((int)w.m, nslice, w.u_sptr, w.u_scol, (const DV*)w.u_diag, uv,
                                               (const V*)r, (V*)q, w.st, w.part_k1, mode);
  return cudaGetLastError();
}

template <int P, class DV>
static cudaError_t uniform_dispatch_g(Work& w, const void* r, void* q, SpmvMode mode) {
  if (w.spmv_lanes == KW_SPMV_UNIFORM_SELL) return uniform_sell_launch<P, DV>(w, r, q, mode);
  switch (w.spmv_lanes - KW_SPMV_UNIFORM) {
    case 1: return uniform_launch<P, DV, 1>(w, r, q, mode);
    case 2: return uniform_launch<P, DV, 2>(w, r, q, mode);
    case 4: return uniform_launch<P, DV, 4>(w, r, q, mode);
    case 8: return uniform_launch<P, DV, 8>(w, r, q, mode);
    default: return uniform_launch<P, DV, 16>(w, r, q, mode);
  }
}

// The diagonal/value type per form: FP64 (kind 0) only in the FP64 form, FP32
// (kind 1) when exact (always in the FP32 form), FP32 pairs (kind 2) in the pair form.
template <int P>
static cudaError_t uniform_dispatch(Work& w, const void* r, void* q, SpmvMode mode) {
  if (!w.u_rowptr || !w.u_col || !w.u_diag) return cudaErrorInvalidValue;
  if constexpr (P == PREC_F64) {
    if (w.u_kind == 1) return uniform_dispatch_g<P, float>(w, r, q, mode);
    return uniform_dispatch_g<P, double>(w, r, q, mode);
  } else if constexpr (P == PREC_C32) {
    return uniform_dispatch_g<P, float>(w, r, q, mode);
  } else {
    if (w.u_kind == 1) return uniform_dispatch_g<P, float>(w, r, q, mode);
    return uniform_dispatch_g<P, df>(w, r, q, mode);
  }
}

template <class DV>
__host__ __forceinline__ DV dv_from_double(double v) {
  if constexpr (std::is_same<DV, double>::value) return v;
  else if constexpr (std::is_same<DV, float>::value) return (float)v;
  else {
    DV d;
    d.hi = (float)v;
    d.lo = (float)(v - (double)d.hi);
    return d;
  }
}

template <int P, class DV>
static cudaError_t spin_launch(Work& w, const void* r, void* q, SpmvMode mode) {
  typedef typename PT<P>::V V;
  const int need = (int)((w.m + 255) / 256);
  if (w.sp_table) {
    if (w.sp_uniform) {
      static int per_sm = 0;
      const int nblk = resident_blocks(per_sm, k_spmv_spin_tab<P, DV, true>, 256, w.num_sms);
      k_spmv_spin_tab<P, DV, true><<<std::max(1, std::min(nblk, need)), 256, 0, w.stream>>>(
          (int)w.m, w.sp_table, (const DV*)w.sp_val, w.sp_nbond, (const DV*)w.u_diag, dv_from_double<DV>(w.u_v),
          (const V*)r, (V*)q, w.st, w.part_k1, mode);
    } else {
      static int per_sm = 0;
      const int nblk = resident_blocks(per_sm, k_spmv_spin_tab<P, DV, false>, 256, w.num_sms);
      k_spmv_spin_tab<P, DV, false><<<std::max(1, std::min(nblk, need)), 256, 0, w.stream>>>(
          (int)w.m, w.sp_table, (const DV*)w.sp_val, w.sp_nbond, (const DV*)w.u_diag, dv_from_double<DV>(w.u_v),
          (const V*)r, (V*)q, w.st, w.part_k1, mode);
    }
    return cudaGetLastError();
  }
  if (w.sp_uniform) {
    static int nblk_per_sm = 0;
    const int nblk = resident_blocks(nblk_per_sm, k_spmv_spin<P, DV, true>, 256, w.num_sms);
    k_spmv_spin<P, DV, true><<<std::max(1, std::min(nblk, need)), 256, 0, w.stream>>>(
        (int)w.m, w.sp_basis, w.sp_binom, w.sp_bond, (const DV*)w.sp_val, w.sp_nbond, (const DV*)w.u_diag,
        dv_from_double<DV>(w.u_v), (const V*)r, (V*)q, w.st, w.part_k1, mode);
  } else {
    static int nblk_per_sm = 0;
    const int nblk = resident_blocks(nblk_per_sm, k_spmv_spin<P, DV, false>, 256, w.num_sms);
    k_spmv_spin<P, DV, false><<<std::max(1, std::min(nblk, need)), 256, 0, w.stream>>>(
        (int)w.m, w.sp_basis, w.sp_binom, w.sp_bond, (const DV*)w.sp_val, w.sp_nbond, (const DV*)w.u_diag,
        dv_from_double<DV>(w.u_v), (const V*)r, (V*)q, w.st, w.part_k1, mode);
  }
  return cudaGetLastError();
}

template <int P, class DV>
static cudaError_t lattice_launch(Work& w, const void* r, void* q, SpmvMode mode) {
  typedef typename PT<P>::V V;
  static int nblk_per_sm = 0;
  const int nblk = resident_blocks(nblk_per_sm, k_spmv_lattice<P, DV>, 256, w.num_sms);
  const int grid = std::max(1, std::min(nblk, (int)((w.m + 255) / 256)));
  k_spmv_lattice<P, DV><<<grid, 256, 0, w.stream>>>((int)w.m, w.lx, w.ly, w.lz, (const DV*)w.u_diag,
                                                   dv_from_double<DV>(w.u_v), (const V*)r, (V*)q, w.st, w.part_k1,
                                                   mode);
  return cudaGetLastError();
}

// Generated operators: the diagonal storage kind selects the value type as in
// the uniform layout (FP64 in the FP64 form unless exact in FP32, FP32 in the
// FP32 form, FP32 pairs in the pair form unless exact in FP32).
template <int P>
static cudaError_t generated_dispatch(Work& w, const void* r, void* q, SpmvMode mode) {
  if (!w.u_diag || (w.op == OP_SPIN && (!w.sp_basis || !w.sp_binom || !w.sp_bond))) return cudaErrorInvalidValue;
#define KW_GEN(DV) (w.op == OP_SPIN ? spin_launch<P, DV>(w, r, q, mode) : lattice_launch<P, DV>(w, r, q, mode))
  if constexpr (P == PREC_F64) {
    if (w.u_kind == 1) return KW_GEN(float);
    return KW_GEN(double);
  } else if constexpr (P == PREC_C32) {
    return KW_GEN(float);
  } else {
    if (w.u_kind == 1) return KW_GEN(float);
    return KW_GEN(df);
  }
#undef KW_GEN
}

// K1 through the caller's matrix-vector callback.
// Under reverse communication the same path is cut in two: phase 1 stages r
// (and records where the caller finds r and puts H r), phase 2 finishes after
// the caller's product.
template <int P>
static cudaError_t matvec_dispatch(Work& w, const void* r, void* q, SpmvMode mode) {
  typedef typename PT<P>::V V;
  typedef typename MvT<P>::H H;
  const void* rin = r;
  void* hq = q;
  if constexpr (P == PREC_DF) {
    void* sr = (w.rci && w.mv_adjoint) ? w.mv_r2 : w.mv_r;
    void* sq = (w.rci && w.mv_adjoint) ? w.mv_q2 : w.mv_q;
    if (!sr || !sq) return cudaErrorInvalidValue;
    if (w.rci_phase != 2) {
      k_pairs_to_c128<<<4 * w.num_sms, 256, 0, w.stream>>>((int)w.m, (const dfc*)r, (double2*)sr, w.st,
                                                          mode.solver);
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) return e;
    }
    rin = sr;
    hq = sq;
  }
  if (w.rci_phase == 1) {     // the caller computes H r between the calls
    if (w.mv_adjoint) {
      w.rci_rt = rin;
      w.rci_qt = hq;
    } else {
      w.rci_r = rin;
      w.rci_q = hq;
    }
    return cudaSuccess;
  }
  if (w.rci_phase != 2) {
    kw_matvec_fn fn = (w.mv_adjoint && w.mv_fn_adj) ? w.mv_fn_adj : w.mv_fn;
    void* user = (w.mv_adjoint && w.mv_fn_adj) ? w.mv_user_adj : w.mv_user;
    if (fn(user, rin, hq, w.m, P == PREC_C32 ? KW_ELEM_C64 : KW_ELEM_C128, (void*)w.stream) != 0) {
      w.mv_failed = 1;
      return cudaErrorUnknown;
    }
  }
  static int nblk_per_sm = 0;
  const int nblk = resident_blocks(nblk_per_sm, k_matvec_finish<P>, 256, w.num_sms);
  const int grid = std::max(1, std::min(nblk, (int)((w.m + 255) / 256)));
  k_matvec_finish<P><<<grid, 256, 0, w.stream>>>((int)w.m, (const V*)r, (const H*)hq, (V*)q, w.st, w.part_k1, mode);
  return cudaGetLastError();
}

template <int P>
static cudaError_t spmv_dispatch(Work& w, const void* r, void* q, SpmvMode mode) {
  if (w.mv_fn || w.rci) return matvec_dispatch<P>(w, r, q, mode);
  if (w.op == OP_SPIN || w.op == OP_LATTICE) return generated_dispatch<P>(w, r, q, mode);
  if (w.spmv_lanes > KW_SPMV_UNIFORM) return uniform_dispatch<P>(w, r, q, mode);
  if constexpr (P == PREC_F64) {
    if (w.val_f32) return spmv_dispatch_v<P, float>(w, r, q, mode);
    return spmv_dispatch_v<P, double>(w, r, q, mode);
  } else if constexpr (P == PREC_C32) {
    return spmv_dispatch_v<P, float>(w, r, q, mode);
  } else {
    if (w.val_f32) return spmv_dispatch_v<P, float>(w, r, q, mode);
    return spmv_dispatch_v<P, df>(w, r, q, mode);
  }
}

template <int P, int NP, int METHOD>
static cudaError_t seed_launch(Work& w, void* rn, void* rm, int parity) {
  typedef typename PT<P>::V V;
  typedef typename PT<P>::R R;
  // shadow buffers rotate like the residual buffers (parity 0: r~_n in rtA)
  const void* rtn = parity ? w.rtB : w.rtA;
  void* rtm = parity ? w.rtA : w.rtB;
  const int ntiles = (int)((w.m + kSeedTile - 1) / kSeedTile);
  // Row-group form (pair form, COCG and CG): by default above nine projection rows
  if constexpr (P == PREC_DF && METHOD != KW_METHOD_BICG && NP > 0) {
    if (w.seed_rg > 0 || (w.seed_rg < 0 && w.nproj > 9)) {
      auto kern = k_seed_update_rg<NP, METHOD>;
      const int dyn = kRgStages * (int)rg_stage_bytes(w.nproj);
      static int attr_bytes = 0, occ_bytes = -1, per_sm = 1;
      cudaError_t e;
      if (dyn > attr_bytes) {
        if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn)) != cudaSuccess)
          return e;
        attr_bytes = dyn;
      }
      if (occ_bytes != dyn) {
        int b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, 256, dyn) != cudaSuccess || b < 1) b = 1;
        per_sm = b;
        occ_bytes = dyn;
      }
      const int grid = std::max(1, std::min(per_sm * w.num_sms, ntiles));
      kern<<<grid, 256, dyn, w.stream>>>((int)w.m, (const dfc*)rn, (const dfc*)w.q, (dfc*)rm, (const df*)w.proj_rows,
                                         w.proj_ld, w.nproj, parity, w.st, w.part, w.w, w.bulk == 2 ? 16u : 0u);
      return cudaGetLastError();
    }
  }
  // Staged form: the FP32 and FP32-pair forms, whose update is bound by memory
  // latency, not by the FP64 pipe; the BiCG shadow keeps plain loads.
  if constexpr (P != PREC_F64 && METHOD != KW_METHOD_BICG) {
    // auto (bulk < 0): staged when more than 9 projection rows make the plain kernel register-bound
    const bool staged = w.bulk > 0 || (w.bulk < 0 && w.nproj > 9);
    if (staged && w.m >= kSeedTile) {
      const uint32_t stage = seed_stage_bytes<V, R>(w.nproj);
      const int nstage = 3 * stage <= 72 * 1024 ? 3 : 2;
      const int dyn = nstage * (int)stage;
      static int attr_bytes = 0, occ_bytes = -1, per_sm = 1;
      auto kern = k_seed_update<P, NP, METHOD, true>;
      cudaError_t e;
      if (dyn > attr_bytes) {
        if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn)) != cudaSuccess)
          return e;
        attr_bytes = dyn;
      }
      if (occ_bytes != dyn) {
        int b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, 256, dyn) != cudaSuccess || b < 1) b = 1;
        per_sm = b;
        occ_bytes = dyn;
      }
      const int grid = std::max(1, std::min(per_sm * w.num_sms, ntiles));
      kern<<<grid, 256, dyn, w.stream>>>((int)w.m, (const V*)rn, (const V*)w.q, (V*)rm, (const R*)w.proj_rows,
                                         w.proj_ld, w.nproj, parity, w.st, w.part, w.w, (const V*)rtn,
                                         (const V*)w.qt, (V*)rtm, nstage, w.bulk == 2 ? 16u : 0u);
      return cudaGetLastError();
    }
  }
  static int nblk_per_sm = 0;
  const int nblk = resident_blocks(nblk_per_sm, k_seed_update<P, NP, METHOD, false>, 256, w.num_sms);
  const int grid = std::max(1, std::min(nblk, ntiles));
  return launch_k12(k_seed_update<P, NP, METHOD, false>, grid, w.num_sms, w.stream, (int)w.m, (const V*)rn,
                    (const V*)w.q, (V*)rm, (const R*)w.proj_rows, w.proj_ld, w.nproj, parity, w.st, w.part, w.w,
                    (const V*)rtn, (const V*)w.qt, (V*)rtm, 1, 0u);
}

template <int P, int METHOD>
static cudaError_t seed_dispatch_m(Work& w, void* rn, void* rm, int parity) {
  const int np = w.nproj;
  if (np == 0) return seed_launch<P, 0, METHOD>(w, rn, rm, parity);
  if (np <= 2) return seed_launch<P, 2, METHOD>(w, rn, rm, parity);
  if (np <= 5) return seed_launch<P, 5, METHOD>(w, rn, rm, parity);
  if (np <= 9) return seed_launch<P, 9, METHOD>(w, rn, rm, parity);
  if (np <= 17) return seed_launch<P, 17, METHOD>(w, rn, rm, parity);
  return seed_launch<P, KW_MAX_PROJ, METHOD>(w, rn, rm, parity);
}

template <int P>
static cudaError_t seed_dispatch(Work& w, void* rn, void* rm, int parity) {
  if (w.method == KW_METHOD_BICG) {
    if (!w.rtA || !w.rtB || !w.qt) return cudaErrorInvalidValue;
    return seed_dispatch_m<P, KW_METHOD_BICG>(w, rn, rm, parity);
  }
  if (w.method == KW_METHOD_CG) return seed_dispatch_m<P, KW_METHOD_CG>(w, rn, rm, parity);
  return seed_dispatch_m<P, KW_METHOD_COCG>(w, rn, rm, parity);
}

// K1 of iteration n+1 for the solver of Table 1 on r (and r~ for BiCG):
// COCG r^T q, CG r^dagger q; BiCG the product on r, the adjoint product on r~
// (conjugate seed shift; the adjoint callback when given) and r~^dagger q.
template <int P>
static cudaError_t k1_dispatch(Work& w, void* r, void* rt) {
  typedef typename PT<P>::V V;
  SpmvMode mode;
  mode.solver = 1;
  mode.zs = make_double2(0.0, 0.0);
  mode.zs_pair = make_float4(0.f, 0.f, 0.f, 0.f);
  mode.t_out = nullptr;
  if (w.method != KW_METHOD_BICG) {
    mode.conj_dot = w.method == KW_METHOD_CG;
    return spmv_dispatch<P>(w, r, w.q, mode);
  }
  if (!rt || !w.qt) return cudaErrorInvalidValue;
  mode.dot = 0;
  cudaError_t e = spmv_dispatch<P>(w, r, w.q, mode);
  if (e != cudaSuccess) return e;
  SpmvMode ms = mode;
  ms.conj_zs = 1;
  w.mv_adjoint = 1;   // the callback path takes the adjoint callback for this product
  e = spmv_dispatch<P>(w, rt, w.qt, ms);
  w.mv_adjoint = 0;
  if (e != cudaSuccess) return e;
  if (w.rci_phase == 1) return cudaSuccess;   // the products are the caller's to make first
  SpmvMode md = mode;
  md.dot = 1;
  static int nblk_per_sm = 0;
  const int nblk = resident_blocks(nblk_per_sm, k_dot_tail<P>, 256, w.num_sms);
  const int grid = std::max(1, std::min(nblk, (int)((w.m + 255) / 256)));
  k_dot_tail<P><<<grid, 256, 0, w.stream>>>((int)w.m, (const V*)rt, (const V*)w.q, w.st, w.part_k1, md);
  return cudaGetLastError();
}

// K4 with w.xp_tile shifts per tile (4, 8 or 16; the autotuner's pick) on the
// form's or the FP32 shift storage.  No more blocks than (shift tile, row
// chunk) items at full activity: every block takes part in the arrival count,
// so idle blocks would only add to it.
template <int P, int TS, bool XP32>
static cudaError_t update_xp_launch(Work& w, const void* r1, State* st, int parity, cudaStream_t s) {
  typedef typename XT<P, XP32>::V XV;
  typedef typename PT<P>::V V;
  static int nblk_per_sm = 0;
  // two complex FP32 elements per thread (FP32 storage, or the FP32 form) when both bases are 16-byte
  // aligned (x may be the caller's memory)
  const int pairs = std::is_same<XV, float2>::value && (reinterpret_cast<uintptr_t>(w.X) & 15) == 0 &&
                    (reinterpret_cast<uintptr_t>(w.P) & 15) == 0;
  const long long nunit = pairs ? w.m / 2 + 1 : w.m;
  const long long items = (long long)((w.K + TS - 1) / TS) * ((nunit + 255) / 256);
  const int nblk = (int)std::max<long long>(
      1, std::min<long long>(resident_blocks(nblk_per_sm, k_update_xp<P, TS, XP32>, 256, w.num_sms), items));
  const size_t c0 = (size_t)parity * 3 * w.K;
  k_update_xp<P, TS, XP32><<<nblk, 256, 0, s>>>((int)w.m, w.list + (size_t)parity * w.K, w.coef + c0,
                                                  w.coef_pair + c0, (XV*)w.X, (XV*)w.P, (const V*)r1, st, parity,
                                                  pairs);
  return cudaGetLastError();
}

template <int P>
cudaError_t launch_update_xp(Work& w, const void* r1, State* st, int parity, cudaStream_t s) {
  const int ts = w.xp_tile;
  if (w.xp32) {
    if (ts == 4) return update_xp_launch<P, 4, true>(w, r1, st, parity, s);
    if (ts == 16) return update_xp_launch<P, 16, true>(w, r1, st, parity, s);
    return update_xp_launch<P, 8, true>(w, r1, st, parity, s);
  }
  if (ts == 4) return update_xp_launch<P, 4, false>(w, r1, st, parity, s);
  if (ts == 16) return update_xp_launch<P, 16, false>(w, r1, st, parity, s);
  return update_xp_launch<P, 8, false>(w, r1, st, parity, s);
}

// One iteration n on three streams (K1(n) was enqueued by the previous
// iteration or by launch_init):
//   stream:  [wait K3(n-1)] [wait K4(n-2)] K2(n) [record ev_k2] K1(n+1)
//   stream2: [wait ev_k2] K3(n) [record ev_k3]
//   stream3: [wait ev_k3] K4(n) [record ev_k4[n & 1]]
// K1(n+1) needs only r_{n+1}; K3(n) needs only K2(n)'s scalars; K4(n) needs
// K3(n)'s coefficients and list and r_{n+1}.  K2(n+1) waits for K3(n) only: a
// seed switch decided by K3(n) reaches K1(n+1)'s product through K2(n+1)'s
// correction, and K4(n) runs beside K2(n+1), K3(n+1) and K1(n+2).  K4(n)'s
// inputs stay intact until K2(n+2): its r_{n+1} is the buffer K2(n+2)
// overwrites, and its coefficients, list and list length are in the slots of
// parity n & 1, which K2(n+2) (the length) and K3(n+2) write next.  So K2(n+2)
// waits for K4(n).  If ev is not NULL, ev[0..5] are recorded around K2 and K1
// (stream), K3 (stream2) and K4 (stream3).
template <int P>
cudaError_t launch_iteration(Work& w, int parity, int first, cudaEvent_t* ev, int64_t* launches) {
  typedef typename PT<P>::V V;
  if (!w.st || !w.part || !w.part_k1 || !w.rA || !w.rB || !w.q || !w.z || !w.list || !w.stream2 || !w.ev_k2 ||
      !w.ev_k3 || !w.stream3 || !w.ev_k4[0] || !w.ev_k4[1])
    return cudaErrorInvalidValue;
  // parity 0: r_n in rA, r_{n-1} in rB; parity 1: swapped.  K2 writes r_{n+1} over r_{n-1}.
  void* rn = parity ? w.rB : w.rA;
  void* rm = parity ? w.rA : w.rB;
  cudaError_t e;
#define KW_MARK(i, s) \
  if (ev && (e = cudaEventRecord(ev[i], s)) != cudaSuccess) return e;
  cudaStream_t s2 = w.overlap ? w.stream2 : w.stream;
  cudaStream_t s3 = w.overlap ? w.stream3 : w.stream;
  if (w.overlap && !first && (e = cudaStreamWaitEvent(w.stream, w.ev_k3, 0)) != cudaSuccess) return e;
  if (w.overlap && (w.k4_mask & (1 << parity)) && (e = cudaStreamWaitEvent(w.stream, w.ev_k4[parity], 0)) != cudaSuccess)
    return e;
  KW_MARK(0, w.stream);
  if ((e = seed_dispatch<P>(w, rn, rm, parity)) != cudaSuccess) return e;
  KW_MARK(1, w.stream);
  if (w.overlap && (e = cudaEventRecord(w.ev_k2, w.stream)) != cudaSuccess) return e;
  // K1(n+1) on r_{n+1} (and r~_{n+1}, which K2 wrote over r~_{n-1})
  if ((e = k1_dispatch<P>(w, rm, parity ? w.rtA : w.rtB)) != cudaSuccess) return e;
  KW_MARK(2, w.stream);

  if (w.overlap && (e = cudaStreamWaitEvent(s2, w.ev_k2, 0)) != cudaSuccess) return e;
  KW_MARK(3, s2);
  ShiftArgs a;
  a.K = w.K;
  a.np = w.nproj;
  a.full = w.full ? 1 : 0;
  a.parity = parity;
  a.z = w.z;
  a.pi1 = w.pi1;
  a.pi0 = w.pi0;
  a.active = w.active;
  a.conv_iter = w.conv_iter;
  a.final_res = w.final_res;
  a.coef = w.coef + (size_t)parity * 3 * w.K;
  a.coef_pair = w.coef_pair + (size_t)parity * 3 * w.K;
  a.Y = w.Y;
  a.U = w.U;
  a.w = w.w;
  a.hist = w.hist;
  a.list = w.list + (size_t)parity * w.K;
  a.part = w.part;
  a.log = w.log;
  a.log_max = w.log_max;
  // lanes per shift: one per projection row up to 4; beyond that each lane takes several rows, so
  // that the shift's FP64 scalars are not recomputed on many lanes and the grid (one warp per block,
  // each arriving on the block counter) stays small.  Every choice gives the same numbers.
  const int lps = w.nproj <= 1 ? 1 : w.nproj <= 2 ? 2 : 4;
  const int spw = 32 / lps;
  const int nb3 = (w.K + spw - 1) / spw;
  switch (lps) {
    case 1: k_shift<1><<<nb3, 32, 0, s2>>>(a, w.st); break;
    case 2: k_shift<2><<<nb3, 32, 0, s2>>>(a, w.st); break;
    case 4: k_shift<4><<<nb3, 32, 0, s2>>>(a, w.st); break;
    case 8: k_shift<8><<<nb3, 32, 0, s2>>>(a, w.st); break;
    case 16: k_shift<16><<<nb3, 32, 0, s2>>>(a, w.st); break;
    default: k_shift<32><<<nb3, 32, 0, s2>>>(a, w.st); break;
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  KW_MARK(4, s2);
  if (w.overlap && (e = cudaEventRecord(w.ev_k3, s2)) != cudaSuccess) return e;
  *launches += (w.mv_fn && P == PREC_DF) ? 4 : 3;
  if (w.full) {
    if (w.overlap && (e = cudaStreamWaitEvent(s3, w.ev_k3, 0)) != cudaSuccess) return e;
    if ((e = launch_update_xp<P>(w, rm, w.st, parity, s3)) != cudaSuccess) return e;
    KW_MARK(5, s3);
    if (w.overlap) {
      if ((e = cudaEventRecord(w.ev_k4[parity], s3)) != cudaSuccess) return e;
      w.k4_mask |= 1 << parity;
    }
    *launches += 1;
  }
#undef KW_MARK
  return cudaSuccess;
}

// K1 on r (and r~ for BiCG) outside the iteration, as launch_init ends: used
// when a stopped solve is resumed.
template <int P>
cudaError_t launch_k1(Work& w, void* r, void* rt) {
  return k1_dispatch<P>(w, r, rt);
}

template <int P>
cudaError_t launch_init(Work& w) {
  typedef typename PT<P>::V V;
  typedef typename PT<P>::R R;
  if (!w.st || !w.part || !w.part_k1 || !w.rA || !w.rB || !w.q || !w.b || !w.pi1 || !w.w0 ||
      (w.full && (!w.X || !w.P)))
    return cudaErrorInvalidValue;
  const int nb = 4 * w.num_sms;
  k_init_vectors<P><<<nb, 256, 0, w.stream>>>((int)w.m, w.nproj, w.b, w.left, (V*)w.rA, (V*)w.rB,
                                              (R*)w.proj_rows, w.proj_ld);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (w.full) {
    if (w.xp32) k_init_xp<float2><<<8 * w.num_sms, 256, 0, w.stream>>>((int)w.m, w.K, w.b, (float2*)w.X, (float2*)w.P);
    else k_init_xp<V><<<8 * w.num_sms, 256, 0, w.stream>>>((int)w.m, w.K, w.b, (V*)w.X, (V*)w.P);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if (w.nproj <= 8)
    k_init_dots<8><<<nb, 256, 0, w.stream>>>((int)w.m, w.nproj, w.b, w.left, w.tol, w.st, w.part, w.w0);
  else
    k_init_dots<KW_MAX_PROJ><<<nb, 256, 0, w.stream>>>((int)w.m, w.nproj, w.b, w.left, w.tol, w.st, w.part, w.w0);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_init_shifts<<<(w.K + 127) / 128, 128, 0, w.stream>>>(w.K, w.nproj, w.pi1, w.pi0, w.active, w.conv_iter,
                                                        w.final_res, w.Y, w.U, w.w0);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (w.method == KW_METHOD_BICG) {   // r~_0 = b~ (default b), r~_{-1} = 0, rho_0 = b~^T b
    if (!w.rtA || !w.rtB || !w.qt) return cudaErrorInvalidValue;
    k_init_shadow<P><<<nb, 256, 0, w.stream>>>((int)w.m, w.btilde ? w.btilde : w.b, w.b, (V*)w.rtA, (V*)w.rtB,
                                               w.st, w.part);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  // K1(0) on r_0 (rA); every iteration then enqueues the next K1 after its K2
  return k1_dispatch<P>(w, w.rA, w.rtA);
}

template <int P>
cudaError_t launch_unfinish_x(Work& w) {
  if constexpr (P == PREC_DF) {
    k_double_to_pairs<<<8 * w.num_sms, 256, 0, w.stream>>>((dfc*)w.X, (long long)w.K * w.m);
    return cudaGetLastError();
  } else {
    return cudaSuccess;
  }
}

// Full-mode outputs: FP32-pair vectors are first converted to FP64 in place
// (the caller's x buffer holds kw_c128 in that form), then projected.
template <int P>
cudaError_t launch_finish_x(Work& w) {
  if constexpr (P == PREC_DF) {
    k_pairs_to_double<<<8 * w.num_sms, 256, 0, w.stream>>>((dfc*)w.X, (long long)w.K * w.m);
    return cudaGetLastError();
  } else {
    return cudaSuccess;
  }
}

template <int P>
cudaError_t launch_project_x(Work& w, double2* out) {
  // after launch_finish_x the FP32-pair form holds FP64 values
  typedef typename std::conditional<P == PREC_C32, float2, double2>::type XV;
  constexpr int PX = P == PREC_C32 ? PREC_C32 : PREC_F64;
  const int np = w.nout;
  if (np <= 8)
    k_project_x<PX, 8><<<w.K, 256, 0, w.stream>>>((int)w.m, np, w.b, w.left, (const XV*)w.X, out);
  else
    k_project_x<PX, KW_MAX_PROJ><<<w.K, 256, 0, w.stream>>>((int)w.m, np, w.b, w.left, (const XV*)w.X, out);
  return cudaGetLastError();
}

template <int P>
cudaError_t launch_spmv_dot(Work& w, const void* r, void* q, double2 zs, float4 zs_pair, double2* t_dev) {
  SpmvMode mode;
  mode.solver = 0;
  mode.zs = zs;
  mode.zs_pair = zs_pair;
  mode.t_out = t_dev;
  return spmv_dispatch<P>(w, r, q, mode);
}

}  // namespace kw
